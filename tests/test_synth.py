"""The synthetic input generator (plumbing shared by both sides): the grid
traversal of many-primitive scenes gives exactly the frames of testing every
primitive."""
import numpy as np

import synth


def test_grid_traversal_equals_testing_every_primitive():
    sc = synth.multistory_scene(width=160, height=120)
    assert len(sc.prims) > 200
    idx = [0, 900, 1800, 2600, 3500, 4400]
    a = sc.render(idx)
    b = sc.render(idx, grid=False)
    assert np.array_equal(a.ids, b.ids)
    assert np.array_equal(a.depth.view(np.uint32), b.depth.view(np.uint32))
    assert np.array_equal(a.labels, b.labels) and np.array_equal(a.tokens, b.tokens)
    assert (a.num_masks > 10).all()


def test_tiny_recipe():
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    assert (sc.width, sc.height, sc.fx, sc.patch_h, sc.patch_w, sc.dim) == (64, 48, 50.0, 6, 8, 512)
    assert fr.depth.shape == (20, 48, 64) and fr.tokens.shape == (20, 48, 512)
    assert (fr.num_masks <= 8).all() and (fr.num_masks >= 4).all()
    # no depth noise: every depth is the exact ray-surface distance of a
    # plane (rendering twice gives the same bits, seeded)
    again = sc.render(range(20))
    assert np.array_equal(fr.depth.view(np.uint32), again.depth.view(np.uint32))
    assert np.array_equal(fr.tokens.view(np.uint32), again.tokens.view(np.uint32))


def _masks_are_the_largest_ids(fr, i, M):
    ids = fr.ids[i]
    vals, cnt = np.unique(ids[ids > 0], return_counts=True)
    order = sorted(zip(-cnt, vals))
    want = [int(v) for _, v in order[:M]]
    got = fr.mask_ids[i][: fr.num_masks[i]].tolist()
    assert got == want
    # label m marks exactly the pixels of the m-th id
    for m, oid in enumerate(got, start=1):
        assert np.array_equal(fr.labels[i] == m, ids == oid)


def test_room_recipe_masks_and_tokens():
    sc = synth.room_scene()
    assert (sc.width, sc.height, sc.fx, sc.patch_h, sc.patch_w, sc.dim, sc.max_masks) == (640, 480, 525.0, 24, 24,
                                                                                            768, 40)
    assert abs(sc.voxel_size - 0.025) < 1e-9 and sc.num_frames == 2000
    fr = sc.render([0, 500, 1000])
    for i in range(len(fr)):
        _masks_are_the_largest_ids(fr, i, sc.max_masks)
        assert fr.num_masks[i] >= 20
        # tokens: the mean of the object at each patch centre plus 0.1 noise
        H, W, Ph, Pw = sc.height, sc.width, sc.patch_h, sc.patch_w
        for p in (0, 137, 575):
            pi, pj = divmod(p, Pw)
            v = (2 * pi + 1) * H // (2 * Ph)
            u = (2 * pj + 1) * W // (2 * Pw)
            mu = sc.object_mean(int(fr.ids[i][v, u]))
            r = fr.tokens[i][p] - mu
            assert abs(float(r.std()) - 0.1) < 0.02 and abs(float(r.mean())) < 0.02


def test_room_depth_noise_is_about_one_percent():
    sc = synth.room_scene()
    clean = synth.room_scene()
    clean.depth_noise = 0.0
    a = sc.render([10])
    b = clean.render([10])
    assert np.array_equal(a.ids, b.ids)
    ok = (b.depth[0] > 0) & np.isfinite(b.depth[0])
    rel = a.depth[0][ok] / b.depth[0][ok] - 1.0
    assert 0.007 < float(rel.std()) < 0.013 and abs(float(rel.mean())) < 0.002
