"""Pins of the oracle's second token grid and the query heatmap.

Reading (Sec. III-A/B, III-C): DINOv2 tokens drive instance association and
CLIP tokens the stored embedding.  With a second grid, each mask's
association feature is the pixel-level mean of that grid's tokens over the
mask; the association cosine gate (and the end-of-trajectory merge) compares
those features, while Eq. 1, the quality terms and the stored embedding stay
on the first grid; the winning observation of a fusion brings both.

Fig. 2's heatmap of a query vector q over a token grid is D_p * cos(f_p, q).
"""
import numpy as np
import pytest

import oracle
import synth
from tests import scenes

PA_H, PA_W, DA = 6, 8, 96


def _box(pid, c, h):
    return (0, pid, tuple(np.asarray(c) + 0.013), tuple(h))


def test_assoc_feature_is_the_pixel_mean_of_the_second_grid():
    sc = synth.tiny_scene()
    fr = sc.render(range(4))
    at = fr.assoc_tokens(PA_H, PA_W, DA)
    m = oracle.OracleMap(**oracle.config_for_scene(sc, assoc_dim=DA, assoc_patch_h=PA_H, assoc_patch_w=PA_W))
    for i in range(len(fr)):
        r = m.integrate(*oracle.frame_args(fr, i), assoc_tokens=at[i])
        H, W = fr.labels[i].shape
        v, u = np.mgrid[0:H, 0:W]
        patch = (v * PA_H // H) * PA_W + (u * PA_W // W)  # pixel -> patch of the second grid
        for k in range(int(fr.num_masks[i])):
            sel = fr.labels[i] == k + 1
            if r["npix"][k] < m.cfg["min_mask_pixels"]:
                assert not np.any(r["A"][k])
                continue
            want = at[i][patch[sel]].astype(np.float64).mean(axis=0)
            np.testing.assert_allclose(r["A"][k], want, rtol=1e-5, atol=1e-6)


def _two_views(seed_a, seed_b, assoc_same):
    prims = [_box(1, (0, 0, 0.2), (0.3, 0.3, 0.2))]
    poses = scenes.orbit((0, 0, 0.2), 1.5, 1.0, 2, sweep=np.deg2rad(5))
    sc_a = scenes.custom_scene(prims, poses, seed=seed_a)
    sc_b = scenes.custom_scene(prims, poses, seed=seed_b)
    fa, fb = sc_a.render([0]), sc_b.render([1])
    aa = fa.assoc_tokens(PA_H, PA_W, DA)[0]
    ab = (sc_a if assoc_same else scenes.custom_scene(prims, poses, seed=seed_a + 10)).render([1])
    ab = ab.assoc_tokens(PA_H, PA_W, DA)[0]
    return sc_a, fa, fb, aa, ab


@pytest.mark.parametrize("clip_same,dino_same", [(False, True), (True, False), (True, True), (False, False)])
def test_association_follows_the_second_grid(clip_same, dino_same):
    sc_a, fa, fb, aa, ab = _two_views(1, 1 if clip_same else 2, dino_same)
    cfg = oracle.config_for_scene(sc_a, assoc_dim=DA, assoc_patch_h=PA_H, assoc_patch_w=PA_W)
    m = oracle.OracleMap(**cfg)
    m.integrate(*oracle.frame_args(fa, 0), assoc_tokens=aa)
    r = m.integrate(*oracle.frame_args(fb, 0), assoc_tokens=ab)
    k = list(fb.mask_ids[0]).index(1)
    assert r["rep"][k] == (0 if dino_same else 1), (clip_same, dino_same)
    # one grid only: the first grid decides
    m1 = oracle.OracleMap(**oracle.config_for_scene(sc_a))
    m1.integrate(*oracle.frame_args(fa, 0))
    r1 = m1.integrate(*oracle.frame_args(fb, 0))
    assert r1["rep"][k] == (0 if clip_same else 1)


def test_fusion_brings_both_embeddings_of_the_winner():
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    at = fr.assoc_tokens(PA_H, PA_W, DA)
    m = oracle.OracleMap(**oracle.config_for_scene(sc, assoc_dim=DA, assoc_patch_h=PA_H, assoc_patch_w=PA_W))
    switched = 0
    for i in range(len(fr)):
        before = m.instances()
        r = m.integrate(*oracle.frame_args(fr, i), assoc_tokens=at[i])
        inst = m.instances()
        for k in range(int(fr.num_masks[i])):
            rid = int(r["rep"][k])
            if rid < 0:
                continue
            # an instance's (E, A) is always one observation's pair
            if np.array_equal(inst["E"][rid], r["E"][k]):
                assert np.array_equal(inst["A"][rid], r["A"][k])
                switched += rid < len(before["parent"])
    assert switched > 0  # some existing instance adopted a later view


def test_heatmap_closed_forms_and_fp64():
    rng = np.random.default_rng(3)
    F = rng.standard_normal((40, 64)).astype(np.float32)
    st = oracle.token_stats(F)
    for j in (0, 7, 39):
        h = oracle.query_heatmap(F, F[j])
        assert h[j] == st["Dp"][j]  # cos(f_j, f_j) = 1
        hn = oracle.query_heatmap(F, -F[j])
        assert hn[j] == -st["Dp"][j]
    # orthogonal support: tokens on the first 32 dims, query on the rest
    G = F.copy()
    G[:, 32:] = 0
    q = np.zeros(64, np.float32)
    q[32:] = 1
    assert not np.any(oracle.query_heatmap(G, q))
    # fp64 brute force
    q = rng.standard_normal(64).astype(np.float32)
    F64 = F.astype(np.float64)
    r = np.linalg.norm(F64 - F64.mean(axis=0), axis=1)
    D64 = r / (r.mean() + 1e-6)
    c64 = F64 @ q / (np.linalg.norm(F64, axis=1) * np.linalg.norm(q))
    np.testing.assert_allclose(oracle.query_heatmap(F, q), D64 * c64, rtol=1e-5, atol=1e-6)
