"""Pins of the oracle's neighbourhood overlap (Sec. III-B: the active set
holds the instances that overlap a new segment "or their immediate
neighborhood").

Reading: with overlap_dilation, a segment voxel overlaps every instance that
labels the voxel itself or one of its 26 neighbours in the map before the
frame, once per instance; the overlap gate and everything after it are
unchanged.  Checked by brute force over Tiny frames (the overlap histogram
recomputed from the exported map with Python sets) and by a wall seen again
one voxel deeper: disjoint from the first view, merged only with dilation.
"""
import numpy as np

import oracle
import synth
from tests import scenes

B = 1 << 17


def _pack(k):
    return ((k[0] + B) << 36) | ((k[1] + B) << 18) | (k[2] + B)


def _neigh(key):
    k = oracle.unpack_key(key)
    return [_pack((k[0] + a, k[1] + b, k[2] + c)) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def test_brute_force_dilated_overlap_on_tiny_frames():
    sc = synth.tiny_scene()
    fr = sc.render(range(0, 12, 2))
    m = oracle.OracleMap(**oracle.config_for_scene(sc, overlap_dilation=1))
    plain = oracle.OracleMap(**oracle.config_for_scene(sc))
    grew = 0
    for i in range(len(fr)):
        keys0, ids0 = m.voxels()
        before = dict(zip(keys0.tolist(), ids0.tolist()))
        r = m.integrate(*oracle.frame_args(fr, i))
        ov = {}
        new = set()
        for mm, k in zip(r["seg_m"].tolist(), r["seg_keys"].tolist()):
            roots = {before[n] for n in _neigh(k) if n in before}
            for root in roots:
                ov[(mm, root)] = ov.get((mm, root), 0) + 1
            if k not in before:
                new.add(k)
        assert r["overlap_pairs"] == len(ov)
        assert r["active_instances"] == len({k for (_, k) in ov})
        assert r["new_voxels"] == len(new)
        keys1, _ = m.voxels()
        assert set(keys1.tolist()) == set(before) | new
        rp = plain.integrate(*oracle.frame_args(fr, i))
        grew += r["overlap_pairs"] > rp["overlap_pairs"]
    assert grew > 0  # the neighbourhood reaches instances the voxels themselves miss


def _wall(z, seed=0):
    H, W, f = 24, 32, 30.0
    depth = scenes.plane_depth(H, W, f, f, W / 2, H / 2, z)
    labels = np.ones((H, W), np.uint16)
    rng = np.random.default_rng(seed)
    tok = rng.standard_normal((12, 16)).astype(np.float32)
    return depth, labels, tok, (f, f, W / 2, H / 2)


def test_wall_one_voxel_deeper_merges_only_with_dilation():
    s = 0.05
    z0 = 1.013  # keys z = 20; z0 + s -> 21, z0 + 2 s -> 22
    pose = scenes.identity_pose()
    for shift, merged_dilated in ((1, True), (2, False)):
        out = {}
        for dil in (0, 1):
            cfg = oracle.default_config(16, 3, 4, s, min_mask_pixels=3, overlap_dilation=dil)
            m = oracle.OracleMap(**cfg)
            d0, l0, t0, intr = _wall(z0)
            m.integrate(d0, l0, t0, pose, intr, 1)
            d1, l1, _, _ = _wall(z0 + shift * s)
            r = m.integrate(d1, l1, t0, pose, intr, 1)  # same tokens: cosine 1
            out[dil] = r
        assert out[0]["overlap_pairs"] == 0 and out[0]["rep"][0] == 1 and out[0]["new_instances"] == 1
        if merged_dilated:
            assert out[1]["overlap_pairs"] == 1 and out[1]["rep"][0] == 0 and out[1]["new_instances"] == 0
        else:
            assert out[1]["overlap_pairs"] == 0 and out[1]["rep"][0] == 1
