"""Pins of the oracle's DBSCAN noise filter (Sec. III-A: segment points are
filtered by DBSCAN before voxelisation).

Reading: core = at least min_pts points of the segment (itself included)
within eps; kept = core or within eps of a core point; the rest is noise.
Checked against a brute-force statement of that definition, exact hand cases
(points on a dyadic grid, so every distance is exact), and a frame whose
outlier pixels must leave exactly as if they had no label.
"""
import numpy as np
import pytest

import oracle
from tests import scenes


def _brute(pts, seg, eps, min_pts):
    pts = np.asarray(pts, np.float32)
    seg = np.asarray(seg)
    e2 = np.float32(eps) * np.float32(eps)
    n = len(pts)
    core = np.zeros(n, bool)
    near = np.zeros((n, n), bool)
    for i in range(n):
        d = pts[i][None, :] - pts  # float32 element-wise, as written
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        near[i] = (d2 <= e2) & (seg == seg[i])
        core[i] = near[i].sum() >= min_pts
    keep = core | (near & core[None, :]).any(axis=1)
    return ~keep


@pytest.mark.parametrize("seed,eps,min_pts", [(0, 0.05, 4), (1, 0.08, 6), (2, 0.03, 3), (3, 0.05, 1)])
def test_matches_brute_force_on_clustered_points(seed, eps, min_pts):
    rng = np.random.default_rng(seed)
    pts, seg = [], []
    for s in range(4):  # a dense cluster and scattered points per segment
        c = rng.uniform(-1, 1, 3)
        pts.append(c + 0.02 * rng.standard_normal((150, 3)))
        pts.append(c + 0.4 * rng.standard_normal((40, 3)))
        seg += [s + 1] * 190
    pts = np.concatenate(pts).astype(np.float32)
    seg = np.array(seg, np.int32)
    got = oracle.dbscan_noise(pts, seg, eps, min_pts)
    want = _brute(pts, seg, eps, min_pts)
    assert np.array_equal(got, want)
    if min_pts == 1:
        assert not got.any()
    else:
        assert 0 < got.sum() < len(pts)


def test_core_border_and_noise_by_hand():
    eps = 0.25
    q = 0.125
    cluster = [(0, 0, 0), (q, 0, 0), (0, q, 0), (q, q, 0)]   # pairwise <= 0.177: 4 neighbours each
    border = (0.375, 0, 0)       # exactly eps from (q, 0, 0), farther from the rest: 2 neighbours
    lone = (1.0, 0, 0)           # nothing within eps
    other = (0.0625, 0, 0)       # inside the cluster but of another segment
    pts = cluster + [border, lone, other]
    seg = [1, 1, 1, 1, 1, 1, 2]
    noise = oracle.dbscan_noise(pts, seg, eps, 4)
    assert noise.tolist() == [False, False, False, False, False, True, True]
    # with a border point one ulp beyond eps it becomes noise
    far = np.nextafter(np.float32(0.375), np.float32(1))
    noise = oracle.dbscan_noise(cluster + [(float(far), 0, 0)], [1] * 5, eps, 4)
    assert noise.tolist() == [False] * 4 + [True]


def _wall_frame(outliers):
    H, W, f = 48, 64, 50.0
    depth = scenes.plane_depth(H, W, f, f, W / 2, H / 2, 2.0)
    labels = np.ones((H, W), np.uint16)
    for (v, u) in outliers:
        depth[v, u] = 1.5  # half a metre in front of the wall
    rng = np.random.default_rng(5)
    tok = rng.standard_normal((48, 16)).astype(np.float32)
    return depth, labels, tok, (f, f, W / 2, H / 2)


def test_frame_outliers_leave_as_if_unlabelled():
    outliers = [(10, 10), (20, 40), (30, 25), (40, 50)]
    depth, labels, tok, intr = _wall_frame(outliers)
    pose = scenes.identity_pose()
    cfg = oracle.default_config(16, 6, 8, 0.05, min_mask_pixels=3)
    # pixels 4 cm apart at 2 m: an interior wall point has itself and 4
    # neighbours within 5 cm (diagonals are 5.7 cm away)
    a = oracle.OracleMap(**dict(cfg, dbscan_eps=0.05, dbscan_min_pts=4))
    ra = a.integrate(depth, labels, tok, pose, intr, 1)
    lab0 = labels.copy()
    for (v, u) in outliers:
        lab0[v, u] = 0
    b = oracle.OracleMap(**cfg)
    rb = b.integrate(depth, lab0, tok, pose, intr, 1)
    assert ra["denoised_pixels"] == len(outliers) and rb["denoised_pixels"] == 0
    assert ra["valid_pixels"] == rb["valid_pixels"]
    assert np.array_equal(ra["seg_keys"], rb["seg_keys"]) and np.array_equal(ra["nvox"], rb["nvox"])
    assert np.array_equal(ra["S"][:, 1].view(np.uint32), rb["S"][:, 1].view(np.uint32))  # S_angle
    ka, ia = a.voxels()
    kb, ib = b.voxels()
    assert np.array_equal(ka, kb) and np.array_equal(ia, ib)
    # min_pts = 1 keeps everything: the outliers are voxelised
    c = oracle.OracleMap(**dict(cfg, dbscan_eps=0.05, dbscan_min_pts=1))
    rc = c.integrate(depth, labels, tok, pose, intr, 1)
    assert rc["denoised_pixels"] == 0 and rc["valid_pixels"] == ra["valid_pixels"] + len(outliers)
