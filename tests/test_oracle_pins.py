"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the CPU oracle against a closed form, an invariant, a special
case that reduces to a textbook computation, or a brute force on tiny inputs:
never against a re-typed copy of its own formula.  Passages: Eq. 1 (the
distinctiveness map), the D-weighted pooling and Eq. 2-3 (view quality) of
Sec. III-C; voxelisation of Sec. III-A; association and merging of Sec. III-B;
Q-replacement fusion of Sec. III-C.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import scenes

RNG = np.random.default_rng(1234)


# ---------------------------------------------------------------- Eq. 1 -----
def test_eq1_constant_tokens_give_zero_distinctiveness():
    F = np.full((48, 32), 0.3, np.float32)
    st = oracle.token_stats(F)
    assert np.all(st["Dp"] == 0.0)
    assert np.all(st["n"] == 0.0)
    assert np.all(st["fbar"] == np.float32(0.3))


def test_eq1_two_values_give_unit_distinctiveness():
    # half the patches equal a, half equal b: every residual norm is |a-b|/2,
    # so D_p = r / (r + eps) for all p
    P, D = 40, 64
    a, b = RNG.standard_normal(D), RNG.standard_normal(D)
    F = np.where(np.arange(P)[:, None] < P // 2, a, b).astype(np.float32)
    st = oracle.token_stats(F, eps=1e-6)
    r = np.linalg.norm(a - b) / 2
    np.testing.assert_allclose(st["Dp"], r / (r + 1e-6), rtol=2e-6)


@pytest.mark.parametrize("P", [5, 48, 576])
def test_eq1_one_distinct_patch(P):
    # P-1 copies of c and one c + delta:
    #   D_distinct = P / 2,  D_other = P / (2 (P - 1))   (eps -> 0)
    D = 32
    c = RNG.standard_normal(D)
    F = np.tile(c, (P, 1)).astype(np.float32)
    F[3 % P] += RNG.standard_normal(D).astype(np.float32)
    st = oracle.token_stats(F, eps=1e-9)
    Dp = st["Dp"]
    assert Dp[3 % P] == pytest.approx(P / 2, rel=1e-5)
    others = np.delete(Dp, 3 % P)
    np.testing.assert_allclose(others, P / (2 * (P - 1)), rtol=1e-4)


def test_eq1_mean_distinctiveness_is_one():
    # (1/P) sum_p D_p = nbar / (nbar + eps) for any tokens
    F = RNG.standard_normal((576, 96)).astype(np.float32) * 3 + 1
    st = oracle.token_stats(F, eps=1e-6)
    nbar = float(np.mean(st["n"].astype(np.float64)))
    assert float(np.mean(st["Dp"].astype(np.float64))) == pytest.approx(nbar / (nbar + 1e-6), rel=1e-6)


def test_eq1_translation_and_scale_invariance():
    F = RNG.standard_normal((48, 64)).astype(np.float32)
    d0 = oracle.token_stats(F, eps=0.0)["Dp"]
    d1 = oracle.token_stats(np.float32(4.0) * F + np.float32(0.75), eps=0.0)["Dp"]
    np.testing.assert_allclose(d1, d0, rtol=1e-5)


def test_eq1_permutation_equivariance_is_bit_exact():
    # sums are exact, so the order of patches cannot change a single bit
    F = RNG.standard_normal((96, 64)).astype(np.float32)
    perm = RNG.permutation(96)
    s0, s1 = oracle.token_stats(F), oracle.token_stats(F[perm])
    assert np.array_equal(s1["Dp"], s0["Dp"][perm])
    assert np.array_equal(s1["cosg"], s0["cosg"][perm])
    assert np.array_equal(s1["fbar"], s0["fbar"])


def test_eq1_matches_fp64_within_fp32_error():
    F = RNG.standard_normal((576, 128)).astype(np.float32)
    st = oracle.token_stats(F)
    cov = np.ones((1, 576), np.int32)
    Dp64, _ = oracle.pool_f64(F, cov, np.array([576], np.int32))
    np.testing.assert_allclose(st["Dp"], Dp64, rtol=2e-6)


def test_token_range_is_rejected():
    F = np.zeros((4, 8), np.float32)
    F[1, 2] = 2000.0
    with pytest.raises(ValueError):
        oracle.token_stats(F)
    F[1, 2] = np.nan
    with pytest.raises(ValueError):
        oracle.token_stats(F)


def test_cosine_closed_forms():
    a = RNG.standard_normal(64).astype(np.float32)
    assert oracle.cosine(a, a) == pytest.approx(1.0, abs=1e-7)
    assert oracle.cosine(a, -a) == pytest.approx(-1.0, abs=1e-7)
    b = np.zeros(64, np.float32)
    b[0], b[1] = 1.0, 0.0
    c = np.zeros(64, np.float32)
    c[1] = 2.0
    assert oracle.cosine(b, c) == 0.0
    assert oracle.cosine(b, np.zeros(64, np.float32)) == 0.0
    # 45 degrees
    c[0] = 2.0
    assert oracle.cosine(b, c) == pytest.approx(np.sqrt(0.5), abs=1e-7)


# ------------------------------------------------------------- coverage -----
def test_coverage_brute_force_ragged_grid():
    H, W, Ph, Pw, M = 37, 53, 5, 7, 6
    lab = RNG.integers(0, M + 2, size=(H, W)).astype(np.uint16)  # includes labels > M
    cov, npix = oracle.mask_coverage(lab, Ph, Pw, M)
    ref = np.zeros((M, Ph * Pw), np.int64)
    for v in range(H):
        for u in range(W):
            m = int(lab[v, u])
            if 1 <= m <= M:
                ref[m - 1, (v * Ph // H) * Pw + (u * Pw // W)] += 1
    assert np.array_equal(cov, ref)
    for m in range(1, M + 1):
        assert npix[m - 1] == int((lab == m).sum())


# --------------------------------------------------------------- pooling ----
def _tiny_frame(i=0):
    sc = synth.tiny_scene()
    fr = sc.render([i])
    return sc, fr


def test_pool_weights_sum_to_one_and_follow_coverage():
    sc, fr = _tiny_frame(3)
    m = oracle.OracleMap(**oracle.config_for_scene(sc))
    r = m.integrate(*oracle.frame_args(fr, 0))
    live = r["npix"] >= max(1, sc.width * sc.height // 1000)
    W = r["W"][live].astype(np.float64)
    np.testing.assert_allclose(W.sum(1), 1.0, atol=1e-6 * W.shape[1])
    assert np.all(W >= 0)
    assert np.all((W > 0) == (r["cov"][live] > 0))


def _single_view_map(D=32, Ph=6, Pw=8):
    return oracle.OracleMap(**oracle.default_config(D, Ph, Pw, 0.05))


def test_pool_mask_inside_one_patch_returns_that_token():
    H, W, Ph, Pw, D = 48, 64, 6, 8, 32
    lab = np.zeros((H, W), np.uint16)
    lab[9:12, 17:20] = 1     # rows 8..15 / cols 16..23 form patch (1, 2)
    F = RNG.standard_normal((Ph * Pw, D)).astype(np.float32)
    depth = np.full((H, W), 2.0, np.float32)
    r = _single_view_map(D, Ph, Pw).integrate(depth, lab, F, np.eye(4), (50, 50, 32, 24), 1)
    assert r["W"][0, 1 * Pw + 2] == 1.0
    np.testing.assert_allclose(r["E"][0], F[1 * Pw + 2], atol=1e-9, rtol=0)


def test_pool_uniform_distinctiveness_is_coverage_mean():
    # two token values on alternating patches -> D constant -> e = sum c f / sum c
    H, W, Ph, Pw, D = 48, 64, 6, 8, 32
    a, b = RNG.standard_normal(D), RNG.standard_normal(D)
    F = np.where((np.arange(Ph * Pw) % 2)[:, None] == 0, a, b).astype(np.float32)
    lab = np.zeros((H, W), np.uint16)
    lab[5:40, 3:50] = 1
    depth = np.full((H, W), 2.0, np.float32)
    r = _single_view_map(D, Ph, Pw).integrate(depth, lab, F, np.eye(4), (50, 50, 32, 24), 1)
    c = r["cov"][0].astype(np.float64)
    ref = (c[:, None] * F.astype(np.float64)).sum(0) / c.sum()
    np.testing.assert_allclose(r["E"][0], ref, rtol=0, atol=1e-6)


def test_pool_constant_tokens_fall_back_to_coverage_weights():
    H, W, Ph, Pw, D = 48, 64, 6, 8, 16
    F = np.full((Ph * Pw, D), -0.625, np.float32)
    lab = np.zeros((H, W), np.uint16)
    lab[10:30, 10:40] = 1
    depth = np.full((H, W), 2.0, np.float32)
    r = _single_view_map(D, Ph, Pw).integrate(depth, lab, F, np.eye(4), (50, 50, 32, 24), 1)
    c = r["cov"][0]
    np.testing.assert_allclose(r["W"][0], c / c.sum(), rtol=1e-7)
    np.testing.assert_allclose(r["E"][0], -0.625, atol=1e-9)
    assert r["S"][0, 3] == 0.5  # S_dist = 0.5 + 0.5 * 0


# ----------------------------------------------------------- Eq. 2 terms ----
@pytest.mark.parametrize("frac,expect", [(1 / 3.3, 1.0), (1 / 6.6, 0.5), (0.9, 1.0), (0.01, 0.033)])
def test_s_size(frac, expect):
    H, W, Ph, Pw, D = 100, 100, 4, 4, 8
    n = int(round(frac * H * W))
    lab = np.zeros(H * W, np.uint16)
    lab[:n] = 1
    lab = lab.reshape(H, W)
    F = RNG.standard_normal((Ph * Pw, D)).astype(np.float32)
    depth = np.full((H, W), 2.0, np.float32)
    r = _single_view_map(D, Ph, Pw).integrate(depth, lab, F, np.eye(4), (100, 100, 50, 50), 1)
    assert r["S"][0, 0] == pytest.approx(expect, abs=2e-3)


def test_s_sem_closed_forms():
    H, W, Ph, Pw, D = 48, 64, 6, 8, 16
    g = RNG.standard_normal(D).astype(np.float32)
    F = np.tile(g, (Ph * Pw, 1))
    lab = np.ones((H, W), np.uint16)
    depth = np.full((H, W), 2.0, np.float32)
    mp = _single_view_map(D, Ph, Pw)
    r = mp.integrate(depth, lab, F, np.eye(4), (50, 50, 32, 24), 1, global_embed=g)
    assert r["S"][0, 2] == pytest.approx(1.0, abs=1e-6)
    r = _single_view_map(D, Ph, Pw).integrate(depth, lab, -F, np.eye(4), (50, 50, 32, 24), 1, global_embed=g)
    assert r["S"][0, 2] == 0.0  # ReLU of cos = -1


def _plane_frame(theta, z0=2.013, H=48, W=64, f=2000.0):
    depth = scenes.plane_depth(H, W, f, f, W / 2, H / 2, z0, theta)
    lab = np.ones((H, W), np.uint16)
    return depth, lab, (f, f, W / 2, H / 2)


def test_s_angle_fronto_parallel_wall_is_one():
    depth, lab, intr = _plane_frame(0.0)
    F = RNG.standard_normal((48, 16)).astype(np.float32)
    r = _single_view_map(16, 6, 8).integrate(depth, lab, F, np.eye(4), intr, 1)
    assert r["S"][0, 1] == pytest.approx(1.0, abs=1e-3)


@pytest.mark.parametrize("deg", [20.0, 45.0, 60.0])
def test_s_angle_rotated_wall_is_cos_theta(deg):
    th = np.deg2rad(deg)
    depth, lab, intr = _plane_frame(th)
    F = RNG.standard_normal((48, 16)).astype(np.float32)
    cfg = oracle.default_config(16, 6, 8, 0.01)
    r = oracle.OracleMap(**cfg).integrate(depth, lab, F, np.eye(4), intr, 1)
    assert r["S"][0, 1] == pytest.approx(np.cos(th), abs=0.02)


# ------------------------------------------------------------- voxel keys ---
def test_keys_closed_form_grid():
    # identity pose, fx = z0 / s: pixel (u, v) lands in voxel (u - cx, v - cy, floor(z0/s))
    H, W, s, z0 = 24, 32, 0.05, 1.013
    fx = z0 / s
    depth = np.full((H, W), z0, np.float32)
    lab = np.ones((H, W), np.uint16)
    F = RNG.standard_normal((4, 8)).astype(np.float32)
    cfg = oracle.default_config(8, 2, 2, s)
    r = oracle.OracleMap(**cfg).integrate(depth, lab, F, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    got = {oracle.unpack_key(k) for k in r["seg_keys"]}
    want = {(u - W // 2, v - H // 2, 20) for u in range(W) for v in range(H)}
    assert got == want
    assert r["new_voxels"] == H * W and r["nvox"][0] == H * W


def test_keys_match_fp64_brute_force_on_tiny_frames():
    # the voxel set equals the unique quantised points of an independent fp64
    # back-projection (faces are placed off the voxel grid)
    sc = synth.tiny_scene()
    fr = sc.render(range(0, 20, 5))
    m = oracle.OracleMap(**oracle.config_for_scene(sc))
    min_px = max(1, sc.width * sc.height // 1000)
    for i in range(len(fr)):
        r = m.integrate(*oracle.frame_args(fr, i))
        lab, z, T = fr.labels[i], fr.depth[i].astype(np.float64), fr.poses[i]
        v, u = np.nonzero(lab)
        npix = np.bincount(lab.ravel(), minlength=256)
        ok = (z[v, u] >= 0.1) & (z[v, u] <= 10.0) & (npix[lab[v, u]] >= min_px)
        v, u = v[ok], u[ok]
        zz = z[v, u]
        xc = (u + 0.5 - sc.cx) * zz / sc.fx
        yc = (v + 0.5 - sc.cy) * zz / sc.fy
        P = (T[:3, :3] @ np.stack([xc, yc, zz]) + T[:3, 3:4]).T
        k = np.floor(P / sc.voxel_size).astype(np.int64)
        want = {(int(lab[vv, uu]), tuple(kk)) for vv, uu, kk in zip(v, u, k)}
        got = {(int(mm), oracle.unpack_key(kk)) for mm, kk in zip(r["seg_m"], r["seg_keys"])}
        assert got == want


def test_depth_validity_and_unlabelled_pixels_are_skipped():
    H, W = 20, 30
    depth = np.full((H, W), 2.0, np.float32)
    depth[0, :] = np.nan
    depth[1, :] = 0.05      # below z_min
    depth[2, :] = 50.0      # above z_max
    lab = np.ones((H, W), np.uint16)
    lab[:, 0] = 0
    F = RNG.standard_normal((4, 8)).astype(np.float32)
    r = oracle.OracleMap(**oracle.default_config(8, 2, 2, 0.05)).integrate(
        depth, lab, F, np.eye(4), (30, 30, 15, 10), 1)
    assert r["valid_pixels"] == (H - 3) * (W - 1)
    assert r["npix"][0] == H * (W - 1)


# ---------------------------------------------------- association / merge ---
def _run(scene, frames=None, **cfg):
    fr = scene.render(range(scene.num_frames) if frames is None else frames)
    m = oracle.OracleMap(**oracle.config_for_scene(scene, **cfg))
    reps = [m.integrate(*oracle.frame_args(fr, i)) for i in range(len(fr))]
    return m, fr, reps


def _box(pid, c, h):
    return (0, pid, tuple(np.asarray(c) + 0.013), tuple(h))


def test_one_box_seen_from_many_poses_stays_one_instance():
    sc = scenes.custom_scene([_box(1, (0, 0, 0.2), (0.3, 0.25, 0.2))],
                             scenes.orbit((0, 0, 0.2), 1.5, 0.9, 20, sweep=np.deg2rad(150)))
    m, fr, reps = _run(sc)
    inst = m.instances()
    live = np.nonzero(inst["parent"] == np.arange(len(inst["parent"])))[0]
    assert len(live) == 1
    for i, r in enumerate(reps):
        for k in range(fr.num_masks[i]):
            if fr.mask_ids[i][k] == 1:
                assert r["rep"][k] == live[0]
    assert inst["n_obs"][live[0]] == 20


def test_two_disjoint_boxes_stay_two_instances():
    prims = [_box(1, (-0.45, 0, 0.2), (0.25, 0.25, 0.2)), _box(2, (0.45, 0, 0.2), (0.25, 0.25, 0.2))]
    sc = scenes.custom_scene(prims, scenes.orbit((0, 0, 0.2), 1.8, 1.0, 12, start=-np.pi / 2,
                                                 sweep=np.deg2rad(60)))
    m, fr, reps = _run(sc)
    keys, ids = m.voxels()
    inst = m.instances()
    live = np.nonzero(inst["parent"] == np.arange(len(inst["parent"])))[0]
    assert len(live) == 2
    # every voxel's instance is one of the two, and each box keeps its own side
    kx = np.array([oracle.unpack_key(k)[0] for k in keys])
    left = set(ids[kx < 0])
    right = set(ids[kx >= 0])
    assert len(left) == 1 and len(right) == 1 and left != right


def test_similarity_gate_blocks_merge_of_dissimilar_segments():
    # identical geometry twice; with independent token means the second view
    # overlaps completely but is dissimilar -> a new instance (Sec. III-B)
    prims = [_box(1, (0, 0, 0.2), (0.3, 0.3, 0.2))]
    poses = scenes.orbit((0, 0, 0.2), 1.5, 1.0, 2, sweep=np.deg2rad(5))
    sc_a = scenes.custom_scene(prims, poses, seed=1)
    sc_b = scenes.custom_scene(prims, poses, seed=2)
    fa, fb = sc_a.render([0]), sc_b.render([1])
    cfg = oracle.config_for_scene(sc_a)
    same = oracle.OracleMap(**cfg)
    same.integrate(*oracle.frame_args(fa, 0))
    r_same = same.integrate(*oracle.frame_args(sc_a.render([1]), 0))
    diff = oracle.OracleMap(**cfg)
    diff.integrate(*oracle.frame_args(fa, 0))
    r_diff = diff.integrate(*oracle.frame_args(fb, 0))
    k_same = list(sc_a.render([1]).mask_ids[0]).index(1)
    k_diff = list(fb.mask_ids[0]).index(1)
    assert r_same["rep"][k_same] == 0 and r_same["new_instances"] == 0
    assert r_diff["rep"][k_diff] == 1 and r_diff["new_instances"] == 1


def test_overlap_gate_is_an_exact_rational_test():
    # second frame: one mask whose voxel set overlaps the first instance in
    # exactly 1/5 of its voxels -> passes at 1/5, fails at 21/100
    H, W, s, z0 = 10, 50, 0.05, 1.013
    fx = z0 / s
    depth = np.full((H, W), z0, np.float32)
    F = np.ones((4, 8), np.float32)
    lab1 = np.zeros((H, W), np.uint16)
    lab1[:, :10] = 1
    lab2 = np.zeros((H, W), np.uint16)
    lab2[:, 8:18] = 1   # 20 of its 100 voxels are old
    for num, den, expect_new in ((1, 5, 0), (21, 100, 1)):
        m = oracle.OracleMap(**oracle.default_config(8, 2, 2, s, ov_num=num, ov_den=den))
        m.integrate(depth, lab1, F, np.eye(4), (fx, fx, W // 2, H // 2), 1)
        r = m.integrate(depth, lab2, F, np.eye(4), (fx, fx, W // 2, H // 2), 1)
        assert r["new_instances"] == expect_new
        assert r["new_voxels"] == 80


def test_overlap_is_normalised_by_the_smaller_set():
    # a 2 x 5 fragment lies entirely inside a new 10 x 10 segment: 10 shared
    # voxels are 1/10 of the segment but all of the fragment -> merged
    H, W, s, z0 = 10, 10, 0.05, 1.013
    fx = z0 / s
    depth = np.full((H, W), z0, np.float32)
    F = np.ones((4, 8), np.float32)
    frag = np.zeros((H, W), np.uint16)
    frag[:5, :2] = 1
    m = oracle.OracleMap(**oracle.default_config(8, 2, 2, s))
    m.integrate(depth, frag, F, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    r = m.integrate(depth, np.ones((H, W), np.uint16), F, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    assert r["rep"][0] == 0 and r["new_instances"] == 0 and r["new_voxels"] == 90
    assert m.instances()["count"][0] == 100


def test_transitive_merge_keeps_the_smallest_id():
    # frame 1: the wall split into two disjoint masks -> instances 0 and 1;
    # frame 2: one mask covering both -> merged into 0 (Sec. III-B refinement)
    H, W, s, z0 = 20, 40, 0.05, 1.013
    fx = z0 / s
    depth = np.full((H, W), z0, np.float32)
    F = np.ones((4, 8), np.float32) + 0.01 * RNG.standard_normal((4, 8)).astype(np.float32)
    lab1 = np.zeros((H, W), np.uint16)
    lab1[:, :20] = 1
    lab1[:, 20:] = 2
    lab2 = np.ones((H, W), np.uint16)
    m = oracle.OracleMap(**oracle.default_config(8, 2, 2, s))
    r1 = m.integrate(depth, lab1, F, np.eye(4), (fx, fx, W // 2, H // 2), 2)
    assert list(r1["rep"]) == [0, 1]
    r2 = m.integrate(depth, lab2, F, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    assert r2["merges"] == 1 and r2["rep"][0] == 0
    inst = m.instances()
    assert list(inst["parent"]) == [0, 0]
    assert inst["count"][0] == H * W and inst["count"][1] == 0
    keys, ids = m.voxels()
    assert np.all(ids == 0)


def test_fusion_switches_to_a_higher_quality_view():
    # a closer view covers more pixels -> larger S_size -> its embedding replaces
    # the stored one (Sec. III-C)
    H, W, s, z0 = 40, 40, 0.05, 1.013
    fx = z0 / s
    depth = np.full((H, W), z0, np.float32)
    base = RNG.standard_normal(8).astype(np.float32)
    F1 = np.tile(base, (4, 1)) + 0.05 * RNG.standard_normal((4, 8)).astype(np.float32)
    F2 = np.tile(base, (4, 1)) + 0.05 * RNG.standard_normal((4, 8)).astype(np.float32)
    small = np.zeros((H, W), np.uint16)
    small[10:20, 10:20] = 1
    big = np.zeros((H, W), np.uint16)
    big[8:23, 8:23] = 1     # 15 x 15 voxels, 100 of them already mapped
    m = oracle.OracleMap(**oracle.default_config(8, 2, 2, s))
    r1 = m.integrate(depth, small, F1, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    r2 = m.integrate(depth, big, F2, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    assert r2["rep"][0] == 0 and r2["S"][0, 4] > r1["S"][0, 4]
    inst = m.instances()
    assert inst["Q"][0] == r2["S"][0, 4]
    assert np.array_equal(inst["E"][0], r2["E"][0])
    # a worse view afterwards does not replace it
    r3 = m.integrate(depth, small, F1, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    assert r3["rep"][0] == 0
    assert np.array_equal(m.instances()["E"][0], r2["E"][0])


def test_fusion_tie_keeps_the_incumbent():
    # swapping two embedding dimensions leaves every Q term bit-identical (all
    # sums are exact) but changes the embedding: strict '>' keeps the old one
    H, W, s, z0 = 40, 40, 0.05, 1.013
    fx = z0 / s
    depth = np.full((H, W), z0, np.float32)
    F1 = RNG.standard_normal((4, 16)).astype(np.float32) + 2.0
    F2 = F1.copy()
    F2[:, [0, 1]] = F2[:, [1, 0]]
    lab = np.zeros((H, W), np.uint16)
    lab[5:30, 5:30] = 1
    m = oracle.OracleMap(**oracle.default_config(16, 2, 2, s))
    r1 = m.integrate(depth, lab, F1, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    r2 = m.integrate(depth, lab, F2, np.eye(4), (fx, fx, W // 2, H // 2), 1)
    assert r2["S"][0, 4] == r1["S"][0, 4]
    assert not np.array_equal(r2["E"][0], r1["E"][0])
    assert r2["rep"][0] == 0
    assert np.array_equal(m.instances()["E"][0], r1["E"][0])


def test_brute_force_overlap_and_new_voxels_on_tiny_frames():
    # recompute the overlap histogram and the new-voxel set from the exported
    # voxel sets and the map before each frame
    sc = synth.tiny_scene()
    fr = sc.render(range(0, 6, 2))
    m = oracle.OracleMap(**oracle.config_for_scene(sc))
    for i in range(len(fr)):
        keys0, ids0 = m.voxels()
        before = dict(zip(keys0.tolist(), ids0.tolist()))
        r = m.integrate(*oracle.frame_args(fr, i))
        ov = {}
        new = set()
        for mm, k in zip(r["seg_m"].tolist(), r["seg_keys"].tolist()):
            if k in before:
                ov[(mm, before[k])] = ov.get((mm, before[k]), 0) + 1
            else:
                new.add(k)
        assert r["overlap_pairs"] == len(ov)
        assert r["new_voxels"] == len(new)
        assert r["active_instances"] == len({k for (_, k) in ov})
        keys1, ids1 = m.voxels()
        after = dict(zip(keys1.tolist(), ids1.tolist()))
        assert set(after) == set(before) | new
        # a new voxel takes the instance of its lowest-index segment
        owner = {}
        for mm, k in zip(r["seg_m"].tolist(), r["seg_keys"].tolist()):
            if k in new and (k not in owner or mm < owner[k]):
                owner[k] = mm
        for k, mm in owner.items():
            assert after[k] == r["rep"][mm - 1]


def test_map_invariants_over_the_tiny_trajectory():
    sc = synth.tiny_scene()
    m, fr, reps = _run(sc)
    inst = m.instances()
    keys, ids = m.voxels()
    parent = inst["parent"]
    assert np.all(parent[parent] == parent)                 # flat
    assert np.all(parent <= np.arange(len(parent)))         # rep = smallest id
    assert np.all(parent[ids] == ids)                       # voxels resolve to roots
    cnt = np.bincount(ids, minlength=len(parent))
    assert np.array_equal(cnt, np.where(parent == np.arange(len(parent)), inst["count"], 0))
    assert len(np.unique(keys)) == len(keys)


@pytest.mark.parametrize("bad", ["fx", "fy", "cx", "pose", "fx0"])
def test_non_finite_camera_or_pose_is_refused(bad):
    # a frame whose intrinsics or pose are not finite numbers (or whose focal
    # length is zero) is refused before the map changes
    H, W, D = 8, 8, 4
    m = oracle.OracleMap(**oracle.default_config(D, 2, 2, 0.05, min_mask_pixels=1))
    depth = np.full((H, W), 1.0, np.float32)
    lab = np.ones((H, W), np.uint16)
    F = np.ones((4, D), np.float32)
    intr = {"fx": (np.nan, 8.0, 4.0, 4.0), "fy": (8.0, np.inf, 4.0, 4.0), "cx": (8.0, 8.0, np.nan, 4.0),
            "pose": (8.0, 8.0, 4.0, 4.0), "fx0": (0.0, 8.0, 4.0, 4.0)}[bad]
    pose = np.eye(4)
    if bad == "pose":
        pose[1, 3] = 1e39  # finite in fp64, infinite once rounded to fp32
    with pytest.raises(RuntimeError):
        m.integrate(depth, lab, F, pose, intr, 1)
    assert m.voxels()[0].size == 0
    m.integrate(depth, lab, F, np.eye(4), (8.0, 8.0, 4.0, 4.0), 1)  # a valid frame still integrates
    assert m.voxels()[0].size > 0
