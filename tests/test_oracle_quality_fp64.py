"""The oracle's per-mask quality terms (Eq. 2-3, Sec. III-C) and segment
voxel sets (Sec. III-A) against an independent float64 restatement on
rendered frames.

The restatement follows the readings of the paper:
  - a pixel counts for mask m when its label is m (1..num_masks) and the mask
    holds at least min_mask_pixels pixels; its point is valid when
    z_min <= z <= z_max;
  - pinhole back-projection with pixel centres at +0.5, camera -> world by
    the pose; voxel key = floor(p / s) per axis;
  - pixel normal: the cross product of the forward differences along v and
    u (a backward difference where the forward neighbour is not a valid point
    of the same mask; no normal without either), normalised and turned to
    face the camera;
  - voxel normal: the normalised sum of its pixels' normals; view ray: the
    unit vector from the camera centre to the voxel centre;
    S_angle = sum_v max(0, -r_v . n_v) / |V_m| (Eq. 3);
  - pooled embedding e_m = sum_p w_p f_p with w_p = c_p D_p / sum c D (the
    coverage mean when every D is zero);
  - S_size = min(lambda |M| / (H W), 1); S_dist = 0.5 + 0.5 * sum_p c_p D_p /
    |M| with D of Eq. 1; S_sem = clamp(sum_p c_p ReLU(cos(f_p, g)) / |M|, 0, 1)
    with g the mean token; Q = S_size S_angle S_sem S_dist (Eq. 2).
Everything is float64, so it differs from the oracle's fp32 path by rounding
(and by the rare point whose fp32 and fp64 keys straddle a voxel face):
the voxel sets must agree but for a few voxels, and every term within the
stated tolerance.
"""
import numpy as np

import oracle
import synth


def _eq1_f64(F, eps):
    F = F.astype(np.float64)
    fbar = F.mean(0)
    n = np.linalg.norm(F - fbar, axis=1)
    return n / (n.mean() + eps), fbar


def quality_f64(depth, labels, tokens, pose, intr, M, cfg, Ph, Pw):
    H, W = depth.shape
    fx, fy, cx, cy = intr
    s, lam, eps = float(cfg["voxel_size"]), float(cfg["lambda_size"]), float(cfg["eps"])
    zmin, zmax, minpx = float(cfg["z_min"]), float(cfg["z_max"]), int(cfg["min_mask_pixels"])
    R, t = np.asarray(pose, np.float64)[:3, :3], np.asarray(pose, np.float64)[:3, 3]
    lab = labels.astype(np.int64)
    lab[lab > M] = 0
    npix = np.bincount(lab.ravel(), minlength=M + 1)[1:]
    kept = np.zeros(M + 1, bool)
    kept[1:] = npix >= minpx
    z = depth.astype(np.float64)
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    xc = (uu + 0.5 - cx) * z / fx
    yc = (vv + 0.5 - cy) * z / fy
    P = np.stack([xc, yc, z], -1) @ R.T + t
    ok = (lab > 0) & kept[lab] & np.isfinite(z) & (z >= zmin) & (z <= zmax)

    def diff(axis):
        # forward difference inside the mask, else backward, else none
        fwd = np.zeros_like(P)
        if axis == 1:
            same_f = np.zeros(ok.shape, bool)
            same_f[:, :-1] = ok[:, :-1] & ok[:, 1:] & (lab[:, :-1] == lab[:, 1:])
            same_b = np.zeros(ok.shape, bool)
            same_b[:, 1:] = ok[:, 1:] & ok[:, :-1] & (lab[:, 1:] == lab[:, :-1])
            fwd[:, :-1] = P[:, 1:] - P[:, :-1]
            bwd = np.zeros_like(P)
            bwd[:, 1:] = P[:, 1:] - P[:, :-1]
        else:
            same_f = np.zeros(ok.shape, bool)
            same_f[:-1] = ok[:-1] & ok[1:] & (lab[:-1] == lab[1:])
            same_b = np.zeros(ok.shape, bool)
            same_b[1:] = ok[1:] & ok[:-1] & (lab[1:] == lab[:-1])
            fwd[:-1] = P[1:] - P[:-1]
            bwd = np.zeros_like(P)
            bwd[1:] = P[1:] - P[:-1]
        d = np.where(same_f[..., None], fwd, bwd)
        good = same_f | same_b
        return d, good

    du, gu = diff(1)
    dv, gv = diff(0)
    nrm = np.cross(dv, du)
    ln = np.linalg.norm(nrm, axis=-1)
    has_n = ok & gu & gv & (ln > 0)
    nrm = np.where(has_n[..., None], nrm / np.where(ln > 0, ln, 1.0)[..., None], 0.0)
    toward = np.einsum("hwc,hwc->hw", nrm, t - P)
    nrm = np.where((toward < 0)[..., None], -nrm, nrm)
    keys = np.floor(P / s).astype(np.int64)
    cov = np.zeros((M, Ph * Pw), np.int64)
    pv = (vv * Ph) // H
    pu = (uu * Pw) // W
    pid = pv * Pw + pu
    for m in range(1, M + 1):
        sel = lab == m
        cov[m - 1] = np.bincount(pid[sel], minlength=Ph * Pw)
    Dp, fbar = _eq1_f64(tokens, eps)
    Fd = tokens.astype(np.float64)
    cosg = Fd @ fbar / (np.linalg.norm(Fd, axis=1) * np.linalg.norm(fbar))
    out = {}
    for m in range(1, M + 1):
        if not kept[m]:
            continue
        sel = ok & (lab == m)
        ks = keys[sel]
        ns = nrm[sel]
        vox = {}
        for k, n in zip(map(tuple, ks), ns):
            vox[k] = vox.get(k, 0.0) + n
        if not vox:
            continue
        acc = 0.0
        for k, n in vox.items():
            ln2 = np.linalg.norm(n)
            if ln2 == 0:
                continue
            c = (np.asarray(k, np.float64) + 0.5) * s
            r = (c - t) / np.linalg.norm(c - t)
            acc += max(0.0, -float(r @ (n / ln2)))
        s_angle = acc / len(vox)
        cm = cov[m - 1].astype(np.float64)
        Mm = float(npix[m - 1])
        # a3: pixel-level D-weighted mean of the tokens (coverage mean when
        # every D is zero)
        a = cm * Dp
        w = a / a.sum() if a.sum() > 0 else cm / cm.sum()
        E = w @ Fd
        s_size = min(lam * Mm / (H * W), 1.0)
        s_dist = 0.5 + 0.5 * float(cm @ Dp) / Mm
        s_sem = min(max(float(cm @ np.maximum(cosg, 0.0)) / Mm, 0.0), 1.0)
        out[m] = dict(keys=set(vox), E=E, S=np.array([s_size, s_angle, s_sem, s_dist,
                                                      s_size * s_angle * s_sem * s_dist]))
    return out


def _compare(sc, idx, tol_angle):
    fr = sc.render(idx)
    cfg = oracle.config_for_scene(sc)
    om = oracle.OracleMap(**cfg)
    worst = np.zeros(5)
    worst_e = 0.0
    masks = 0
    for i in range(len(fr)):
        args = oracle.frame_args(fr, i)
        r = om.integrate(*args)
        q = quality_f64(*args, cfg, sc.patch_h, sc.patch_w)
        live = [m for m in range(1, args[5] + 1) if r["nvox"][m - 1] > 0]
        assert sorted(live) == sorted(q), f"frame {idx[i]}: live masks"
        segs = {}
        for m, k in zip(r["seg_m"].tolist(), r["seg_keys"].tolist()):
            segs.setdefault(m, set()).add(tuple(oracle.unpack_key(k)))
        for m in live:
            sym = len(segs[m] ^ q[m]["keys"])
            assert sym <= max(2, len(q[m]["keys"]) // 500), (idx[i], m, sym)
            e = np.abs(r["S"][m - 1].astype(np.float64) - q[m]["S"])
            worst = np.maximum(worst, e)
            E64 = q[m]["E"]
            rel = np.linalg.norm(r["E"][m - 1].astype(np.float64) - E64) / np.linalg.norm(E64)
            worst_e = max(worst_e, rel)
            masks += 1
    assert masks > 0
    # S_size exact up to fp32 rounding; S_sem and S_dist follow Eq. 1 and the
    # cosines; S_angle and Q also see the few straddling points
    assert worst[0] < 1e-6, worst
    assert worst[2] < 1e-6 and worst[3] < 1e-6, worst
    assert worst[1] < tol_angle and worst[4] < tol_angle, worst
    assert worst_e < 1e-6, worst_e  # the pooled embedding, per vector
    return worst, worst_e, masks


def test_quality_terms_tiny_trajectory():
    _compare(synth.tiny_scene(), list(range(20)), 1e-5)


def test_quality_terms_room_frames():
    sc = synth.room_scene()
    _compare(sc, list(range(0, 60, 12)), 1e-3)


def test_oracle_fp64_pooling_twin_matches_numpy():
    # the oracle's float64 pooling (the reference of every error statement
    # about the fast pooled embedding) against numpy float64, on Room frames
    sc = synth.room_scene()
    fr = sc.render([0, 300])
    for i in range(len(fr)):
        F = fr.tokens[i]
        M = int(fr.num_masks[i])
        cov, npix = oracle.mask_coverage(fr.labels[i], sc.patch_h, sc.patch_w, M)
        Dp, E = oracle.pool_f64(F, cov, npix, 1e-6)
        D64, _ = _eq1_f64(F, 1e-6)
        assert np.max(np.abs(Dp - D64)) < 1e-12
        for m in range(M):
            c = cov[m].astype(np.float64)
            if c.sum() == 0:
                continue
            a = c * D64
            w = a / a.sum()
            e = w @ F.astype(np.float64)
            assert np.linalg.norm(E[m] - e) <= 1e-12 * np.linalg.norm(e)
