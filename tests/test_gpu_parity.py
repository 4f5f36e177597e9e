"""GPU path vs the oracle, element by element, through the C ABI.

Bit-exact: voxel keys, coverage counts, labels, overlap/instance counters,
and every quantity the method computes with exact sums (D, weights, Q terms,
the exact pooled embedding, stored instance embeddings).  The tensor-core
pooled embedding is held to 1e-5 relative error per vector.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import common, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2603_03935_gb300 import _build
    _build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return torch, dev


def _dframe(torch, dev, fr, i):
    from paper_2603_03935_gb300 import device_frame
    sc = fr.scene
    d = torch.from_numpy(fr.depth[i]).to(dev)
    l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[i]).to(dev)
    return device_frame(d, l, t, fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[i])


def _hframe(fr, i):
    from paper_2603_03935_gb300 import host_frame
    sc = fr.scene
    return host_frame(fr.depth[i], fr.labels[i], fr.tokens[i], fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy),
                      fr.num_masks[i])


def run_parity(torch_dev, scene, frames, host=False, **cfg_kw):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    fr = scene.render(frames)
    cfg = common.disc_cfg(scene, **cfg_kw)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    stats = []
    for i in range(len(fr)):
        st = gmap.integrate(_hframe(fr, i) if host else _dframe(torch, dev, fr, i))
        o = omap.integrate(*oracle.frame_args(fr, i))
        common.compare_frame(st, gmap.last_frame(), o, ctx=f"{scene.name} frame {i}")
        stats.append(st)
    common.compare_maps(gmap, omap, ctx=scene.name)
    return gmap, omap, stats


def test_tiny_trajectory_parity(torch_dev):
    run_parity(torch_dev, synth.tiny_scene(), range(20))


def test_tiny_parity_with_host_inputs(torch_dev):
    run_parity(torch_dev, synth.tiny_scene(), range(0, 20, 3), host=True)


@pytest.mark.parametrize("batch", [9, 16])
def test_host_inputs_in_batches_split_in_halves(torch_dev, batch):
    # batches of 8 or more host frames run their stateless part in two halves,
    # the second half's copies under the first half's kernels (9: uneven)
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, host_frame
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    hd = torch.from_numpy(fr.depth).pin_memory()
    hl = torch.from_numpy(fr.labels.view(np.int16)).pin_memory()
    ht = torch.from_numpy(fr.tokens).pin_memory()
    d, l, t = hd.numpy(), hl.numpy().view(np.uint16), ht.numpy()
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    frames = [host_frame(d[i], l[i], t[i], fr.poses[i], intr, fr.num_masks[i]) for i in range(20)]
    cfg = common.disc_cfg(sc, batch_frames=batch)
    gmap = DiscMap(**cfg)
    stats, done, rc = gmap.integrate_frames(frames)
    assert rc == 0 and done == 20
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(20):
        o = omap.integrate(*oracle.frame_args(fr, i))
        for gk, ok in common.COUNT_FIELDS:
            assert stats[i][gk] == o[ok], (i, gk)
    common.compare_maps(gmap, omap, ctx=f"host frames, batches of {batch} in halves")


def test_host_input_halves_of_different_bases(torch_dev):
    # calls of 16 and then 15 host frames: both split their batch in two
    # halves whose second half has 8 frames, starting at slot 8 and at slot 7;
    # each must replay its own captured launch sequence
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, host_frame
    sc = synth.tiny_scene(num_frames=100)
    sizes = [16, 16, 16, 16, 15, 15]
    fr = sc.render(range(sum(sizes)))
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    frames = [host_frame(fr.depth[i], fr.labels[i], fr.tokens[i], fr.poses[i], intr, fr.num_masks[i])
              for i in range(sum(sizes))]
    cfg = common.disc_cfg(sc, batch_frames=16)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    lo = 0
    for n in sizes:
        stats, done, rc = gmap.integrate_frames(frames[lo:lo + n])
        assert rc == 0 and done == n
        for j in range(n):
            o = omap.integrate(*oracle.frame_args(fr, lo + j), report=True)
            for gk, ok in common.COUNT_FIELDS:
                assert stats[j][gk] == o[ok], f"frame {lo + j} {gk}: {stats[j][gk]} vs {o[ok]}"
        lo += n
    common.compare_maps(gmap, omap, ctx="host-input halves of different bases")


def test_host_inputs_in_one_call_of_many_batches(torch_dev):
    # a whole trajectory from pinned host memory in one call: frames lie back
    # to back, so each batch's copies merge into one per input kind and run
    # on the input stream while the previous batch computes (two staging
    # sets); the map must equal the oracle's, frame for frame
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, host_frame
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    hd = torch.from_numpy(fr.depth).pin_memory()
    hl = torch.from_numpy(fr.labels.view(np.int16)).pin_memory()
    ht = torch.from_numpy(fr.tokens).pin_memory()
    d, l, t = hd.numpy(), hl.numpy().view(np.uint16), ht.numpy()
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    frames = [host_frame(d[i], l[i], t[i], fr.poses[i], intr, fr.num_masks[i]) for i in range(20)]
    assert all(f[1][0].ctypes.data == d[i].ctypes.data for i, f in enumerate(frames))  # no copies made
    cfg = common.disc_cfg(sc, batch_frames=3)
    gmap = DiscMap(**cfg)
    stats, done, rc = gmap.integrate_frames(frames)
    assert rc == 0 and done == 20
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(20):
        o = omap.integrate(*oracle.frame_args(fr, i))
        for gk, ok in common.COUNT_FIELDS:
            assert stats[i][gk] == o[ok], (i, gk)
    common.compare_maps(gmap, omap, ctx="one call of 7 batches from pinned host memory")


def test_tiny_parity_with_growth_of_both_tables(torch_dev):
    # tiny initial capacities force rehashing and instance-table growth
    run_parity(torch_dev, synth.tiny_scene(), range(20), voxel_capacity=256, instance_capacity=2)


def test_room_scale_frames_parity(torch_dev):
    # full 640x480 frames, 24x24x768 tokens, 40 masks, 2.5 cm voxels
    sc = synth.room_scene(num_frames=2000)
    run_parity(torch_dev, sc, [0, 1, 2, 3, 250, 251], voxel_capacity=1 << 22, instance_capacity=1024)


def test_tiny_parity_with_neighbourhood_overlap(torch_dev):
    # overlap_dilation: a segment voxel also overlaps the instances of its 26
    # neighbours (the neighbourhood reading of Sec. III-B)
    _, _, stats = run_parity(torch_dev, synth.tiny_scene(), range(20), overlap_dilation=1)
    assert sum(st["overlap_pairs"] for st in stats) > 0


def test_room_batched_parity_with_neighbourhood_overlap(torch_dev):
    # 32 full-size frames in one call: neighbours inserted by earlier frames
    # of the batch must be seen by the later ones
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene(num_frames=2000)
    fr = sc.render(range(32))
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 24, instance_capacity=1 << 16, overlap_dilation=1)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    frames = [_dframe(torch, dev, fr, i) for i in range(32)]
    stats, done, rc = gmap.integrate_frames(frames)
    assert rc == 0 and done == 32
    for j, st in enumerate(stats):
        o = omap.integrate(*oracle.frame_args(fr, j), report=True)
        for gk, ok in common.COUNT_FIELDS:
            assert st[gk] == o[ok], f"frame {j} {gk}: {st[gk]} vs {o[ok]}"
    common.compare_maps(gmap, omap, ctx="room batched, neighbourhood overlap")


def test_room_trajectory_batched_parity(torch_dev):
    # the launch configuration the benchmark times: 32 consecutive full-size
    # frames per disc_integrate_frames call, device-resident inputs
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene(num_frames=2000)
    fr = sc.render(range(64))
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 24, instance_capacity=1 << 16)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for lo in (0, 32):
        frames = [_dframe(torch, dev, fr, i) for i in range(lo, lo + 32)]
        stats, done, rc = gmap.integrate_frames(frames)
        assert rc == 0 and done == 32
        for j, st in enumerate(stats):
            o = omap.integrate(*oracle.frame_args(fr, lo + j), report=True)
            for gk, ok in common.COUNT_FIELDS:
                assert st[gk] == o[ok], f"frame {lo + j} {gk}: {st[gk]} vs {o[ok]}"
    common.compare_maps(gmap, omap, ctx="room batched")


def test_ragged_token_grid_and_odd_frame(torch_dev):
    # P = 7 x 5 = 35 (ragged last GEMM chunk), D = 200 (ragged last tile),
    # 50 x 37 pixels (patch bands of uneven height)
    prims = [(0, 1, (0.013, 0.013, 0.213), (0.3, 0.25, 0.2)),
             (1, 2, (0.6, 0.5, 0.25), (0.2, 0.2, 0.25))]
    sc = scenes.custom_scene(prims, scenes.orbit((0.2, 0.2, 0.2), 1.6, 0.9, 6, sweep=np.deg2rad(60)),
                             width=50, height=37, f=40.0, dim=200, patch=(7, 5), voxel=0.04, max_masks=5)
    run_parity(torch_dev, sc, range(6))


def test_equal_results_alone_and_batched(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    cfg = common.disc_cfg(sc)
    a, b = DiscMap(**cfg), DiscMap(**cfg)
    for i in range(20):
        a.integrate(_dframe(torch, dev, fr, i))
    frames = [_dframe(torch, dev, fr, i) for i in range(20)]
    stats, done, rc = b.integrate_frames(frames)
    assert rc == 0 and done == 20
    ka, ia = a.voxels()
    kb, ib = b.voxels()
    assert np.array_equal(ka, kb) and np.array_equal(ia, ib)
    ea, eb = a.instances(), b.instances()
    for k in ("parent", "count", "n_obs"):
        assert np.array_equal(ea[k], eb[k])
    assert np.array_equal(ea["E"], eb["E"])


def test_empty_and_degenerate_frames(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, host_frame
    sc = synth.tiny_scene()
    cfg = common.disc_cfg(sc)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    H, W, P, D = sc.height, sc.width, sc.patch_h * sc.patch_w, sc.dim
    rng = np.random.default_rng(3)
    tok = rng.standard_normal((P, D)).astype(np.float32)
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    pose = sc.poses[0]
    cases = [
        ("no masks", np.full((H, W), 2.0, np.float32), np.zeros((H, W), np.uint16), 0),
        ("all depth invalid", np.full((H, W), np.nan, np.float32), np.ones((H, W), np.uint16), 1),
        ("labels above num_masks", np.full((H, W), 2.0, np.float32), np.full((H, W), 5, np.uint16), 2),
        ("masks below the size filter", np.full((H, W), 2.0, np.float32),
         np.pad(np.ones((1, 2), np.uint16), ((0, H - 1), (0, W - 2))), 1),
        ("constant tokens", np.full((H, W), 2.0, np.float32), np.ones((H, W), np.uint16), 1),
    ]
    for name, depth, lab, M in cases:
        t = np.full_like(tok, 0.5) if name == "constant tokens" else tok
        st = gmap.integrate(host_frame(depth, lab, t, pose, intr, M))
        o = omap.integrate(depth, lab, t, pose, intr, M)
        common.compare_frame(st, gmap.last_frame(), o, ctx=name)
    common.compare_maps(gmap, omap, ctx="degenerate")


def test_maximum_mask_count(torch_dev):
    # 256 masks per frame (the largest a frame may carry): a wall cut into a
    # 16 x 16 grid of regions, seen from three slightly shifted poses; every
    # mask is live, so the new-id scan and the pooling GEMM run at full width
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, host_frame
    H, W, f = 96, 128, 120.0
    Ph, Pw, D = 12, 16, 64
    rng = np.random.default_rng(11)
    means = rng.standard_normal((257, D)).astype(np.float32)
    v, u = np.mgrid[0:H, 0:W]
    lab = (1 + (v * 16 // H) * 16 + (u * 16 // W)).astype(np.uint16)  # 1..256
    cfg = dict(voxel_size=0.02, z_min=0.1, z_max=10.0, eps=1e-6, tau_cos=0.75, lambda_size=3.3, ov_num=1,
               ov_den=5, embed_dim=D, patch_h=Ph, patch_w=Pw, max_width=W, max_height=H, max_masks=256,
               min_mask_pixels=12, voxel_capacity=1 << 16, max_load=0.5, instance_capacity=1024)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    intr = (f, f, W / 2, H / 2)
    for i in range(3):
        depth = scenes.plane_depth(H, W, f, f, W / 2, H / 2, 1.513 + 0.004 * i)
        pose = scenes.identity_pose()
        pose[0, 3] = 0.003 * i
        pv, pu = np.mgrid[0:Ph, 0:Pw]
        pid = lab[((2 * pv + 1) * H) // (2 * Ph), ((2 * pu + 1) * W) // (2 * Pw)].reshape(-1)
        tok = (means[pid] + 0.1 * rng.standard_normal((Ph * Pw, D))).astype(np.float32)
        st = gmap.integrate(host_frame(depth, lab, tok, pose, intr, 256))
        o = omap.integrate(depth, lab, tok, pose, intr, 256)
        common.compare_frame(st, gmap.last_frame(), o, ctx=f"256 masks frame {i}")
        assert st["live_segments"] == 256
    common.compare_maps(gmap, omap, ctx="256 masks")
    assert len(gmap.instances()["parent"]) >= 256


def test_token_range_error_leaves_the_map_unchanged(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, host_frame
    sc = synth.tiny_scene()
    fr = sc.render(range(3))
    gmap = DiscMap(**common.disc_cfg(sc))
    gmap.integrate(_hframe(fr, 0))
    k0, i0 = gmap.voxels()
    bad = fr.tokens[1].copy()
    bad[3, 7] = np.inf
    st = gmap.integrate(host_frame(fr.depth[1], fr.labels[1], bad, fr.poses[1], (sc.fx, sc.fy, sc.cx, sc.cy),
                                   fr.num_masks[1]), check=False)
    assert st["rc"] == -7 and st["status"] == -7
    k1, i1 = gmap.voxels()
    assert np.array_equal(k0, k1) and np.array_equal(i0, i1)
    # and a batch stops at the failing frame
    frames = [_hframe(fr, 2), host_frame(fr.depth[1], fr.labels[1], bad, fr.poses[1],
                                         (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[1]), _hframe(fr, 0)]
    stats, done, rc = gmap.integrate_frames(frames, check=False)
    assert rc == -7 and done == 1


def test_borderline_cosines_are_rescored_exactly(torch_dev):
    # put tau_cos exactly on a cosine the oracle computes for a real
    # (segment, instance) pair: the fast tensor-core score lands inside the
    # error band and the exact re-score must reproduce the oracle's decision
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(3))
    probe = oracle.OracleMap(**oracle.config_for_scene(sc))
    probe.integrate(*oracle.frame_args(fr, 0))
    E0 = probe.instances()["E"]
    r1 = probe.integrate(*oracle.frame_args(fr, 1))
    m = int(np.argmax(r1["nvox"]))
    k = int(r1["rep"][m]) if r1["rep"][m] < len(E0) else 0
    tau = oracle.cosine(r1["E"][m], E0[k])
    for t in (tau, np.nextafter(np.float32(tau), np.float32(2))):
        cfg = common.disc_cfg(sc, tau_cos=float(t))
        gmap = DiscMap(**cfg)
        omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
        border = 0
        for i in range(3):
            st = gmap.integrate(_dframe(torch, dev, fr, i))
            o = omap.integrate(*oracle.frame_args(fr, i))
            common.compare_frame(st, gmap.last_frame(), o, ctx=f"tau={t} frame {i}")
            border += st["borderline_rescored"]
        common.compare_maps(gmap, omap, ctx=f"tau={t}")
        assert border >= 1


def test_checkpoint_resume_equals_uninterrupted(torch_dev, tmp_path):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(12))
    cfg = common.disc_cfg(sc)
    full = DiscMap(**cfg)
    for i in range(12):
        full.integrate(_dframe(torch, dev, fr, i))
    part = DiscMap(**cfg)
    for i in range(6):
        part.integrate(_dframe(torch, dev, fr, i))
    part.save(tmp_path / "map.bin")
    part.close()
    res = DiscMap.load(tmp_path / "map.bin")
    for i in range(6, 12):
        res.integrate(_dframe(torch, dev, fr, i))
    ka, ia = full.voxels()
    kb, ib = res.voxels()
    assert np.array_equal(ka, kb) and np.array_equal(ia, ib)
    ea, eb = full.instances(), res.instances()
    for k in ("parent", "count", "n_obs", "Q", "E"):
        assert np.array_equal(ea[k], eb[k])


def test_queries(torch_dev):
    torch, dev = torch_dev
    sc = synth.tiny_scene()
    gmap, omap, _ = run_parity(torch_dev, sc, range(8))
    inst = omap.instances()
    live = np.nonzero(inst["parent"] == np.arange(len(inst["parent"])))[0]
    # query = an instance's own embedding -> that instance first, cosine 1
    q = inst["E"][live[:4]]
    ids, scores = gmap.query_topk(q, 3)
    assert np.array_equal(ids[:, 0], live[:4])
    np.testing.assert_allclose(scores[:, 0], 1.0, atol=1e-5)
    # scores against an fp64 recomputation
    E = inst["E"][live].astype(np.float64)
    for qi in range(len(q)):
        c = E @ q[qi].astype(np.float64) / (np.linalg.norm(E, axis=1) * np.linalg.norm(q[qi]))
        order = np.lexsort((live, -c))[:3]
        np.testing.assert_allclose(scores[qi], c[order], atol=1e-5)
    # point queries: voxel centres map to their instance, far points to -1
    keys, vids = omap.voxels()
    ks = np.array([oracle.unpack_key(k) for k in keys[:200]], np.float64)
    pts = ((ks + 0.5) * sc.voxel_size).astype(np.float32)
    got = gmap.query_points(np.vstack([pts, [[100.0, 100.0, 100.0]]]))
    assert np.array_equal(got[:-1], vids[:200]) and got[-1] == -1


def test_bf16_tokens_parity(torch_dev):
    # bf16 tokens widen exactly to fp32: the oracle, given those fp32 values,
    # must match bit for bit
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.tiny_scene()
    fr = sc.render(range(10))
    cfg = common.disc_cfg(sc)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    for i in range(len(fr)):
        t16 = torch.from_numpy(fr.tokens[i]).to(dev).to(torch.bfloat16).contiguous()
        t32 = t16.float().cpu().numpy()
        d = torch.from_numpy(fr.depth[i]).to(dev)
        l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
        st = gmap.integrate(device_frame(d, l, t16, fr.poses[i], intr, fr.num_masks[i]))
        o = omap.integrate(fr.depth[i], fr.labels[i], t32, fr.poses[i], intr, fr.num_masks[i])
        common.compare_frame(st, gmap.last_frame(), o, ctx=f"bf16 frame {i}")
    common.compare_maps(gmap, omap, ctx="bf16 tokens")


# BF16 precision: the fast pooled embedding (bf16 operands, fp32 accumulation
# on the tensor cores) and the bf16 scoring copies only decide which pairs get
# an exact re-score, so labels, counts and stored embeddings stay identical
# to the oracle; the fast embedding's error against the fp64 pooling twin
# stays within the bound the re-score band is built from.
BF16_ETA = 2 * 2.0 ** -9 + 2.0 ** -18


def _bf16_fast_error(rep, tokens, scene):
    Dp64, E64 = oracle.pool_f64(tokens, rep["cov"], rep["npix"])
    worst = 0.0
    for m in range(len(rep["npix"])):
        if rep["npix"][m] < 1 or not np.any(rep["W"][m]):
            continue  # masks below the size filter carry no weights
        # sum_p w_p ||f_p||
        w = rep["W"][m].astype(np.float64)
        bsum = float(np.sum(w * np.linalg.norm(tokens.astype(np.float64), axis=1)))
        K = (scene.patch_h * scene.patch_w + 31) // 32 * 32
        bound = (BF16_ETA + 3 * K * 2.0 ** -24) * bsum
        err = float(np.linalg.norm(rep["E_fast"][m].astype(np.float64) - E64[m]))
        assert err <= bound, f"mask {m}: |E_fast - E_fp64| = {err} > {bound}"
        worst = max(worst, err / max(float(np.linalg.norm(E64[m])), 1e-30))
    return worst


def test_bf16_precision_parity_and_fp64_error(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    cfg = common.disc_cfg(sc, precision=1)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    worst = 0.0
    for i in range(len(fr)):
        st = gmap.integrate(_dframe(torch, dev, fr, i))
        o = omap.integrate(*oracle.frame_args(fr, i))
        rep = gmap.last_frame()
        common.compare_frame(st, rep, o, ctx=f"bf16 precision frame {i}", efast_tol=2e-2)
        worst = max(worst, _bf16_fast_error(rep, fr.tokens[i], sc))
    common.compare_maps(gmap, omap, ctx="bf16 precision")
    print(f"bf16 tiny: worst |E_fast - E64| / |E64| = {worst:.5f}")
    assert worst < 1e-2, worst


def test_bf16_precision_borderline_rescored(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(3))
    probe = oracle.OracleMap(**oracle.config_for_scene(sc))
    probe.integrate(*oracle.frame_args(fr, 0))
    E0 = probe.instances()["E"]
    r1 = probe.integrate(*oracle.frame_args(fr, 1))
    m = int(np.argmax(r1["nvox"]))
    k = int(r1["rep"][m]) if r1["rep"][m] < len(E0) else 0
    tau = oracle.cosine(r1["E"][m], E0[k])
    for t in (tau, np.nextafter(np.float32(tau), np.float32(2))):
        cfg = common.disc_cfg(sc, tau_cos=float(t), precision=1)
        gmap = DiscMap(**cfg)
        omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
        border = 0
        for i in range(3):
            st = gmap.integrate(_dframe(torch, dev, fr, i))
            o = omap.integrate(*oracle.frame_args(fr, i))
            common.compare_frame(st, gmap.last_frame(), o, ctx=f"bf16 tau={t} frame {i}", efast_tol=2e-2)
            border += st["borderline_rescored"]
        common.compare_maps(gmap, omap, ctx=f"bf16 tau={t}")
        assert border >= 1


def test_bf16_precision_checkpoint_and_mixed_group(torch_dev, tmp_path):
    # a bf16-precision map next to fp32 maps in one group; its checkpoint
    # reloads to the same scoring behaviour
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscGroup, DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(12))
    frames = [_dframe(torch, dev, fr, i) for i in range(12)]
    a32, a16 = DiscMap(**common.disc_cfg(sc)), DiscMap(**common.disc_cfg(sc, precision=1))
    grp = DiscGroup(max_maps=2, frames_per_map=4, embed_dim=sc.dim, patch_h=sc.patch_h, patch_w=sc.patch_w,
                    max_width=sc.width, max_height=sc.height, max_masks=sc.max_masks)
    _, done, rc = grp.integrate([a32, a16], [frames[:6], frames[:6]])
    assert rc == 0 and done == [6, 6]
    a16.save(tmp_path / "m16.disc")
    b16 = DiscMap.load(tmp_path / "m16.disc")
    _, done, rc = grp.integrate([a32, b16], [frames[6:], frames[6:]])
    assert rc == 0
    for m in (a16,):
        _, d, rc1 = m.integrate_frames(frames[6:])
        assert rc1 == 0
    for x, y, ctx in ((a32, b16, "fp32 vs bf16"), (a16, b16, "bf16 alone vs reloaded in a group")):
        kx, ix = x.voxels()
        ky, iy = y.voxels()
        assert np.array_equal(kx, ky) and np.array_equal(ix, iy), ctx
        ex, ey = x.instances(), y.instances()
        assert np.array_equal(ex["E"].view(np.uint32), ey["E"].view(np.uint32)), ctx


# FP8 precision: E4M3 operands with power-of-two per-vector scales (per
# token, per weight row, per stored embedding) and fp32 accumulation.  The
# weights kernel bounds |E_fast - e| per mask from the actual rounding
# residues; the test checks that bound against e = sum_p w_p f_p taken in
# fp64, checks a looser a-priori bound that follows from the format alone
# (3 mantissa bits: relative rounding 2^-4, subnormal step 2^-9 of the
# scale), and states the error against the fp64 pooling twin.
def _fp8_apriori(n_patches, D, K):
    sub = 2.0 ** -10 * n_patches * np.sqrt(D) / 112.0  # weight rows' subnormal rounding
    tok = 2.0 ** -4 + np.sqrt(D) * 2.0 ** -10 / 224.0  # token rounding, relative to ||f_p||
    acc = (K / 32 + 2) * 2.0 ** -12
    return ((1 + tok) * (2.0 ** -4 + sub) + tok + 2 * acc) * 1.01


def _fp8_fast_error(rep, tokens, scene):
    F = tokens.astype(np.float64)
    _, E64 = oracle.pool_f64(tokens, rep["cov"], rep["npix"])
    K = (scene.patch_h * scene.patch_w + 31) // 32 * 32
    worst, tight = 0.0, []
    for m in range(len(rep["npix"])):
        if rep["npix"][m] < 1 or not np.any(rep["W"][m]):
            continue
        w = rep["W"][m].astype(np.float64)
        e = w @ F  # sum_p w_p f_p with the frame's fp32 weights, in fp64
        err = float(np.linalg.norm(rep["E_fast"][m].astype(np.float64) - e))
        bound = float(rep["E_bound"][m])
        assert err <= bound, f"mask {m}: |E_fast - e| = {err} > device bound {bound}"
        bsum = float(np.sum(w * np.linalg.norm(F, axis=1)))
        apri = _fp8_apriori(int(np.count_nonzero(w)), F.shape[1], K) * bsum
        assert bound <= apri, f"mask {m}: device bound {bound} above the a-priori bound {apri}"
        tight.append(bound / apri)
        worst = max(worst, float(np.linalg.norm(rep["E_fast"][m] - E64[m])) / max(float(np.linalg.norm(E64[m])), 1e-30))
    return worst, tight


def test_fp8_precision_parity_and_fp64_error(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    cfg = common.disc_cfg(sc, precision=2)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    worst, tight, border = 0.0, [], 0
    for i in range(len(fr)):
        st = gmap.integrate(_dframe(torch, dev, fr, i))
        o = omap.integrate(*oracle.frame_args(fr, i))
        rep = gmap.last_frame()
        common.compare_frame(st, rep, o, ctx=f"fp8 precision frame {i}", efast_tol=0.15)
        w, t = _fp8_fast_error(rep, fr.tokens[i], sc)
        worst, tight, border = max(worst, w), tight + t, border + st["borderline_rescored"]
    common.compare_maps(gmap, omap, ctx="fp8 precision")
    inst = gmap.instances()
    ea = omap.instances()["E"]
    assert np.array_equal(inst["E"].view(np.uint32), ea.view(np.uint32))
    # E4M3 keeps 3 mantissa bits: a few percent against fp64, and the
    # device's residue-based bound well inside the format's worst case
    print(f"fp8 tiny: worst |E_fast - E64| / |E64| = {worst:.4f}, device bound / a-priori bound <= "
          f"{max(tight):.3f} (median {float(np.median(tight)):.3f}), re-scored pairs {border}")
    assert 1e-3 < worst < 0.1, worst
    assert max(tight) < 0.8, max(tight)


def test_fp8_precision_room_scale(torch_dev):
    # full 640x480 frames, 24x24x768 tokens, 40 masks: labels and stored
    # embeddings identical to the oracle; the E4M3 fast embedding within the
    # device bound of every mask, and that bound within the format's worst case
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene(num_frames=2000)
    idx = [0, 1, 2, 3, 250, 251]
    fr = sc.render(idx)
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 22, instance_capacity=1024, precision=2)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    worst, tight, border = 0.0, [], 0
    for i in range(len(idx)):
        st = gmap.integrate(_dframe(torch, dev, fr, i))
        o = omap.integrate(*oracle.frame_args(fr, i))
        rep = gmap.last_frame()
        common.compare_frame(st, rep, o, ctx=f"fp8 room frame {idx[i]}", efast_tol=0.15)
        w, t = _fp8_fast_error(rep, fr.tokens[i], sc)
        worst, tight, border = max(worst, w), tight + t, border + st["borderline_rescored"]
    common.compare_maps(gmap, omap, ctx="fp8 room")
    print(f"fp8 room: worst |E_fast - E64| / |E64| = {worst:.4f}, device bound / a-priori bound <= "
          f"{max(tight):.3f} (median {float(np.median(tight)):.3f}), re-scored pairs {border}")
    assert worst < 0.1


def test_fp8_precision_borderline_rescored(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(3))
    probe = oracle.OracleMap(**oracle.config_for_scene(sc))
    probe.integrate(*oracle.frame_args(fr, 0))
    E0 = probe.instances()["E"]
    r1 = probe.integrate(*oracle.frame_args(fr, 1))
    m = int(np.argmax(r1["nvox"]))
    k = int(r1["rep"][m]) if r1["rep"][m] < len(E0) else 0
    tau = oracle.cosine(r1["E"][m], E0[k])
    for t in (tau, np.nextafter(np.float32(tau), np.float32(2)), np.nextafter(np.float32(tau), np.float32(0))):
        cfg = common.disc_cfg(sc, tau_cos=float(t), precision=2)
        gmap = DiscMap(**cfg)
        omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
        border = 0
        for i in range(3):
            st = gmap.integrate(_dframe(torch, dev, fr, i))
            o = omap.integrate(*oracle.frame_args(fr, i))
            common.compare_frame(st, gmap.last_frame(), o, ctx=f"fp8 tau={t} frame {i}", efast_tol=0.15)
            border += st["borderline_rescored"]
        common.compare_maps(gmap, omap, ctx=f"fp8 tau={t}")
        assert border >= 1


def test_fp8_precision_checkpoint_and_mixed_group(torch_dev, tmp_path):
    # fp32, bf16 and fp8 maps side by side in one group give one and the same
    # map; an fp8 checkpoint reloads with rebuilt E4M3 scoring copies
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscGroup, DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(12))
    frames = [_dframe(torch, dev, fr, i) for i in range(12)]
    maps = [DiscMap(**common.disc_cfg(sc, precision=p)) for p in (0, 1, 2)]
    grp = DiscGroup(max_maps=3, frames_per_map=4, embed_dim=sc.dim, patch_h=sc.patch_h, patch_w=sc.patch_w,
                    max_width=sc.width, max_height=sc.height, max_masks=sc.max_masks)
    _, done, rc = grp.integrate(maps, [frames[:6]] * 3)
    assert rc == 0 and done == [6, 6, 6]
    maps[2].save(tmp_path / "m8.disc")
    b8 = DiscMap.load(tmp_path / "m8.disc")
    _, done, rc = grp.integrate(maps[:2] + [b8], [frames[6:]] * 3)
    assert rc == 0
    _, _, rc1 = maps[2].integrate_frames(frames[6:])
    assert rc1 == 0
    for y, ctx in ((maps[1], "bf16"), (b8, "fp8 reloaded in a group"), (maps[2], "fp8 alone")):
        kx, ix = maps[0].voxels()
        ky, iy = y.voxels()
        assert np.array_equal(kx, ky) and np.array_equal(ix, iy), ctx
        ex, ey = maps[0].instances(), y.instances()
        for k in ("parent", "count", "n_obs"):
            assert np.array_equal(ex[k], ey[k]), (ctx, k)
        assert np.array_equal(ex["E"].view(np.uint32), ey["E"].view(np.uint32)), ctx


def test_multistory_bf16_parity(torch_dev):
    # the multi-story building: up to 100 masks, 5 cm voxels, depth to 20 m,
    # bf16 tokens at BF16 precision, a voxel table of 2^27 slots; consecutive
    # frames on each of the three floors
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.multistory_scene()
    idx = [0, 1, 2, 3, 1700, 1701, 1702, 3400, 3401, 3402]
    fr = sc.render(idx)
    assert int(fr.num_masks.max()) == 100
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 27, instance_capacity=1 << 14, precision=1)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    for j in range(len(idx)):
        t16 = torch.from_numpy(fr.tokens[j]).to(dev).to(torch.bfloat16).contiguous()
        t32 = t16.float().cpu().numpy()
        d = torch.from_numpy(fr.depth[j]).to(dev)
        l = torch.from_numpy(fr.labels[j].view(np.int16)).to(dev)
        st = gmap.integrate(device_frame(d, l, t16, fr.poses[j], intr, fr.num_masks[j]))
        o = omap.integrate(fr.depth[j], fr.labels[j], t32, fr.poses[j], intr, fr.num_masks[j])
        common.compare_frame(st, gmap.last_frame(), o, ctx=f"multistory frame {idx[j]}", efast_tol=2e-2)
    common.compare_maps(gmap, omap, ctx="multistory")
    assert gmap.cfg["voxel_capacity"] >= 1 << 27


def test_overlapped_batches_equal_sequential(torch_dev):
    # serial_sms > 0: the stateless steps of the next batch overlap the serial
    # steps of this one (two streams, SM partitions); results must not change
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene()
    fr = sc.render(range(40))
    frames = [_dframe(torch, dev, fr, i) for i in range(40)]
    kw = dict(voxel_capacity=1 << 22, instance_capacity=1 << 12, batch_frames=8)
    a = DiscMap(**common.disc_cfg(sc, **kw))
    b = DiscMap(**common.disc_cfg(sc, serial_sms=48, **kw))
    for lo in (0, 24):
        sa, da, ra = a.integrate_frames(frames[lo:lo + 16] if lo == 0 else frames[lo:])
        sb, db, rb = b.integrate_frames(frames[lo:lo + 16] if lo == 0 else frames[lo:])
        assert ra == rb == 0 and da == db
        for x, y in zip(sa, sb):
            for k in ("unique_seg_voxels", "new_voxels", "new_instances", "merges", "overlap_pairs"):
                assert x[k] == y[k]
    ka, ia = a.voxels()
    kb, ib = b.voxels()
    assert np.array_equal(ka, kb) and np.array_equal(ia, ib)
    ea, eb = a.instances(), b.instances()
    for k in ("parent", "count", "n_obs"):
        assert np.array_equal(ea[k], eb[k])
    assert np.array_equal(ea["E"].view(np.uint32), eb["E"].view(np.uint32))


@pytest.mark.parametrize("eps,min_pts", [(0.05, 6), (0.08, 12)])
def test_dbscan_tiny_trajectory_parity(torch_dev, eps, min_pts):
    # Sec. III-A noise filter: Tiny frames have 3-5 cm between pixels, so
    # segment edges and thin objects produce noise points
    sc = synth.tiny_scene()
    gmap, omap, stats = run_parity(torch_dev, sc, range(20), dbscan_eps=eps, dbscan_min_pts=min_pts)
    assert sum(s["denoised_pixels"] for s in stats) > 0


def test_dbscan_room_frames_batched_parity(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene()
    fr = sc.render(range(40))
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 22, instance_capacity=1 << 12, dbscan_eps=0.05,
                          dbscan_min_pts=10)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for lo, hi in ((0, 32), (32, 40)):  # a full batch, then a partial one reusing the slots
        frames = [_dframe(torch, dev, fr, i) for i in range(lo, hi)]
        stats, done, rc = gmap.integrate_frames(frames)
        assert rc == 0 and done == hi - lo
        for j, st in enumerate(stats):
            o = omap.integrate(*oracle.frame_args(fr, lo + j), report=True)
            for gk, ok in common.COUNT_FIELDS:
                assert st[gk] == o[ok], f"frame {lo + j} {gk}: {st[gk]} vs {o[ok]}"
    common.compare_maps(gmap, omap, ctx="room dbscan")


def test_dbscan_wall_outliers(torch_dev):
    from paper_2603_03935_gb300 import DiscMap, host_frame
    H, W, f = 48, 64, 50.0
    depth = scenes.plane_depth(H, W, f, f, W / 2, H / 2, 2.0)
    labels = np.ones((H, W), np.uint16)
    outliers = [(10, 10), (20, 40), (30, 25), (40, 50)]
    for (v, u) in outliers:
        depth[v, u] = 1.5
    tok = np.random.default_rng(5).standard_normal((48, 16)).astype(np.float32)
    intr = (f, f, W / 2, H / 2)
    cfg = dict(voxel_size=0.05, embed_dim=16, patch_h=6, patch_w=8, max_width=W, max_height=H, max_masks=2,
               min_mask_pixels=3, voxel_capacity=1 << 14, instance_capacity=16, dbscan_eps=0.05, dbscan_min_pts=4)
    gmap = DiscMap(**cfg)
    ocfg = oracle.default_config(16, 6, 8, 0.05, min_mask_pixels=3, dbscan_eps=0.05, dbscan_min_pts=4)
    omap = oracle.OracleMap(**ocfg)
    st = gmap.integrate(host_frame(depth, labels, tok, np.eye(4), intr, 1))
    o = omap.integrate(depth, labels, tok, np.eye(4), intr, 1)
    assert st["denoised_pixels"] == o["denoised_pixels"] == len(outliers)
    common.compare_frame(st, gmap.last_frame(), o, ctx="wall outliers")
    common.compare_maps(gmap, omap, ctx="wall outliers")
