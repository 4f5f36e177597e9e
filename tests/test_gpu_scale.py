"""Parity at the sizes the benchmark times, through the C ABI.

* Room-scale: 800 consecutive 640x480 frames in 32-frame disc_integrate_frames
  calls, from a voxel table of 2^16 slots and an instance table of 64 ids, so
  the table is rehashed and the instance arrays double several times on the
  way; every frame's counters and the final map equal the oracle's.
* Multi-story: 220 consecutive frames that leave the ground floor for the
  first floor (the path changes floor after frame 1666), bf16 tokens at BF16
  precision, up to 100 masks, a 2^27-slot voxel table.
* Served: maps of mixed sizes and precisions, each walking its own
  trajectory, submitted from several client threads into one server; every
  frame's counters and each final map equal the oracle's, and each query
  returns the top-k of the oracle's instances at that point.
* Past the shared capacities: checkpoints whose instances are cut into many
  small pieces make a frame join more edge roots or overlap more pairs than
  the association kernel keeps in shared memory; the frame takes the map's
  global pair hash and union region, with the same result as the oracle.
"""
import threading

import numpy as np
import pytest

import oracle
import synth
from tests import common

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2603_03935_gb300 import _build
    _build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return torch, dev


def _counters_equal(st, o, ctx):
    for gk, ok in common.COUNT_FIELDS:
        assert st[gk] == o[ok], f"{ctx} {gk}: {st[gk]} vs {o[ok]}"


def test_room_800_frames_with_table_growth(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.room_scene(num_frames=2000)
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 16, instance_capacity=64)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    B, N = 32, 800
    for lo in range(0, N, B):
        fr = sc.render(range(lo, lo + B))
        d = torch.from_numpy(fr.depth).to(dev)
        l = torch.from_numpy(fr.labels.view(np.int16)).to(dev)
        t = torch.from_numpy(fr.tokens).to(dev)
        frames = [device_frame(d[j], l[j], t[j], fr.poses[j], intr, fr.num_masks[j]) for j in range(B)]
        stats, done, rc = gmap.integrate_frames(frames)
        assert rc == 0 and done == B
        for j in range(B):
            o = omap.integrate(*oracle.frame_args(fr, j), report=True)
            _counters_equal(stats[j], o, f"room frame {lo + j}")
        if lo + B == N // 2:
            common.compare_maps(gmap, omap, ctx=f"room after {lo + B} frames")
    common.compare_maps(gmap, omap, ctx=f"room after {N} frames")
    nv, nid = gmap.counts()
    assert nv > (1 << 16) // 2 * 16 and nid > 64 * 4  # both tables grew several times


def test_multistory_220_frames_across_a_floor_change(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.multistory_scene()
    lo, hi = 1500, 1720
    assert sc.poses[lo][2, 3] < 3.0 < sc.poses[hi - 1][2, 3]  # ground floor, then the first floor
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 27, instance_capacity=1 << 10, precision=1)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    B = 32
    saw_100 = False
    for a in range(lo, hi, B):
        idx = list(range(a, min(a + B, hi)))
        fr = sc.render(idx)
        saw_100 |= int(fr.num_masks.max()) == 100
        t16 = torch.from_numpy(fr.tokens).to(dev).to(torch.bfloat16).contiguous()
        t32 = t16.float().cpu().numpy()
        d = torch.from_numpy(fr.depth).to(dev)
        l = torch.from_numpy(fr.labels.view(np.int16)).to(dev)
        frames = [device_frame(d[j], l[j], t16[j], fr.poses[j], intr, fr.num_masks[j]) for j in range(len(idx))]
        stats, done, rc = gmap.integrate_frames(frames)
        assert rc == 0 and done == len(idx)
        for j in range(len(idx)):
            o = omap.integrate(fr.depth[j], fr.labels[j], t32[j], fr.poses[j], intr, fr.num_masks[j])
            _counters_equal(stats[j], o, f"multistory frame {idx[j]}")
    assert saw_100
    common.compare_maps(gmap, omap, ctx="multistory 1500..1719")


def _oracle_topk(inst, q, k):
    """Top-k of the live instances (own parent, observed) by the float64
    cosine: (ids, scores), score descending, id ascending on ties."""
    live = np.nonzero((inst["parent"] == np.arange(len(inst["parent"]))) & (inst["n_obs"] > 0))[0]
    E = inst["E"][live].astype(np.float64)
    out_ids, out_sc = [], []
    for v in np.asarray(q, np.float64):
        s = E @ v / (np.linalg.norm(E, axis=1) * np.linalg.norm(v))
        order = np.lexsort((live, -s))[:k]
        out_ids.append(live[order])
        out_sc.append(s[order])
    return out_ids, out_sc


def test_served_maps_equal_the_oracle(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscServer, host_frame
    # four room-scale maps of different frame sizes, object counts and mask
    # limits, at FP32, BF16 and FP8 E4M3 precision (the fast score's
    # precision changes no decision)
    kinds = [(640, 480, 80, 40, 0), (320, 240, 20, 12, 2), (480, 360, 60, 30, 1), (320, 240, 40, 25, 2)]
    scs = [synth.room_scene(seed=31 + g, width=w, height=h, n_objects=o, max_masks=m)
           for g, (w, h, o, m, _) in enumerate(kinds)]
    nfr = [40, 48, 36, 44]
    starts = [0, 300, 700, 1100]  # each map walks its own stretch of its path
    frs = [s.render(range(a, a + n)) for s, a, n in zip(scs, starts, nfr)]
    srv = DiscServer(32 << 30, max_maps=len(scs), frames_per_map=4, embed_dim=scs[0].dim,
                     patch_h=scs[0].patch_h, patch_w=scs[0].patch_w, max_width=640, max_height=480,
                     max_masks=40, device=dev.index)
    cfgs = [common.disc_cfg(s, voxel_capacity=1 << 20, instance_capacity=256, precision=k[4])
            for s, k in zip(scs, kinds)]
    ids = [srv.open_map(**c) for c in cfgs]
    queries = [fr.tokens[0][:3] for fr in frs]
    q_at = [n // 2 for n in nfr]
    results = [None] * len(scs)

    def client(g):
        fr, sc = frs[g], scs[g]
        intr = (sc.fx, sc.fy, sc.cx, sc.cy)
        tickets, tq = [], None
        for i in range(nfr[g]):
            tickets.append(srv.submit_frame(ids[g], host_frame(fr.depth[i], fr.labels[i], fr.tokens[i],
                                                               fr.poses[i], intr, fr.num_masks[i])))
            if i + 1 == q_at[g]:
                tq = srv.submit_query(ids[g], queries[g], 5)
        results[g] = ([srv.wait_frame(t) for t in tickets], srv.wait_query(tq))

    th = [threading.Thread(target=client, args=(g,)) for g in range(len(scs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    rep = srv.stats()
    assert rep["batches"] < sum(nfr)  # frames of different maps shared batches
    for g, (sc, fr) in enumerate(zip(scs, frs)):
        stats, (qrc, qids, qsc, _) = results[g]
        assert all(s["rc"] == 0 for s in stats), f"map {g}"
        assert qrc == 0
        om = oracle.OracleMap(**common.to_oracle_cfg(cfgs[g]))
        for i in range(nfr[g]):
            o = om.integrate(*oracle.frame_args(fr, i), report=True)
            _counters_equal(stats[i], o, f"served map {g} frame {i}")
            if i + 1 == q_at[g]:
                oids, osc = _oracle_topk(om.instances(), queries[g], 5)
                for r in range(len(queries[g])):
                    n = len(oids[r])
                    assert np.all(qids[r][n:] == -1)
                    np.testing.assert_allclose(qsc[r][:n], osc[r], rtol=0, atol=1e-5)
                    # ids agree wherever the oracle's scores are not a near-tie
                    for j in range(n):
                        near = [abs(osc[r][j] - osc[r][x]) <= 1e-5 for x in range(n) if x != j]
                        if not any(near):
                            assert qids[r][j] == oids[r][j], f"map {g} query {r} rank {j}"
        common.compare_maps(srv.map(ids[g]), om, ctx=f"served map {g}")
    srv.close()


def _split_state(omap, S):
    """The oracle map's voxels with each instance cut into up to S pieces by
    a hash of the voxel key (every piece its own instance with the parent's
    embedding and Q): (keys, labels, parent, count, Q, E, n_obs)."""
    keys, ids = omap.voxels()
    inst = omap.instances()
    h = (keys * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
    new = ids.astype(np.int64) * S + (h % np.uint64(S)).astype(np.int64)
    uniq, inv = np.unique(new, return_inverse=True)
    nid = len(uniq)
    old = (uniq // S).astype(np.int64)
    labels = inv.astype(np.int32)
    return (keys, labels, np.arange(nid, dtype=np.int32), np.bincount(labels, minlength=nid).astype(np.int64),
            inst["Q"][old].astype(np.float32), np.ascontiguousarray(inst["E"][old], np.float32),
            np.ones(nid, np.int32))


def _write_checkpoint(path, cfg, state):
    import struct
    from paper_2603_03935_gb300 import binding as b
    keys, labels, parent, count, Q, E, obs = state
    c = b.Config(**b.config_default(**cfg))
    with open(path, "wb") as f:
        f.write(b"DISCMAP1" + bytes(c) + struct.pack("<qi", len(keys), len(parent)))
        for a, dt in ((keys, np.uint64), (labels, np.int32), (parent, np.int32), (count, np.int64), (Q, np.float32),
                      (E, np.float32), (obs, np.int32)):
            f.write(np.ascontiguousarray(a, dt).tobytes())


@pytest.mark.parametrize("kind,S,before", [("tiny", 200, 10), ("room", 60, 8)])
def test_frames_past_the_shared_capacities(torch_dev, tmp_path, kind, S, before):
    # maps whose instances are cut into many small pieces: the next frame
    # overlaps hundreds to thousands of them and its segments join most, so
    # its edge roots (tiny: ~600) or its pairs (room: ~2000) pass what the
    # association kernel keeps in shared memory and the frame runs on the
    # map's global pair hash and union region; loaded through a checkpoint
    # into the library and set into the oracle, both must agree
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.tiny_scene() if kind == "tiny" else synth.room_scene(num_frames=2000)
    fr = sc.render(range(before + 2))
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 20, instance_capacity=1 << 14)
    ocfg = common.to_oracle_cfg(cfg)
    base = oracle.OracleMap(**ocfg)
    for i in range(before):
        base.integrate(*oracle.frame_args(fr, i))
    state = _split_state(base, S)
    omap = oracle.OracleMap(**ocfg)
    omap.set_state(*state)
    path = tmp_path / "split.ckpt"
    _write_checkpoint(path, cfg, state)
    gmap = DiscMap.load(path)
    common.compare_maps(gmap, omap, ctx=f"{kind} split state loaded")
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    d = torch.from_numpy(fr.depth).to(dev)
    l = torch.from_numpy(fr.labels.view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens).to(dev)
    frames = [device_frame(d[j], l[j], t[j], fr.poses[j], intr, fr.num_masks[j]) for j in (before, before + 1)]
    stats, done, rc = gmap.integrate_frames(frames)
    assert rc == 0 and done == 2
    for j in range(2):
        o = omap.integrate(*oracle.frame_args(fr, before + j), report=True)
        _counters_equal(stats[j], o, f"{kind} split frame {before + j}")
        if j == 0:
            assert o["merges"] > 512 if kind == "tiny" else o["overlap_pairs"] > 1536
    common.compare_maps(gmap, omap, ctx=f"{kind} split, after two frames")
