"""The serving loop (disc_server_*): continuous batching over resident maps.

Clients on several host threads submit frames and queries for different maps
at once; the server batches whatever is pending.  Every map must end
bit-identical to the same frames integrated alone, every query must return
what it returns against the map alone at the same point, and a failing frame
must fail alone.
"""
import threading

import numpy as np
import pytest

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


def _hframe(fr, i, tokens=None):
    from paper_2603_03935_gb300 import host_frame
    sc = fr.scene
    return host_frame(fr.depth[i], fr.labels[i], fr.tokens[i] if tokens is None else tokens, fr.poses[i],
                      (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[i])


def _scenes():
    a = synth.tiny_scene(seed=0)
    b = synth.tiny_scene(seed=3)
    prims = [(0, 1, (0.013, 0.013, 0.213), (0.3, 0.25, 0.2)),
             (1, 2, (0.7, 0.45, 0.25), (0.2, 0.2, 0.25)),
             (0, 3, (-0.6, 0.5, 0.15), (0.15, 0.3, 0.15))]
    c = scenes.custom_scene(prims, scenes.orbit((0.1, 0.2, 0.2), 1.7, 0.9, 12, sweep=np.deg2rad(150)),
                            width=80, height=60, f=60.0, dim=512, patch=(6, 8), voxel=0.04, max_masks=6)
    d = scenes.custom_scene(prims[:2], scenes.orbit((0.2, 0.1, 0.2), 1.4, 1.0, 10, sweep=np.deg2rad(90)),
                            width=48, height=36, f=40.0, dim=512, patch=(6, 8), voxel=0.05, max_masks=3)
    return [a, b, c, d]


def _server(scs, budget=8 << 30, workers=0, **kw):
    from paper_2603_03935_gb300 import DiscServer
    g = dict(max_maps=len(scs), frames_per_map=2, embed_dim=scs[0].dim, patch_h=scs[0].patch_h,
             patch_w=scs[0].patch_w, max_width=max(s.width for s in scs), max_height=max(s.height for s in scs),
             max_masks=max(s.max_masks for s in scs))
    g.update(kw)
    return DiscServer(budget, workers=workers, **g)


def _same_map(a, b, ctx):
    ka, ia = a.voxels()
    kb, ib = b.voxels()
    assert np.array_equal(ka, kb) and np.array_equal(ia, ib), f"{ctx}: voxels"
    ea, eb = a.instances(), b.instances()
    for k in ("parent", "count", "n_obs"):
        assert np.array_equal(ea[k], eb[k]), f"{ctx}: {k}"
    assert np.array_equal(ea["E"].view(np.uint32), eb["E"].view(np.uint32)), f"{ctx}: embeddings"
    assert np.array_equal(ea["Q"].view(np.uint32), eb["Q"].view(np.uint32)), f"{ctx}: Q"


@pytest.mark.parametrize("workers,borrow", [(1, False), (2, False), (4, False), (2, True)])
def test_concurrent_clients_equal_each_map_alone(torch_dev, workers, borrow):
    # with several workers, batches of different maps run at once; a map is
    # in one batch at a time, so every result still equals the map alone;
    # borrowed frames are read in place when their batch runs
    from paper_2603_03935_gb300 import DiscMap
    scs = _scenes()
    nfr = [20, 14, 12, 10]
    frs = [s.render(range(n)) for s, n in zip(scs, nfr)]
    srv = _server(scs, workers=workers)
    ids = [srv.open_map(**common.disc_cfg(s)) for s in scs]
    queries = [fr.tokens[0][:3] for fr in frs]  # three patch tokens of each map's first frame
    q_at = [n // 2 for n in nfr]                # each map is queried after half its frames
    results = [None] * len(scs)

    def client(g):
        tickets = []
        tq = None
        held = []  # borrowed inputs stay alive until their waits return
        for i in range(nfr[g]):
            if borrow:
                held.append(_hframe(frs[g], i))
                tickets.append(srv.submit_frame_borrowed(ids[g], held[-1]))
            else:
                tickets.append(srv.submit_frame(ids[g], _hframe(frs[g], i)))
            if i + 1 == q_at[g]:
                tq = srv.submit_query(ids[g], queries[g], 3)
        stats = [srv.wait_frame(t) for t in tickets]
        results[g] = (stats, srv.wait_query(tq))

    threads = [threading.Thread(target=client, args=(g,)) for g in range(len(scs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    rep = srv.stats()
    assert rep["frames"] == sum(nfr) and rep["queries"] == len(scs) and rep["pending"] == 0
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    for g, sc in enumerate(scs):
        stats, (qrc, qids, qsc, _) = results[g]
        assert all(s["rc"] == 0 for s in stats), f"map {g}: {[s['rc'] for s in stats]}"
        alone = DiscMap(**common.disc_cfg(sc))
        a_stats = []
        for i in range(q_at[g]):
            a_stats.append(alone.integrate(_hframe(frs[g], i)))
        aids, asc = alone.query_topk(queries[g], 3)
        for i in range(q_at[g], nfr[g]):
            a_stats.append(alone.integrate(_hframe(frs[g], i)))
        assert qrc == 0 and np.array_equal(qids, aids) and np.array_equal(qsc.view(np.uint32), asc.view(np.uint32)), \
            f"map {g}: query"
        for i, (s1, s2) in enumerate(zip(stats, a_stats)):
            for k in ("unique_seg_voxels", "new_voxels", "new_instances", "merges", "overlap_pairs"):
                assert s1[k] == s2[k], f"map {g} frame {i} {k}"
        _same_map(srv.map(ids[g]), alone, f"map {g}")
    assert rep["batches"] < sum(nfr)  # frames of different maps shared batches
    srv.close()


def test_failing_frame_fails_alone(torch_dev):
    from paper_2603_03935_gb300 import DiscMap
    scs = _scenes()[:3]
    frs = [s.render(range(8)) for s in scs]
    srv = _server(scs, frames_per_map=4)
    ids = [srv.open_map(**common.disc_cfg(s)) for s in scs]
    bad = frs[0].tokens[3].copy()
    bad[2, 5] = np.nan
    tickets = []
    for i in range(8):  # interleaved submission, one map's frame 3 is bad
        for g in range(3):
            tok = bad if (g == 0 and i == 3) else None
            tickets.append((g, i, srv.submit_frame(ids[g], _hframe(frs[g], i, tok))))
    out = {(g, i): srv.wait_frame(t) for g, i, t in tickets}
    for (g, i), st in out.items():
        assert st["rc"] == (-7 if (g == 0 and i == 3) else 0), (g, i, st["rc"])
    for g, sc in enumerate(scs):
        alone = DiscMap(**common.disc_cfg(sc))
        for i in range(8):
            tok = bad if (g == 0 and i == 3) else None
            alone.integrate(_hframe(frs[g], i, tok), check=False)
        _same_map(srv.map(ids[g]), alone, f"map {g}")
    srv.close()


def test_admission_by_device_memory_budget(torch_dev):
    scs = _scenes()[:2]
    probe = _server(scs)
    base = probe.stats()["resident_bytes"]
    mid = probe.open_map(**common.disc_cfg(scs[0]))
    one = probe.stats()["resident_bytes"] - base
    probe.close()
    assert one > 0
    srv = _server(scs, budget=base + one + one // 2)
    first = srv.open_map(**common.disc_cfg(scs[0]))
    rc, _ = srv.try_open_map(**common.disc_cfg(scs[0]))
    assert rc == -6  # DISC_ERR_BUDGET: a second map does not fit
    srv.close_map(first)
    rc, second = srv.try_open_map(**common.disc_cfg(scs[0]))
    assert rc == 0 and second >= 0
    srv.close()


def test_second_grid_and_precisions_in_one_server(torch_dev):
    # maps with and without a second token grid, at FP32, BF16 and FP8, served
    # side by side (the server copies every input, second grid included, at
    # submission); each equals the same frames integrated alone
    from paper_2603_03935_gb300 import DiscMap, host_frame
    GRID = dict(assoc_dim=96, assoc_patch_h=6, assoc_patch_w=8)
    scs = _scenes()[:2]
    frs = [s.render(range(10)) for s in scs]
    ats = [fr.assoc_tokens(6, 8, 96) for fr in frs]
    srv = _server(scs, frames_per_map=3, **GRID)
    kinds = [(0, 2, True), (1, 0, False), (0, 1, False), (1, 2, True)]  # (scene, precision, second grid)
    cfgs = [common.disc_cfg(scs[s], precision=p, **(GRID if a else {})) for s, p, a in kinds]
    ids = [srv.open_map(**c) for c in cfgs]

    def frame(g, i):
        s, _, a = kinds[g]
        fr, sc = frs[s], scs[s]
        return host_frame(fr.depth[i], fr.labels[i], fr.tokens[i], fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy),
                          fr.num_masks[i], assoc_tokens=ats[s][i] if a else None)

    tickets = [(g, srv.submit_frame(ids[g], frame(g, i))) for i in range(10) for g in range(len(kinds))]
    for g, t in tickets:
        assert srv.wait_frame(t)["rc"] == 0, g
    for g, c in enumerate(cfgs):
        alone = DiscMap(**c)
        for i in range(10):
            alone.integrate(frame(g, i))
        _same_map(srv.map(ids[g]), alone, f"map {g} {kinds[g]}")
        if kinds[g][2]:
            assert np.array_equal(srv.map(ids[g]).instances()["A"].view(np.uint32),
                                  alone.instances()["A"].view(np.uint32))
    srv.close()
