"""Groups of maps (disc_group_integrate) vs the oracle, map by map.

Maps of different frame sizes, mask counts, token grids' contents and frame
counts are integrated side by side; every map must end bit-identical to the
oracle run on that map alone, and a failing frame must stop only its own map.
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


def _dframe(torch, dev, fr, i, tokens=None):
    from paper_2603_03935_gb300 import device_frame
    sc = fr.scene
    d = torch.from_numpy(fr.depth[i]).to(dev)
    l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[i] if tokens is None else tokens).to(dev)
    return device_frame(d, l, t, fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[i])


def _mixed_scenes():
    """Same token grid (6 x 8 x 512), different frame sizes and contents."""
    a = synth.tiny_scene(seed=0)
    b = synth.tiny_scene(seed=5)
    prims = [(0, 1, (0.013, 0.013, 0.213), (0.3, 0.25, 0.2)),
             (1, 2, (0.7, 0.45, 0.25), (0.2, 0.2, 0.25)),
             (0, 3, (-0.6, 0.5, 0.15), (0.15, 0.3, 0.15))]
    c = scenes.custom_scene(prims, scenes.orbit((0.1, 0.2, 0.2), 1.7, 0.9, 9, sweep=np.deg2rad(120)),
                            width=80, height=60, f=60.0, dim=512, patch=(6, 8), voxel=0.04, max_masks=6)
    d = scenes.custom_scene(prims[:2], scenes.orbit((0.2, 0.1, 0.2), 1.4, 1.0, 3, sweep=np.deg2rad(40)),
                            width=48, height=36, f=40.0, dim=512, patch=(6, 8), voxel=0.05, max_masks=3)
    return [a, b, c, d]


def _group(sc_list, frames_per_map):
    from paper_2603_03935_gb300 import DiscGroup
    return DiscGroup(max_maps=len(sc_list), frames_per_map=frames_per_map, embed_dim=sc_list[0].dim,
                     patch_h=sc_list[0].patch_h, patch_w=sc_list[0].patch_w,
                     max_width=max(s.width for s in sc_list), max_height=max(s.height for s in sc_list),
                     max_masks=max(s.max_masks for s in sc_list))


def test_group_maps_equal_the_oracle_map_by_map(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    scs = _mixed_scenes()
    counts = [20, 13, 9, 3]
    frs = [s.render(range(n)) for s, n in zip(scs, counts)]
    maps = [DiscMap(**common.disc_cfg(s)) for s in scs]
    omaps = [oracle.OracleMap(**common.to_oracle_cfg(m.cfg)) for m in maps]
    grp = _group(scs, 4)
    # two calls: frames [0, 7) of every map, then the rest (a map may sit out)
    for lo, hi in ((0, 7), (7, 20)):
        per = [[_dframe(torch, dev, fr, i) for i in range(lo, min(hi, n))] for fr, n in zip(frs, counts)]
        stats, done, rc = grp.integrate(maps, per)
        assert rc == 0 and done == [len(p) for p in per]
        for g, (fr, om) in enumerate(zip(frs, omaps)):
            for j, st in enumerate(stats[g]):
                o = om.integrate(*oracle.frame_args(fr, lo + j), report=True)
                for gk, ok in common.COUNT_FIELDS:
                    assert st[gk] == o[ok], f"map {g} frame {lo + j} {gk}: {st[gk]} vs {o[ok]}"
    for g, (m, om) in enumerate(zip(maps, omaps)):
        common.compare_maps(m, om, ctx=f"group map {g}")


def test_group_equals_each_map_alone(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    scs = _mixed_scenes()
    counts = [20, 13, 9, 3]
    frs = [s.render(range(n)) for s, n in zip(scs, counts)]
    together = [DiscMap(**common.disc_cfg(s)) for s in scs]
    alone = [DiscMap(**common.disc_cfg(s)) for s in scs]
    grp = _group(scs, 8)
    per = [[_dframe(torch, dev, fr, i) for i in range(n)] for fr, n in zip(frs, counts)]
    _, done, rc = grp.integrate(together, per)
    assert rc == 0 and done == counts
    for m, frames in zip(alone, per):
        _, d1, rc1 = m.integrate_frames(frames)
        assert rc1 == 0
    for g, (a, b) in enumerate(zip(together, alone)):
        ka, ia = a.voxels()
        kb, ib = b.voxels()
        assert np.array_equal(ka, kb) and np.array_equal(ia, ib), f"map {g} voxels"
        ea, eb = a.instances(), b.instances()
        for k in ("parent", "count", "n_obs"):
            assert np.array_equal(ea[k], eb[k]), f"map {g} {k}"
        assert np.array_equal(ea["E"].view(np.uint32), eb["E"].view(np.uint32)), f"map {g} embeddings"
        assert np.array_equal(ea["Q"].view(np.uint32), eb["Q"].view(np.uint32)), f"map {g} Q"


def test_group_error_stops_only_its_own_map(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    scs = _mixed_scenes()[:3]
    counts = [6, 6, 6]
    frs = [s.render(range(n)) for s, n in zip(scs, counts)]
    maps = [DiscMap(**common.disc_cfg(s)) for s in scs]
    grp = _group(scs, 4)
    per = [[_dframe(torch, dev, fr, i) for i in range(n)] for fr, n in zip(frs, counts)]
    bad = frs[1].tokens[2].copy()
    bad[5, 9] = np.inf
    per[1][2] = _dframe(torch, dev, frs[1], 2, tokens=bad)
    stats, done, rc = grp.integrate(maps, per, check=False)
    assert rc == -7
    assert done == [6, 2, 6]
    assert stats[1][2]["status"] == -7 and all(s["status"] == -7 for s in stats[1][3:])
    for g, (m, fr) in enumerate(zip(maps, frs)):
        om = oracle.OracleMap(**common.to_oracle_cfg(m.cfg))
        for i in range(done[g]):
            om.integrate(*oracle.frame_args(fr, i))
        common.compare_maps(m, om, ctx=f"map {g} after the failure")


def test_group_rejects_duplicate_and_mismatched_maps(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    scs = _mixed_scenes()[:2]
    frs = [s.render(range(2)) for s in scs]
    maps = [DiscMap(**common.disc_cfg(s)) for s in scs]
    grp = _group(scs, 2)
    per = [[_dframe(torch, dev, fr, i) for i in range(2)] for fr in frs]
    _, done, rc = grp.integrate([maps[0], maps[0]], per, check=False)
    assert rc == -1 and done == [0, 0]
    other = DiscMap(**common.disc_cfg(scs[0], embed_dim=256))
    _, done, rc = grp.integrate([maps[0], other], per, check=False)
    assert rc == -1
    assert maps[0].counts() == (0, 0)


def test_group_room_scale_maps(torch_dev):
    # the batched benchmark's launch shape: several room-scale maps, a few
    # frames of each per batch
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    scs = [synth.room_scene(seed=s) for s in (1, 2, 3)]
    n = 6
    frs = [s.render(range(n)) for s in scs]
    maps = [DiscMap(**common.disc_cfg(s, voxel_capacity=1 << 22, instance_capacity=1 << 12)) for s in scs]
    omaps = [oracle.OracleMap(**common.to_oracle_cfg(m.cfg)) for m in maps]
    grp = _group(scs, 4)
    per = [[_dframe(torch, dev, fr, i) for i in range(n)] for fr in frs]
    stats, done, rc = grp.integrate(maps, per)
    assert rc == 0 and done == [n] * 3
    for g, (fr, om) in enumerate(zip(frs, omaps)):
        for j in range(n):
            o = om.integrate(*oracle.frame_args(fr, j), report=True)
            for gk, ok in common.COUNT_FIELDS:
                assert stats[g][j][gk] == o[ok], f"room map {g} frame {j} {gk}"
        common.compare_maps(maps[g], om, ctx=f"room map {g}")


def test_schedules_leave_results_unchanged_and_autotune_picks_one(torch_dev):
    # the launch schedule (frames per geometry launch, serial CTA counts,
    # lanes per key of the voxel lookup, CTAs per map of the association
    # kernel) changes no result; the autotuner times fresh maps and keeps the
    # tuned map and group untouched
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscGroup, DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(16))
    frames = [_dframe(torch, dev, fr, i) for i in range(16)]
    omap = oracle.OracleMap(**common.to_oracle_cfg(common.disc_cfg(sc)))
    for i in range(16):
        omap.integrate(*oracle.frame_args(fr, i))
    for geo, q, pw, ac, bsp in ((4, 4, 1, 0, 0), (1, 1, 2, 1, 1), (2, 8, 4, 2, 2), (8, 2, 8, 8, 4),
                                (32, 32, 1, 4, 8)):
        for bf in (8, 16):  # a call of 16 frames: two batches, or one cut into bsp
            m = DiscMap(**common.disc_cfg(sc, batch_frames=bf))
            m.set_schedule(geo, q, pw, ac, bsp)
            _, done, rc = m.integrate_frames(frames)
            assert rc == 0 and done == 16
            common.compare_maps(m, omap, ctx=f"schedule {geo}/{q}/{pw}/{ac}/{bsp}, batches of {bf}")
    m = DiscMap(**common.disc_cfg(sc, batch_frames=8))
    rep = m.autotune(frames[:8], reps=1)
    assert rep["candidates"] == 20 and rep["best_ms"] <= rep["default_ms"]
    assert rep["geometry_chunk"] in (2, 4, 8) and rep["probe_width"] in (1, 2, 4)
    assert rep["assoc_cluster"] in (0, 4) and rep["batch_split"] in (0, 1, 4)
    assert m.counts()[0] == 0
    _, done, rc = m.integrate_frames(frames)
    assert rc == 0
    common.compare_maps(m, omap, ctx="after autotune")
    # a group tuned on two maps' sample, then used
    a, b = DiscMap(**common.disc_cfg(sc)), DiscMap(**common.disc_cfg(sc))
    grp = DiscGroup(max_maps=2, frames_per_map=4, embed_dim=sc.dim, patch_h=sc.patch_h, patch_w=sc.patch_w,
                    max_width=sc.width, max_height=sc.height, max_masks=sc.max_masks)
    from paper_2603_03935_gb300 import binding
    arr = (binding.Frame * 4)()
    for i in range(4):
        arr[i] = frames[i][0]
    grep = grp.autotune([a, b], [arr, arr], [4, 4], reps=1)
    assert grep["candidates"] == 20 and a.counts()[0] == 0 and b.counts()[0] == 0
    _, done, rc = grp.integrate([a, b], [frames, frames])
    assert rc == 0 and done == [16, 16]
    common.compare_maps(a, omap, ctx="tuned group, map a")
    common.compare_maps(b, omap, ctx="tuned group, map b")
