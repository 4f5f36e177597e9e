"""Asynchronous calls (disc_integrate_frames_async, disc_group_integrate_async)
against the oracle, through the C ABI.

Two calls stay unfinished at a time, so a call's last frames still associate
while the next call's per-frame kernels run; the results must be those of
integrating the same frames one by one (Sec. III-B: every frame meets the map
its predecessors left):
* Room-scale frames in 32-frame asynchronous calls, from a small voxel table
  (it grows on the way) and from the benchmark's 2^26-slot one, and a small
  instance table, with the map read in the middle (an implicit finish),
  every frame's counters and the final map against the oracle;
* a frame that fails on the device stops the rest of its call and every call
  enqueued while that one was unfinished; a frame that fails the host checks
  makes the call synchronous;
* group calls: several maps, three asynchronous calls in flight order, each
  map against the oracle.
"""
import ctypes

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


def _dframes(torch, dev, fr, idx, bad=None):
    from paper_2603_03935_gb300 import device_frame
    sc = fr.scene
    out = []
    for i in idx:
        tok = fr.tokens[i] if bad is None or i != bad[0] else bad[1]
        d = torch.from_numpy(fr.depth[i]).to(dev)
        l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
        t = torch.from_numpy(np.ascontiguousarray(tok)).to(dev)
        out.append(device_frame(d, l, t, fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[i]))
    return out


def _counters_equal(st, o, ctx):
    for gk, ok in common.COUNT_FIELDS:
        assert st[gk] == o[ok], f"{ctx} {gk}: {st[gk]} vs {o[ok]}"


@pytest.mark.parametrize("table_log2", [16, 26])
def test_async_room_calls_equal_the_oracle(torch_dev, table_log2):
    # 2^16 slots: the table grows under the calls (room checks with a round
    # trip); 2^26, the benchmark's table: the host bound always fits, so no
    # call waits for a room check
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene(num_frames=400)
    cfg = common.disc_cfg(sc, voxel_capacity=1 << table_log2, instance_capacity=64)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    B, N, MID = 32, 256, 160
    fr = sc.render(range(N))
    handles, reports = [], []

    def oracle_to(n):
        while len(reports) < n:
            reports.append(omap.integrate(*oracle.frame_args(fr, len(reports)), report=True))

    for lo in range(0, N, B):
        handles.append(gmap.integrate_frames_async(_dframes(torch, dev, fr, range(lo, lo + B))))
        if lo + B == MID:
            # reading the map finishes the calls before it
            oracle_to(MID)
            common.compare_maps(gmap, omap, ctx=f"room after {MID} frames")
    assert gmap.wait() == 0
    oracle_to(N)
    for c, h in enumerate(handles):
        stats, done, rc = h.result()
        assert rc == 0 and done == B
        for j in range(B):
            _counters_equal(stats[j], reports[c * B + j], f"room frame {c * B + j}")
    common.compare_maps(gmap, omap, ctx=f"room after {N} frames")
    nv, nid = gmap.counts()
    assert nv > (1 << 16) and nid > 64  # past the small table's and the instance table's first capacities
    gmap.close()


def test_async_device_error_stops_the_calls_enqueued_behind_it(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(16))
    cfg = common.disc_cfg(sc)
    gmap = DiscMap(**cfg)
    bad = fr.tokens[5].copy()
    bad[2, 3] = np.inf  # fails frame 5 on the device (DISC_ERR_RANGE)
    h1 = gmap.integrate_frames_async(_dframes(torch, dev, fr, range(0, 8), bad=(5, bad)))
    h2 = gmap.integrate_frames_async(_dframes(torch, dev, fr, range(8, 12)))
    _s1, done1, rc1 = h1.result(check=False)
    _s2, done2, rc2 = h2.result(check=False)
    assert (rc1, done1) == (-7, 5)
    assert (rc2, done2) == (-7, 0)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(5):
        omap.integrate(*oracle.frame_args(fr, i))
    common.compare_maps(gmap, omap, ctx="after the failed frame")
    # once finished, a new call starts from the map as it stands
    h3 = gmap.integrate_frames_async(_dframes(torch, dev, fr, range(8, 16)))
    stats, done3, rc3 = h3.result()
    assert (rc3, done3) == (0, 8)
    for i in range(8, 16):
        o = omap.integrate(*oracle.frame_args(fr, i), report=True)
        _counters_equal(stats[i - 8], o, f"frame {i} after the error")
    common.compare_maps(gmap, omap, ctx="after the later call")
    gmap.close()


def test_async_host_check_failure_runs_synchronously(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, binding
    sc = synth.tiny_scene()
    fr = sc.render(range(10))
    cfg = common.disc_cfg(sc)
    gmap = DiscMap(**cfg)
    h1 = gmap.integrate_frames_async(_dframes(torch, dev, fr, range(0, 4)))
    frames = _dframes(torch, dev, fr, range(4, 10))
    arr = (binding.Frame * 6)()
    for i, (f, _k) in enumerate(frames):
        arr[i] = f
    arr[2].fx = float("nan")  # frame 6 fails the host checks
    stats = (binding.Stats * 6)()
    done, res = ctypes.c_int32(-1), ctypes.c_int32(1)
    rc = gmap.integrate_frames_async_raw(arr, 6, stats, done, res)
    # written before returning, after the earlier call finished
    assert rc == -1 and res.value == -1 and done.value == 2
    _s1, done1, rc1 = h1.result()
    assert (rc1, done1) == (0, 4)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(6):
        o = omap.integrate(*oracle.frame_args(fr, i), report=True)
        if i >= 4:
            _counters_equal(stats[i - 4].as_dict(), o, f"frame {i}")
    common.compare_maps(gmap, omap, ctx="after the refused frame")
    gmap.close()


def test_group_async_calls_equal_the_oracle(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscGroup, DiscMap, binding
    scs = [synth.tiny_scene(seed=s) for s in (0, 3, 7)]
    counts = [20, 14, 9]
    frs = [s.render(range(n)) for s, n in zip(scs, counts)]
    maps = [DiscMap(**common.disc_cfg(s)) for s in scs]
    omaps = [oracle.OracleMap(**common.to_oracle_cfg(m.cfg)) for m in maps]
    grp = DiscGroup(max_maps=3, frames_per_map=4, embed_dim=scs[0].dim, patch_h=scs[0].patch_h,
                    patch_w=scs[0].patch_w, max_width=max(s.width for s in scs),
                    max_height=max(s.height for s in scs), max_masks=max(s.max_masks for s in scs))
    calls = []
    for lo, hi in ((0, 4), (4, 11), (11, 20)):  # the third call finishes the first
        per, arrs, sts, cnts = [], [], [], []
        for fr, n in zip(frs, counts):
            fl = _dframes(torch, dev, fr, range(lo, min(hi, n)))
            a = (binding.Frame * max(len(fl), 1))()
            for i, (f, _k) in enumerate(fl):
                a[i] = f
            per.append(fl)
            arrs.append(a)
            sts.append((binding.Stats * max(len(fl), 1))())
            cnts.append(len(fl))
        done = (ctypes.c_int32 * 3)()
        res = ctypes.c_int32(1)
        assert grp.integrate_async_raw(maps, arrs, cnts, sts, done, res) == 0
        calls.append((lo, per, sts, cnts, done, res))
    assert grp.wait() == 0
    for lo, per, sts, cnts, done, res in calls:
        assert res.value == 0 and list(done) == cnts
        for g, (fr, om) in enumerate(zip(frs, omaps)):
            for j in range(cnts[g]):
                o = om.integrate(*oracle.frame_args(fr, lo + j), report=True)
                _counters_equal(sts[g][j].as_dict(), o, f"map {g} frame {lo + j}")
    for g, (m, om) in enumerate(zip(maps, omaps)):
        common.compare_maps(m, om, ctx=f"group map {g}")
    grp.close()
    for m in maps:
        m.close()
