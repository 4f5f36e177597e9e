"""Failure paths on the GPU, made without a GPU fault: a device wait that runs
out (its limit is about a second), device allocations that fail (injected on
the host), and a determinism check (the same frames twice, bit for bit).

After each failure the call returns its status, the map is as it was before
the failing frame, and the context stays usable: integration resumes and ends
equal to the oracle."""
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


def _dframe(torch, dev, fr, i):
    from paper_2603_03935_gb300 import device_frame
    sc = fr.scene
    d = torch.from_numpy(fr.depth[i]).to(dev)
    l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[i]).to(dev)
    return device_frame(d, l, t, fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[i])


def _state(m):
    k, i = m.voxels()
    e = m.instances()
    return k, i, {x: e[x].copy() for x in ("parent", "count", "Q", "E", "n_obs")}


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for x in a[2]:
        assert np.array_equal(a[2][x].view(np.uint8), b[2][x].view(np.uint8)), x


def test_device_wait_runs_out_and_the_map_survives(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    from paper_2603_03935_gb300.binding import debug_gemm_stall
    sc = synth.tiny_scene()
    fr = sc.render(range(6))
    cfg = common.disc_cfg(sc)
    m = DiscMap(**cfg)
    for i in range(3):
        m.integrate(_dframe(torch, dev, fr, i))
    before = _state(m)
    debug_gemm_stall(True)
    try:
        st = m.integrate(_dframe(torch, dev, fr, 3), check=False)
    finally:
        debug_gemm_stall(False)
    assert st["rc"] == -5  # DISC_ERR_TIMEOUT
    _same(_state(m), before)
    for i in range(3, 6):
        assert m.integrate(_dframe(torch, dev, fr, i))["rc"] == 0
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(6):
        omap.integrate(*oracle.frame_args(fr, i))
    common.compare_maps(m, omap, ctx="after a timed-out frame")


def test_allocation_failures_are_reported_and_the_map_survives(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscError, DiscMap
    from paper_2603_03935_gb300.binding import debug_fail_alloc_after
    sc = synth.tiny_scene()
    fr = sc.render(range(12))
    cfg = common.disc_cfg(sc, voxel_capacity=256, instance_capacity=4)  # both tables must grow
    # creation: out of memory at every point of the map's allocations
    for n in (0, 1, 5):
        debug_fail_alloc_after(n)
        try:
            with pytest.raises(DiscError) as e:
                DiscMap(**cfg)
            assert e.value.code == -2
        finally:
            debug_fail_alloc_after(-1)
    m = DiscMap(**cfg)
    assert m.integrate(_dframe(torch, dev, fr, 0))["rc"] == 0
    grew = 0
    for i in range(1, 12):
        before = _state(m)
        debug_fail_alloc_after(0)
        try:
            st = m.integrate(_dframe(torch, dev, fr, i), check=False)
        finally:
            debug_fail_alloc_after(-1)
        if st["rc"] != 0:
            assert st["rc"] == -2  # DISC_ERR_OOM: a table had to grow
            _same(_state(m), before)
            grew += 1
            assert m.integrate(_dframe(torch, dev, fr, i))["rc"] == 0  # the same frame, allocations back
    assert grew > 0
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(12):
        omap.integrate(*oracle.frame_args(fr, i))
    common.compare_maps(m, omap, ctx="after refused growth")


def test_same_frames_twice_give_the_same_bits(torch_dev):
    # races in the lowest-index-wins claims or the atomics would show here
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    sc = synth.room_scene(num_frames=2000)
    fr = sc.render(range(40))
    frames = [_dframe(torch, dev, fr, i) for i in range(40)]
    out = []
    for _ in range(2):
        m = DiscMap(**common.disc_cfg(sc, voxel_capacity=1 << 22, instance_capacity=1 << 12))
        _, done, rc = m.integrate_frames(frames)
        assert rc == 0 and done == 40
        out.append((_state(m), m.last_frame()))
    _same(out[0][0], out[1][0])
    for k in ("E", "E_fast", "W", "S", "cov"):
        assert np.array_equal(np.asarray(out[0][1][k]).view(np.uint8), np.asarray(out[1][1][k]).view(np.uint8)), k


def _bad_intrinsics(sc, bad):
    intr = [sc.fx, sc.fy, sc.cx, sc.cy]
    pose_fix = None
    if bad == "fx_nan":
        intr[0] = float("nan")
    elif bad == "fy_inf":
        intr[1] = float("inf")
    elif bad == "fx_zero":
        intr[0] = 0.0
    elif bad == "pose_1e39":
        pose_fix = 1e39  # finite in fp64, infinite once rounded to fp32
    return tuple(intr), pose_fix


@pytest.mark.parametrize("bad", ["fx_nan", "fy_inf", "fx_zero", "pose_1e39"])
def test_non_finite_camera_or_pose_is_refused_by_the_library(torch_dev, bad):
    # a frame with a non-finite intrinsic or pose entry, or a zero focal
    # length, is refused with DISC_ERR_INVALID_ARG before the map changes;
    # the next valid frame integrates and the map ends equal to the oracle's
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.tiny_scene()
    fr = sc.render(range(3))
    cfg = common.disc_cfg(sc)
    gmap = DiscMap(**cfg)
    gmap.integrate(_dframe(torch, dev, fr, 0))
    before = _state(gmap)
    intr, pose_fix = _bad_intrinsics(sc, bad)
    pose = fr.poses[1].copy()
    if pose_fix is not None:
        pose[1, 3] = pose_fix
    d = torch.from_numpy(fr.depth[1]).to(dev)
    l = torch.from_numpy(fr.labels[1].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[1]).to(dev)
    st = gmap.integrate(device_frame(d, l, t, pose, intr, fr.num_masks[1]), check=False)
    assert st["rc"] == -1
    after = _state(gmap)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    for k in before[2]:
        assert np.array_equal(before[2][k], after[2][k]), k
    # in a call of several frames, the frames before the bad one integrate
    frames = [_dframe(torch, dev, fr, 1), device_frame(d, l, t, pose, intr, fr.num_masks[1])]
    _, done, rc = gmap.integrate_frames(frames, check=False)
    assert rc == -1 and done == 1
    gmap.integrate(_dframe(torch, dev, fr, 2))
    om = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(3):
        om.integrate(*oracle.frame_args(fr, i))
    common.compare_maps(gmap, om, ctx=f"after a refused frame ({bad})")


def test_non_finite_camera_in_a_group_stops_only_its_own_map(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscGroup, DiscMap, device_frame
    scs = [synth.tiny_scene(seed=0), synth.tiny_scene(seed=5), synth.tiny_scene(seed=7)]
    frs = [s.render(range(5)) for s in scs]
    maps = [DiscMap(**common.disc_cfg(s)) for s in scs]
    grp = DiscGroup(max_maps=3, frames_per_map=4, embed_dim=scs[0].dim, patch_h=scs[0].patch_h,
                    patch_w=scs[0].patch_w, max_width=scs[0].width, max_height=scs[0].height,
                    max_masks=scs[0].max_masks)
    per = [[_dframe(torch, dev, fr, i) for i in range(5)] for fr in frs]
    sc, fr = scs[1], frs[1]
    d = torch.from_numpy(fr.depth[2]).to(dev)
    l = torch.from_numpy(fr.labels[2].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[2]).to(dev)
    per[1][2] = device_frame(d, l, t, fr.poses[2], (float("nan"), sc.fy, sc.cx, sc.cy), fr.num_masks[2])
    stats, done, rc = grp.integrate(maps, per, check=False)
    assert rc == -1
    assert done == [5, 2, 5]
    for g, (m, f) in enumerate(zip(maps, frs)):
        om = oracle.OracleMap(**common.to_oracle_cfg(m.cfg))
        for i in range(done[g]):
            om.integrate(*oracle.frame_args(f, i))
        common.compare_maps(m, om, ctx=f"map {g} after a refused frame in the group")
