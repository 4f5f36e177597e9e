"""The second token grid (association on its features) and the Fig. 2 query
heatmap on the GPU against the oracle, through the C ABI.

Bit-exact: everything the single-grid parity holds, plus the exact pooled
association feature of every mask and every instance's association feature.
The tensor-core association feature stays within its stated bound.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import common

pytestmark = pytest.mark.gpu

PA_H, PA_W, DA = 6, 8, 96
GRID = dict(assoc_dim=DA, assoc_patch_h=PA_H, assoc_patch_w=PA_W)


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2603_03935_gb300 import _build
    _build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return torch, dev


def _aframe(torch, dev, fr, at, i, host=False):
    from paper_2603_03935_gb300 import device_frame, host_frame
    sc = fr.scene
    intr = (sc.fx, sc.fy, sc.cx, sc.cy)
    if host:
        return host_frame(fr.depth[i], fr.labels[i], fr.tokens[i], fr.poses[i], intr, fr.num_masks[i],
                          assoc_tokens=at[i])
    d = torch.from_numpy(fr.depth[i]).to(dev)
    l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[i]).to(dev)
    a = torch.from_numpy(at[i]).to(dev)
    return device_frame(d, l, t, fr.poses[i], intr, fr.num_masks[i], assoc_tokens=a)


def _check_assoc(rep, o, ctx, tol):
    assert np.array_equal(rep["A"].view(np.uint32), o["A"].view(np.uint32)), f"{ctx}: association features differ"
    live = np.asarray(o["npix"]) >= 1
    if live.any():
        assert common.rel_err_rows(rep["A_fast"][live], o["A"][live]) <= tol, f"{ctx}: tensor-core A"


def _run(torch_dev, sc, idx, precision=0, host=False, **kw):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap
    fr = sc.render(idx)
    at = fr.assoc_tokens(PA_H, PA_W, DA)
    cfg = common.disc_cfg(sc, precision=precision, **GRID, **kw)
    gmap = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    tol = (1e-5, 2e-2, 0.15)[precision]
    for i in range(len(idx)):
        st = gmap.integrate(_aframe(torch, dev, fr, at, i, host))
        o = omap.integrate(*oracle.frame_args(fr, i), assoc_tokens=at[i])
        rep = gmap.last_frame()
        common.compare_frame(st, rep, o, ctx=f"assoc frame {idx[i]}", efast_tol=tol)
        _check_assoc(rep, o, f"assoc frame {idx[i]}", tol)
    common.compare_maps(gmap, omap, ctx="assoc")
    ga, oa = gmap.instances(), omap.instances()
    assert np.array_equal(ga["A"].view(np.uint32), oa["A"].view(np.uint32))
    assert np.array_equal(ga["E"].view(np.uint32), oa["E"].view(np.uint32))
    return gmap, omap, fr, at


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_tiny_trajectory_with_second_grid(torch_dev, precision):
    _run(torch_dev, synth.tiny_scene(), range(20), precision=precision)


def test_second_grid_from_host_memory(torch_dev):
    _run(torch_dev, synth.tiny_scene(), range(0, 20, 2), host=True)


def test_room_frames_with_second_grid(torch_dev):
    sc = synth.room_scene(num_frames=2000)
    _run(torch_dev, sc, [0, 1, 2, 3, 250, 251], voxel_capacity=1 << 22, instance_capacity=1024)


def test_second_grid_checkpoint_finalize_and_group(torch_dev, tmp_path):
    # an fp8 map with a second grid: reloaded from a checkpoint, integrated on
    # in a group beside a single-grid map, then finalised; equal to the
    # oracle throughout
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscGroup, DiscMap
    sc = synth.tiny_scene()
    fr = sc.render(range(16))
    at = fr.assoc_tokens(PA_H, PA_W, DA)
    cfg = common.disc_cfg(sc, precision=2, **GRID)
    a = DiscMap(**cfg)
    omap = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    for i in range(8):
        a.integrate(_aframe(torch, dev, fr, at, i))
        omap.integrate(*oracle.frame_args(fr, i), assoc_tokens=at[i])
    a.save(tmp_path / "a.disc")
    b = DiscMap.load(tmp_path / "a.disc")
    plain = DiscMap(**common.disc_cfg(sc))
    oplain = oracle.OracleMap(**common.to_oracle_cfg(common.disc_cfg(sc)))
    grp = DiscGroup(max_maps=2, frames_per_map=4, embed_dim=sc.dim, patch_h=sc.patch_h, patch_w=sc.patch_w,
                    max_width=sc.width, max_height=sc.height, max_masks=sc.max_masks, **GRID)
    from tests.test_gpu_parity import _dframe
    _, done, rc = grp.integrate([b, plain], [[_aframe(torch, dev, fr, at, i) for i in range(8, 16)],
                                             [_dframe(torch, dev, fr, i) for i in range(16)]])
    assert rc == 0 and done == [8, 16]
    for i in range(8, 16):
        omap.integrate(*oracle.frame_args(fr, i), assoc_tokens=at[i])
    for i in range(16):
        oplain.integrate(*oracle.frame_args(fr, i))
    common.compare_maps(b, omap, ctx="second grid, reloaded, in a group")
    common.compare_maps(plain, oplain, ctx="single grid beside it")
    assert np.array_equal(b.instances()["A"].view(np.uint32), omap.instances()["A"].view(np.uint32))
    rg = b.finalize(min_voxels=20, contact_num=1, contact_den=10, tau_cos=0.5)
    ro = omap.finalize(min_voxels=20, contact_num=1, contact_den=10, tau_cos=0.5)
    for k in ("contact_pairs", "merged", "removed", "removed_voxels"):
        assert rg[k] == ro[k], (k, rg, ro)
    common.compare_maps(b, omap, ctx="finalised")


def test_query_heatmap_matches_oracle(torch_dev):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import query_heatmap
    for sc, n in ((synth.tiny_scene(), 3), (synth.room_scene(num_frames=2000), 2)):
        fr = sc.render(range(n))
        for i in range(n):
            F = fr.tokens[i]
            q = sc.object_mean(int(fr.mask_ids[i][0]))  # an object's mean token as the query
            want = oracle.query_heatmap(F, q)
            got = query_heatmap(torch.from_numpy(F).to(dev), torch.from_numpy(q).to(dev)).cpu().numpy()
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), sc.name
            # the object's own patches light up
            assert want.max() > 0.5
