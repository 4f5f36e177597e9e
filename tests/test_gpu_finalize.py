"""End-of-trajectory finalisation on the GPU (disc_map_finalize) vs the oracle.

Exact map states built by hand (the oracle pins' situations, loaded through a
checkpoint file) and maps grown from real trajectories are finalised on both
sides; reports, voxel ids and instance tables must agree bit for bit.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests import common
from tests import test_oracle_finalize as pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2603_03935_gb300 import _build
    _build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return torch, dev


def _write_checkpoint(path, cfg, keys, labels, parent, count, Q, E, n_obs):
    """A map file in the layout disc_map_load reads."""
    from paper_2603_03935_gb300 import binding
    c = binding.Config(**binding.config_default(**cfg))
    with open(path, "wb") as f:
        f.write(b"DISCMAP1")
        f.write(bytes(c))
        f.write(np.int64(len(keys)).tobytes())
        f.write(np.int32(len(parent)).tobytes())
        f.write(np.asarray(keys, np.uint64).tobytes())
        f.write(np.asarray(labels, np.int32).tobytes())
        f.write(np.asarray(parent, np.int32).tobytes())
        f.write(np.asarray(count, np.int64).tobytes())
        f.write(np.asarray(Q, np.float32).tobytes())
        f.write(np.asarray(E, np.float32).tobytes())
        f.write(np.asarray(n_obs, np.int32).tobytes())


def _gpu_cfg():
    o = pins._cfg()
    return dict(voxel_size=o["voxel_size"], z_min=o["z_min"], z_max=o["z_max"], eps=o["eps"], tau_cos=o["tau_cos"],
                lambda_size=o["lambda_size"], ov_num=o["ov_num"], ov_den=o["ov_den"], embed_dim=o["embed_dim"],
                patch_h=o["patch_h"], patch_w=o["patch_w"], max_width=8, max_height=8, max_masks=4,
                min_mask_pixels=1, voxel_capacity=1 << 12, instance_capacity=16)


def _pair(tmp_path, instances, **kw):
    """The same hand-built state in the oracle and in a GPU map."""
    from paper_2603_03935_gb300 import DiscMap
    om = pins._build(instances, **kw)
    keys, ids = om.voxels()   # resolved ids = labels here (flat parents)
    inst = om.instances()
    # labels as stored: the builder labels each voxel with its own instance id
    labels = []
    for i, (vox, _) in enumerate(instances):
        labels += [i] * len(vox)
    raw_keys = [pins._key(*v) for vox, _ in instances for v in vox]
    path = tmp_path / "state.disc"
    _write_checkpoint(path, _gpu_cfg(), raw_keys, labels, inst["parent"], inst["count"], inst["Q"], inst["E"],
                      inst["n_obs"])
    return om, DiscMap.load(path)


def _same(gm, om, ctx):
    common.compare_maps(gm, om, ctx=ctx)


CASES = [
    ("fragment", lambda: dict(instances=[(pins._plate(0, 6, 0, 6), pins._vec(1)),
                                         (pins._plate(6, 8, 0, 1), pins._vec(2, pins._vec(1), 0.05))]),
     dict(min_voxels=1)),
    ("dissimilar", lambda: dict(instances=[(pins._plate(0, 6, 0, 6), pins._vec(1)),
                                           (pins._plate(6, 8, 0, 1), -pins._vec(1))]), dict(min_voxels=1)),
    ("rational 6/5", lambda: dict(instances=[(pins._plate(0, 6, 0, 6), pins._vec(1)),
                                             ([(6, y, 0) for y in range(10)], pins._vec(1))]),
     dict(min_voxels=1, contact_num=6, contact_den=5)),
    ("rational 7/5", lambda: dict(instances=[(pins._plate(0, 6, 0, 6), pins._vec(1)),
                                             ([(6, y, 0) for y in range(10)], pins._vec(1))]),
     dict(min_voxels=1, contact_num=7, contact_den=5)),
    ("chain", lambda: dict(instances=[(pins._plate(0, 4, 0, 4), pins._vec(3)),
                                      (pins._plate(4, 5, 0, 4), pins._vec(4, pins._vec(3), 0.05)),
                                      (pins._plate(5, 9, 0, 4), pins._vec(5, pins._vec(3), 0.05))],
                           Q=[0.3, 0.3, 0.3]), dict(min_voxels=1)),
    ("filter", lambda: dict(instances=[(pins._plate(0, 6, 0, 6), pins._vec(6)),
                                       ([(20, 0, 0), (21, 0, 0)], pins._vec(7)),
                                       (pins._plate(6, 7, 0, 2), pins._vec(8, pins._vec(6), 0.05))]),
     dict(min_voxels=3)),
    ("two levels", lambda: dict(instances=[(pins._plate(0, 4, 0, 4), pins._vec(9)),
                                           (pins._plate(4, 5, 0, 4), pins._vec(9)),
                                           (pins._plate(5, 6, 0, 4), pins._vec(9))], parent=[0, 1, 1]),
     dict(min_voxels=1)),
]


@pytest.mark.parametrize("name,make,fin", CASES, ids=[c[0] for c in CASES])
def test_finalize_hand_built_states(torch_dev, tmp_path, name, make, fin):
    om, gm = _pair(tmp_path, **make())
    ro = om.finalize(**fin)
    rg = gm.finalize(**fin)
    assert {k: rg[k] for k in ro} == ro, name
    _same(gm, om, name)


@pytest.mark.parametrize("scene,n,fin", [
    ("tiny", 20, dict(min_voxels=40, contact_num=1, contact_den=10, tau_cos=0.5)),
    ("room", 24, dict(min_voxels=30, contact_num=1, contact_den=5, tau_cos=0.75)),
])
def test_finalize_after_trajectory(torch_dev, scene, n, fin):
    torch, dev = torch_dev
    from paper_2603_03935_gb300 import DiscMap, device_frame
    sc = synth.tiny_scene() if scene == "tiny" else synth.room_scene()
    fr = sc.render(range(n))
    kw = {} if scene == "tiny" else dict(voxel_capacity=1 << 22, instance_capacity=1 << 12)
    cfg = common.disc_cfg(sc, **kw)
    gm = DiscMap(**cfg)
    om = oracle.OracleMap(**common.to_oracle_cfg(cfg))
    frames = []
    for i in range(n):
        d = torch.from_numpy(fr.depth[i]).to(dev)
        l = torch.from_numpy(fr.labels[i].view(np.int16)).to(dev)
        t = torch.from_numpy(fr.tokens[i]).to(dev)
        frames.append(device_frame(d, l, t, fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy), fr.num_masks[i]))
        om.integrate(*oracle.frame_args(fr, i), report=False)
    _, done, rc = gm.integrate_frames(frames)
    assert rc == 0 and done == n
    ro = om.finalize(**fin)
    rg = gm.finalize(**fin)
    assert {k: rg[k] for k in ro} == ro
    assert ro["contact_pairs"] > 0
    _same(gm, om, f"{scene} finalised")
    # final: integration refused, queries skip dropped instances and voxels
    st = gm.integrate(frames[0], check=False)
    assert st["rc"] == -1
    keys, ids = gm.voxels()
    if (ids == -1).any():
        k = int(keys[np.argmax(ids == -1)])
        kx, ky, kz = (int(v) for v in oracle.unpack_key(k))
        s = cfg["voxel_size"]
        assert gm.query_points(np.array([[(kx + 0.5) * s, (ky + 0.5) * s, (kz + 0.5) * s]]))[0] == -1
    inst = gm.instances()
    ids_q, _ = gm.query_topk(inst["E"][:4], 8)
    dropped = set(np.nonzero((inst["parent"] == np.arange(len(inst["parent"]))) & (inst["n_obs"] == 0))[0].tolist())
    assert not (set(ids_q.ravel().tolist()) & dropped)


def test_final_map_checkpoint_reloads_final(torch_dev, tmp_path):
    from paper_2603_03935_gb300 import DiscMap
    om, gm = _pair(tmp_path, **CASES[5][1]())
    gm.finalize(min_voxels=3)
    gm.save(tmp_path / "final.disc")
    g2 = DiscMap.load(tmp_path / "final.disc")
    om.finalize(min_voxels=3)
    _same(g2, om, "reloaded final map")
    assert g2.finalize(min_voxels=3, check=False)["rc"] == -1
