"""The C ABI library builds, loads and exports every entry point of
include/disc.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdisc():
    from paper_2603_03935_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "disc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**(disc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("disc_map_create", "disc_integrate_frame", "disc_integrate_frames", "disc_query_topk",
                     "disc_query_points", "disc_map_destroy", "disc_map_export_voxels", "disc_map_save",
                     "disc_map_load", "disc_integrate_frames_async", "disc_map_wait", "disc_group_integrate_async",
                     "disc_group_wait"):
        assert required in names


def test_library_exports_every_declared_symbol(libdisc):
    missing = [n for n in declared_functions() if not hasattr(libdisc, n)]
    assert not missing, missing


def test_host_only_entry_points(libdisc):
    import paper_2603_03935_gb300 as pkg
    cfg = pkg.config_default()
    assert cfg["lambda_size"] == pytest.approx(3.3)
    assert cfg["tau_cos"] == pytest.approx(0.75)
    assert (cfg["ov_num"], cfg["ov_den"]) == (1, 5)
    assert pkg.status_str(0) == "ok"
    assert pkg.status_str(-7) == "token out of range"
    # key packing agrees with the oracle's independent packing
    import oracle
    for k in [(0, 0, 0), (-1, 2, -3), (131071, -131072, 5)]:
        key = pkg.pack_key(*k)
        assert oracle.unpack_key(key) == k
    assert pkg.pack_key(1, 2, 3) == oracle.point_key(1.01, 2.01, 3.01, 1.0)


def test_asynchronous_entry_points_refuse_bad_arguments_without_a_device(libdisc):
    # argument checks come before any device call, so they run here
    from paper_2603_03935_gb300 import binding as b
    L = b.lib()
    res, done = ctypes.c_int32(7), ctypes.c_int32(7)
    assert L.disc_integrate_frames_async(None, None, 0, None, ctypes.byref(done), ctypes.byref(res)) == -1
    assert L.disc_map_wait(None) == -1
    assert L.disc_group_integrate_async(None, None, 0, None, None, None, None, ctypes.byref(res)) == -1
    assert L.disc_group_wait(None) == -1
    assert (res.value, done.value) == (7, 7)  # nothing was enqueued, nothing written


def test_product_path_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    import paper_2603_03935_gb300.binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        b.lib()


def test_create_without_device_fails_cleanly(libdisc):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_2603_03935_gb300 as pkg
    with pytest.raises(pkg.DiscError):
        pkg.DiscMap()


def test_corrupt_checkpoints_are_refused_before_any_allocation(libdisc, tmp_path):
    # disc_map_load checks the header's config and that its sizes account for
    # the whole file before it allocates or touches a device
    import struct
    import paper_2603_03935_gb300 as pkg
    from paper_2603_03935_gb300 import binding as b
    L = b.lib()
    c = b.Config(**b.config_default(embed_dim=8, patch_h=2, patch_w=2, max_width=8, max_height=8,
                                    max_masks=4, voxel_capacity=1 << 10, instance_capacity=16))
    head = b"DISCMAP1" + bytes(c)

    def load(blob):
        p = tmp_path / "ck.bin"
        p.write_bytes(blob)
        h = ctypes.c_void_p()
        return L.disc_map_load(str(p).encode(), None, ctypes.byref(h)), h.value

    nv, nid = 3, 2
    body = _checkpoint_body([5, 9, 2], [0, 1, 1], [0, 1], [1, 2], [0.5, 0.25], np.zeros((2, 8), np.float32), [1, 1])
    good = head + struct.pack("<qi", nv, nid) + body
    assert load(b"NOTAMAP1" + good[8:]) == (-1, None)              # magic
    assert load(good[:-1]) == (-1, None)                           # one byte short
    assert load(good + b"\0") == (-1, None)                        # one byte long
    assert load(head + struct.pack("<qi", 1 << 41, nid) + body) == (-1, None)   # absurd voxel count
    assert load(head + struct.pack("<qi", nv, -1) + body) == (-1, None)
    bad = b.Config.from_buffer_copy(bytes(c))
    bad.max_load = 0.0                                             # would never stop doubling the table
    assert load(b"DISCMAP1" + bytes(bad) + struct.pack("<qi", nv, nid) + body) == (-1, None)
    assert load(b"DISCMAP1" + bytes(c)[:10]) == (-1, None)         # truncated header
    import torch
    if not torch.cuda.is_available():
        # the well-formed file passes every check and fails only at the device
        rc, h = load(good)
        assert rc != -1 and h is None


def _checkpoint_body(keys, ids, parent, count, Q, E, obs):
    """The arrays of a checkpoint file after its header, in file order."""
    return b"".join([np.asarray(keys, np.uint64).tobytes(), np.asarray(ids, np.int32).tobytes(),
                     np.asarray(parent, np.int32).tobytes(), np.asarray(count, np.int64).tobytes(),
                     np.asarray(Q, np.float32).tobytes(), np.asarray(E, np.float32).tobytes(),
                     np.asarray(obs, np.int32).tobytes()])


def test_checkpoints_with_bad_contents_are_refused_before_any_allocation(libdisc, tmp_path):
    # labels and parents index the instance arrays on the device and keys
    # fill the voxel table: each bad value is refused on the host
    import struct
    from paper_2603_03935_gb300 import binding as b
    L = b.lib()
    c = b.Config(**b.config_default(embed_dim=8, patch_h=2, patch_w=2, max_width=8, max_height=8,
                                    max_masks=4, voxel_capacity=1 << 10, instance_capacity=16))
    E = np.zeros((2, 8), np.float32)
    good = dict(keys=[5, 9, 2], ids=[0, 1, 1], parent=[0, 1], count=[1, 2], Q=[0.5, 0.25], E=E, obs=[1, 1])

    def load(magic=b"DISCMAP1", **change):
        a = dict(good, **change)
        blob = magic + bytes(c) + struct.pack("<qi", len(a["keys"]), len(a["parent"])) + _checkpoint_body(**a)
        p = tmp_path / "ck.bin"
        p.write_bytes(blob)
        h = ctypes.c_void_p()
        return L.disc_map_load(str(p).encode(), None, ctypes.byref(h)), h.value

    bad = [dict(ids=[0, 2, 1]),                       # label = nid
           dict(ids=[0, -1, 1]),                      # unlabelled voxel in a map that is not final
           dict(ids=[0, -2, 1]),
           dict(parent=[0, 7]),                       # parent out of range
           dict(parent=[-1, 1]),
           dict(parent=[1, 0]),                       # not flat: the parent of 0's parent is not 0's parent
           dict(count=[1, -3]),
           dict(obs=[-1, 1]),
           dict(Q=[np.nan, 0.25]),
           dict(keys=[5, 0xFFFFFFFFFFFFFFFF, 2]),     # the table's empty marker
           dict(keys=[5, 1 << 54, 2]),                # not a packed key
           dict(keys=[5, 9, 5]),                      # repeated key
           dict(E=np.full((2, 8), np.inf, np.float32)),
           dict(E=np.full((2, 8), 2048.0, np.float32))]
    for change in bad:
        assert load(**change) == (-1, None), change
    bad_final = dict(ids=[0, -2, 1])
    assert load(b"DISCMAPF", **bad_final) == (-1, None)
    import torch
    if not torch.cuda.is_available():
        # well-formed contents (a finalised map may hold unlabelled voxels)
        # pass every check and fail only at the device
        for magic, change in ((b"DISCMAP1", {}), (b"DISCMAPF", dict(ids=[0, -1, 1]))):
            rc, h = load(magic, **change)
            assert rc != -1 and h is None, (magic, change)


def test_server_worker_count_is_checked_before_any_device_use(libdisc):
    from paper_2603_03935_gb300 import binding as b
    L = b.lib()
    for workers in (-1, 5):
        c = b.ServerConfig()
        L.disc_group_config_default(ctypes.byref(c.group))
        c.hbm_budget_bytes = 1 << 30
        c.max_queue = 16
        c.workers = workers
        h = ctypes.c_void_p()
        assert L.disc_server_create(ctypes.byref(c), ctypes.byref(h)) == -1 and h.value is None
