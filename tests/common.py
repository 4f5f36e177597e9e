"""Shared helpers of the GPU parity tests: one scene, two implementations.

The seeded frames come from ``synth``; the oracle and the CUDA library each
integrate them with the same configuration and their per-frame intermediates
and final maps are compared.
"""
import numpy as np

import oracle


def oracle_cfg(scene, **kw):
    return oracle.config_for_scene(scene, **kw)


def disc_cfg(scene, **kw):
    o = oracle_cfg(scene)
    c = dict(voxel_size=o["voxel_size"], z_min=o["z_min"], z_max=o["z_max"], eps=o["eps"],
             tau_cos=o["tau_cos"], lambda_size=o["lambda_size"], ov_num=o["ov_num"], ov_den=o["ov_den"],
             embed_dim=scene.dim, patch_h=scene.patch_h, patch_w=scene.patch_w,
             max_width=scene.width, max_height=scene.height, max_masks=scene.max_masks,
             min_mask_pixels=o["min_mask_pixels"], voxel_capacity=1 << 16, max_load=0.5,
             instance_capacity=64)
    c.update(kw)
    return c


def to_oracle_cfg(dcfg):
    keys = ("voxel_size", "z_min", "z_max", "eps", "tau_cos", "lambda_size", "ov_num", "ov_den",
            "embed_dim", "patch_h", "patch_w", "min_mask_pixels")
    out = {k: dcfg[k] for k in keys}
    out["dbscan_eps"] = dcfg.get("dbscan_eps", 0.0)
    out["dbscan_min_pts"] = dcfg.get("dbscan_min_pts", 1)
    out["overlap_dilation"] = dcfg.get("overlap_dilation", 0)
    for k in ("assoc_dim", "assoc_patch_h", "assoc_patch_w"):
        out[k] = dcfg.get(k, 0)
    return out


EXACT_FIELDS = ("fbar", "Dp", "cosg", "cov", "npix", "W", "E", "S", "nvox", "rep")
COUNT_FIELDS = (("valid_pixels", "valid_pixels"), ("dropped_pixels", "dropped_pixels"),
                ("new_voxels", "new_voxels"), ("active_instances", "active_instances"),
                ("new_instances", "new_instances"), ("merges", "merges"),
                ("live_segments", "live_segments"), ("overlap_pairs", "overlap_pairs"),
                ("unique_seg_voxels", "n_seg"), ("denoised_pixels", "denoised_pixels"))


def rel_err_rows(a, b):
    """max over rows of ||a - b|| / ||b|| (rows with ||b|| == 0 use ||a||)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    num = np.linalg.norm(a - b, axis=-1)
    den = np.linalg.norm(b, axis=-1)
    r = np.where(den > 0, num / np.where(den > 0, den, 1), num)
    return float(r.max()) if r.size else 0.0


def compare_frame(g_stats, g_rep, o_rep, ctx="", efast_tol=1e-5):
    for k in EXACT_FIELDS:
        a, b = np.asarray(g_rep[k]), np.asarray(o_rep[k])
        assert a.shape == b.shape, f"{ctx} {k}: shape {a.shape} vs {b.shape}"
        if not np.array_equal(a.view(np.uint8) if a.dtype.kind == "f" else a,
                              b.view(np.uint8) if b.dtype.kind == "f" else b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{ctx} {k} differs at {bad[:5].tolist()}: {a[tuple(bad[0])] if len(bad) else ''} "
                                 f"vs {b[tuple(bad[0])] if len(bad) else ''}")
    assert np.array_equal(g_rep["seg_m"], o_rep["seg_m"]), f"{ctx} segment labels of voxel pairs differ"
    assert np.array_equal(g_rep["seg_keys"], o_rep["seg_keys"]), f"{ctx} voxel keys differ"
    for gk, ok in COUNT_FIELDS:
        assert g_stats[gk] == o_rep[ok], f"{ctx} {gk}: {g_stats[gk]} vs {o_rep[ok]}"
    live = np.asarray(o_rep["npix"]) >= 1
    if live.any():
        assert rel_err_rows(g_rep["E_fast"][live], o_rep["E"][live]) <= efast_tol, f"{ctx} tensor-core pooling error"


def compare_maps(gmap, omap, ctx=""):
    gk, gi = gmap.voxels()
    ok_, oi = omap.voxels()
    assert np.array_equal(gk, ok_), f"{ctx} voxel key sets differ ({len(gk)} vs {len(ok_)})"
    assert np.array_equal(gi, oi), f"{ctx} voxel instance ids differ"
    ga, oa = gmap.instances(), omap.instances()
    for k in ("parent", "count", "n_obs"):
        assert np.array_equal(ga[k], oa[k]), f"{ctx} instance {k} differs"
    assert np.array_equal(ga["Q"].view(np.uint32), oa["Q"].view(np.uint32)), f"{ctx} instance Q differs"
    assert np.array_equal(ga["E"].view(np.uint32), oa["E"].view(np.uint32)), f"{ctx} instance embeddings differ"
