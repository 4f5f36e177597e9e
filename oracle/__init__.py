"""ORACLE for the DISC integration step -- test infrastructure only.

A plain single-threaded C++ restatement of the paper's per-frame step (Sec.
III-A to III-C, Eq. 1-3), loaded through ctypes.  Only ``tests/``, the package
smoke check and the benchmark's CPU-baseline leg may import this module; the
CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdisc_oracle.so")
_SRC = [os.path.join(_HERE, "disc_oracle.cpp"), os.path.join(_HERE, "disc_oracle.h")]


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, no FMA contraction)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17",
                               "-fPIC", "-shared", "-o", _SO, _SRC[0]])
    return _SO


class Config(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("z_min", ctypes.c_float), ("z_max", ctypes.c_float),
                ("eps", ctypes.c_float), ("tau_cos", ctypes.c_float), ("lambda_size", ctypes.c_float),
                ("ov_num", ctypes.c_int32), ("ov_den", ctypes.c_int32),
                ("embed_dim", ctypes.c_int32), ("patch_h", ctypes.c_int32), ("patch_w", ctypes.c_int32),
                ("min_mask_pixels", ctypes.c_int32), ("dbscan_eps", ctypes.c_float),
                ("dbscan_min_pts", ctypes.c_int32), ("overlap_dilation", ctypes.c_int32),
                ("assoc_dim", ctypes.c_int32), ("assoc_patch_h", ctypes.c_int32), ("assoc_patch_w", ctypes.c_int32)]


class Frame(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("T_world_cam", ctypes.c_double * 16),
                ("depth", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("tokens", ctypes.c_void_p),
                ("num_masks", ctypes.c_int32), ("global_embed", ctypes.c_void_p),
                ("assoc_tokens", ctypes.c_void_p)]


class Report(ctypes.Structure):
    _fields_ = [("fbar", ctypes.c_void_p), ("Dp", ctypes.c_void_p), ("cosg", ctypes.c_void_p),
                ("cov", ctypes.c_void_p), ("npix", ctypes.c_void_p), ("W", ctypes.c_void_p),
                ("E", ctypes.c_void_p), ("S", ctypes.c_void_p), ("nvox", ctypes.c_void_p),
                ("rep", ctypes.c_void_p), ("seg_keys", ctypes.c_void_p), ("seg_m", ctypes.c_void_p),
                ("seg_cap", ctypes.c_int64), ("n_seg", ctypes.c_int64),
                ("valid_pixels", ctypes.c_int32), ("dropped_pixels", ctypes.c_int32),
                ("new_voxels", ctypes.c_int32), ("active_instances", ctypes.c_int32),
                ("new_instances", ctypes.c_int32), ("merges", ctypes.c_int32),
                ("live_segments", ctypes.c_int32), ("overlap_pairs", ctypes.c_int32),
                ("denoised_pixels", ctypes.c_int32), ("A", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        L.oracle_map_create.restype = vp
        L.oracle_map_create.argtypes = [ctypes.POINTER(Config)]
        L.oracle_map_destroy.argtypes = [vp]
        L.oracle_integrate_frame.restype = ctypes.c_int
        L.oracle_integrate_frame.argtypes = [vp, ctypes.POINTER(Frame), ctypes.POINTER(Report)]
        L.oracle_num_voxels.restype = i64
        L.oracle_num_voxels.argtypes = [vp]
        L.oracle_export_voxels.argtypes = [vp, vp, vp]
        L.oracle_num_ids.restype = i32
        L.oracle_num_ids.argtypes = [vp]
        L.oracle_export_instances.argtypes = [vp, vp, vp, vp, vp, vp]
        L.oracle_token_stats.restype = ctypes.c_int
        L.oracle_token_stats.argtypes = [vp, i32, i32, vp, f32, vp, vp, vp, vp]
        L.oracle_mask_coverage.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp]
        L.oracle_point_key.restype = ctypes.c_int
        L.oracle_point_key.argtypes = [f32, f32, f32, f32, ctypes.POINTER(ctypes.c_uint64)]
        L.oracle_unpack_key.argtypes = [ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                        ctypes.POINTER(i32)]
        L.oracle_cosine.restype = f32
        L.oracle_cosine.argtypes = [vp, vp, i32]
        L.oracle_pool_f64.argtypes = [vp, i32, i32, vp, vp, i32, ctypes.c_double, vp, vp]
        L.oracle_dbscan_noise.argtypes = [vp, vp, i64, f32, i32, vp]
        L.oracle_finalize.restype = ctypes.c_int
        L.oracle_finalize.argtypes = [vp, ctypes.POINTER(FinalizeConfig), ctypes.POINTER(FinalizeReport)]
        L.oracle_set_state.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, i32]
        L.oracle_set_assoc.argtypes = [vp, vp, i32]
        L.oracle_export_assoc.argtypes = [vp, vp]
        L.oracle_query_heatmap.restype = ctypes.c_int
        L.oracle_query_heatmap.argtypes = [vp, i32, i32, vp, f32, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def default_config(D: int, Ph: int, Pw: int, voxel: float, **kw) -> dict:
    c = dict(voxel_size=voxel, z_min=0.1, z_max=10.0, eps=1e-6, tau_cos=0.75, lambda_size=3.3,
             ov_num=1, ov_den=5, embed_dim=D, patch_h=Ph, patch_w=Pw, min_mask_pixels=1,
             dbscan_eps=0.0, dbscan_min_pts=1, overlap_dilation=0, assoc_dim=0, assoc_patch_h=0,
             assoc_patch_w=0)
    c.update(kw)
    return c


def config_for_scene(scene, **kw) -> dict:
    npx = scene.width * scene.height
    c = default_config(scene.dim, scene.patch_h, scene.patch_w, scene.voxel_size,
                       z_min=scene.z_min, z_max=scene.z_max, min_mask_pixels=max(1, npx // 1000))
    c.update(kw)
    return c


class FinalizeConfig(ctypes.Structure):
    _fields_ = [("min_voxels", ctypes.c_int32), ("contact_num", ctypes.c_int32), ("contact_den", ctypes.c_int32),
                ("tau_cos", ctypes.c_float)]


class FinalizeReport(ctypes.Structure):
    _fields_ = [("contact_pairs", ctypes.c_int32), ("merged", ctypes.c_int32), ("removed", ctypes.c_int32),
                ("removed_voxels", ctypes.c_int64)]


class OracleMap:
    """One map integrated frame by frame on the CPU."""

    def __init__(self, **cfg):
        self.cfg = dict(cfg)
        c = Config(**cfg)
        self._h = lib().oracle_map_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("bad oracle config")
        self.D = cfg["embed_dim"]
        self.P = cfg["patch_h"] * cfg["patch_w"]
        self.Da = int(cfg.get("assoc_dim", 0))
        self.Pa = int(cfg.get("assoc_patch_h", 0)) * int(cfg.get("assoc_patch_w", 0))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_map_destroy(h)
            self._h = None

    def finalize(self, min_voxels, contact_num=1, contact_den=5, tau_cos=None):
        """End-of-trajectory orphan merge and noise filter; returns the report."""
        c = FinalizeConfig(int(min_voxels), int(contact_num), int(contact_den),
                           float(self.cfg["tau_cos"] if tau_cos is None else tau_cos))
        r = FinalizeReport()
        rc = lib().oracle_finalize(self._h, ctypes.byref(c), ctypes.byref(r))
        if rc != 0:
            raise ValueError(f"oracle_finalize: {rc}")
        return {k: int(getattr(r, k)) for k, _ in FinalizeReport._fields_}

    def set_state(self, keys, labels, parent, count, Q, E, n_obs, A=None):
        """Replace the map's voxels and instances (exact test situations)."""
        keys = np.ascontiguousarray(keys, np.uint64)
        labels = np.ascontiguousarray(labels, np.int32)
        parent = np.ascontiguousarray(parent, np.int32)
        count = np.ascontiguousarray(count, np.int64)
        Q = np.ascontiguousarray(Q, np.float32)
        E = np.ascontiguousarray(E, np.float32).reshape(len(parent), self.D)
        n_obs = np.ascontiguousarray(n_obs, np.int32)
        lib().oracle_set_state(self._h, keys.ctypes.data, labels.ctypes.data, len(keys), parent.ctypes.data,
                               count.ctypes.data, Q.ctypes.data, E.ctypes.data, n_obs.ctypes.data, len(parent))
        if A is not None:
            A = np.ascontiguousarray(A, np.float32).reshape(len(parent), self.Da)
            lib().oracle_set_assoc(self._h, A.ctypes.data, len(parent))

    def integrate(self, depth, labels, tokens, pose, intr, num_masks, global_embed=None,
                  report: bool = True, assoc_tokens=None):
        """Integrate one frame; returns a dict of intermediates when report=True.
        assoc_tokens: the second token grid [Pa][Da] when the map has one."""
        H, W = depth.shape
        depth = np.ascontiguousarray(depth, np.float32)
        labels = np.ascontiguousarray(labels, np.uint16)
        tokens = np.ascontiguousarray(tokens, np.float32).reshape(self.P, self.D)
        g = None if global_embed is None else np.ascontiguousarray(global_embed, np.float32)
        f = Frame()
        f.width, f.height = W, H
        f.fx, f.fy, f.cx, f.cy = [float(x) for x in intr]
        for i, v in enumerate(np.asarray(pose, np.float64).reshape(16)):
            f.T_world_cam[i] = float(v)
        f.depth, f.labels, f.tokens = depth.ctypes.data, labels.ctypes.data, tokens.ctypes.data
        f.num_masks = int(num_masks)
        f.global_embed = _p(g)
        at = None
        if self.Da > 0:
            at = np.ascontiguousarray(assoc_tokens, np.float32).reshape(self.Pa, self.Da)
            f.assoc_tokens = at.ctypes.data
        M, P, D = int(num_masks), self.P, self.D
        out = None
        rep = Report()
        if report:
            Mx = max(M, 1)
            cap = int((labels > 0).sum()) + 1
            out = dict(fbar=np.zeros(D, np.float32), Dp=np.zeros(P, np.float32), cosg=np.zeros(P, np.float32),
                       cov=np.zeros((Mx, P), np.int32), npix=np.zeros(Mx, np.int32),
                       W=np.zeros((Mx, P), np.float32), E=np.zeros((Mx, D), np.float32),
                       S=np.zeros((Mx, 5), np.float32), nvox=np.zeros(Mx, np.int32),
                       rep=np.zeros(Mx, np.int32), seg_keys=np.zeros(cap, np.uint64),
                       seg_m=np.zeros(cap, np.int32))
            for k in ("fbar", "Dp", "cosg", "cov", "npix", "W", "E", "S", "nvox", "rep", "seg_keys", "seg_m"):
                setattr(rep, k, out[k].ctypes.data)
            if self.Da > 0:
                out["A"] = np.zeros((Mx, self.Da), np.float32)
                rep.A = out["A"].ctypes.data
            rep.seg_cap = cap
        rc = lib().oracle_integrate_frame(self._h, ctypes.byref(f), ctypes.byref(rep) if report else None)
        if rc != 0:
            raise RuntimeError(f"oracle_integrate_frame failed: {rc}")
        if report:
            n = int(rep.n_seg)
            for k in ("cov", "npix", "W", "E", "S", "nvox", "rep", "A"):
                if k in out:
                    out[k] = out[k][:M]
            out["seg_keys"] = out["seg_keys"][:n]
            out["seg_m"] = out["seg_m"][:n]
            for k in ("valid_pixels", "dropped_pixels", "new_voxels", "active_instances", "new_instances",
                      "merges", "live_segments", "overlap_pairs", "denoised_pixels"):
                out[k] = int(getattr(rep, k))
            out["n_seg"] = n
        return out

    def voxels(self):
        n = int(lib().oracle_num_voxels(self._h))
        keys = np.zeros(n, np.uint64)
        ids = np.zeros(n, np.int32)
        if n:
            lib().oracle_export_voxels(self._h, keys.ctypes.data, ids.ctypes.data)
        return keys, ids

    def instances(self):
        n = int(lib().oracle_num_ids(self._h))
        parent = np.zeros(n, np.int32)
        count = np.zeros(n, np.int64)
        Q = np.zeros(n, np.float32)
        E = np.zeros((n, self.D), np.float32)
        obs = np.zeros(n, np.int32)
        if n:
            lib().oracle_export_instances(self._h, parent.ctypes.data, count.ctypes.data, Q.ctypes.data,
                                          E.ctypes.data, obs.ctypes.data)
        out = dict(parent=parent, count=count, Q=Q, E=E, n_obs=obs)
        if self.Da > 0:
            A = np.zeros((n, self.Da), np.float32)
            if n:
                lib().oracle_export_assoc(self._h, A.ctypes.data)
            out["A"] = A
        return out


def query_heatmap(F: np.ndarray, q: np.ndarray, eps: float = 1e-6) -> np.ndarray:
    """Fig. 2 heatmap: D_p * cos(f_p, q) over a token grid [P][D]."""
    F = np.ascontiguousarray(F, np.float32)
    P, D = F.shape
    q = np.ascontiguousarray(q, np.float32).reshape(D)
    heat = np.zeros(P, np.float32)
    rc = lib().oracle_query_heatmap(F.ctypes.data, P, D, q.ctypes.data, eps, heat.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_query_heatmap: {rc}")
    return heat


def token_stats(F: np.ndarray, g=None, eps: float = 1e-6):
    F = np.ascontiguousarray(F, np.float32)
    P, D = F.shape
    fbar, n, Dp, cosg = (np.zeros(D, np.float32), np.zeros(P, np.float32), np.zeros(P, np.float32),
                         np.zeros(P, np.float32))
    gg = None if g is None else np.ascontiguousarray(g, np.float32)
    rc = lib().oracle_token_stats(F.ctypes.data, P, D, _p(gg), eps, fbar.ctypes.data, n.ctypes.data,
                                  Dp.ctypes.data, cosg.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_token_stats: {rc}")
    return dict(fbar=fbar, n=n, Dp=Dp, cosg=cosg)


def mask_coverage(labels: np.ndarray, Ph: int, Pw: int, M: int):
    labels = np.ascontiguousarray(labels, np.uint16)
    H, W = labels.shape
    cov = np.zeros((max(M, 1), Ph * Pw), np.int32)
    npix = np.zeros(max(M, 1), np.int32)
    lib().oracle_mask_coverage(labels.ctypes.data, H, W, Ph, Pw, M, cov.ctypes.data, npix.ctypes.data)
    return cov[:M], npix[:M]


def point_key(x, y, z, voxel):
    k = ctypes.c_uint64(0)
    ok = lib().oracle_point_key(float(x), float(y), float(z), float(voxel), ctypes.byref(k))
    return int(k.value) if ok else None


def unpack_key(key):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    lib().oracle_unpack_key(ctypes.c_uint64(int(key)), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def cosine(a, b):
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return float(lib().oracle_cosine(a.ctypes.data, b.ctypes.data, a.shape[0]))


def pool_f64(F, cov, npix, eps=1e-6):
    F = np.ascontiguousarray(F, np.float32)
    cov = np.ascontiguousarray(cov, np.int32)
    npix = np.ascontiguousarray(npix, np.int32)
    P, D = F.shape
    M = cov.shape[0]
    Dp = np.zeros(P, np.float64)
    E = np.zeros((max(M, 1), D), np.float64)
    lib().oracle_pool_f64(F.ctypes.data, P, D, cov.ctypes.data, npix.ctypes.data, M, eps,
                          Dp.ctypes.data, E.ctypes.data)
    return Dp, E[:M]


def frame_args(frames, i):
    """(depth, labels, tokens, pose, intrinsics, num_masks) of frame i of a synth.Frames."""
    sc = frames.scene
    return (frames.depth[i], frames.labels[i], frames.tokens[i], frames.poses[i],
            (sc.fx, sc.fy, sc.cx, sc.cy), int(frames.num_masks[i]))


def dbscan_noise(points, seg, eps, min_pts):
    """Noise flags of the per-segment DBSCAN filter (Sec. III-A)."""
    pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    sg = np.ascontiguousarray(seg, np.int32)
    out = np.zeros(len(pts), np.uint8)
    if len(pts):
        lib().oracle_dbscan_noise(pts.ctypes.data, sg.ctypes.data, len(pts), float(eps), int(min_pts),
                                  out.ctypes.data)
    return out.astype(bool)
