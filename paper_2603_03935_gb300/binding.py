"""ctypes binding of libdisc (include/disc.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdisc.so")

c_i32, c_i64, c_f32, c_f64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_void_p

STATUS = {0: "DISC_OK", -1: "DISC_ERR_INVALID_ARG", -2: "DISC_ERR_OOM", -3: "DISC_ERR_TABLE_FULL",
          -4: "DISC_ERR_CUDA", -5: "DISC_ERR_TIMEOUT", -6: "DISC_ERR_BUDGET", -7: "DISC_ERR_RANGE",
          -8: "DISC_ERR_CAPACITY"}


class DiscError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = int(code)
        super().__init__(f"{what}: {STATUS.get(self.code, self.code)}")


class Config(ctypes.Structure):
    _fields_ = [("voxel_size", c_f32), ("z_min", c_f32), ("z_max", c_f32), ("eps", c_f32),
                ("tau_cos", c_f32), ("lambda_size", c_f32), ("ov_num", c_i32), ("ov_den", c_i32),
                ("embed_dim", c_i32), ("patch_h", c_i32), ("patch_w", c_i32),
                ("max_width", c_i32), ("max_height", c_i32), ("max_masks", c_i32),
                ("min_mask_pixels", c_i32), ("voxel_capacity", c_i64), ("max_load", c_f32),
                ("instance_capacity", c_i32), ("precision", c_i32), ("cuda_stream", c_vp),
                ("device", c_i32), ("batch_frames", c_i32), ("dbscan_eps", c_f32), ("dbscan_min_pts", c_i32),
                ("serial_sms", c_i32), ("overlap_dilation", c_i32), ("assoc_dim", c_i32),
                ("assoc_patch_h", c_i32), ("assoc_patch_w", c_i32)]


class Frame(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32),
                ("cy", c_f32), ("T_world_cam", c_f64 * 16), ("depth", c_vp), ("labels", c_vp),
                ("tokens", c_vp), ("token_dtype", c_i32), ("num_masks", c_i32),
                ("global_embed", c_vp), ("inputs_on_device", c_i32), ("assoc_tokens", c_vp)]


class Stats(ctypes.Structure):
    _fields_ = [(k, c_i32) for k in ("valid_pixels", "dropped_pixels", "unique_seg_voxels", "new_voxels",
                                     "active_instances", "overlap_pairs", "new_instances", "merges",
                                     "live_segments", "borderline_rescored", "max_probe", "status",
                                     "denoised_pixels", "scored_pairs", "embedding_copies")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class GroupConfig(ctypes.Structure):
    _fields_ = [("max_maps", c_i32), ("frames_per_map", c_i32), ("embed_dim", c_i32), ("patch_h", c_i32),
                ("patch_w", c_i32), ("max_width", c_i32), ("max_height", c_i32), ("max_masks", c_i32),
                ("cuda_stream", c_vp), ("device", c_i32), ("serial_sms", c_i32), ("assoc_dim", c_i32),
                ("assoc_patch_h", c_i32), ("assoc_patch_w", c_i32)]


class Schedule(ctypes.Structure):
    _fields_ = [("geometry_chunk", c_i32), ("serial_ctas", c_i32), ("probe_width", c_i32), ("assoc_cluster", c_i32),
                ("batch_split", c_i32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("best", Schedule), ("best_ms", c_f64), ("default_ms", c_f64), ("candidates", c_i32)]

    def as_dict(self):
        return {"geometry_chunk": int(self.best.geometry_chunk), "serial_ctas": int(self.best.serial_ctas),
                "probe_width": int(self.best.probe_width), "assoc_cluster": int(self.best.assoc_cluster),
                "batch_split": int(self.best.batch_split),
                "best_ms": float(self.best_ms), "default_ms": float(self.default_ms),
                "candidates": int(self.candidates)}


class ServerConfig(ctypes.Structure):
    _fields_ = [("group", GroupConfig), ("hbm_budget_bytes", c_i64), ("max_queue", c_i32), ("workers", c_i32)]


class ServerReport(ctypes.Structure):
    _fields_ = [("frames", c_i64), ("queries", c_i64), ("batches", c_i64), ("pending", c_i64),
                ("resident_bytes", c_i64), ("busy_ms", c_f64), ("wall_ms", c_f64), ("p50_ms", c_f64),
                ("p99_ms", c_f64)]


class FinalizeConfig(ctypes.Structure):
    _fields_ = [("min_voxels", c_i32), ("contact_num", c_i32), ("contact_den", c_i32), ("tau_cos", c_f32)]


class FinalizeReport(ctypes.Structure):
    _fields_ = [("contact_pairs", c_i32), ("merged", c_i32), ("removed", c_i32), ("removed_voxels", c_i64)]


class Report(ctypes.Structure):
    _fields_ = [("fbar", c_vp), ("Dp", c_vp), ("cosg", c_vp), ("cov", c_vp), ("npix", c_vp), ("W", c_vp),
                ("E", c_vp), ("E_fast", c_vp), ("S", c_vp), ("nvox", c_vp), ("rep", c_vp),
                ("seg_keys", c_vp), ("seg_m", c_vp), ("seg_cap", c_i64), ("n_seg", c_i64),
                ("num_masks", c_i32), ("E_bound", c_vp), ("A", c_vp), ("A_fast", c_vp)]


_lib = None


def lib():
    """Load libdisc.so; raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdisc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.disc_config_default.argtypes = [P(Config)]
        L.disc_config_default.restype = None
        L.disc_map_create.argtypes = [P(Config), P(Config), P(c_vp)]
        L.disc_integrate_frame.argtypes = [c_vp, P(Frame), P(Stats)]
        L.disc_integrate_frames.argtypes = [c_vp, P(Frame), c_i32, P(Stats), P(c_i32)]
        L.disc_integrate_frames_async.argtypes = [c_vp, P(Frame), c_i32, P(Stats), P(c_i32), P(c_i32)]
        L.disc_map_wait.argtypes = [c_vp]
        L.disc_map_last_frame.argtypes = [c_vp, P(Report)]
        L.disc_query_topk.argtypes = [c_vp, c_vp, c_i32, c_i32, c_vp, c_vp]
        L.disc_query_points.argtypes = [c_vp, c_vp, c_i64, c_vp]
        L.disc_map_counts.argtypes = [c_vp, P(c_i64), P(c_i32)]
        L.disc_map_export_voxels.argtypes = [c_vp, c_vp, c_vp, c_i64]
        L.disc_map_export_instances.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i32]
        L.disc_map_save.argtypes = [c_vp, ctypes.c_char_p]
        L.disc_map_load.argtypes = [ctypes.c_char_p, P(Config), P(c_vp)]
        L.disc_pack_key.argtypes = [c_i32, c_i32, c_i32]
        L.disc_pack_key.restype = ctypes.c_uint64
        L.disc_map_get_config.argtypes = [c_vp, P(Config)]
        L.disc_map_get_config.restype = ctypes.c_int
        L.disc_map_kernel_launches.argtypes = [c_vp]
        L.disc_map_kernel_launches.restype = c_i64
        L.disc_map_set_phase_timing.argtypes = [c_vp, c_i32]
        L.disc_map_set_phase_timing.restype = ctypes.c_int
        L.disc_map_phase_times.argtypes = [c_vp, c_vp, c_vp, c_vp, c_i32]
        L.disc_map_phase_times.restype = ctypes.c_int
        L.disc_phase_name.argtypes = [c_i32]
        L.disc_phase_name.restype = ctypes.c_char_p
        L.disc_token_stats_static.argtypes = [c_vp, c_i32, c_i32, c_i32, c_vp, c_f32, c_vp, c_vp, c_vp]
        L.disc_token_stats_static.restype = ctypes.c_int
        L.disc_query_heatmap.argtypes = [c_vp, c_i32, c_i32, c_i32, c_vp, c_f32, c_vp, c_vp]
        L.disc_query_heatmap.restype = ctypes.c_int
        L.disc_map_export_assoc.argtypes = [c_vp, c_vp, c_i32]
        L.disc_debug_fail_alloc_after.argtypes = [c_i64]
        L.disc_debug_fail_alloc_after.restype = None
        L.disc_debug_gemm_stall.argtypes = [c_i32, c_i32]
        L.disc_debug_gemm_stall.restype = ctypes.c_int
        L.disc_map_set_schedule.argtypes = [c_vp, P(Schedule)]
        L.disc_group_set_schedule.argtypes = [c_vp, P(Schedule)]
        L.disc_map_autotune.argtypes = [c_vp, c_vp, c_i32, c_i32, P(TuneReport)]
        L.disc_group_autotune.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp, c_i32, P(TuneReport)]
        for f in ("disc_map_set_schedule", "disc_group_set_schedule", "disc_map_autotune", "disc_group_autotune"):
            getattr(L, f).restype = ctypes.c_int
        L.disc_map_export_assoc.restype = ctypes.c_int
        L.disc_map_device_bytes.argtypes = [c_vp]
        L.disc_map_device_bytes.restype = c_i64
        L.disc_map_destroy.argtypes = [c_vp]
        L.disc_map_destroy.restype = None
        L.disc_status_str.argtypes = [c_i32]
        L.disc_status_str.restype = ctypes.c_char_p
        L.disc_group_config_default.argtypes = [P(GroupConfig)]
        L.disc_group_config_default.restype = None
        L.disc_group_create.argtypes = [P(GroupConfig), P(c_vp)]
        L.disc_group_integrate.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]
        L.disc_group_integrate_async.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, P(c_i32)]
        L.disc_group_wait.argtypes = [c_vp]
        L.disc_group_set_phase_timing.argtypes = [c_vp, c_i32]
        L.disc_group_phase_times.argtypes = [c_vp, c_vp, c_vp, c_vp, c_i32]
        L.disc_group_kernel_launches.argtypes = [c_vp]
        L.disc_group_kernel_launches.restype = c_i64
        L.disc_group_device_bytes.argtypes = [c_vp]
        L.disc_group_device_bytes.restype = c_i64
        L.disc_group_destroy.argtypes = [c_vp]
        L.disc_group_destroy.restype = None
        L.disc_map_finalize.argtypes = [c_vp, P(FinalizeConfig), P(FinalizeReport)]
        L.disc_server_create.argtypes = [P(ServerConfig), P(c_vp)]
        L.disc_server_open_map.argtypes = [c_vp, P(Config), P(c_i32)]
        L.disc_server_close_map.argtypes = [c_vp, c_i32]
        L.disc_server_map.argtypes = [c_vp, c_i32]
        L.disc_server_map.restype = c_vp
        L.disc_server_submit_frame.argtypes = [c_vp, c_i32, P(Frame), P(c_i64)]
        L.disc_server_submit_frame_borrowed.argtypes = [c_vp, c_i32, P(Frame), P(c_i64)]
        L.disc_server_submit_query.argtypes = [c_vp, c_i32, c_vp, c_i32, c_i32, P(c_i64)]
        L.disc_server_wait.argtypes = [c_vp, c_i64, P(Stats), c_vp, c_vp, P(c_f64)]
        L.disc_server_stats.argtypes = [c_vp, P(ServerReport)]
        L.disc_server_reset_stats.argtypes = [c_vp]
        L.disc_server_destroy.argtypes = [c_vp]
        L.disc_server_destroy.restype = None
        for f in ("disc_map_create", "disc_integrate_frame", "disc_integrate_frames", "disc_map_last_frame",
                  "disc_query_topk", "disc_query_points", "disc_map_counts", "disc_map_export_voxels",
                  "disc_map_export_instances", "disc_map_save", "disc_map_load", "disc_group_create",
                  "disc_group_integrate", "disc_group_set_phase_timing", "disc_group_phase_times",
                  "disc_server_create", "disc_server_open_map", "disc_server_close_map", "disc_server_submit_frame",
                  "disc_server_submit_query", "disc_server_wait", "disc_server_stats", "disc_server_reset_stats",
                  "disc_map_finalize", "disc_integrate_frames_async", "disc_map_wait",
                  "disc_group_integrate_async", "disc_group_wait"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().disc_status_str(int(code)).decode()


def pack_key(kx: int, ky: int, kz: int) -> int:
    return int(lib().disc_pack_key(kx, ky, kz))


def config_default(**overrides) -> dict:
    c = Config()
    lib().disc_config_default(ctypes.byref(c))
    d = {k: getattr(c, k) for k, _ in Config._fields_}
    d.update(overrides)
    return d


def _check(code, what):
    if code != 0:
        raise DiscError(code, what)


def _fill_frame(fr: Frame, width, height, intr, pose):
    fr.width, fr.height = int(width), int(height)
    fr.fx, fr.fy, fr.cx, fr.cy = (float(x) for x in intr)
    for i, v in enumerate(np.asarray(pose, np.float64).reshape(16)):
        fr.T_world_cam[i] = float(v)


def host_frame(depth, labels, tokens, pose, intr, num_masks, global_embed=None, assoc_tokens=None):
    """A disc_frame over host numpy arrays (kept alive by the returned tuple);
    assoc_tokens: the second token grid, same dtype as tokens."""
    depth = np.ascontiguousarray(depth, np.float32)
    labels = np.ascontiguousarray(labels, np.uint16)
    if tokens.dtype == np.float32:
        tokens = np.ascontiguousarray(tokens)
        tdt = 0
    else:  # bfloat16 bits as uint16
        tokens = np.ascontiguousarray(tokens, np.uint16)
        tdt = 1
    g = None if global_embed is None else np.ascontiguousarray(global_embed, np.float32)
    fr = Frame()
    _fill_frame(fr, depth.shape[1], depth.shape[0], intr, pose)
    fr.depth, fr.labels, fr.tokens = depth.ctypes.data, labels.ctypes.data, tokens.ctypes.data
    fr.token_dtype = tdt
    fr.num_masks = int(num_masks)
    fr.global_embed = None if g is None else g.ctypes.data
    fr.inputs_on_device = 0
    at = None
    if assoc_tokens is not None:
        at = np.ascontiguousarray(assoc_tokens, tokens.dtype)
        fr.assoc_tokens = at.ctypes.data
    return fr, (depth, labels, tokens, g, at)


def device_frame(depth, labels, tokens, pose, intr, num_masks, global_embed=None, assoc_tokens=None):
    """A disc_frame over device tensors (torch CUDA tensors or raw pointers).

    depth: float32 [H, W]; labels: int16/uint16 [H, W]; tokens: float32 or
    bfloat16 [P, D]; all contiguous on the map's device."""
    import torch
    H, W = depth.shape
    fr = Frame()
    _fill_frame(fr, W, H, intr, pose)
    fr.depth, fr.labels, fr.tokens = depth.data_ptr(), labels.data_ptr(), tokens.data_ptr()
    fr.token_dtype = 1 if tokens.dtype == torch.bfloat16 else 0
    fr.num_masks = int(num_masks)
    fr.global_embed = None if global_embed is None else global_embed.data_ptr()
    fr.inputs_on_device = 1
    if assoc_tokens is not None:
        fr.assoc_tokens = assoc_tokens.data_ptr()
    return fr, (depth, labels, tokens, global_embed, assoc_tokens)


def token_stats_static(tokens, global_embed=None, eps=1e-6, stream=None):
    """Eq. 1 distinctiveness and cosine to the global embedding for one token
    grid (torch CUDA tensor [P, D], fp32 or bf16) with no device allocation.
    Returns (Dp, cosg) as new CUDA tensors allocated by the caller here."""
    import torch
    P, D = tokens.shape
    Dp = torch.empty(P, dtype=torch.float32, device=tokens.device)
    cosg = torch.empty(P, dtype=torch.float32, device=tokens.device)
    s = torch.cuda.current_stream(tokens.device) if stream is None else stream
    rc = lib().disc_token_stats_static(tokens.data_ptr(), 1 if tokens.dtype == torch.bfloat16 else 0, P, D,
                                       None if global_embed is None else global_embed.data_ptr(), float(eps),
                                       Dp.data_ptr(), cosg.data_ptr(), s.cuda_stream)
    _check(rc, "disc_token_stats_static")
    return Dp, cosg


def debug_fail_alloc_after(n: int):
    """Test hook: after n more device allocations the library's allocations
    fail as out of memory (n < 0: off)."""
    lib().disc_debug_fail_alloc_after(int(n))


def debug_gemm_stall(on: bool, device: int = 0):
    """Test hook: the pooling GEMM issues no MMA, so its bounded waits run out
    (~1 s) and the frames it serves fail with DISC_ERR_TIMEOUT."""
    _check(lib().disc_debug_gemm_stall(int(device), 1 if on else 0), "disc_debug_gemm_stall")


def query_heatmap(tokens, query, eps=1e-6, stream=None):
    """Fig. 2 heatmap D_p * cos(f_p, q) of a query vector (CUDA tensor [D])
    over a token grid (CUDA tensor [P, D], fp32 or bf16); no device allocation
    in the library.  Returns a new CUDA tensor [P]."""
    import torch
    P, D = tokens.shape
    heat = torch.empty(P, dtype=torch.float32, device=tokens.device)
    s = torch.cuda.current_stream(tokens.device) if stream is None else stream
    rc = lib().disc_query_heatmap(tokens.data_ptr(), 1 if tokens.dtype == torch.bfloat16 else 0, P, D,
                                  query.data_ptr(), float(eps), heat.data_ptr(), s.cuda_stream)
    _check(rc, "disc_query_heatmap")
    return heat


class AsyncFrames:
    """The pending results of one disc_integrate_frames_async call: the
    counters, frames done and status, valid once the call is finished."""

    def __init__(self, gmap, frames, n):
        self.map = gmap
        self.keep = frames  # the frames' input buffers stay alive with the handle
        self.stats = (Stats * max(n, 1))()
        self.done = c_i32(0)
        self.rc = c_i32(0)
        self.n = n

    def result(self, check: bool = True):
        """Wait for the map's asynchronous calls, then (stats dicts, frames
        done, status), as integrate_frames returns them."""
        self.map.wait()
        if check:
            _check(self.rc.value, "disc_integrate_frames_async")
        return [self.stats[i].as_dict() for i in range(self.n)], int(self.done.value), int(self.rc.value)


class DiscMap:
    """One map resident on one GPU (disc_map_create ... disc_map_destroy)."""

    def __init__(self, **cfg):
        c = Config(**config_default(**cfg))
        resolved = Config()
        h = c_vp()
        _check(lib().disc_map_create(ctypes.byref(c), ctypes.byref(resolved), ctypes.byref(h)),
               "disc_map_create")
        self._h = h
        self.cfg = {k: getattr(resolved, k) for k, _ in Config._fields_}
        self.D = int(resolved.embed_dim)
        self.P = int(resolved.patch_h * resolved.patch_w)

    @classmethod
    def _from_handle(cls, h):
        self = cls.__new__(cls)
        self._h = h
        c = Config()
        _check(lib().disc_map_get_config(h, ctypes.byref(c)), "disc_map_get_config")
        self.cfg = {k: getattr(c, k) for k, _ in Config._fields_}
        self.D = int(c.embed_dim)
        self.P = int(c.patch_h * c.patch_w)
        return self

    def close(self):
        h = getattr(self, "_h", None)
        if h and getattr(self, "_owned", True):
            lib().disc_map_destroy(h)  # finishes the map's asynchronous calls first
        self._h = None

    __del__ = close

    def integrate(self, frame, check: bool = True) -> dict:
        """frame: (Frame, keepalive) from host_frame/device_frame."""
        fr, _keep = frame
        st = Stats()
        rc = lib().disc_integrate_frame(self._h, ctypes.byref(fr), ctypes.byref(st))
        if check:
            _check(rc, "disc_integrate_frame")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def integrate_frames(self, frames, check: bool = True):
        n = len(frames)
        arr = (Frame * n)()
        for i, (fr, _k) in enumerate(frames):
            arr[i] = fr
        st = (Stats * n)()
        done = c_i32(0)
        rc = lib().disc_integrate_frames(self._h, arr, n, st, ctypes.byref(done))
        if check:
            _check(rc, "disc_integrate_frames")
        return [s.as_dict() for s in st], int(done.value), rc

    def integrate_frames_raw(self, arr, n, stats):
        """Pre-built ctypes arrays (no per-call marshalling); returns the status."""
        return lib().disc_integrate_frames(self._h, arr, n, stats, None)

    def integrate_frames_async_raw(self, arr, n, stats, n_done=None, result=None):
        """disc_integrate_frames_async on pre-built ctypes arrays.  stats (a
        Stats array), n_done and result (c_int32 objects, or None) are written
        when the call is finished; the caller keeps them and the frames'
        input buffers alive until then.  Returns the status of the call."""
        return lib().disc_integrate_frames_async(self._h, arr, n, stats,
                                                 None if n_done is None else ctypes.byref(n_done),
                                                 None if result is None else ctypes.byref(result))

    def integrate_frames_async(self, frames) -> "AsyncFrames":
        """Enqueue frames (a list of (Frame, keepalive)) and return at once;
        AsyncFrames.result() waits and gives what integrate_frames gives."""
        n = len(frames)
        arr = (Frame * n)()
        for i, (fr, _k) in enumerate(frames):
            arr[i] = fr
        h = AsyncFrames(self, frames, n)
        rc = self.integrate_frames_async_raw(arr, n, h.stats, h.done, h.rc)
        _check(rc, "disc_integrate_frames_async")
        # the library writes into the handle when the call is finished, which
        # may be as late as the map's destruction: the map holds it till then
        if not hasattr(self, "_pending"):
            self._pending = []
        self._pending.append(h)
        return h

    def wait(self) -> int:
        """disc_map_wait: finish the map's asynchronous calls; returns the
        first status among them that is not DISC_OK (0 if none)."""
        rc = lib().disc_map_wait(self._h)
        self._pending = []
        return rc

    def set_schedule(self, geometry_chunk=8, serial_ctas=4, probe_width=1, assoc_cluster=0, batch_split=0):
        _check(lib().disc_map_set_schedule(self._h, ctypes.byref(Schedule(geometry_chunk, serial_ctas, probe_width,
                                                                          assoc_cluster, batch_split))),
               "disc_map_set_schedule")

    def autotune(self, frames, reps=3) -> dict:
        """Time the candidate launch schedules on sample frames (list of
        (Frame, keepalive), or a ctypes Frame array) and keep the fastest."""
        if isinstance(frames, list):
            arr = (Frame * len(frames))()
            for i, (fr, _k) in enumerate(frames):
                arr[i] = fr
        else:
            arr = frames
        r = TuneReport()
        _check(lib().disc_map_autotune(self._h, arr, len(arr), reps, ctypes.byref(r)), "disc_map_autotune")
        return r.as_dict()

    def last_frame(self) -> dict:
        M_cap = int(self.cfg["max_masks"])
        P, D = self.P, self.D
        npx = int(self.cfg["max_width"]) * int(self.cfg["max_height"])
        out = dict(fbar=np.zeros(D, np.float32), Dp=np.zeros(P, np.float32), cosg=np.zeros(P, np.float32),
                   cov=np.zeros((max(M_cap, 1), P), np.int32), npix=np.zeros(max(M_cap, 1), np.int32),
                   W=np.zeros((max(M_cap, 1), P), np.float32), E=np.zeros((max(M_cap, 1), D), np.float32),
                   E_fast=np.zeros((max(M_cap, 1), D), np.float32), S=np.zeros((max(M_cap, 1), 5), np.float32),
                   nvox=np.zeros(max(M_cap, 1), np.int32), rep=np.zeros(max(M_cap, 1), np.int32),
                   seg_keys=np.zeros(npx, np.uint64), seg_m=np.zeros(npx, np.int32),
                   E_bound=np.zeros(max(M_cap, 1), np.float32))
        Da = int(self.cfg.get("assoc_dim", 0))
        if Da > 0:
            out["A"] = np.zeros((max(M_cap, 1), Da), np.float32)
            out["A_fast"] = np.zeros((max(M_cap, 1), Da), np.float32)
        r = Report()
        for k in ("fbar", "Dp", "cosg", "cov", "npix", "W", "E", "E_fast", "S", "nvox", "rep", "seg_keys", "seg_m",
                  "E_bound", "A", "A_fast"):
            if k in out:
                setattr(r, k, out[k].ctypes.data)
        r.seg_cap = npx
        _check(lib().disc_map_last_frame(self._h, ctypes.byref(r)), "disc_map_last_frame")
        M = int(r.num_masks)
        n = int(r.n_seg)
        for k in ("cov", "npix", "W", "E", "E_fast", "S", "nvox", "rep", "E_bound", "A", "A_fast"):
            if k in out:
                out[k] = out[k][:M]
        order = np.lexsort((out["seg_keys"][:n], out["seg_m"][:n]))
        out["seg_keys"] = out["seg_keys"][:n][order]
        out["seg_m"] = out["seg_m"][:n][order]
        out["n_seg"] = n
        out["num_masks"] = M
        return out

    def counts(self):
        nv, nid = c_i64(0), c_i32(0)
        _check(lib().disc_map_counts(self._h, ctypes.byref(nv), ctypes.byref(nid)), "disc_map_counts")
        return int(nv.value), int(nid.value)

    def voxels(self):
        nv, _ = self.counts()
        keys = np.zeros(max(nv, 1), np.uint64)
        ids = np.zeros(max(nv, 1), np.int32)
        _check(lib().disc_map_export_voxels(self._h, keys.ctypes.data, ids.ctypes.data, nv), "export_voxels")
        return keys[:nv], ids[:nv]

    def instances(self):
        _, n = self.counts()
        parent = np.zeros(max(n, 1), np.int32)
        count = np.zeros(max(n, 1), np.int64)
        Q = np.zeros(max(n, 1), np.float32)
        E = np.zeros((max(n, 1), self.D), np.float32)
        obs = np.zeros(max(n, 1), np.int32)
        _check(lib().disc_map_export_instances(self._h, parent.ctypes.data, count.ctypes.data, Q.ctypes.data,
                                                E.ctypes.data, obs.ctypes.data, n), "export_instances")
        out = dict(parent=parent[:n], count=count[:n], Q=Q[:n], E=E[:n], n_obs=obs[:n])
        Da = int(self.cfg.get("assoc_dim", 0))
        if Da > 0:
            A = np.zeros((max(n, 1), Da), np.float32)
            _check(lib().disc_map_export_assoc(self._h, A.ctypes.data, max(n, 1)), "export_assoc")
            out["A"] = A[:n]
        return out

    def query_topk(self, queries, k):
        q = np.ascontiguousarray(queries, np.float32).reshape(-1, self.D)
        ids = np.zeros((q.shape[0], k), np.int32)
        sc = np.zeros((q.shape[0], k), np.float32)
        _check(lib().disc_query_topk(self._h, q.ctypes.data, q.shape[0], k, ids.ctypes.data, sc.ctypes.data),
               "disc_query_topk")
        return ids, sc

    def query_points(self, xyz):
        x = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
        ids = np.zeros(x.shape[0], np.int32)
        _check(lib().disc_query_points(self._h, x.ctypes.data, x.shape[0], ids.ctypes.data), "disc_query_points")
        return ids

    def kernel_launches(self) -> int:
        return int(lib().disc_map_kernel_launches(self._h))

    def set_phase_timing(self, enable: bool):
        _check(lib().disc_map_set_phase_timing(self._h, 1 if enable else 0), "disc_map_set_phase_timing")

    def phase_times(self) -> dict:
        n = 16
        ms = np.zeros(n, np.float64)
        la = np.zeros(n, np.int64)
        ca = np.zeros(n, np.int64)
        _check(lib().disc_map_phase_times(self._h, ms.ctypes.data, la.ctypes.data, ca.ctypes.data, n),
               "disc_map_phase_times")
        return {lib().disc_phase_name(i).decode(): dict(ms=float(ms[i]), launches=int(la[i]), calls=int(ca[i]))
                for i in range(n)}

    def device_bytes(self) -> int:
        return int(lib().disc_map_device_bytes(self._h))

    def finalize(self, min_voxels, contact_num=1, contact_den=5, tau_cos=None, check: bool = True):
        """End-of-trajectory orphan merge and voxel-count filter; the report."""
        c = FinalizeConfig(int(min_voxels), int(contact_num), int(contact_den),
                           float(self.cfg["tau_cos"] if tau_cos is None else tau_cos))
        r = FinalizeReport()
        rc = lib().disc_map_finalize(self._h, ctypes.byref(c), ctypes.byref(r))
        if check:
            _check(rc, "disc_map_finalize")
        out = {k: int(getattr(r, k)) for k, _ in FinalizeReport._fields_}
        out["rc"] = rc
        return out

    def save(self, path):
        _check(lib().disc_map_save(self._h, str(path).encode()), "disc_map_save")

    @classmethod
    def load(cls, path, **override):
        c = Config(**config_default(**override)) if override else None
        h = c_vp()
        _check(lib().disc_map_load(str(path).encode(), ctypes.byref(c) if c is not None else None,
                                   ctypes.byref(h)), "disc_map_load")
        return cls._from_handle(h)


class DiscGroup:
    """Batches over many maps (disc_group_create ... disc_group_destroy)."""

    def __init__(self, **cfg):
        c = GroupConfig()
        lib().disc_group_config_default(ctypes.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        h = c_vp()
        _check(lib().disc_group_create(ctypes.byref(c), ctypes.byref(h)), "disc_group_create")
        self._h = h
        self.cfg = {k: getattr(c, k) for k, _ in GroupConfig._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().disc_group_destroy(h)
            self._h = None

    __del__ = close

    def integrate_raw(self, maps, frame_arrays, counts, stats_arrays=None, n_done=None):
        """maps: [DiscMap]; frame_arrays: [ctypes Frame array]; counts: [int];
        stats_arrays: [ctypes Stats array] or None; returns the status."""
        n = len(maps)
        hm = (c_vp * n)(*[m._h.value for m in maps])
        hf = (c_vp * n)(*[ctypes.cast(a, c_vp).value if a is not None else None for a in frame_arrays])
        hc = (c_i32 * n)(*counts)
        hs = (c_vp * n)(*[ctypes.cast(a, c_vp).value if a is not None else None for a in stats_arrays]) \
            if stats_arrays is not None else None
        return lib().disc_group_integrate(self._h, hm, n, hf, hc, hs, n_done)

    def integrate_async_raw(self, maps, frame_arrays, counts, stats_arrays=None, n_done=None, result=None):
        """disc_group_integrate_async; stats_arrays, n_done (a c_int32 array)
        and result (a c_int32) are written when the call is finished and must
        stay alive until then.  Returns the status of the call."""
        n = len(maps)
        hm = (c_vp * n)(*[m._h.value for m in maps])
        hf = (c_vp * n)(*[ctypes.cast(a, c_vp).value if a is not None else None for a in frame_arrays])
        hc = (c_i32 * n)(*counts)
        hs = (c_vp * n)(*[ctypes.cast(a, c_vp).value if a is not None else None for a in stats_arrays]) \
            if stats_arrays is not None else None
        return lib().disc_group_integrate_async(self._h, hm, n, hf, hc, hs, n_done,
                                                None if result is None else ctypes.byref(result))

    def wait(self) -> int:
        """disc_group_wait: finish the group's asynchronous calls."""
        return lib().disc_group_wait(self._h)

    def set_schedule(self, geometry_chunk=8, serial_ctas=4, probe_width=1, assoc_cluster=0, batch_split=0):
        _check(lib().disc_group_set_schedule(self._h, ctypes.byref(Schedule(geometry_chunk, serial_ctas, probe_width,
                                                                            assoc_cluster, batch_split))),
               "disc_group_set_schedule")

    def autotune(self, maps, frame_arrays, counts, reps=3) -> dict:
        """Time the candidate launch schedules on a sample (per map a ctypes
        Frame array and a count; fresh maps of the same configurations take
        the frames) and keep the fastest for this group."""
        n = len(maps)
        hm = (c_vp * n)(*[m._h.value for m in maps])
        hf = (c_vp * n)(*[ctypes.cast(a, c_vp).value for a in frame_arrays])
        hc = (c_i32 * n)(*counts)
        r = TuneReport()
        _check(lib().disc_group_autotune(self._h, hm, n, hf, hc, reps, ctypes.byref(r)), "disc_group_autotune")
        return r.as_dict()

    def integrate(self, maps, frames_per_map, check: bool = True):
        """frames_per_map: per map a list of (Frame, keepalive).  Returns
        (per-map list of stats dicts, per-map frames done, status)."""
        n = len(maps)
        arrs, sts = [], []
        for frames in frames_per_map:
            k = len(frames)
            a = (Frame * max(k, 1))()
            for i, (fr, _keep) in enumerate(frames):
                a[i] = fr
            arrs.append(a)
            sts.append((Stats * max(k, 1))())
        done = (c_i32 * max(n, 1))()
        rc = self.integrate_raw(maps, arrs, [len(f) for f in frames_per_map], sts, done)
        if check:
            _check(rc, "disc_group_integrate")
        stats = [[sts[g][i].as_dict() for i in range(len(frames_per_map[g]))] for g in range(n)]
        return stats, [int(done[g]) for g in range(n)], rc

    def kernel_launches(self) -> int:
        return int(lib().disc_group_kernel_launches(self._h))

    def device_bytes(self) -> int:
        return int(lib().disc_group_device_bytes(self._h))

    def set_phase_timing(self, enable: bool):
        _check(lib().disc_group_set_phase_timing(self._h, 1 if enable else 0), "disc_group_set_phase_timing")

    def phase_times(self) -> dict:
        n = 16
        ms = np.zeros(n, np.float64)
        la = np.zeros(n, np.int64)
        ca = np.zeros(n, np.int64)
        _check(lib().disc_group_phase_times(self._h, ms.ctypes.data, la.ctypes.data, ca.ctypes.data, n),
               "disc_group_phase_times")
        return {lib().disc_phase_name(i).decode(): dict(ms=float(ms[i]), launches=int(la[i]), calls=int(ca[i]))
                for i in range(n)}


class DiscServer:
    """Request loop over resident maps (disc_server_create ... disc_server_destroy)."""

    def __init__(self, hbm_budget_bytes, max_queue=4096, workers=0, **group):
        c = ServerConfig()
        lib().disc_group_config_default(ctypes.byref(c.group))
        for k, v in group.items():
            setattr(c.group, k, v)
        c.hbm_budget_bytes = int(hbm_budget_bytes)
        c.max_queue = int(max_queue)
        c.workers = int(workers)
        h = c_vp()
        _check(lib().disc_server_create(ctypes.byref(c), ctypes.byref(h)), "disc_server_create")
        self._h = h
        self.D = int(c.group.embed_dim)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().disc_server_destroy(h)
            self._h = None

    __del__ = close

    def open_map(self, **cfg) -> int:
        c = Config(**config_default(**cfg))
        mid = c_i32(-1)
        rc = lib().disc_server_open_map(self._h, ctypes.byref(c), ctypes.byref(mid))
        _check(rc, "disc_server_open_map")
        return int(mid.value)

    def try_open_map(self, **cfg):
        """(status, map id or -1) without raising."""
        c = Config(**config_default(**cfg))
        mid = c_i32(-1)
        rc = lib().disc_server_open_map(self._h, ctypes.byref(c), ctypes.byref(mid))
        return rc, int(mid.value)

    def close_map(self, map_id: int):
        _check(lib().disc_server_close_map(self._h, map_id), "disc_server_close_map")

    def map(self, map_id: int) -> DiscMap:
        """A non-owning view of the map (export, queries) between requests."""
        h = lib().disc_server_map(self._h, map_id)
        if not h:
            raise DiscError(-1, "disc_server_map")
        m = DiscMap._from_handle(c_vp(h))
        m._owned = False
        return m

    def submit_frame(self, map_id: int, frame) -> int:
        fr, _keep = frame
        t = c_i64(0)
        _check(lib().disc_server_submit_frame(self._h, map_id, ctypes.byref(fr), ctypes.byref(t)),
               "disc_server_submit_frame")
        return int(t.value)

    def submit_frame_borrowed(self, map_id: int, frame) -> int:
        """Queue a frame whose buffers the server reads in place: they (the
        keepalive of `frame` included) must stay unchanged until the ticket's
        wait returns."""
        fr, _keep = frame
        t = c_i64(0)
        _check(lib().disc_server_submit_frame_borrowed(self._h, map_id, ctypes.byref(fr), ctypes.byref(t)),
               "disc_server_submit_frame_borrowed")
        return int(t.value)

    def submit_frame_raw(self, map_id: int, fr) -> int:
        t = c_i64(0)
        rc = lib().disc_server_submit_frame(self._h, map_id, ctypes.byref(fr), ctypes.byref(t))
        return int(t.value) if rc == 0 else rc

    def submit_query(self, map_id: int, queries, k: int) -> int:
        q = np.ascontiguousarray(queries, np.float32).reshape(-1, self.D)
        t = c_i64(0)
        _check(lib().disc_server_submit_query(self._h, map_id, q.ctypes.data, q.shape[0], k, ctypes.byref(t)),
               "disc_server_submit_query")
        return int(t.value), q.shape[0], k

    def wait_frame(self, ticket: int):
        st = Stats()
        lat = c_f64(0.0)
        rc = lib().disc_server_wait(self._h, ticket, ctypes.byref(st), None, None, ctypes.byref(lat))
        d = st.as_dict()
        d["rc"] = rc
        d["latency_ms"] = float(lat.value)
        return d

    def wait_query(self, tq):
        ticket, nq, k = tq
        ids = np.zeros((nq, k), np.int32)
        sc = np.zeros((nq, k), np.float32)
        lat = c_f64(0.0)
        rc = lib().disc_server_wait(self._h, ticket, None, ids.ctypes.data, sc.ctypes.data, ctypes.byref(lat))
        return rc, ids, sc, float(lat.value)

    def stats(self) -> dict:
        r = ServerReport()
        _check(lib().disc_server_stats(self._h, ctypes.byref(r)), "disc_server_stats")
        return {k: getattr(r, k) for k, _ in ServerReport._fields_}

    def reset_stats(self):
        _check(lib().disc_server_reset_stats(self._h), "disc_server_reset_stats")
