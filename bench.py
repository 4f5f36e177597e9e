"""Benchmark of the DISC per-frame integration step on GB300.

Workload (the Room-scale configuration): a 10x8x3 m synthetic room with 80
random boxes/ellipsoids, a 2000-frame closed camera path, 640x480 fp32 depth
with 1 % noise, 40 masks per frame, 24x24x768 fp32 patch tokens, 2.5 cm
voxels.  A step integrates B consecutive frames of the trajectory into one
resident map through disc_integrate_frames (all steps a1-a10 per frame).

Reported: frames/s (whole job, all ranks), voxel-updates/s, p50/p99 single-
frame latency, the roofline of the dominant kernel (per-phase CUDA events on
the map's stream), an end-to-end figure through the same C ABI with pinned
host buffers (H2D inside the timed region), and the CPU oracle's throughput on
a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & voxel-updates/s on 1 GB300 (plain vs batched/served); p50/p99 frame ms"
WORKLOAD = "Room-scale plain: 10x8x3 m room, 80 boxes/ellipsoids, 640x480 fp32 depth (1% noise), " \
           "40 masks/frame, tokens 24x24x768 fp32, voxel 2.5 cm, FP32"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames-per-step", type=int, default=32)
    ap.add_argument("--latency-frames", type=int, default=64)
    ap.add_argument("--timing-batches", type=int, default=4)
    ap.add_argument("--batch-frames", type=int, default=0,
                    help="frames per internal batch of a call (0: the map's default)")
    ap.add_argument("--serial-sms", type=int, default=0,
                    help="SMs of the serial part of overlapped batches (0: default, < 0: no overlap)")
    ap.add_argument("--batched-maps", type=int, default=64)
    ap.add_argument("--batched-frames", type=int, default=4, help="frames of each map per batch")
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--batched-history", default="0,16,64,256",
                    help="frames each batched map integrates before the timed frames, cycling over the maps")
    ap.add_argument("--same-maps", type=int, default=16,
                    help="maps of the same-workload batched line (Room-scale 640x480 fp32, as the plain path; 0: skip)")
    ap.add_argument("--same-frames", type=int, default=8, help="frames of each map per batch of that line")
    ap.add_argument("--multistory-steps", type=int, default=16,
                    help="timed 32-frame steps of the Multi-story configuration (0: skip)")
    ap.add_argument("--tiny", type=int, default=1, help="1: time the Tiny configuration")
    ap.add_argument("--served-maps", type=int, default=32)
    ap.add_argument("--served-rates", default="4000,8000,12000,16000", help="offered frames/s, comma separated")
    ap.add_argument("--served-repeats", type=int, default=2, help="measurements per offered rate")
    ap.add_argument("--served-frames", type=int, default=96,
                    help="frames of each served map's path; the measurements together take every frame once")
    ap.add_argument("--batch-split", type=int, default=0,
                    help="smaller batches per 32-frame call of the plain path (0: the library's automatic choice)")
    ap.add_argument("--table-log2", type=int, default=26,
                    help="initial voxel-table slots of the plain path's map, as a power of two")
    ap.add_argument("--assoc-cluster", type=int, default=0,
                    help="CTAs per map of the plain path's association kernel (0: automatic)")
    ap.add_argument("--geometry-chunk", type=int, default=0,
                    help="frames per back-projection launch of the plain path (0: the library's default, 8)")
    ap.add_argument("--batched-tune", type=int, default=1, help="1: autotune the group's launch schedule first")
    ap.add_argument("--served-workers", type=int, default=2, help="batches the server runs at once")
    ap.add_argument("--served-borrow", type=int, default=1,
                    help="1: clients hand over pinned frames read in place; 0: the server copies each frame")
    ap.add_argument("--served-precision", type=int, default=2, help="0 fp32, 1 bf16, 2 fp8 e4m3")
    ap.add_argument("--precision", type=int, default=0,
                    help="fast pooling/scoring precision of the plain path: 0 fp32 (the Room-scale "
                         "configuration), 1 bf16, 2 fp8 e4m3")
    ap.add_argument("--assoc-steps", type=int, default=5,
                    help="steps with a second (24x32x1024) token grid driving association (0: skip)")
    ap.add_argument("--dilation-steps", type=int, default=20,
                    help="steps of the same workload with the 26-neighbour overlap (0: skip)")
    ap.add_argument("--dbscan-steps", type=int, default=20,
                    help="steps of the same workload with the DBSCAN filter on (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--finalize", type=int, default=1,
                    help="1: time the end-of-trajectory step on the main map once its frames are in")
    ap.add_argument("--heatmap-calls", type=int, default=100, help="timed query-heatmap calls (0: skip)")
    ap.add_argument("--watchdog-s", type=float, default=600.0,
                    help="a run still going after this long prints the sections it finished and ends")
    return ap.parse_args()


def rank_env():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(rank: int) -> int:
    """Replicas only: every rank integrates its own map of its own scene."""
    return 1 + rank


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's value (the job ends when its last rank does)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def guarded(name, fn):
    """A section of the line after the main measurement: its result, or an
    {"error": ...} entry if it raises, so that the line still carries every
    section that finished."""
    try:
        return fn()
    except Exception as ex:  # recorded, the rest of the line stands
        print(f"bench: section {name} failed: {ex!r}", file=sys.stderr, flush=True)
        return {"error": repr(ex)}


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank does the same work)."""
    return units_per_rank * world / (max_ms / 1e3)


def room_cfg(scene):
    from tests import common
    return common.disc_cfg(scene, voxel_capacity=1 << 24, instance_capacity=1 << 16)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples, started before the warm-up (the tool
    takes a moment to start) and kept only inside the timed window."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0, period_ms=20):
        self.proc = None
        self.path = None
        self.idx = device_index
        self.period = period_ms
        self.window = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, t0, t1):
        """The timed window, in time.time() seconds."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        samples = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                if "." in parts[0]:
                    ts += float("0." + parts[0].split(".")[1])
                samples.append((ts, float(parts[2]), float(parts[3]),
                                {n for n, v in zip(names, parts[6:10]) if v.lower() == "active"}))
            except ValueError:
                continue
        os.unlink(self.path)
        if not samples:
            return None
        inside = samples
        if self.window:
            t0, t1 = self.window
            inside = [x for x in samples if t0 - 0.02 <= x[0] <= t1 + 0.02]
            if not inside:  # window shorter than the sampling period: the nearest sample
                mid = 0.5 * (t0 + t1)
                inside = [min(samples, key=lambda x: abs(x[0] - mid))]
        reasons = set()
        for x in inside:
            reasons |= x[3]
        return {"sm_mhz": float(np.median([x[1] for x in inside])), "sm_max_mhz": float(max(x[2] for x in inside)),
                "reasons": sorted(reasons), "samples": len(inside), "period_ms": self.period}


def measured_traffic(kernel, frames_per_launch):
    """DRAM bytes of one launch of `kernel` over frames_per_launch frames,
    from its committed ncu summary (profiles/<kernel>_room_640x480.md: the
    bytes of one captured launch over its frames, scaled per frame), or None
    when there is none or the kernel's source changed since the counters were
    taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_room_640x480.md")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith(("|", "#", " ")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        src = os.path.join(ROOT, kv["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != kv["source_sha256"]:
            return None
        return int(kv["traffic_bytes_per_launch"]) / int(kv["frames_per_launch"]) * frames_per_launch
    except Exception:
        return None


# The method's algorithmic bytes per frame (what the step must move, each
# datum once): the inputs (depth fp32 and labels u16 per pixel, the token grid
# at its dtype), 12 B per unique (segment, voxel) probe of the map (8 B key +
# 4 B label), 12 B per new voxel written, one instance embedding read per
# (segment, instance) pair whose cosine is taken (at the scoring copy's
# width), and one fp32 embedding written per adopted segment.  Scratch the
# kernels use for themselves (hash slots, lists, partial sums) is not counted.
def step_bytes(s, H, W, P, D, tok_b=4, emb_b=4):
    """Algorithmic bytes of one frame (s: its stats)."""
    return (6 * H * W + P * D * tok_b + 12 * s["unique_seg_voxels"] + 12 * s["new_voxels"]
            + D * emb_b * s["scored_pairs"] + 4 * D * s["embedding_copies"])


def algorithmic_bytes(phase, sts, H, W, P, D, tok_b=4, emb_b=4, lookup_in_entries=False):
    """The part of step_bytes each phase is credited with, summed over the
    frames of the timed batches (sts: per-frame stats).  Divided by the
    phase's launches it gives the bytes per launch.  Phases that move none of
    the step's bytes (scratch only) report 0."""
    per_frame = {
        "backproject": lambda s: 6 * H * W,
        "coverage": lambda s: 2 * H * W,
        "token_stats": lambda s: P * D * tok_b,
        "pool_exact": lambda s: P * D * tok_b,
        "pool_gemm": lambda s: P * D * tok_b,
        "lookup": lambda s: 12 * s["unique_seg_voxels"],
        "entries": lambda s: 12 * s["unique_seg_voxels"] if lookup_in_entries else 0,
        "associate": lambda s: D * emb_b * s["scored_pairs"] + 4 * D * s["embedding_copies"],
        "commit": lambda s: 12 * s["new_voxels"],
        "score": lambda s: D * emb_b * s["scored_pairs"],
        "apply": lambda s: 12 * s["new_voxels"] + 4 * D * s["embedding_copies"],
    }
    if phase not in per_frame:
        return 0.0
    return float(sum(per_frame[phase](s_) for s_ in sts))


def host_cpu():
    """Model name of the host CPU and its core count."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return model, os.cpu_count() or 1


BATCHED = "Batched: {G} independent room-scale maps of uneven size (320x240..640x480 frames, 20-120 objects, " \
          "5-60 masks/frame, voxel 2.5 cm; {hist} frames of history before the timed frames, cycling over the " \
          "maps), bf16 tokens 24x24x768, {J} frames of every map per batch"


def batched_scenes(G, seed0):
    """G room scenes of uneven size: frame sizes, object counts and mask limits
    cycle through fixed lists (seeded per map)."""
    import synth
    sizes = ((640, 480), (480, 360), (320, 240), (560, 420))
    objs = (80, 20, 120, 50, 100)
    masks = (40, 5, 60, 25, 12, 50)
    return [synth.room_scene(seed=seed0 + g, width=sizes[g % 4][0], height=sizes[g % 4][1],
                             n_objects=objs[g % 5], max_masks=masks[g % 6]) for g in range(G)]


def _group_async_steps(torch, stream, binding, grp, maps, steps, J, flush):
    """Time steps (per step a list of per-map Frame arrays of J frames) as
    disc_group_integrate_async calls in one timed region, the L2 flush
    enqueued between the steps; returns (ms, unique segment-voxel pairs)."""
    G, T = len(maps), len(steps)
    sts = [[(binding.Stats * J)() for _ in range(G)] for _ in range(T)]
    done = [(ctypes.c_int32 * G)() for _ in range(T)]
    res = [ctypes.c_int32(1) for _ in range(T)]
    flush.fill_(-1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(T):
        if s:
            flush.fill_(float(s))
        rc = grp.integrate_async_raw(maps, steps[s], [J] * G, sts[s], done[s], res[s])
        assert rc == 0, rc
    rc = grp.wait()
    e1.record(stream)
    e1.synchronize()
    assert rc == 0 and all(r.value == 0 for r in res) and all(list(d) == [J] * G for d in done), rc
    upd = sum(sts[s][g][j].unique_seg_voxels for s in range(T) for g in range(G) for j in range(J))
    return e0.elapsed_time(e1), upd


def run_batched(args, torch, dev, stream, rank):
    """The batched form: every map's frames j..j+J of a step in one group call,
    device-resident bf16 inputs; timed as asynchronous calls
    (disc_group_integrate_async), then as synchronous ones for the latency."""
    from paper_2603_03935_gb300 import DiscGroup, DiscMap, binding
    from tests import common
    G, J, T = args.batched_maps, args.batched_frames, args.batched_steps
    scs = batched_scenes(G, 1000 + 97 * rank)
    hist = [int(x) for x in args.batched_history.split(",") if x] or [0]
    hg = [hist[g % len(hist)] for g in range(G)]  # frames each map integrated before the timed frames
    nf = (1 + 2 * T) * J
    frs = [s.render(range(h, h + nf)) for s, h in zip(scs, hg)]
    dd = [torch.from_numpy(f.depth).to(dev) for f in frs]
    ll = [torch.from_numpy(f.labels.view(np.int16)).to(dev) for f in frs]
    tt = [torch.from_numpy(f.tokens).to(dev).to(torch.bfloat16).contiguous() for f in frs]
    maps = [DiscMap(**common.disc_cfg(s, voxel_capacity=1 << 21, instance_capacity=1 << 12)) for s in scs]
    grp = DiscGroup(max_maps=G, frames_per_map=J, embed_dim=scs[0].dim, patch_h=scs[0].patch_h,
                    patch_w=scs[0].patch_w, max_width=max(s.width for s in scs),
                    max_height=max(s.height for s in scs), max_masks=max(s.max_masks for s in scs),
                    cuda_stream=stream.cuda_stream, device=dev.index)
    # history: each map first integrates the start of its own path (untimed,
    # through the group, 32 frames of every map with history per call), so
    # the maps enter the measurement at uneven sizes
    for lo in range(0, max(hg), 32):
        part = [g for g in range(G) if hg[g] > lo]
        keep, arrs, cnts = [], [], []
        for g in part:
            hf = scs[g].render(range(lo, min(hg[g], lo + 32)))
            a, k = _device_frames(torch, dev, binding, scs[g], hf, range(len(hf.depth)), bf16=True)
            keep.append(k)
            arrs.append(a)
            cnts.append(len(hf.depth))
        hst = [(binding.Stats * 32)() for _ in part]
        rc = grp.integrate_raw([maps[g] for g in part], arrs, cnts, hst)
        assert rc == 0, rc
    torch.cuda.synchronize()
    vox0 = [m.counts()[0] for m in maps]

    def arrays(lo):
        out = []
        for g in range(G):
            a = (binding.Frame * J)()
            sc, fr = scs[g], frs[g]
            for j in range(J):
                i = lo + j
                f = a[j]
                f.width, f.height = sc.width, sc.height
                f.fx, f.fy, f.cx, f.cy = sc.fx, sc.fy, sc.cx, sc.cy
                for q, v in enumerate(fr.poses[i].reshape(16)):
                    f.T_world_cam[q] = float(v)
                f.depth, f.labels, f.tokens = dd[g][i].data_ptr(), ll[g][i].data_ptr(), tt[g][i].data_ptr()
                f.token_dtype = 1
                f.num_masks = int(fr.num_masks[i])
                f.global_embed = None
                f.inputs_on_device = 1
            out.append(a)
        return out

    steps = [arrays(s * J) for s in range(1 + 2 * T)]
    sts = [(binding.Stats * J)() for _ in range(G)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    # the launch schedule the autotuner picks on the first step's frames
    # (fresh maps of the same configurations; the timed maps stay untouched)
    tune = grp.autotune(maps, steps[0], [J] * G, reps=2) if args.batched_tune else None
    l0 = grp.kernel_launches()
    assert grp.integrate_raw(maps, steps[0], [J] * G, sts) == 0
    torch.cuda.synchronize()
    # the timed steps as asynchronous group calls (a batch's frame chains
    # overlap the next batch's per-frame kernels), one timed region
    async_ms, upd = _group_async_steps(torch, stream, binding, grp, maps, steps[1:1 + T], J, flush)
    # the next T steps of every map as synchronous calls, each timed alone:
    # a frame's result is ready when its call returns (the latency figures)
    times = []
    for s in range(1 + T, 1 + 2 * T):
        flush.fill_(float(s))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = grp.integrate_raw(maps, steps[s], [J] * G, sts)
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        times.append(e0.elapsed_time(e1))
    total_ms = float(np.sum(times))
    out = {"workload": BATCHED.format(G=G, J=J, hist=args.batched_history),
           "frames_per_s": T * G * J / (async_ms / 1e3),
           "mode": "one disc_group_integrate_async call per batch, disc_group_wait after the last; one timed region",
           "sync_calls": {"frames_per_s": T * G * J / (total_ms / 1e3),
                          "mode": "one synchronous disc_group_integrate call per batch, each timed alone"},
           "map_voxels_at_start": {"min": int(min(vox0)), "median": int(np.median(vox0)), "max": int(max(vox0))},
           "voxel_updates_per_s": upd / (async_ms / 1e3), "maps": G, "frames_per_map_per_batch": J,
           "steps": T, "ms_per_batch": async_ms / T,
           "frame_latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                                "mode": "a frame's result is ready when its batch ends"},
           "gpu_launches_per_batch": (grp.kernel_launches() - l0) // (1 + 2 * T),
           "schedule": tune,
           "device_gb": (grp.device_bytes() + sum(m.device_bytes() for m in maps)) / 1e9}
    grp.close()
    for m in maps:
        m.close()
    return out


SAME = "Batched, same per-frame work as the plain line: {G} independent Room-scale maps (10x8x3 m room, " \
       "80 boxes/ellipsoids, 640x480 fp32 depth with 1% noise, 40 masks/frame, tokens 24x24x768 fp32, voxel " \
       "2.5 cm, FP32), {J} frames of every map per group call, each map {W} frames into its own trajectory"


def _device_frames(torch, dev, binding, sc, fr, idx, bf16=False):
    """A ctypes Frame array over device copies of frames idx of fr (the
    tensors are returned too, to keep them alive)."""
    d = torch.from_numpy(fr.depth[idx]).to(dev)
    l = torch.from_numpy(fr.labels[idx].view(np.int16)).to(dev)
    t = torch.from_numpy(fr.tokens[idx]).to(dev)
    if bf16:
        t = t.to(torch.bfloat16).contiguous()
    a = (binding.Frame * len(idx))()
    for j, i in enumerate(idx):
        f = a[j]
        f.width, f.height = sc.width, sc.height
        f.fx, f.fy, f.cx, f.cy = sc.fx, sc.fy, sc.cx, sc.cy
        for q, v in enumerate(fr.poses[i].reshape(16)):
            f.T_world_cam[q] = float(v)
        f.depth, f.labels, f.tokens = d[j].data_ptr(), l[j].data_ptr(), t[j].data_ptr()
        f.token_dtype = 1 if bf16 else 0
        f.num_masks = int(fr.num_masks[i])
        f.global_embed = None
        f.inputs_on_device = 1
    return a, (d, l, t)


def run_same_workload_batched(args, torch, dev, stream, rank):
    """The batched form on the plain line's workload: G Room-scale maps
    (seeds 2.., FP32, fp32 tokens), each first integrating W frames of its
    own trajectory untimed, then T group calls of J frames per map timed as
    asynchronous calls in one region, then T more as synchronous calls, each
    timed alone."""
    import synth
    from paper_2603_03935_gb300 import DiscGroup, DiscMap, binding
    from tests import common
    G, J, T, W = args.same_maps, args.same_frames, 3, 32
    scs = [synth.room_scene(seed=2 + 97 * rank + g) for g in range(G)]
    maps = [DiscMap(**common.disc_cfg(s, voxel_capacity=1 << 22, instance_capacity=1 << 12,
                                      cuda_stream=stream.cuda_stream, device=dev.index)) for s in scs]
    grp = DiscGroup(max_maps=G, frames_per_map=J, embed_dim=scs[0].dim, patch_h=scs[0].patch_h,
                    patch_w=scs[0].patch_w, max_width=scs[0].width, max_height=scs[0].height,
                    max_masks=scs[0].max_masks, cuda_stream=stream.cuda_stream, device=dev.index)
    sts = [(binding.Stats * J)() for _ in range(G)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step(lo):
        frs = [sc.render(range(lo, lo + J)) for sc in scs]
        return [_device_frames(torch, dev, binding, sc, fr, list(range(J))) for sc, fr in zip(scs, frs)]

    for lo in range(0, W, J):  # untimed: the maps' first W frames
        arrs = step(lo)
        assert grp.integrate_raw(maps, [a for a, _ in arrs], [J] * G, sts) == 0
        del arrs
    timed = [step(W + s * J) for s in range(T)]  # resident before the timed region
    torch.cuda.synchronize()
    async_ms, upd = _group_async_steps(torch, stream, binding, grp, maps, [[a for a, _ in st] for st in timed], J,
                                       flush)
    del timed
    times, pairs, newv, supd = [], 0, 0, 0
    for s in range(T, 2 * T):
        arrs = step(W + s * J)
        torch.cuda.synchronize()
        flush.fill_(float(s))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = grp.integrate_raw(maps, [a for a, _ in arrs], [J] * G, sts)
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        times.append(e0.elapsed_time(e1))
        for g in range(G):
            for j in range(J):
                supd += sts[g][j].unique_seg_voxels
                pairs += sts[g][j].overlap_pairs
                newv += sts[g][j].new_voxels
        del arrs
    total_ms = float(np.sum(times))
    nfr = T * G * J
    out = {"workload": SAME.format(G=G, J=J, W=W), "frames_per_s": nfr / (async_ms / 1e3),
           "mode": "one disc_group_integrate_async call per batch, disc_group_wait after the last; one timed region",
           "sync_calls": {"frames_per_s": nfr / (total_ms / 1e3),
                          "mode": "the next batches as synchronous disc_group_integrate calls, each timed alone"},
           "voxel_updates_per_s": upd / (async_ms / 1e3), "maps": G, "frames_per_map_per_batch": J,
           "steps": T, "ms_per_batch": async_ms / T,
           "per_frame": {"voxel_updates": supd / nfr, "overlap_pairs": pairs / nfr, "new_voxels": newv / nfr},
           "frame_latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                                "mode": "a frame's result is ready when its (synchronous) batch ends"}}
    grp.close()
    for m in maps:
        m.close()
    return out


MULTISTORY = "Multi-story: 3 floors of 40x30 m, 1000 objects, 640x480 depth (to 20 m, 1% noise), up to 100 " \
             "masks/frame, tokens 24x24x768 bf16, voxel 5 cm, a 2^27-slot voxel table, BF16 pooling and " \
             "scoring with FP32 accumulation and exact re-score near the threshold"


def run_multistory(args, torch, dev, stream, rank, cpu):
    """The Multi-story configuration: 32-frame calls along its serpentine
    path (device-resident bf16 tokens), two untimed warm-up steps, then the
    timed steps; the oracle (bf16-rounded tokens, one host core) on its first
    frames for about cpu_seconds."""
    import oracle
    import synth
    from paper_2603_03935_gb300 import DiscMap, binding
    from tests import common
    B, K, Wm = 32, args.multistory_steps, 2
    sc = synth.multistory_scene()
    cfg = common.disc_cfg(sc, voxel_capacity=1 << 27, instance_capacity=1 << 14, precision=1,
                          cuda_stream=stream.cuda_stream, device=dev.index)
    m = DiscMap(**cfg)
    stats = (binding.Stats * B)()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    times, upd, pairs, masks, cfr = [], 0, 0, 0, None
    for s in range(Wm + K):
        fr = sc.render(range(s * B, (s + 1) * B))
        if s == 0:
            cfr = fr
        a, keep = _device_frames(torch, dev, binding, sc, fr, list(range(B)), bf16=True)
        torch.cuda.synchronize()
        flush.fill_(float(s))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = m.integrate_frames_raw(a, B, stats)
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        if s >= Wm:
            times.append(e0.elapsed_time(e1))
            upd += sum(stats[j].unique_seg_voxels for j in range(B))
            pairs += sum(stats[j].overlap_pairs for j in range(B))
            masks += int(fr.num_masks.sum())
    nv, nid = m.counts()
    m.close()
    total_ms = float(np.sum(times))
    out = {"workload": MULTISTORY, "frames_per_s": K * B / (total_ms / 1e3),
           "voxel_updates_per_s": upd / (total_ms / 1e3), "frames": K * B, "first_frame": Wm * B,
           "step_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                       "mode": "one 32-frame disc_integrate_frames call"},
           "per_frame": {"voxel_updates": upd / (K * B), "overlap_pairs": pairs / (K * B), "masks": masks / (K * B)},
           "map": {"voxels": nv, "instances": nid}}
    if cpu and args.cpu_seconds > 0:
        om = oracle.OracleMap(**common.to_oracle_cfg(cfg))
        t16 = torch.from_numpy(cfr.tokens).to(torch.bfloat16).float().numpy()
        intr = (sc.fx, sc.fy, sc.cx, sc.cy)
        t0 = time.perf_counter()
        n = 0
        while n < B and (n == 0 or time.perf_counter() - t0 < args.cpu_seconds):
            om.integrate(cfr.depth[n], cfr.labels[n], t16[n], cfr.poses[n], intr, cfr.num_masks[n], report=False)
            n += 1
        dt = time.perf_counter() - t0
        model, nproc = host_cpu()
        out["cpu_baseline"] = {"value": n / dt, "unit": "frames/s", "cores": 1, "kind": "oracle", "cpu_model": model,
                               "nproc": nproc, "sample": f"frames 0..{n - 1} of the Multi-story path, fresh map"}
    return out


TINY = "Tiny: 4x4x3 m room with 4 boxes, 20 orbit frames of 64x48 (fx = fy = 50), <= 8 masks, tokens 8x6x512 " \
       "fp32, voxel 5 cm, FP32"


def run_tiny(args, torch, dev, stream, cpu):
    """The Tiny configuration: its 20 frames in one call on a fresh map,
    repeated; the oracle over the same 20 frames."""
    import oracle
    import synth
    from paper_2603_03935_gb300 import DiscMap, binding
    from tests import common
    sc = synth.tiny_scene()
    fr = sc.render(range(20))
    a, keep = _device_frames(torch, dev, binding, sc, fr, list(range(20)))
    cfg = common.disc_cfg(sc, cuda_stream=stream.cuda_stream, device=dev.index)
    stats = (binding.Stats * 20)()
    times = []
    for r in range(8):
        m = DiscMap(**cfg)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = m.integrate_frames_raw(a, 20, stats)
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        if r >= 3:
            times.append(e0.elapsed_time(e1))
        m.close()
    ms = float(np.median(times))
    out = {"workload": TINY, "frames_per_s": 20 / (ms / 1e3), "ms_per_trajectory": ms,
           "mode": "one disc_integrate_frames call of the 20 frames on a fresh map (median of 5, after 3)"}
    if cpu:
        om_t = []
        for r in range(3):
            om = oracle.OracleMap(**common.to_oracle_cfg(cfg))
            t0 = time.perf_counter()
            for i in range(20):
                om.integrate(*oracle.frame_args(fr, i), report=False)
            om_t.append(time.perf_counter() - t0)
        model, nproc = host_cpu()
        out["cpu_baseline"] = {"value": 20 / float(np.median(om_t)), "unit": "frames/s", "cores": 1, "kind": "oracle",
                               "cpu_model": model, "nproc": nproc, "sample": "the 20 frames, fresh map, median of 3"}
    return out


SERVED = "Served: {G} resident room-scale maps of mixed size (320x240..640x480, 5-60 masks, bf16 tokens, " \
         "{prec} pooling and scoring), " \
         "Poisson arrivals, integrate:query 9:1 (top-5 of 4 vectors), each map walking on along its own path " \
         "({F} frames, none taken twice), 4 client threads, frame inputs {sub}, continuous batching of up to {J} " \
         "frames per map per batch, {W} batches in flight"


def run_served(args, torch, dev, rank):
    """The served form: requests from client threads at Poisson arrival times
    into disc_server_*; p50/p99 frame latency (submission to completion) and
    completed frames/s per offered rate."""
    import threading
    from paper_2603_03935_gb300 import DiscServer, binding
    from tests import common
    G, F, J = args.served_maps, args.served_frames, 4
    scs = batched_scenes(G, 5000 + 97 * rank)
    frs = [sc.render(range(F)) for sc in scs]
    bf = []
    for sc, fr in zip(scs, frs):
        t16 = torch.from_numpy(fr.tokens).to(torch.bfloat16).view(torch.int16)
        if args.served_borrow:
            # the clients' frames sit in pinned host memory, read in place
            dp = torch.from_numpy(fr.depth).pin_memory().numpy()
            lp = torch.from_numpy(fr.labels.view(np.int16)).pin_memory().numpy().view(np.uint16)
            tp = t16.pin_memory().numpy().view(np.uint16)
        else:
            dp, lp, tp = fr.depth, fr.labels, t16.numpy().view(np.uint16)
        bf.append([binding.host_frame(dp[i], lp[i], tp[i], fr.poses[i], (sc.fx, sc.fy, sc.cx, sc.cy),
                                      fr.num_masks[i]) for i in range(F)])
    srv = DiscServer(64 << 30, max_queue=1 << 16, workers=args.served_workers, max_maps=G, frames_per_map=J,
                     embed_dim=scs[0].dim,
                     patch_h=scs[0].patch_h, patch_w=scs[0].patch_w, max_width=max(s.width for s in scs),
                     max_height=max(s.height for s in scs), max_masks=max(s.max_masks for s in scs),
                     device=dev.index)
    # the served maps score in FP8 (E4M3 embeddings with per-vector scales)
    ids = [srv.open_map(**common.disc_cfg(sc, voxel_capacity=1 << 21, instance_capacity=1 << 12,
                                          precision=args.served_precision)) for sc in scs]
    queries = [fr.tokens[0][:4] for fr in frs]
    # warm-up: every map takes its first 4 frames; the measured requests
    # then walk on along each map's path from there
    nxt = [0] * G
    for g in range(G):
        for i in range(4):
            srv.wait_frame(srv.submit_frame(ids[g], bf[g][i]))
        nxt[g] = 4
    rng = np.random.default_rng(11 + rank)
    out = []
    levels = [float(x) for x in args.served_rates.split(",") if x]
    runs = [r for r in levels for _ in range(args.served_repeats)]
    per_run = (F - 4) // len(runs)  # frames of each map per measurement: no frame is taken twice
    for rate in runs:
        # requests of this measurement: per_run frames of every map in a
        # random order of maps, one query per nine frames at random places
        # (9:1), Poisson arrivals
        which = rng.permutation(np.repeat(np.arange(G), per_run))
        qs = rng.integers(0, G, len(which) // 9)
        n = len(which) + len(qs)
        is_q = np.zeros(n, bool)
        is_q[rng.choice(n, len(qs), replace=False)] = True
        order = np.empty(n, np.int64)
        order[~is_q] = which
        order[is_q] = qs
        which = order
        gaps = rng.exponential(1.0 / (rate / 0.9), n)
        when = np.cumsum(gaps)
        plan = []
        for r in range(n):
            g = int(which[r])
            if is_q[r]:
                plan.append((when[r], g, -1))
            else:
                plan.append((when[r], g, nxt[g]))
                nxt[g] += 1
        srv.reset_stats()
        fail, newv = [], []

        def client(c):
            # client c submits the requests of maps g with g % 4 == c, so a
            # map's frames go in in the order of its path
            tk = []
            t0 = start
            for r in range(n):
                at, g, i = plan[r]
                if g % 4 != c:
                    continue
                d = t0 + at - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                if i < 0:
                    tk.append((True, srv.submit_query(ids[g], queries[g], 5)))
                elif args.served_borrow:
                    tk.append((False, srv.submit_frame_borrowed(ids[g], bf[g][i])))
                else:
                    tk.append((False, srv.submit_frame(ids[g], bf[g][i])))
            for q, t in tk:
                if q:
                    rc = srv.wait_query(t)[0]
                else:
                    st_ = srv.wait_frame(t)
                    rc = st_["rc"]
                    newv.append(st_["new_voxels"])
                if rc != 0:
                    fail.append(rc)

        start = time.perf_counter()
        th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        wall = time.perf_counter() - start
        rep = srv.stats()
        out.append({"offered_frames_per_s": rate, "frames_per_s": (rep["frames"] - len(fail)) / wall,
                    "refused": len(fail), "refused_codes": sorted(set(fail))[:5],
                    "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "frames": rep["frames"],
                    "queries": rep["queries"], "batches": rep["batches"],
                    "worker_busy": rep["busy_ms"] / (1e3 * wall * max(args.served_workers, 1)),
                    "frames_per_batch": rep["frames"] / max(rep["batches"], 1),
                    "new_voxels_per_frame": float(np.mean(newv)) if newv else 0.0})
    srv.close()
    prec = ("fp32", "bf16", "fp8 e4m3")[args.served_precision]
    # the knee: the highest offered rate whose median achieved rate keeps up
    # with 95 % of it
    knee = 0.0
    for rate in levels:
        got = [o["frames_per_s"] for o in out if o["offered_frames_per_s"] == rate]
        if got and float(np.median(got)) >= 0.95 * rate:
            knee = rate
    sub = "borrowed from pinned host memory" if args.served_borrow else "copied at submission"
    return {"workload": SERVED.format(G=G, F=F, J=J, prec=prec, W=args.served_workers, sub=sub), "rates": out, "knee_offered_frames_per_s": knee,
            "repeats": args.served_repeats}


def run_reference(args, rank):
    """The oracle, as it stands, on the host cores: same workload and metric.
    Its warm-up integrates the frames the GPU arm's warm-up steps take
    (warmup x frames-per-step, untimed); its timed steps then take
    the next frames, two per step, as a bounded sample of the frames the GPU
    arm times."""
    import oracle
    import synth
    if rank != 0:
        return
    scene = synth.room_scene(seed=replica_seed(0))
    per_step = 2
    start = args.warmup * args.frames_per_step
    n = start + args.steps * per_step
    fr = scene.render(range(n))
    m = oracle.OracleMap(**oracle.config_for_scene(scene))
    k = 0
    while k < start:
        m.integrate(*oracle.frame_args(fr, k), report=False)
        k += 1
    t0 = time.perf_counter()
    upd = 0
    for _ in range(args.steps):
        for _ in range(per_step):
            r = m.integrate(*oracle.frame_args(fr, k), report=True)
            upd += r["n_seg"]
            k += 1
    dt = time.perf_counter() - t0
    fps = args.steps * per_step / dt
    out = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded room trajectory)",
           "config": {"workload": WORKLOAD, "frames_per_step": per_step, "l2": "n/a (CPU)"},
           "voxel_updates_per_s": upd / dt,
           "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                            "cpu_model": host_cpu()[0], "nproc": host_cpu()[1],
                            "sample": f"frames {start}..{k - 1} of the Room trajectory (the first frames the GPU "
                                      f"arm times), map built through frames 0..{start - 1} untimed"},
           "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cpu_baseline(scene, fr, budget_s, start):
    """The oracle on one host core over the first frames the GPU arm times
    (from frame `start`, for about budget_s seconds), on a map built through
    frames 0..start-1 untimed."""
    import oracle
    m = oracle.OracleMap(**oracle.config_for_scene(scene))
    for i in range(start):
        m.integrate(*oracle.frame_args(fr, i), report=False)
    t0 = time.perf_counter()
    n = start
    upd = 0
    while n < len(fr) and (n == start or time.perf_counter() - t0 < budget_s):
        r = m.integrate(*oracle.frame_args(fr, n), report=True)
        upd += r["n_seg"]
        n += 1
    dt = time.perf_counter() - t0
    model, nproc = host_cpu()
    return {"value": (n - start) / dt, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "cpu_model": model, "nproc": nproc,
            "sample": f"frames {start}..{n - 1} of the Room trajectory (the first frames the GPU arm times), "
                      f"map built through frames 0..{start - 1} untimed ({upd / dt:.3g} voxel-updates/s)"}


class Watchdog:
    """Prints the line assembled so far and ends the process when the run
    outlives its budget, so that a later section that stalls (the many-map
    batched or served forms, say) cannot take the finished measurements with
    it.  Unfinished sections carry an "error" entry; without the main
    measurement nothing is printed and the exit status is 1."""

    def __init__(self, budget_s, assemble):
        self.assemble = assemble
        self.lock = threading.Lock()
        self.printed = False
        self.done = threading.Event()
        threading.Thread(target=self._run, args=(budget_s,), daemon=True).start()

    def _run(self, budget_s):
        if self.done.wait(budget_s):
            return
        with self.lock:
            if self.printed:
                return
            line = self.assemble(unfinished="did not finish within the run's %.0f s budget" % budget_s)
            if line is not None:
                print(json.dumps(line), flush=True)
                self.printed = True
        os._exit(0 if self.printed else 1)

    def emit(self, line):
        with self.lock:
            if not self.printed:
                print(json.dumps(line), flush=True)
                self.printed = True
        self.done.set()


def main():
    args = parse()
    rank, world, local = rank_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import synth
    from paper_2603_03935_gb300 import DiscMap, binding

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if not os.path.exists(binding.LIB_PATH):
        if rank == 0:
            import __graft_entry__
            __graft_entry__.build()
        if world > 1:
            dist.barrier()

    B, K, Wm = args.frames_per_step, args.steps, args.warmup
    # the line's sections as they finish (the watchdog prints what is here)
    state = {}
    SECTIONS = ("sync_calls", "dbscan", "assoc_grid", "dilation", "latency_ms", "finalize", "heatmap",
                "phases_ms_per_frame", "roofline", "roofline_critical_path", "roofline_step", "cpu_baseline", "e2e",
                "batched", "batched_same_workload", "tiny", "multistory", "served")

    def assemble(unfinished=None):
        core = state.get("core")
        if core is None:
            return None
        total_ms = core["total_ms"]
        out = {"metric": METRIC, "value": whole_job_rate(K * B, world, total_ms), "unit": "frames/s",
               "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": total_ms / K,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded room trajectory; stands in for the paper's HM3D/Replica trajectories)",
               "config": {"workload": WORKLOAD if args.precision == 0 else
                          WORKLOAD.replace(", FP32", ", %s fast pooling and scoring (fp32 tokens)" %
                                           ("BF16", "FP8 E4M3")[args.precision - 1]),
                          "frames_per_step": B, "frames_timed": K * B,
                          "batch_split": args.batch_split or "automatic",
                          "assoc_cluster": args.assoc_cluster or "automatic",
                          "geometry_chunk": args.geometry_chunk or 8,
                          "voxel_table_slots": 1 << args.table_log2,
                          "trajectory_frames": core["n_render"],
                          "l2": "flushed between timed steps (258 MB write)", "replicas": world},
               "voxel_updates_per_s": core["updates"] * world / (total_ms / 1e3),
               "new_voxels_per_s": core["new_vox"] * world / (total_ms / 1e3),
               "frame_ms_batched": total_ms / (K * B),
               "gpu_launches": int(core["launches"]),
               "clocks": core["clk"]}
        for k in SECTIONS:
            out[k] = state[k] if k in state else ({"error": unfinished} if unfinished else None)
        return out

    dog = Watchdog(args.watchdog_s, assemble) if rank == 0 and args.watchdog_s > 0 else None
    # replicas only: every rank integrates its own map of its own scene; the
    # camera path is closed, so frames past its end continue on the next lap
    scene = synth.room_scene(seed=replica_seed(rank))
    n_main = (Wm + K) * B
    n_extra = args.timing_batches * B + args.latency_frames
    n_render = min(scene.num_frames, n_main + n_extra)
    fr = scene.render(range(n_render))
    H, W_, P, D = scene.height, scene.width, scene.patch_h * scene.patch_w, scene.dim
    intr = (scene.fx, scene.fy, scene.cx, scene.cy)

    # a dedicated stream: the map enqueues on it, the timing events are
    # recorded on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    cfg = room_cfg(scene)
    cfg["voxel_capacity"] = 1 << args.table_log2
    if args.batch_frames > 0:
        cfg["batch_frames"] = args.batch_frames
    cfg["serial_sms"] = args.serial_sms
    cfg["precision"] = args.precision
    cfg["cuda_stream"] = stream.cuda_stream
    cfg["device"] = local
    depth = torch.from_numpy(fr.depth).to(dev)
    labels = torch.from_numpy(fr.labels.view(np.int16)).to(dev)
    tokens = torch.from_numpy(fr.tokens).to(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def plain_map(c):
        m = DiscMap(**c)
        if args.batch_split or args.assoc_cluster or args.geometry_chunk:
            m.set_schedule(geometry_chunk=args.geometry_chunk or 8, assoc_cluster=args.assoc_cluster,
                           batch_split=args.batch_split)
        return m

    def frame_array(lo, hi, on_device=True, host=None):
        n = hi - lo
        arr = (binding.Frame * n)()
        for j in range(n):
            i = (lo + j) % n_render
            f = arr[j]
            f.width, f.height = W_, H
            f.fx, f.fy, f.cx, f.cy = intr
            for q, v in enumerate(fr.poses[i].reshape(16)):
                f.T_world_cam[q] = float(v)
            if on_device:
                f.depth, f.labels, f.tokens = depth[i].data_ptr(), labels[i].data_ptr(), tokens[i].data_ptr()
            else:
                hd, hl, ht = host
                f.depth, f.labels, f.tokens = hd[i].data_ptr(), hl[i].data_ptr(), ht[i].data_ptr()
            f.token_dtype = 0
            f.num_masks = int(fr.num_masks[i])
            f.global_embed = None
            f.inputs_on_device = 1 if on_device else 0
        return arr

    steps = [frame_array(s * B, (s + 1) * B) for s in range(Wm + K)]
    stats = (binding.Stats * B)()

    clocks = ClockSampler(local)
    clocks.start()
    gmap = plain_map(cfg)
    for s in range(Wm):
        rc = gmap.integrate_frames_raw(steps[s], B, stats)
        assert rc == 0, rc
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    time.sleep(0.5)  # the sampler is running by now
    launches0 = gmap.kernel_launches()
    wall0 = time.time()
    # K steps, each one disc_integrate_frames_async call of B frames: a
    # step's last frames associate while the next step's per-frame kernels
    # run (two calls unfinished at most).  One timed region from before the
    # first call to the end of the last (disc_map_wait), with the L2 flush
    # enqueued between the steps inside it.
    astats = [(binding.Stats * B)() for _ in range(K)]
    adone = [ctypes.c_int32(-1) for _ in range(K)]
    ares = [ctypes.c_int32(1) for _ in range(K)]
    flush.fill_(float(Wm))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i, s in enumerate(range(Wm, Wm + K)):
        if i:
            flush.fill_(float(s))       # L2 flush between timed steps
        rc = gmap.integrate_frames_async_raw(steps[s], B, astats[i], adone[i], ares[i])
        assert rc == 0, rc
    rc = gmap.wait()
    e1.record(stream)
    e1.synchronize()
    assert rc == 0 and all(r.value == 0 for r in ares) and all(d.value == B for d in adone), rc
    updates = sum(astats[i][j].unique_seg_voxels for i in range(K) for j in range(B))
    new_vox = sum(astats[i][j].new_voxels for i in range(K) for j in range(B))
    launches = gmap.kernel_launches() - launches0
    clocks.mark(wall0, time.time())
    total_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    clk = clocks.stop()
    frames_all = K * B * world
    state["core"] = {"total_ms": total_ms, "updates": updates, "new_vox": new_vox, "launches": launches,
                     "clk": clk, "n_render": n_render}

    def variant(extra, nsteps, vsteps=None):
        """The same steps (or vsteps) on a fresh map with config changes;
        frames/s and the per-frame counters averaged."""
        steps_ = steps if vsteps is None else vsteps
        vmap = DiscMap(**dict(cfg, **extra))
        for s_ in range(Wm):
            assert vmap.integrate_frames_raw(steps_[s_], B, stats) == 0
        torch.cuda.synchronize()
        dt_ms, nf, sums = 0.0, 0, {}
        for s_ in range(Wm, Wm + min(nsteps, K)):
            flush.fill_(float(s_))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = vmap.integrate_frames_raw(steps_[s_], B, stats)
            e1.record(stream)
            e1.synchronize()
            assert rc == 0, rc
            dt_ms += e0.elapsed_time(e1)
            for j in range(B):
                for k_, v_ in stats[j].as_dict().items():
                    sums[k_] = sums.get(k_, 0) + v_
            nf += B
        vmap.close()
        return nf / (dt_ms / 1e3), nf, {k_: v_ / nf for k_, v_ in sums.items()}

    # the same steps as synchronous calls on a fresh map, each timed alone
    # (the call returns once its frames are done; L2 flushed before each)
    fps_sync, nf_sync, _ = variant({}, K)
    state["sync_calls"] = {"frames_per_s": whole_job_rate(nf_sync, world, nf_sync / fps_sync * 1e3),
                           "frames": nf_sync,
                           "mode": "one synchronous disc_integrate_frames call per step, each step timed alone"}
    # the same workload with the Sec. III-A DBSCAN filter on (eps 5 cm, 10 points)
    dbscan = None
    if args.dbscan_steps > 0:
        fps_, nf, per = variant(dict(dbscan_eps=0.05, dbscan_min_pts=10), args.dbscan_steps)
        dbscan = {"frames_per_s": fps_, "eps_m": 0.05, "min_pts": 10, "frames": nf,
                  "denoised_pixels_per_frame": per["denoised_pixels"]}
    state["dbscan"] = dbscan
    # and with a second token grid driving association (1024-dim ViT-L
    # features on a 24 x 32 patch grid, fp32), generated for the frames used
    assoc = None
    if args.assoc_steps > 0:
        import dataclasses
        A_H, A_W, A_D = 24, 32, 1024
        nsa = Wm + min(args.assoc_steps, K)
        nfa = min(nsa * B, n_render)
        sub = dataclasses.replace(fr, index=fr.index[:nfa], ids=fr.ids[:nfa])
        atok = torch.from_numpy(sub.assoc_tokens(A_H, A_W, A_D)).to(dev)
        asteps = []
        for s_ in range(nsa):
            arr = frame_array(s_ * B, (s_ + 1) * B)
            for j in range(B):
                arr[j].assoc_tokens = atok[(s_ * B + j) % nfa].data_ptr()
            asteps.append(arr)
        fps_, nf, per = variant(dict(assoc_dim=A_D, assoc_patch_h=A_H, assoc_patch_w=A_W), args.assoc_steps, asteps)
        assoc = {"frames_per_s": fps_, "frames": nf, "grid": f"{A_H}x{A_W}x{A_D} fp32",
                 "merges_per_frame": per["merges"], "new_instances_per_frame": per["new_instances"]}
        del atok
    state["assoc_grid"] = assoc

    # and with the neighbourhood overlap (26-neighbour dilation, Sec. III-B)
    dilation = None
    if args.dilation_steps > 0:
        fps_, nf, per = variant(dict(overlap_dilation=1), args.dilation_steps)
        dilation = {"frames_per_s": fps_, "frames": nf, "overlap_pairs_per_frame": per["overlap_pairs"],
                    "merges_per_frame": per["merges"], "new_instances_per_frame": per["new_instances"]}
    state["dilation"] = dilation

    # per-phase device time on the following batches (event-record nodes
    # around each phase, inside the batch's graph)
    lo = n_main
    TB = args.timing_batches
    gmap.set_phase_timing(True)
    ph_stats = (binding.Stats * (TB * B))()
    rc = gmap.integrate_frames_raw(frame_array(lo, lo + TB * B), TB * B, ph_stats)
    assert rc == 0, rc
    phases = gmap.phase_times()
    gmap.set_phase_timing(False)
    lo += TB * B

    # single-frame latency (disc_integrate_frame, one synchronisation per frame)
    lat = []
    for i in range(lo, lo + args.latency_frames):
        a = frame_array(i, i + 1)
        st1 = binding.Stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = binding.lib().disc_integrate_frame(gmap._h, a, ctypes.byref(st1))
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        lat.append(e0.elapsed_time(e1))
    state["latency_ms"] = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "frames": len(lat), "mode": "disc_integrate_frame, one frame per call"}

    # the end-of-trajectory step (orphan merge and voxel-count filter) on the
    # map the measured frames built, one synchronous call
    fin = None
    if args.finalize:
        try:
            nv_, nid_ = gmap.counts()
            torch.cuda.synchronize()
            t0_ = time.perf_counter()
            rep_ = gmap.finalize(min_voxels=100)
            fin_ms = (time.perf_counter() - t0_) * 1e3
            fin = {"ms": fin_ms, "voxels": nv_, "instances": nid_, "voxels_per_s": nv_ / (fin_ms / 1e3),
                   "min_voxels": 100, "report": rep_, "mode": "disc_map_finalize, one call, host clock"}
        except Exception as ex:  # recorded, the rest of the line stands
            fin = {"error": repr(ex)}
    state["finalize"] = fin
    gmap.close()

    # the Fig. 2 query heatmap over one Room token grid (576 x 768 fp32)
    heat = None
    if args.heatmap_calls > 0:
        try:
            from paper_2603_03935_gb300 import query_heatmap
            q_ = tokens[0][7].contiguous()
            for _ in range(3):
                query_heatmap(tokens[0], q_, stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.heatmap_calls):
                query_heatmap(tokens[0], q_, stream=stream)
            e1.record(stream)
            e1.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / args.heatmap_calls
            heat = {"us_per_call": us, "calls": args.heatmap_calls, "grid": f"{P}x{D} fp32",
                    "token_gb_per_s": P * D * 4 / (us * 1e-6) / 1e9,
                    "mode": "disc_query_heatmap calls back to back on one stream, each synchronising "
                            "(a call's latency; tokens L2-resident)"}
        except Exception as ex:
            heat = {"error": repr(ex)}
    state["heatmap"] = heat

    # the dominant single-kernel phase (most device time) and its roofline:
    # the step bytes it is credited with over its event-timed duration
    peak, peak_kind = peaks()
    per_frame = {k: v["ms"] / (TB * B) for k, v in phases.items()}
    single = ("backproject", "coverage", "pool_gemm", "pool_exact", "associate", "commit")
    dom = max(single, key=lambda k: phases[k]["ms"])
    st_list = [{k: getattr(ph_stats[j], k) for k, _ in binding.Stats._fields_} for j in range(TB * B)]
    emb_b = (4, 2, 1)[args.precision]

    def kernel_roofline(name):
        alg_total = algorithmic_bytes(name, st_list, H, W_, P, D, tok_b=4, emb_b=emb_b)
        calls = max(phases[name]["calls"], 1)
        launch_ms = phases[name]["ms"] / calls
        achieved = alg_total / (phases[name]["ms"] / 1e3) / 1e9 if phases[name]["ms"] > 0 and alg_total > 0 else 0.0
        return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": measured_traffic(name, TB * B / calls), "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_total / calls, "launch_us": launch_ms * 1e3,
                "launches_per_frame": calls / (TB * B)}

    roofline = kernel_roofline(dom)
    # the stateless kernel with the most event time: with asynchronous calls
    # the frame chain runs beside the stateless kernels, which set the pace
    crit = max(("backproject", "coverage", "pool_gemm", "pool_exact"), key=lambda k: phases[k]["ms"])
    state["roofline_critical_path"] = kernel_roofline(crit)
    # the whole step against the same peak: algorithmic bytes per frame (mean
    # over the phase-timed frames) times the frames/s of the timed steps
    bpf = float(np.mean([step_bytes(x, H, W_, P, D, tok_b=4, emb_b=emb_b) for x in st_list]))
    rate = whole_job_rate(K * B, world, total_ms)
    state["roofline_step"] = {"bytes_per_frame": bpf, "frames_per_s": rate, "achieved": bpf * rate / 1e9,
                              "peak": peak, "unit": "GB/s", "frac": bpf * rate / 1e9 / peak, "peak_kind": peak_kind}
    state["phases_ms_per_frame"] = {k: round(v, 5) for k, v in per_frame.items()}
    state["roofline"] = roofline
    # the oracle on the host cores (GPU idle meanwhile), before the sections
    # that follow
    state["cpu_baseline"] = cpu_baseline(scene, fr, args.cpu_seconds, Wm * B) if rank == 0 and world == 1 else None

    # end to end through the C ABI with pinned host buffers (H2D inside)
    def run_e2e():
        hd = torch.from_numpy(fr.depth).pin_memory()
        hl = torch.from_numpy(fr.labels.view(np.int16)).pin_memory()
        ht = torch.from_numpy(fr.tokens).pin_memory()
        hsteps = [frame_array(s * B, (s + 1) * B, on_device=False, host=(hd, hl, ht)) for s in range(Wm + K)]
        # one asynchronous call per step, as the plain line: the H2D copies
        # of a step's inputs (pinned host memory) and the read-back of its
        # counters are inside the timed region, and overlap the kernels of
        # the step before
        m1 = plain_map(cfg)
        for s in range(Wm):
            assert m1.integrate_frames_raw(hsteps[s], B, stats) == 0
        hst = [(binding.Stats * B)() for _ in range(K)]
        hdone = [ctypes.c_int32(-1) for _ in range(K)]
        hres = [ctypes.c_int32(1) for _ in range(K)]
        torch.cuda.synchronize()
        flush.fill_(float(Wm))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, s in enumerate(range(Wm, Wm + K)):
            if i:
                flush.fill_(float(s))
            rc = m1.integrate_frames_async_raw(hsteps[s], B, hst[i], hdone[i], hres[i])
            assert rc == 0, rc
        rc = m1.wait()
        e1.record(stream)
        e1.synchronize()
        assert rc == 0 and all(r.value == 0 for r in hres) and all(d.value == B for d in hdone), rc
        async_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        m1.close()
        # the same steps as synchronous calls, each timed alone
        m2 = plain_map(cfg)
        for s in range(Wm):
            assert m2.integrate_frames_raw(hsteps[s], B, stats) == 0
        torch.cuda.synchronize()
        et = []
        for s in range(Wm, Wm + K):
            flush.fill_(float(s))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = m2.integrate_frames_raw(hsteps[s], B, stats)
            e1.record(stream)
            e1.synchronize()
            assert rc == 0, rc
            et.append(e0.elapsed_time(e1))
        # the same K steps as one call (a trajectory handed over at once): the
        # copies of batch b + 1 overlap the kernels of batch b
        m2.close()
        m3 = plain_map(cfg)
        for s in range(Wm):
            assert m3.integrate_frames_raw(hsteps[s], B, stats) == 0
        allf = frame_array(Wm * B, (Wm + K) * B, on_device=False, host=(hd, hl, ht))
        allst = (binding.Stats * (K * B))()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = m3.integrate_frames_raw(allf, K * B, allst)
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        traj_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        m3.close()
        e2e_ms = max_over_ranks(float(np.sum(et)), world, dev)
        e2e = {"value": whole_job_rate(K * B, world, async_ms), "unit": "frames/s",
               "h2d_bytes_per_step": B * (H * W_ * 6 + P * D * 4),
               "d2h_bytes_per_step": B * 96 + 8,  # per frame its 96-byte counters, and the map's voxel count
               "calls": "one disc_integrate_frames_async call per step (32 frames) from pinned host buffers, "
                        "disc_map_wait after the last; one timed region",
               "sync_calls": {"value": whole_job_rate(K * B, world, e2e_ms), "unit": "frames/s",
                              "mode": "one synchronous disc_integrate_frames call per step, each timed alone",
                              "call_ms": {"p50": float(np.median(et)), "min": float(np.min(et)),
                                          "max": float(np.max(et))}},
               "one_call_trajectory": {"value": whole_job_rate(K * B, world, traj_ms), "unit": "frames/s",
                                       "frames": K * B}}
        return e2e

    # (with several ranks a failure would leave the others in a collective: not caught there)
    state["e2e"] = None if args.no_e2e else (guarded("e2e", run_e2e) if world == 1 else run_e2e())

    # the batched and served forms last: their many maps and threads come
    # after every single-map measurement
    # (no collective inside them: a failure is recorded and the other ranks go on)
    state["batched"] = (guarded("batched", lambda: run_batched(args, torch, dev, stream, rank))
                        if args.batched_maps > 0 else None)
    state["batched_same_workload"] = (
        guarded("batched_same_workload", lambda: run_same_workload_batched(args, torch, dev, stream, rank))
        if args.same_maps > 0 else None)
    state["tiny"] = (guarded("tiny", lambda: run_tiny(args, torch, dev, stream, rank == 0 and world == 1))
                     if args.tiny else None)
    state["multistory"] = (
        guarded("multistory", lambda: run_multistory(args, torch, dev, stream, rank, rank == 0 and world == 1))
        if args.multistory_steps > 0 else None)
    state["served"] = guarded("served", lambda: run_served(args, torch, dev, rank)) if args.served_maps > 0 else None

    if rank == 0:
        line = assemble()
        if dog is not None:
            dog.emit(line)
        else:
            print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
