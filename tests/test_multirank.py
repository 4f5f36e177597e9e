"""The benchmark's multi-rank path on the CPU: two gloo ranks (replicas, no
data-path collective) meet only for the max-over-ranks timing; the job rate
counts every rank's frames over the slowest rank's time; the oracle arm runs
on rank 0 alone."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_env()
    local_ms = 100.0 + 50.0 * rank
    mx = bench.max_over_ranks(local_ms, w, torch.device("cpu"))
    rate = bench.whole_job_rate(320, w, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, mx, rate, bench.replica_seed(r)))


def test_two_gloo_ranks_max_time_and_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert all(o[3] == 150.0 for o in out)                    # the slowest rank's time
    assert all(abs(o[4] - 640 / 0.150) < 1e-9 for o in out)  # 2 x 320 frames over it
    assert out[0][5] != out[1][5]                             # each replica its own scene


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    args = bench.parse()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=1)
    assert buf.getvalue() == ""


def test_reference_arm_prints_one_contract_line(monkeypatch):
    # the oracle arm on rank 0: one JSON line with the contract's keys, the
    # oracle timed on the host cores (its cpu_baseline is the line's own value)
    import json
    import bench
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    args = bench.parse()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=0)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_byte_model_of_the_dominant_kernel():
    # the numerator of the benchmark's rooflines: per frame, depth (fp32) and
    # labels (u16) once, the token grid once, 12 B per unique (segment, voxel)
    # probe, 12 B per new voxel, one instance embedding per scored pair and
    # one fp32 embedding per adopted segment; each phase is credited with its
    # part; scratch (hash slots, lists) is not counted
    import bench
    H, W, P, D = 480, 640, 576, 768
    sts = [{"unique_seg_voxels": 20000, "new_voxels": 7000, "overlap_pairs": 30, "scored_pairs": 12,
            "embedding_copies": 2},
           {"unique_seg_voxels": 18000, "new_voxels": 6000, "overlap_pairs": 25, "scored_pairs": 9,
            "embedding_copies": 0}]
    assert bench.algorithmic_bytes("backproject", sts, H, W, P, D) == 2 * 6 * H * W
    assert bench.algorithmic_bytes("token_stats", sts, H, W, P, D) == 2 * 4 * P * D
    assert bench.algorithmic_bytes("pool_gemm", sts, H, W, P, D, tok_b=2) == 2 * 2 * P * D
    assert bench.algorithmic_bytes("lookup", sts, H, W, P, D) == 12 * (20000 + 18000)
    assert bench.algorithmic_bytes("associate", sts, H, W, P, D, emb_b=1) == D * (12 + 9) + 4 * D * 2
    assert bench.algorithmic_bytes("commit", sts, H, W, P, D) == 12 * (7000 + 6000)
    assert bench.algorithmic_bytes("entries", sts, H, W, P, D) == 0.0
    assert bench.algorithmic_bytes("entries", sts, H, W, P, D, lookup_in_entries=True) == 12 * (20000 + 18000)
    assert bench.algorithmic_bytes("union", sts, H, W, P, D) == 0.0
    # the step: the sum of the parts, each datum once
    total = bench.step_bytes(sts[0], H, W, P, D)
    assert total == 6 * H * W + 4 * P * D + 12 * 20000 + 12 * 7000 + 4 * D * 12 + 4 * D * 2
    parts = sum(bench.algorithmic_bytes(ph, sts[:1], H, W, P, D)
                for ph in ("backproject", "token_stats", "lookup", "associate", "commit"))
    assert parts == total
