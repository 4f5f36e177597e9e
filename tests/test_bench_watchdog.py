"""The benchmark's watchdog on the CPU (child processes, since it ends the
process): a run that outlives its budget prints the sections it finished,
the rest marked unfinished, and exits 0; without the main measurement it
prints nothing and exits 1; a run that finishes first prints exactly one
line; a section that raises is recorded as an error entry."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, time
sys.path.insert(0, %r)
import bench
mode = sys.argv[1]
def assemble(unfinished=None):
    if mode == "nocore":
        return None
    return {"value": 1.0, "served": {"error": unfinished} if unfinished else {"p99_ms": 1.0}}
dog = bench.Watchdog(0.3, assemble)
if mode == "finish":
    dog.emit(assemble())
time.sleep(3.0)
print("still here")
"""


def _run(mode):
    p = subprocess.run([sys.executable, "-c", SCRIPT % ROOT, mode], capture_output=True, text=True, timeout=60)
    return p.returncode, [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_budget_passed_prints_finished_sections():
    rc, lines = _run("stall")
    assert rc == 0 and len(lines) == 1
    d = json.loads(lines[0])
    assert d["value"] == 1.0 and "budget" in d["served"]["error"]


def test_no_main_measurement_prints_nothing():
    rc, lines = _run("nocore")
    assert rc == 1 and lines == []


def test_finished_run_prints_once():
    rc, lines = _run("finish")
    assert rc == 0 and len(lines) == 2 and json.loads(lines[0]) == {"value": 1.0, "served": {"p99_ms": 1.0}}
    assert lines[1] == "still here"


def test_a_failing_section_is_recorded_and_the_line_goes_on():
    sys.path.insert(0, ROOT)
    import bench

    def boom():
        raise RuntimeError("section failed")

    assert bench.guarded("served", lambda: {"p99_ms": 1.0}) == {"p99_ms": 1.0}
    out = bench.guarded("served", boom)
    assert set(out) == {"error"} and "section failed" in out["error"]
