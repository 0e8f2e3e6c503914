"""bench.py --impl reference (the oracle timed on the host) on a small sample: one JSON
line with the contract's keys on rank 0, nothing on other ranks.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--p", "3", "--n", "4", "--cpu-sample-s", "0.5"]
    return subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # a step is the bounded sample: its wall time, not the extrapolated solve time
    assert 0 < d["ms_per_step"] < 120e3
    assert abs(d["extrapolated_solve_s"] * d["value"] - 1.0) < 1e-12


def test_reference_arm_other_ranks_print_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


def test_all_cores_cpu_baseline_sums_concurrent_samples():
    """run_cpu_leg_all_cores: one single-threaded oracle sample per process, run together;
    the reported throughput is the sum of the per-process rates (replica semantics)."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.run_cpu_leg_all_cores(2, 3, 0.3, 20, 2)
    one = bench.run_cpu_leg(2, 3, 0, 0.3, 20)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0
    assert 0.5 / one["solve_s"] < r["value"] < 4.0 / one["solve_s"], (r["value"], 1.0 / one["solve_s"])
