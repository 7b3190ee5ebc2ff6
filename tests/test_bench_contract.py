"""The bench's JSON line contract, checked on the CPU through its reference
arm (the FP64 oracle timed on the host, which needs no GPU): one JSON line
with the keys the contract names, the oracle's own values in cpu_baseline,
and an e2e object with zero copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert "workload" in d["config"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_file_is_read_only_for_the_current_kernel_source():
    """profiles/traffic.json holds read + write bytes per captured launch;
    bench.py reports them only while the stream-collide source still hashes
    to the capture's source_sha."""
    sys.path.insert(0, ROOT)
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for st, e in d["lb_kernel"].items():
        assert e["traffic_bytes_per_launch"] == e["read_bytes"] + e["write_bytes"]
        got = bench.ncu_traffic(st)
        if e["source_sha"] == bench.lb_source_sha():
            assert got == e["traffic_bytes_per_launch"]
        else:
            assert got is None
    assert bench.ncu_traffic("no-such-storage") is None


def test_in_step_reduction_of_traced_steps():
    """bench.in_step: each kernel's time is its first start to its end (the
    next kernel's first start), medians over steps; the membrane share is
    the traced span minus the stream-collide kernel."""
    sys.path.insert(0, ROOT)
    import bench
    names = ("force", "spread", "lb", "interp", "vc")

    def step(starts, end):
        ends = list(starts[1:]) + [end]
        return {k: {"first_start_us": s, "median_start_us": s, "last_start_us": s, "end_us": e, "warps": 4}
                for k, s, e in zip(names, starts, ends)}

    tr = [step((0.0, 8.0, 16.0, 48.0, 54.0), 60.0), step((0.0, 9.0, 17.0, 50.0, 57.0), 64.0),
          step((0.0, 8.5, 16.5, 49.0, 55.0), 61.0)]
    out = bench.in_step(tr)
    assert out["steps"] == 3
    assert out["force"] == 8.5 and out["spread"] == 8.0 and out["lb"] == 32.5
    assert out["interp"] == 6.0 and out["vc"] == 6.0
    assert out["span"] == 61.0
    assert out["membrane"] == 61.0 - 32.5


def test_whole_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_mlups(2_000_000, 100, 100.0, 1) == 2000.0
    assert bench.whole_job_mlups(2_000_000, 100, 100.0, 4) == 8000.0
