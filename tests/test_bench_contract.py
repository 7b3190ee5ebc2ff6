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
