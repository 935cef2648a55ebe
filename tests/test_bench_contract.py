"""The benchmark's output contract on the CPU: the reference arm (the CPU
oracle) prints one JSON line with every key the benchmark line carries, and
the DRAM traffic of a step kernel is reported only for the kernel, workload
and kernel sources it was captured on."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def test_reference_arm_prints_one_json_line(oracle_mod):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert KEYS <= set(out), KEYS - set(out)
    assert out["impl"] == "reference" and out["metric"] == "2-species MLUPS" and out["unit"] == "MLUPS"
    assert out["value"] > 0 and out["higher_is_better"] is True and out["steps"] == 2 and out["warmup"] == 1
    # the oracle on every host core (its OpenMP row loops; 1 without OpenMP)
    assert out["cpu_baseline"]["kind"] == "oracle" and 1 <= out["cpu_baseline"]["cores"] <= (os.cpu_count() or 1)
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]
    assert out["config"]["workload"] == "laplace_sweep_24"


def test_traffic_is_keyed_by_kernel_workload_and_sources():
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        entries = json.load(f)
    sha = bench.kernel_source_sha1()
    for e in entries:
        got = bench.kernel_traffic(e["workload"], e["kernel"])
        current = [d for d in entries if d["workload"] == e["workload"] and d["kernel"] == e["kernel"]
                   and d["kernel_source_sha1"] == sha]
        if current:
            assert got == float(current[0]["bytes_per_launch"])
        else:
            assert got is None
    e = entries[0]
    assert bench.kernel_traffic("no_such_workload", e["kernel"]) is None
    assert bench.kernel_traffic(e["workload"], "k_collide<float, 4>") is None
