"""The JSON line of bench.py's reference arm (the oracle timed on the host),
run end to end on the CPU: one line on stdout with the keys and types the
benchmark contract names, the metric of the GPU arm, and a cpu_baseline and
e2e describing the same run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "pr1", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key, kind in [("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                      ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                      ("dtype", str), ("data", str), ("impl", str), ("config", dict), ("cpu_baseline", dict),
                      ("e2e", dict)]:
        assert isinstance(d[key], kind), key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["metric"] == "points/s (displace+render)" and d["unit"] == "points/s" and d["higher_is_better"]
    assert d["vs_baseline"] is None
    assert d["config"]["workload"] == "pr1_65536pts_512x512"
    assert d["value"] > 0 and abs(d["value"] - 2 * 65536 / (2 * d["ms_per_step"] / 1e3)) < 1e-6 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["value"] == d["value"] and cb["kind"] == "oracle" and cb["cores"] == 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
