"""bench.py's reference arm (the oracle timed on the host cores) keeps the JSON contract
of the bench line, on the CPU: each step one restart cycle of the oracle's own solve, the
value the mean cycle time times the cycle count that solve took (measured in the same run)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--grid", "40"], capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    cycles = d["config"]["cycles_per_solve"]
    assert d["value"] > 0 and d["steps"] == 1 and cycles >= 1
    assert abs(d["value"] - d["ms_per_step"] * cycles) <= 1e-9 * d["value"]
    # the whole solve was measured in the same run: its time and the scaled cycle time agree
    assert 0.5 < d["config"]["whole_solve_ms"] / d["value"] < 2.0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("3-D convection-diffusion 40^3")
