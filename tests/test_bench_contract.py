"""The benchmark's reference arm on CPU: one JSON line with the keys the
benchmark contract names (metric, value, unit, steps, warmup, scaling, the
CPU baseline description and an end-to-end entry), on a small grid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
         "--nt", "6", "--steps", "1", "--warmup", "0", "--ref-seconds", "0.5"],
        capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("acoustic 24^3 SO8")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
    # a bench step of this arm is the timed sample itself, not an extrapolation
    assert 0 < d["ms_per_step"] < 600_000
    if not os.environ.get("OMP_NUM_THREADS"):
        assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert "measured time" in d["cpu_baseline"]["sample"]
