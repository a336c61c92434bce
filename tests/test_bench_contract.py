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


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_is_reported_only_for_the_kernel_source_it_was_measured_on(tmp_path, monkeypatch):
    """The roofline's `traffic` comes from a committed ncu figure only when
    that figure was taken on the same step-kernel source, tile and schedule;
    otherwise the line reports null."""
    b = _bench_module()
    os.makedirs(tmp_path / "profiles")
    entry = {"kernel_hash": "h-current", "tile": [64, 8], "schedule": "waves",
             "dram_bytes_per_launch": 123}
    stale = dict(entry, kernel_hash="h-old", dram_bytes_per_launch=456)
    with open(tmp_path / "profiles" / "ncu_traffic.json", "w") as f:
        json.dump({"wl": [stale, entry]}, f)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "_kernel_hash", lambda: "h-current")
    assert b._traffic("wl", [64, 8], "waves") == 123
    assert b._traffic("wl", [64, 8], "shares") is None
    assert b._traffic("wl", [64, 16], "waves") is None
    assert b._traffic("other", [64, 8], "waves") is None
    monkeypatch.setattr(b, "_kernel_hash", lambda: "h-new")
    assert b._traffic("wl", [64, 8], "waves") is None


def test_committed_traffic_entries_name_their_kernel_and_command():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    for entries in d.values():
        for e in entries:
            assert len(e["kernel_hash"]) == 16 and e["dram_bytes_per_launch"] > 0
            assert e["schedule"] in ("waves", "shares") and len(e["tile"]) == 2
            assert e["source"].startswith("ncu ") and "--clock-control none" in e["source"]
