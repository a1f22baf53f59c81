"""Host-side pieces of bench.py, without a GPU: the reference arm's band sizing and the JSON
line it prints (the FP64 oracle on the small workload)."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_band_rows():
    b = _bench()
    # ample time: capped at 1/8 of the rows (384 / 8 = 48), a multiple of the unit
    assert b.reference_band_rows(384, 4, 1e-4, 25) == 48
    # one unit of rows takes too long for the step count: never fewer than one unit
    assert b.reference_band_rows(384, 4, 1.0, 1005) == 4
    # in between: budget / steps / seconds per unit = 120 / 60 / 0.25 = 8 units
    assert b.reference_band_rows(384, 4, 0.25, 60) == 32
    # small images: the 1/8 cap never goes below 8 rows
    assert b.reference_band_rows(96, 4, 1e-4, 1) == 8
    for args in ((384, 4, 0.01, 30), (96, 2, 0.05, 7), (1080, 4, 0.3, 1000)):
        rows = b.reference_band_rows(*args)
        assert rows % args[1] == 0 and args[1] <= rows <= max(8, args[0] // 8)


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_default_launch_mode_and_traced_steps(monkeypatch):
    """No flags: the step is replayed as a CUDA graph and the per-kernel events are recorded on
    every 10th timed step; --direct and --trace-every change both."""
    b = _bench()
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = b.parse()
    assert a.graph and not a.direct and a.trace_every == 10 and a.steps >= 20 and a.warmup >= 3
    monkeypatch.setattr(sys, "argv", ["bench.py", "--direct", "--trace-every", "1"])
    a = b.parse()
    assert not a.graph and a.trace_every == 1
