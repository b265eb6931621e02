"""bench.py's native arm on a GPU: one JSON line with the contract's keys and
sane values (small grid; the extras run at their own sizes)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_native_bench_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--grid", "1024",
                        "--euler-steps", "40", "--steps", "2", "--warmup", "3",
                        "--no-cpu-baseline"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "clocks", "gpu_launches"):
        assert key in line, key
    assert line["value"] > 0 and line["n_gpus"] == 1 and line["steps"] == 2
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    rf = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in rf, key
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] < 2
    e2e = line["e2e"]
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in e2e, key
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    clk = line["clocks"]
    for key in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert key in clk, key
    # the launches it claims: 40 steps of the single-step kernel plus 200 seeds and one
    # health check per bench step
    assert line["gpu_launches"] == 2 * (40 + 200 + 1)
    for key in ("temporal_blocking_gcups", "storage_modes_gcups", "batch_sweep", "serving",
                "serving_loaded", "render"):
        assert key in line, key
    assert line["serving"]["frames"] == 64 * 100 and line["serving"]["p99_ms"] > 0
    ld = line["serving_loaded"]
    assert ld["frames"] == 64 * 180 and ld["peak_sessions"] == 64 and ld["p99_ms"] > 0
    sw = line["batch_sweep"]
    assert sw["gcups_healthy_grids_only"] <= sw["gcups"]
    assert set(sw["first_bad"]) == {str(i) for i in sw["unhealthy_grids"]}
    assert set(line["temporal_blocking_gcups"]) == {str(k) for k in range(1, 9)}
