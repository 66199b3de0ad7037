"""The benchmark's own arm on a GB300, on the small workload with every
section but the single-stream one switched off: one JSON line whose keys,
units and internal arithmetic follow the result contract."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_own_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--workload", "tiny", "--steps", "20", "--warmup", "3",
                        "--e2e-steps", "10", "--cpu-sample", "4096", "--cpu-budget-s", "3",
                        "--batch-rounds", "0", "--serve", "0", "--fov-reps", "0", "--reproj-steps", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks", "resolve_error", "first_pass"):
        assert k in d, k
    assert d["unit"] == "ms/frame" and d["higher_is_better"] is False and d["n_gpus"] == 1
    assert d["steps"] == 20 and d["warmup"] == 3 and d["gpu_launches"] == 20
    assert d["value"] > 0 and abs(d["ms_per_step"] - d["value"]) < 1e-3
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    e = d["e2e"]
    assert e["unit"] == "ms/frame" and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 256 * 256 * 12
    assert d["resolve_error"]["within_tolerance"] is True
    # the timed frames sit in a fixed window of stream ages whatever --steps is
    assert d["first_pass"]["frames"] == 8 and d["stream_age_frames"] == "8..27"
    assert d["config_240_frame_mean_ms"] == d["first_pass"]["ms_per_frame_1_to_end"]
    assert d["cpu_baseline"]["single_thread"]["cores"] == 1
    assert d["cpu_baseline"]["single_thread"]["value"] > 0
    assert d["precision"] is None  # the FP16 form is timed beside the 4k workload only
