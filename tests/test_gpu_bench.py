"""bench.py's one JSON line on a GB300: a short run (2 timed steps after 3
warm-up steps, no autotuning, no configs block) must print every key of the
line's contract, with values that agree with each other."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = K = 16384


def test_bench_line_carries_its_contract():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "2", "--warmup", "3", "--no-tune",
                        "--no-configs"], cwd=ROOT, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 3)
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["device_status"] == 0
    # whole-job effective n^2 k GOPS from the timed step
    assert line["value"] == pytest.approx(N * N * K / (line["ms_per_step"] * 1e-3) / 1e9, rel=1e-9)
    assert "workload" in line["config"]
    rf = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in rf, key
    assert rf["bound"] == "tensor" and rf["unit"] == "TFLOP/s"
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert 0.2 < rf["frac"] < 1.5          # a real leaf rate, not an empty kernel
    assert rf["traffic"] > 0
    # the leaf's launches inside the timed steps: five products per step
    assert rf["launches"] == 5 * line["steps"]
    assert line["gpu_launches"] >= rf["launches"]
    e2e = line["e2e"]
    assert e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == N * K * 4
    assert e2e["d2h_bytes_per_step"] > 0
    assert e2e["ms_per_step"] > line["ms_per_step"] * 0.9   # copies are inside its region
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
    assert line["clocks"]["sm_max_mhz"] is None or line["clocks"]["sm_max_mhz"] > 0
