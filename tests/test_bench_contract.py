"""The benchmark's JSON contract and per-unit work on CPU: the reference arm
(the FP64 oracle on the host cores) prints one line whose baseline block
describes that same run, and the work counts behind the rooflines match their
closed forms."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, check=True,
                         timeout=600, cwd=ROOT)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    for k in ("metric", "value", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["config"]["workload"] and d["unit"] == "frames/s" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"]
    assert cb["cores"] == len(os.sched_getaffinity(0))          # every host core the process may use
    assert "2 timed steps after 1 warm-up" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # one colour of each sweep per step: two colours of 28-40 positions on this recipe
    assert 56 <= d["frames_per_step"] <= 80
    assert d["value"] == pytest.approx(d["frames_per_step"] / (d["ms_per_step"] / 1e3), rel=1e-9)


def test_work_per_position_and_peak():
    import bench
    n, M, p, r = 128, 32, 16, 13
    # full sweep: 2-D FFT and its adjoint (5 N log2 N per length-N transform, 2n of them each way)
    # plus 26 flops of element-wise work per pixel
    assert bench.flops_full_position(n) == 2 * 2 * n * 5 * n * math.log2(n) + 26 * n * n
    assert bench.flops_full_position(n) == pytest.approx(2.72e6, rel=2e-3)
    # 2 (n + M) (4 n r + 5 r p log2 p + 8 M r) + 14 n^2 + 12 M^2
    assert bench.flops_pft_position(n, M, p, r) == 2 * (n + M) * (4 * n * r + 5 * r * p * 4 + 8 * M * r) + 14 * n * n + 12 * M * M
    assert bench.flops_pft_position(n, M, p, r) == pytest.approx(4.77e6, rel=1e-3)
    # the derived FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz
    assert bench.alu_peak_tflops() == pytest.approx(80.54784, rel=1e-12)
