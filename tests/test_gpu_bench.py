"""bench.py's JSON line on the 20^3 patch: the keys every run reports, the
roofline, end-to-end and CPU-baseline objects, and the FP64 main path rated
against the FP64 FMA rate (not the FP32 peak)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bench_line_mixed():
    n = 20 ** 3
    line = _bench("--config", "c1", "--steps", "3", "--warmup", "3", "--fp64-steps", "1", "--e2e-steps", "2",
                  "--mode-steps", "1")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline",
              "roofline_pair_sum", "e2e", "cpu_baseline", "fp64_path", "other_pair_mode", "phase_ms_per_step"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["config"]["particles"] == n and "workload" in line["config"]
    assert line["gpu_launches"] >= 3 * 10
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(line["clocks"])
    r = line["roofline"]
    assert r["bound"] in ("hbm", "alu") and r["peak"] > 0 and r["achieved"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-9 * r["frac"]
    m = line["roofline_pair_sum"]
    assert m["bound"] == "alu" and m["flops_per_pair"] == 70 and m["peak"] > m["peak_fma_measured"] * 0.9
    e = line["e2e"]
    # the whole state in and out every step: 13 fields, the permutation, the dt state
    assert e["value"] > 0 and e["steps"] == 2
    assert e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] >= (13 * 8 + 4) * n
    c = line["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["sample"]
    f = line["fp64_path"]["roofline_pair_sum"]
    assert f["kernel"] == "k_momentum_fp64" and f["flops_per_pair"] == 56


def test_bench_line_fp64_main_path():
    line = _bench("--config", "c1", "--precision", "fp64", "--steps", "3", "--no-cpu", "--e2e-steps", "0",
                  "--mode-steps", "0", "--fp64-steps", "0")
    assert line["dtype"] == "f64"
    m = line["roofline_pair_sum"]
    assert m["kernel"] == "k_momentum_fp64" and m["flops_per_pair"] == 56
    assert m["peak"] == m["peak_fma_measured"] and m["peak"] < 10.0   # TFLOP/s: the FP64 rate
    assert abs(m["frac"] - m["achieved"] / m["peak"]) <= 1e-9 * m["frac"]
