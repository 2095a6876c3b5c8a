"""Host-side arithmetic of the benchmark's roofline lines (no GPU)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_uneven_class_roofline(bench):
    # 3 instances, k = 60/100/80: flops 2mn(240), A's bf16 copy once per
    # iteration for k_max = 100 iterations -> AI = 240 / 100 = 2.4 flop/B
    m, n = 1120, 3072
    r = bench.uneven_class_roofline(m, n, [60, 100, 80], 0.05, 1887.9, 6780.0)
    assert r["instances"] == 3 and r["k_max"] == 100
    assert r["ai_flop_per_byte"] == pytest.approx(2.4)
    assert r["tflops"] == pytest.approx(2.0 * m * n * 240 / 0.05 / 1e12)
    assert r["bound"] == "hbm" and r["roof_tflops"] == pytest.approx(2.4 * 6.78)
    assert r["frac"] == pytest.approx(r["tflops"] / r["roof_tflops"])
    assert r["a_stream_gbs"] == pytest.approx(2.0 * m * n * 100 / 0.05 / 1e9)
    # above the ridge the tensor peak bounds it
    t = bench.uneven_class_roofline(64, 64, [10] * 1000, 1.0, 100.0, 6780.0)
    assert t["bound"] == "tensor" and t["roof_tflops"] == 100.0
