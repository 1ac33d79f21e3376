"""Host-side arithmetic of bench.py that otherwise runs only on a GPU: the roofline of the
tensor-core product, from a fixed set of timings (no GPU)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_roofline_tc_counts_fp64_a_as_the_algorithmic_bytes():
    import bench
    n, s, kp = 4096, 32, 32
    r = bench.roofline_tc(n, s, kp, 0.04338, 0.0498, 0.0666, 5514.3, {"hbm_gbs": 6791.0}, 136314880, 20)
    json.dumps(r)  # one JSON line
    alg = 8 * n * n + 16 * n * kp  # FP64 A once, P in, A P out
    assert r["algorithmic_bytes"] == alg
    assert r["algorithmic_flops"] == 2 * n * n * s
    assert r["achieved"] == pytest.approx(alg / 0.04338e-3 / 1e9, rel=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / 6791.0, abs=1e-4)
    assert r["frac"] == pytest.approx(0.4627, abs=1e-3)
    assert r["frac_of_read_ceiling"] == pytest.approx(r["achieved"] / 5514.3, abs=1e-4)
    assert r["fp64_equiv_tflops"] == pytest.approx(2 * n * n * s / 0.04338e-3 / 1e12, abs=1e-3)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6791.0 and r["traffic"] == 136314880
    assert r["product_call_frac"] == pytest.approx(alg / 0.0666e-3 / 1e9 / 6791.0, abs=1e-4)
    assert bench.roofline_tc(n, s, kp, 0.04338, 0.0498, 0.0666, 5514.3, {}, None, 20)["peak_note"] == "fallback"
