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
    r = bench.roofline_tc(n, s, kp, 0.05843, 0.06485, 0.08281, 5514.3, {"hbm_gbs": 6791.0}, 271159808, 20)
    json.dumps(r)  # one JSON line
    alg = 8 * n * n + 16 * n * kp  # FP64 A once, P in, A P out
    assert r["algorithmic_bytes"] == alg and r["digit_stream_bytes"] == 16 * n * n + 16 * n * kp
    assert r["algorithmic_flops"] == 2 * n * n * s
    assert r["achieved"] == pytest.approx(alg / 0.05843e-3 / 1e9, rel=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / 6791.0, abs=1e-4)
    assert r["frac"] == pytest.approx(0.3435, abs=1e-3)
    # the 16-byte digit stream the kernel reads: twice the algorithmic bytes
    assert r["digit_stream_gbs"] == pytest.approx(2 * r["achieved"], rel=0.01)
    assert r["digit_stream_frac_of_read_ceiling"] == pytest.approx(0.8397, abs=1e-3)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6791.0 and r["traffic"] == 271159808
    assert r["product_call_frac"] == pytest.approx(alg / 0.08281e-3 / 1e9 / 6791.0, abs=1e-4)
    assert bench.roofline_tc(n, s, kp, 0.05843, 0.06485, 0.08281, 5514.3, {}, None, 20)["peak_note"] == "fallback"
