"""Host-side logic of bench.py that otherwise runs only on a GPU, checked without one: the roofline
of the tensor-core product from a fixed set of timings, the clock record of the timed region, and
the rule that drops a recorded DRAM traffic figure once its kernel's sources change."""
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


def test_clock_summary_reads_the_throttle_reasons():
    """The clock record of the timed region: median SM clock, the maximum, and every throttle reason
    that was active in any sample (the lines are nvidia-smi's CSV, fields as ClockSampler asks)."""
    import bench
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1401.2, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = bench.ClockSampler.summary(cs)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    cs.lines = []
    assert bench.ClockSampler.summary(cs) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_recorded_traffic_is_dropped_when_the_kernel_sources_change(tmp_path, monkeypatch):
    """A DRAM traffic figure taken by ncu is reported only while the sources it was taken from are
    unchanged (their hash is stored beside it); any edit to one of them makes it null."""
    import bench
    csrc = tmp_path / "paper_2608_07327_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES["k_dense_tc"]:
        (csrc / f).write_text("// " + f + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("k_dense_tc")
    assert h == bench.kernel_source_hash("k_dense_tc") and len(h) == 16
    rec = tmp_path / "traffic.json"
    rec.write_text(json.dumps({"k_dense_tc:dense4096:s32": {"dram_bytes_per_launch": 123, "source_hash": h}}))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(rec))
    assert bench.recorded_traffic("k_dense_tc", "dense4096", 32) == 123
    assert bench.recorded_traffic("k_dense_tc", "dense4096", 16) is None  # no record for that width
    (csrc / bench.KERNEL_SOURCES["k_dense_tc"][-1]).write_text("// changed\n")
    assert bench.kernel_source_hash("k_dense_tc") != h
    assert bench.recorded_traffic("k_dense_tc", "dense4096", 32) is None

