"""Host-side pieces of the benchmark that need no GPU: the roofline denominators and the
per-launch traffic table keyed by the kernel sources."""
from __future__ import annotations

import hashlib
import os

import pytest

import bench

PEAKS = {"hbm_gbs": 6794.5, "bf16_tflops": 1906.9, "bf16_tflops_sustained": 1697.7, "source": "measured"}


def test_tensor_peak_burst_and_sustained():
    assert bench.tensor_peak(PEAKS, "bf16")[0] == 1906.9
    assert bench.tensor_peak(PEAKS, "bf16", sustained=True)[0] == 1697.7
    # FP8 takes the nominal dense ratio of 4.5 / 2.25 PFLOP/s over the measured BF16 figure.
    assert bench.tensor_peak(PEAKS, "fp8")[0] == pytest.approx(2 * 1906.9)
    assert bench.tensor_peak(PEAKS, "fp8", sustained=True)[0] == pytest.approx(2 * 1697.7)
    assert "sustained" in bench.tensor_peak(PEAKS, "bf16", sustained=True)[1]
    # Without a sustained figure the burst one is used and named.
    only_burst = {k: v for k, v in PEAKS.items() if k != "bf16_tflops_sustained"}
    peak, src = bench.tensor_peak(only_burst, "bf16", sustained=True)
    assert peak == 1906.9 and "burst" in src


def test_fp32_alu_peak():
    # 152 SMs x 128 FMA lanes x 2 FLOP at 2070 MHz.
    assert bench.fp32_alu_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_measured_peaks_has_the_denominators():
    p = bench.measured_peaks()
    for key in ("hbm_gbs", "bf16_tflops"):
        assert p[key] > 0
    assert p["source"] in ("measured", "fallback")


def test_threshold_traffic_follows_the_kernel_sources():
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(bench.ROOT, "paper_2504_13445_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    entry = bench.THRESHOLD_TRAFFIC.get(h.hexdigest())
    for workload in ("mf-2m-k10", "mf-500k", "no-such-workload"):
        got = bench.threshold_traffic(workload)
        assert got == (entry or {}).get(workload)
        # A figure, when present, is DRAM bytes of one launch: above the algorithmic bytes
        # of the operands, below a terabyte.
        assert got is None or 1e8 < got < 1e12
    assert bench.threshold_traffic("no-such-workload") is None
