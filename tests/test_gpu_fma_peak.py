"""Measured FMA throughput of the GPU (tests/cuda/fma_peak.cu): scalar FP32,
packed FP32 pairs (fma.rn.f32x2) and FP64.  The FP32 screen's roofline is
reported against the unit-count peak (SMs x 128 lanes x 2 flops x maximum
clock); this test checks that the measured rates are of that order, so the
derived peak is one the hardware reaches, and prints them."""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_measured_fma_peaks_reach_the_unit_count_peak():
    from paper_1101_3228_gb300.build import _nvcc
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "fma_peak")
        subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                        os.path.join(HERE, "cuda", "fma_peak.cu"), "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    print(out)
    rates = {}
    sms = mhz = None
    for ln in out.splitlines():
        p = ln.split()
        if p[:2] == ["fma_peak", "sms"]:
            sms, mhz = int(p[2]), float(p[4])
        elif p and p[0] == "fma_peak":
            rates[p[1]] = float(p[2])
    assert sms and mhz
    unit_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    # the clock under a long FMA loop may sit below the maximum; the packed form
    # carries two lanes per instruction (at most twice the scalar lane rate)
    assert 0.5 * unit_peak < rates["f32"] <= 1.05 * unit_peak, (rates, unit_peak)
    assert 0.5 * unit_peak < rates["f32x2"] <= 2.1 * unit_peak, (rates, unit_peak)
    assert 0 < rates["f64"] < rates["f32"]
