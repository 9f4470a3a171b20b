"""The benchmark's roofline arithmetic (bench.py), on the CPU.

The algorithmic work of a search is 2d flops per candidate distance (d
multiply-adds; the comparison is not counted): N_k + N_{k+1} candidates per
sample.layer for Algorithm III, N_{k+1} for Algorithm II.  The tensor-core
pipe's own work counts K operand columns per candidate."""
import bench
import qt_workloads as W


def test_candidates_and_flops_per_sample_layer():
    # 2-factor OU: N_0 = 1, N_k = 500 -> (1 + 500 + 99 * 1000) / 100 candidates
    m = W.ou2()
    assert bench.candidates_per_sample_layer(m) == (501 + 99 * 1000) / 100
    assert bench.flops_per_sample_layer(m) == bench.candidates_per_sample_layer(m) * 2 * 2
    assert bench.candidates_per_sample_layer(m, pathwise=True) == 500
    # 8-d chain: (1 + 4000 + 49 * 8000) / 50 = 7920.02 candidates, 16 flops each
    m8 = W.ar8()
    c8 = (4001 + 49 * 8000) / 50
    assert bench.candidates_per_sample_layer(m8) == c8
    assert bench.flops_per_sample_layer(m8) == c8 * 16
    # the tensor pipe: K = 32 columns at d = 8 (the FP16 head/tail split), 16 at d = 4
    assert bench.tc_pipe_flops_per_sample_layer(m8) == c8 * 2 * 32
    m4 = W.basket4()
    assert bench.tc_pipe_flops_per_sample_layer(m4) == bench.candidates_per_sample_layer(m4) * 2 * 16


def test_rooflines_are_work_over_time_over_peak():
    m8 = W.ar8()
    units = m8.n * m8.M
    peaks = {"bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2000.0}
    r = bench.tensor_roofline(m8, units, 4000.0, peaks)
    assert abs(r["achieved"] - (4001 + 49 * 8000) / 50 * 16 * units / 4.0 / 1e12) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 1700.0) < 1e-15
    assert abs(r["mma_frac"] / r["frac"] - 4.0) < 1e-12          # 2K = 64 pipe flops against 2d = 16
    a = bench.alu_roofline(m8, units, 4000.0, peaks, 152)
    assert abs(a["peak"] - 152 * 128 * 2 * 2000.0e6 / 1e12) < 1e-12
    assert abs(a["frac"] - a["achieved"] / a["peak"]) < 1e-15


def test_job_value_and_replica_seeds():
    assert bench.job_value(4, 10**9, 500.0) == 4 * 10**9 / 0.5
    m = W.ou2()
    assert len({bench.replica_seed(m, r) for r in range(8)}) == 8
