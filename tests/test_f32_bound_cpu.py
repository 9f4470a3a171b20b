"""The FP32 screen's error bound, checked on the CPU.

The FP32 screen scores candidate g_j against sample x as a chain of FP32 fused
multiply-adds, s~_j = fma(xa_{d-1}, g~_{j,d-1}, ... fma(xa_0, g~_{j,0}, cc~_j)),
with g~ = fl32(g - mu), cc~ = fl32(|g - mu|^2) and xa = -2 fl32(x - mu).  Its
certificate assumes, for every j,

    |s~_j - s_j| <= E(r_j),   E(r) = (d + 2) 2^-24 (1 + 2^-10) (r^2 + 2 A r),

with s_j = |g_j - mu|^2 - 2 (x - mu).(g_j - mu) the exact score, A = |x - mu| and
r_j = |g_j - mu| (both inflated by 2^-18 as the kernel does).  This test evaluates
the FMA chain with one rounding per step (the product and sum in extended precision,
then rounded to FP32) and checks the bound for every candidate.
"""
import math

import numpy as np
import pytest

f32 = np.float32
LD = np.longdouble


def fma32(a, b, c):
    # a*b is exact in extended precision (48-bit product); the sum is rounded once to
    # extended precision and then to FP32 (a double rounding that only matters when the
    # extended result lands exactly on an FP32 tie, far rarer than this test's sample)
    return f32(LD(a) * LD(b) + LD(c))


def e_bound(d, A, r):
    return (d + 2) * 2.0 ** -24 * (1 + 2.0 ** -10) * (r * r + 2.0 * A * r)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 10, 16])
@pytest.mark.parametrize("scale", [1e-3, 1.0, 1e3])
def test_fp32_score_error_within_bound(d, scale):
    rng = np.random.default_rng(500 * d + int(math.log10(scale) + 5))
    N = 129
    mu32 = (rng.standard_normal(d) * scale).astype(f32)
    grid = mu32.astype(np.float64) + rng.standard_normal((N, d)) * scale
    t = grid - mu32.astype(np.float64)
    g32 = t.astype(f32)
    cc32 = np.sum(t * t, axis=1).astype(f32)
    samples = [rng.standard_normal(d) * scale * s for s in (0.1, 1.0, 3.0, 30.0) for _ in range(5)]
    samples += [t[i] + rng.standard_normal(d) * scale * 1e-6 for i in range(4)]
    worst = 0.0
    for xs in samples:
        x32 = (mu32.astype(np.float64) + xs).astype(f32)
        ax = (x32.astype(np.float64) - mu32.astype(np.float64)).astype(f32)
        xa = (f32(-2.0) * ax).astype(f32)
        a = x32.astype(LD) - mu32.astype(LD)
        g = grid.astype(LD) - mu32.astype(LD)
        exact = (np.sum(g * g, axis=1) - 2.0 * (g @ a)).astype(np.float64)
        A = float(np.sqrt(np.sum(ax.astype(np.float64) ** 2))) * (1 + 2.0 ** -18)
        for j in range(N):
            s = cc32[j]
            for l in range(d):
                s = fma32(xa[l], g32[j, l], s)
            r = float(np.sqrt(np.sum(g[j].astype(np.float64) ** 2))) * (1 + 2.0 ** -18)
            ratio = abs(float(s) - exact[j]) / e_bound(d, A, r)
            assert ratio <= 1.0, (d, scale, j, ratio)
            worst = max(worst, ratio)
    assert worst < 1.0
