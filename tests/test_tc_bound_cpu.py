"""The tensor-core screen's error bound, checked on the CPU.

The tensor-core form scores candidate g_j of a grid against sample x as one MMA
row: both sides centred on the grid's FP32 centre, scaled by sigma = 2^e (the grid
in [-1, 1]), split into an FP16 head and tail, multiplied exactly (an FP16 x FP16
product fits FP32) and summed in FP32.  Its certificate assumes, for every j,

    |s~_j / sigma^2 - s_j| <= E_TC(r_j),
    E_TC(r) = 1.5 2^-18 (r^2 + 2 A r) + (2^-23 sqrt(d) (A + r) sigma + 2^-24) / sigma^2,

with s_j = |g_j - mu|^2 - 2 (x - mu).(g_j - mu) the exact score, A = |x - mu| and
r_j = |g_j - mu| (both inflated by 2^-18 as the kernel does).  This test rebuilds
the roundings of the record preparation, the draw pass and the operand tiles in
numpy and checks the bound for every candidate, on grids of very different scales,
on samples near and far from the grid, and for two summation orders of the FP32
accumulation (left to right, and pairwise).
"""
import math

import numpy as np
import pytest

f32 = np.float32
f16 = np.float16


def dm_class(d):
    return 2 if d <= 2 else (4 if d <= 4 else (6 if d <= 6 else (8 if d <= 8 else 10)))


def tc_bound(d, A, r, sigma):
    inv = 1.0 / sigma
    return 1.5 * 2.0 ** -18 * (r * r + 2.0 * A * r) + (2.0 ** -23 * math.sqrt(d) * (A + r) * sigma + 2.0 ** -24) * inv * inv


def split16(v32):
    h = v32.astype(f16)
    lo = (v32 - h.astype(f32)).astype(f32).astype(f16)
    return h, lo


def fp32_sum(terms, pairwise):
    """Sum FP32 terms in FP32, left to right or as a balanced tree."""
    t = [f32(v) for v in terms]
    if not pairwise:
        acc = f32(0.0)
        for v in t:
            acc = f32(acc + v)
        return acc
    while len(t) > 1:
        nxt = [f32(t[i] + t[i + 1]) for i in range(0, len(t) - 1, 2)]
        if len(t) % 2:
            nxt.append(t[-1])
        t = nxt
    return t[0]


def tc_scores(grid, mu32, x32, d, pairwise):
    DM = dm_class(d)
    # record preparation: centred coordinates rounded to FP32, cc = FP64 sum of squares rounded
    t = grid - mu32.astype(np.float64)
    g32 = t.astype(f32)
    cc32 = np.sum(t * t, axis=1).astype(f32)
    R = float(np.max(np.sqrt(np.sum(g32.astype(np.float64) ** 2, axis=1))))
    e = -math.frexp(R)[1] if R > 0 else 0
    sigma = 2.0 ** e
    # sample side: -2 (x - mu) rounded to FP32, scaled, split
    ax = (x32.astype(np.float64) - mu32.astype(np.float64)).astype(f32)
    xa = (f32(-2.0) * ax).astype(f32)
    vx = (f32(sigma) * xa).astype(f32)
    if np.any(np.abs(vx) > 16384.0):
        return None, sigma, ax
    ah, al = split16(vx)
    # grid side
    vg = (f32(sigma) * g32).astype(f32)
    gh, gl = split16(vg)
    c = (f32(sigma * sigma) * cc32).astype(f32)
    ch, cl = split16(c)
    out = np.empty(len(grid))
    for j in range(len(grid)):
        terms = []
        for l in range(DM):   # columns [a_hi g_hi], [a_hi g_lo], [a_lo g_hi], cc_hi, cc_lo (zero padded)
            terms.append(f32(ah[l]) * f32(gh[j, l]) if l < d else f32(0.0))
        for l in range(DM):
            terms.append(f32(ah[l]) * f32(gl[j, l]) if l < d else f32(0.0))
        for l in range(DM):
            terms.append(f32(al[l]) * f32(gh[j, l]) if l < d else f32(0.0))
        terms += [f32(ch[j]), f32(cl[j])]
        out[j] = float(fp32_sum(terms, pairwise))
    return out, sigma, ax


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 10])
@pytest.mark.parametrize("scale", [1e-3, 1.0, 1e3])
def test_tensor_core_score_error_within_bound(d, scale):
    rng = np.random.default_rng(1000 * d + int(math.log10(scale) + 5))
    N = 257
    mu32 = (rng.standard_normal(d) * scale).astype(f32)
    grid = mu32.astype(np.float64) + rng.standard_normal((N, d)) * scale
    samples = [rng.standard_normal(d) * scale * s for s in (0.1, 1.0, 3.0, 30.0) for _ in range(6)]
    samples += [grid[i] + rng.standard_normal(d) * scale * 1e-6 for i in range(4)]
    worst = 0.0
    checked = 0
    for xs in samples:
        x32 = (mu32.astype(np.float64) + xs).astype(f32)
        for pairwise in (False, True):
            s_tc, sigma, ax = tc_scores(grid, mu32, x32, d, pairwise)
            if s_tc is None:
                continue          # outside the FP16 range: the kernel skips the screen for this sample
            a = x32.astype(np.longdouble) - mu32.astype(np.longdouble)
            g = grid.astype(np.longdouble) - mu32.astype(np.longdouble)
            exact = np.sum(g * g, axis=1) - 2.0 * (g @ a)
            A = float(np.sqrt(np.sum(ax.astype(np.float64) ** 2))) * (1 + 2.0 ** -18)
            r = np.sqrt(np.sum(g.astype(np.float64) ** 2, axis=1)) * (1 + 2.0 ** -18)
            err = np.abs(s_tc / sigma ** 2 - exact.astype(np.float64))
            bound = np.array([tc_bound(d, A, rj, sigma) for rj in r])
            assert np.all(err <= bound), (d, scale, float(np.max(err / bound)))
            worst = max(worst, float(np.max(err / bound)))
            checked += 1
    assert checked > 0
    assert worst < 1.0
