"""Pins of the CPU oracle against things other than itself.

Each test checks one oracle function against a library routine, a closed form,
a textbook method, brute force on a hand-made case, or a statistical law, so
that a dropped term, a wrong sign or index, or a transposed operand fails.
Citations are to Pages & Wilbertz, arXiv:1101.3228.
"""
import ctypes
import math
import os
import shutil

import numpy as np
import pytest
from scipy import integrate, special, stats
from scipy.spatial import cKDTree

import oracle
import qt_workloads as W

def _find_curand():
    """cuRAND's shared library: the loader's search path first, then the toolkit under CUDA_HOME."""
    import ctypes.util
    import glob
    name = ctypes.util.find_library("curand")
    if name:
        return name
    nvcc = shutil.which("nvcc")
    homes = [os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"),
             os.path.dirname(os.path.dirname(nvcc)) if nvcc else None]
    for h in homes:
        if h:
            hits = sorted(glob.glob(os.path.join(h, "lib*", "libcurand.so*")))
            if hits:
                return hits[0]
    return None


CURAND = _find_curand()


# --------------------------------------------------------------------------- Philox (Sec. 3.1 generator)

def _curand_host_blocks(seed: int, offset_words: int, nblocks: int) -> np.ndarray:
    lib = ctypes.CDLL(CURAND)
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4 * nblocks)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(nblocks, 4)


@pytest.mark.skipif(CURAND is None, reason="libcurand not installed")
@pytest.mark.parametrize("seed,offset_blocks", [
    (0, 0), (0x0123456789ABCDEF, 0), (0xDEADBEEF12345678, (3 << 48) + 65536 * 9 + 11),
    (0x0000C0FFEE000002, 65536 * 77 + 5)])
def test_philox_matches_curand_host_generator(seed, offset_blocks):
    # cuRAND's host Philox4_32_10 emits block b from counter
    # ((b div 65536) in words 0-1, b mod 65536 in word 2, 0) under key = seed.
    nb = 1 << 17
    ref = _curand_host_blocks(seed, 4 * offset_blocks, nb)
    b = offset_blocks + np.arange(nb, dtype=np.uint64)
    hi = b // np.uint64(65536)
    ctr = np.zeros((nb, 4), dtype=np.uint32)
    ctr[:, 0] = (hi & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (hi >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = (b % np.uint64(65536)).astype(np.uint32)
    mine = oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    np.testing.assert_array_equal(mine, ref)


# --------------------------------------------------------------------------- ln / sincos used by Box-Muller

def test_ln_f32_against_library_log():
    rng = np.random.default_rng(1)
    j = rng.integers(0, 1 << 23, size=20000)
    u = ((2 * j + 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    u = np.concatenate([u, np.float32([2.0 ** -24, 1 - 2.0 ** -24, 0.5, 0.70710677, 0.7071068])])
    mine = np.array([oracle.ln_f32(float(x)) for x in u])
    ref = np.log(u.astype(np.float64))
    # within 2 ulp of the binary32 result, plus e*ln2 rounding
    tol = 2.0 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 1e-7 * np.abs(ref) / 8
    assert np.all(np.abs(mine - ref) <= tol)


def test_ln_f64_against_library_log():
    rng = np.random.default_rng(2)
    u = np.concatenate([rng.random(20000), [2.0 ** -53, 1 - 2.0 ** -53, 0.5, 0.7071067811865476]])
    u = u[u > 0]
    mine = np.array([oracle.ln_f64(float(x)) for x in u])
    ref = np.log(u)
    assert np.all(np.abs(mine - ref) <= 4.0 * np.spacing(np.abs(ref)))


def test_sincos2pi_against_library():
    rng = np.random.default_rng(3)
    j = rng.integers(0, 1 << 23, size=20000)
    u = (2 * j + 1).astype(np.float64) * 2.0 ** -24
    for x in list(u) + [0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 2.0 ** -24, 1 - 2.0 ** -24]:
        s, c = oracle.sincos2pi_f32(float(x))
        assert abs(s - math.sin(2 * math.pi * x)) <= 4e-7
        assert abs(c - math.cos(2 * math.pi * x)) <= 4e-7
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    for x in rng.random(5000):
        s, c = oracle.sincos2pi_f64(float(x))
        rs = float(mpmath.sinpi(2 * mpmath.mpf(float(x))))
        rc = float(mpmath.cospi(2 * mpmath.mpf(float(x))))
        assert abs(s - rs) <= 2 * np.spacing(abs(rs)) + 2.0 ** -56
        assert abs(c - rc) <= 2 * np.spacing(abs(rc)) + 2.0 ** -56


# --------------------------------------------------------------------------- uniforms and normals

def test_pi_experiment_table2():
    """Sec. 3.1, Table 2: Monte Carlo estimate of pi from pairs of uniforms.
    The estimator 4 * #{u0^2 + u1^2 <= 1} / n has mean pi and std 4 sqrt(p(1-p)/n), p = pi/4."""
    n, reps = 200000, 100
    est = []
    for rep in range(reps):
        u = oracle.uniforms_f32(seed=rep + 11, k=0, r=0, m0=0, M=n // 2).astype(np.float64)
        pts = np.concatenate([u[:, :2], u[:, 2:]], axis=0)
        est.append(4.0 * np.mean(np.sum(pts * pts, axis=1) <= 1.0))
    est = np.array(est)
    p = math.pi / 4
    sd = 4 * math.sqrt(p * (1 - p) / n)
    assert abs(est.mean() - math.pi) < 4 * sd / math.sqrt(reps)
    assert 0.75 * sd < est.std(ddof=1) < 1.25 * sd


@pytest.mark.parametrize("prec", [oracle.PREC_F32, oracle.PREC_F64])
def test_normals_are_standard_normal(prec):
    g = oracle.normals(prec, seed=99, k=3, m0=0, M=200000, count=8)
    for q in range(8):
        assert stats.kstest(g[:, q], "norm").pvalue > 1e-4
    C = np.corrcoef(g.T)
    assert np.max(np.abs(C - np.eye(8))) < 0.02
    # a different layer or sample range is a different stream
    g2 = oracle.normals(prec, seed=99, k=4, m0=0, M=1000, count=8)
    assert not np.array_equal(g[:1000], g2)


def test_box_muller_pairs_the_published_way():
    """Box & Muller: z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = ... sin(2 pi u1), with u from the
    FP32 uniform map; checked against library log/sin/cos on the same Philox words."""
    M = 4000
    u = oracle.uniforms_f32(seed=5, k=2, r=0, m0=100, M=M).astype(np.float64)
    g = oracle.normals(oracle.PREC_F32, seed=5, k=2, m0=100, M=M, count=4)
    r01 = np.sqrt(-2 * np.log(u[:, 0]))
    r23 = np.sqrt(-2 * np.log(u[:, 2]))
    ref = np.stack([r01 * np.cos(2 * np.pi * u[:, 1]), r01 * np.sin(2 * np.pi * u[:, 1]),
                    r23 * np.cos(2 * np.pi * u[:, 3]), r23 * np.sin(2 * np.pi * u[:, 3])], axis=1)
    np.testing.assert_allclose(g, ref, rtol=0, atol=2e-5)


# --------------------------------------------------------------------------- pair sampling (Prop. 1)

@pytest.mark.parametrize("prec", [oracle.PREC_F32, oracle.PREC_F64])
def test_pair_sampling_moments(prec):
    rng = np.random.default_rng(7)
    d = 3
    mk = rng.standard_normal(d)
    Lk = np.tril(rng.standard_normal((d, d))) + 2 * np.eye(d)
    Ak = rng.standard_normal((d, d)) * 0.5
    bk = rng.standard_normal(d)
    Tk = np.tril(rng.standard_normal((d, d))) * 0.3 + 0.5 * np.eye(d)
    M = 400000
    X, Y = oracle.sample_pairs(d, prec, 17, 4, 0, M, mk, Lk, Ak, bk, Tk)
    se = 5.0 / math.sqrt(M)
    S = Lk @ Lk.T
    assert np.all(np.abs(X.mean(0) - mk) < se * np.sqrt(np.diag(S)))
    np.testing.assert_allclose(np.cov(X.T), S, atol=0.02 * np.max(S))
    R = Y - X @ Ak.T - bk                           # = T eps, independent of X
    Q = Tk @ Tk.T
    np.testing.assert_allclose(np.cov(R.T), Q, atol=0.02 * np.max(Q))
    cross = (X - X.mean(0)).T @ (R - R.mean(0)) / M
    assert np.max(np.abs(cross)) < 0.02 * math.sqrt(np.max(S) * np.max(Q))
    assert stats.kstest((X[:, 0] - mk[0]) / math.sqrt(S[0, 0]), "norm").pvalue > 1e-4


def test_pair_sampling_upper_triangle_ignored():
    d = 2
    mk, bk = np.zeros(d), np.zeros(d)
    L1 = np.array([[1.0, 0.0], [0.3, 1.0]])
    L2 = L1.copy()
    L2[0, 1] = 123.0
    A = np.eye(d)
    X1, Y1 = oracle.sample_pairs(d, 1, 3, 0, 0, 100, mk, L1, A, bk, L1)
    X2, Y2 = oracle.sample_pairs(d, 1, 3, 0, 0, 100, mk, L2, A, bk, L2)
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(Y1, Y2)


def test_fp32_samples_are_fp32_values():
    m = W.ou2(M=1000)
    X, Y = oracle.sample_pairs(2, 1, m.seed, 5, 0, 1000, m.m[5], m.L[5], m.A[5], m.b[5], m.T[5])
    np.testing.assert_array_equal(X, X.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(Y, Y.astype(np.float32).astype(np.float64))


# --------------------------------------------------------------------------- nearest neighbour (Sec. 2)

def test_nearest_hand_made_ties_go_low():
    grid = np.array([[-1.0], [0.0], [1.0]])
    Z = np.array([[-0.5], [0.5], [-2.0], [2.0], [0.0], [0.49], [0.51], [-0.51]])
    np.testing.assert_array_equal(oracle.nearest(grid, Z), [0, 1, 0, 2, 1, 1, 2, 0])
    g2 = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    Z2 = np.array([[0.5, 0.5], [0.9, 0.1], [0.5, 0.0], [0.2, 0.7], [1.0, 0.5]])
    np.testing.assert_array_equal(oracle.nearest(g2, Z2), [0, 1, 0, 2, 1])


def test_nearest_1d_is_binary_search_on_midpoints():
    rng = np.random.default_rng(4)
    grid = np.sort(rng.standard_normal(300))
    Z = rng.standard_normal(100000) * 1.5
    mids = 0.5 * (grid[1:] + grid[:-1])
    far = np.min(np.abs(Z[:, None] - mids[None, :]), axis=1) > 1e-9
    ref = np.searchsorted(mids, Z[far])
    np.testing.assert_array_equal(oracle.nearest(grid[:, None], Z[far, None]), ref)


@pytest.mark.parametrize("d", [2, 4, 10])
def test_nearest_matches_kdtree(d):
    rng = np.random.default_rng(10 + d)
    grid = rng.standard_normal((500, d))
    Z = rng.standard_normal((20000, d)) * 1.3
    _, ref = cKDTree(grid).query(Z, k=1)
    np.testing.assert_array_equal(oracle.nearest(grid, Z), ref)
    dist = oracle.nearest_dist(grid, Z)
    np.testing.assert_allclose(dist, np.sum((Z - grid[ref]) ** 2, axis=1), rtol=1e-14, atol=0)


def test_counts_match_library_assignment_and_permutation():
    rng = np.random.default_rng(5)
    gA = rng.standard_normal((40, 2))
    gB = rng.standard_normal((60, 2))
    X = rng.standard_normal((50000, 2))
    Y = X * 0.9 + 0.3 * rng.standard_normal((50000, 2))
    c = oracle.counts_from_samples(gA, gB, X, Y)
    _, i = cKDTree(gA).query(X)
    _, j = cKDTree(gB).query(Y)
    ref = np.zeros((40, 60), dtype=np.int64)
    np.add.at(ref, (i, j), 1)
    np.testing.assert_array_equal(c, ref)
    assert c.sum() == 50000
    pa, pb = rng.permutation(40), rng.permutation(60)
    cp = oracle.counts_from_samples(gA[pa], gB[pb], X, Y)
    np.testing.assert_array_equal(cp, c[np.ix_(pa, pb)])


# --------------------------------------------------------------------------- Algorithm III counts, 1-d law

def _bivariate_cell_prob(mu1, s1, b, tau, lo_i, hi_i, lo_j, hi_j):
    """P(X in [lo_i, hi_i), X + b + tau eps in [lo_j, hi_j)), X ~ N(mu1, s1^2), by quadrature."""
    def f(x):
        return stats.norm.pdf(x, mu1, s1) * (special.ndtr((hi_j - x - b) / tau) - special.ndtr((lo_j - x - b) / tau))
    a = max(lo_i, mu1 - 12 * s1)
    c = min(hi_i, mu1 + 12 * s1)
    if a >= c:
        return 0.0
    return integrate.quad(f, a, c, epsabs=1e-13, epsrel=1e-10, limit=200)[0]


def test_counts_follow_exact_transition_law_1d():
    """Counts of one layer are Multinomial(M, P(X_k in C_i, X_{k+1} in C_j)) (eq. (defPi))."""
    m = W.bs1d()
    grids = W.layer_grids(m)
    off = m.offsets()
    M = 400000
    k = 3
    mdl = m
    c = oracle.transitions(mdl, grids, M, seed=2024, prec=oracle.PREC_F64)[k]
    gA = grids[off[k]:off[k + 1], 0]
    gB = grids[off[k + 1]:off[k + 2], 0]
    bA = np.concatenate([[-np.inf], 0.5 * (gA[1:] + gA[:-1]), [np.inf]])
    bB = np.concatenate([[-np.inf], 0.5 * (gB[1:] + gB[:-1]), [np.inf]])
    mu, s = m.m[k, 0], m.L[k, 0, 0]
    b, tau = m.b[k, 0], m.T[k, 0, 0]
    # rows i with enough mass; cells within the band where the law is not negligible
    zs = []
    for i in range(40, 60):
        for j in range(len(gB)):
            if abs(j - i) > 25:
                continue
            p = _bivariate_cell_prob(mu, s, b, tau, bA[i], bA[i + 1], bB[j], bB[j + 1])
            if M * p < 20:
                continue
            zs.append((c[i, j] - M * p) / math.sqrt(M * p * (1 - p)))
    zs = np.array(zs)
    assert len(zs) > 100
    assert np.max(np.abs(zs)) < 5.5
    assert abs(zs.mean()) < 4.0 / math.sqrt(len(zs))
    assert 0.8 < zs.std() < 1.2


# --------------------------------------------------------------------------- backward induction (Sec. 2)

def test_backward_hand_made_tree():
    # n = 2, N = (1, 2, 2); counts chosen by hand
    N = np.array([1, 2, 2])
    c0 = np.array([[3, 1]])
    c1 = np.array([[2, 2], [0, 0]])                 # row 1 empty -> V_1(1) = phi_1(1)
    phi = np.array([0.1, 0.5, 0.2, 1.0, 3.0])       # phi_0 | phi_1 | phi_2
    V = oracle.backward(N, [c0, c1], phi)
    V2 = np.array([1.0, 3.0])
    V1 = np.array([max(0.5, 0.5 * 1.0 + 0.5 * 3.0), 0.2])
    V0 = max(0.1, 0.75 * V1[0] + 0.25 * V1[1])
    np.testing.assert_allclose(V, [V0, *V1, *V2], rtol=1e-15)
    assert oracle.price(N, [c0, c1], phi) == V[0]


def test_price_with_random_root_weights_root_cells():
    N = np.array([2, 2])
    c0 = np.array([[1, 2], [3, 4]])
    phi = np.array([0.0, 0.0, 1.0, 2.0])
    V = oracle.backward(N, [c0], phi)
    np.testing.assert_allclose(V[:2], [(1 * 1 + 2 * 2) / 3, (3 * 1 + 4 * 2) / 7])
    np.testing.assert_allclose(oracle.price(N, [c0], phi), 0.3 * V[0] + 0.7 * V[1])


def _bs_put(S, K, r, sig, T):
    d1 = (math.log(S / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    return K * math.exp(-r * T) * special.ndtr(-d2) - S * special.ndtr(-d1)


def _crr_bermudan_put(S, K, r, sig, T, steps, dates):
    dt = T / steps
    u = math.exp(sig * math.sqrt(dt))
    dn = 1 / u
    p = (math.exp(r * dt) - dn) / (u - dn)
    disc = math.exp(-r * dt)
    j = np.arange(steps + 1)
    ST = S * u ** (steps - 2 * j)
    V = np.maximum(K - ST, 0.0)
    ex = {int(round(steps * q / dates)) for q in range(1, dates + 1)}
    for s in range(steps - 1, -1, -1):
        V = disc * (p * V[:-1] + (1 - p) * V[1:])
        if s in ex:
            Ss = S * u ** (s - 2 * np.arange(s + 1))
            V = np.maximum(V, K - Ss)
    return float(V[0])


@pytest.fixture(scope="module")
def bs1d_counts():
    m = W.bs1d()
    grids = W.layer_grids(m)
    counts = oracle.transitions(m, grids, m.M, m.seed, oracle.PREC_F64)
    return m, grids, counts


def test_counts_invariants_bs1d(bs1d_counts):
    m, grids, counts = bs1d_counts
    for k, c in enumerate(counts):
        assert c.shape == (m.N[k], m.N[k + 1])
        assert c.sum() == m.M                       # every sample lands in one cell pair
        assert np.all(c >= 0)
        row = c.sum(axis=1)
        pi = np.divide(c, row[:, None], where=row[:, None] > 0, out=np.zeros(c.shape))
        ok = row > 0
        np.testing.assert_allclose(pi[ok].sum(axis=1), 1.0, atol=m.N[k + 1] * 2.0 ** -53)


def test_european_special_case_matches_closed_form(bs1d_counts):
    """Only t_n exercisable: V^_0 = E phi(X^_n) under the tree; with the exact pi this is
    sum_j P(X_n in C_j) phi(x_j) (law of total probability), and it is close to Black-Scholes."""
    m, grids, counts = bs1d_counts
    phi = W.payoff_values(m, grids)
    v_mc = oracle.price(m.N, counts, W.european_phi(m, phi))
    off = m.offsets()
    g = grids[off[m.n]:, 0]
    bnd = np.concatenate([[-np.inf], 0.5 * (g[1:] + g[:-1]), [np.inf]])
    z = (bnd - m.m[m.n, 0]) / m.L[m.n, 0, 0]
    q = np.diff(special.ndtr(z))
    v_exact = float(np.sum(q * phi[off[m.n]:]))
    assert abs(v_mc - v_exact) < 0.02              # ~3 sigma of the M = 10^6 estimate
    bs = _bs_put(100.0, 100.0, 0.05, 0.2, 1.0)
    assert abs(bs - 5.573526) < 1e-6
    assert abs(v_exact - bs) < 0.01                # quantization bias of a 100-point grid


def test_bermudan_matches_binomial_tree(bs1d_counts):
    m, grids, counts = bs1d_counts
    phi = W.payoff_values(m, grids)
    v = oracle.price(m.N, counts, phi)
    crr = _crr_bermudan_put(100.0, 100.0, 0.05, 0.2, 1.0, 10000, 10)
    assert abs(crr - 6.0335) < 1e-3
    assert abs(v - crr) < 0.02
    V = oracle.backward(m.N, counts, phi)
    assert np.all(V >= phi - 1e-15)                 # V_k >= phi_k


def test_bermudan_error_decreases_with_N():
    crr = _crr_bermudan_put(100.0, 100.0, 0.05, 0.2, 1.0, 10000, 10)
    errs = []
    for N in (10, 30, 100):
        m = W.bs1d(M=400000)
        m.N[1:] = N
        grids = W.layer_grids(m)
        counts = oracle.transitions(m, grids, m.M, m.seed, oracle.PREC_F64)
        errs.append(abs(oracle.price(m.N, counts, W.payoff_values(m, grids)) - crr))
    assert errs[0] > errs[2]
    assert errs[2] < 0.03


# --------------------------------------------------------------------------- grid recipe sanity

def test_lloyd_1d_grid_is_stationary():
    x = W.lloyd_gaussian_1d(100)
    lo = np.concatenate([[-np.inf], 0.5 * (x[1:] + x[:-1])])
    hi = np.concatenate([0.5 * (x[1:] + x[:-1]), [np.inf]])
    mass = np.where(hi <= 0, special.ndtr(hi) - special.ndtr(lo), special.ndtr(-lo) - special.ndtr(-hi))
    mean = (stats.norm.pdf(lo) - stats.norm.pdf(hi)) / mass
    assert np.max(np.abs(mean - x)) < 1e-12
    D = W.distortion_1d(x)
    assert abs(100 ** 2 * D - 2.6671) < 1e-3       # Zador asymptote sqrt(3) pi / 2 = 2.72


# --------------------------------------------------------------------------- router network reference

def test_router_mlp_gradient_matches_finite_differences():
    from oracle import router_mlp as R
    rng = np.random.default_rng(21)
    d, B = 5, 37
    P = rng.standard_normal(R.count(d)) * 0.3
    Z = rng.standard_normal((B, d))
    y = rng.integers(0, 64, B)
    L, g = R.loss_and_grad(P, Z, y)
    assert abs(L - R.loss(P, Z, y)) < 1e-12
    idx = rng.choice(P.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (R.loss(Pp, Z, y) - R.loss(Pm, Z, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_router_mlp_zero_network_is_uniform():
    from oracle import router_mlp as R
    d = 3
    P = np.zeros(R.count(d))
    Z = np.random.default_rng(1).standard_normal((10, d))
    L, g = R.loss_and_grad(P, Z, np.arange(10))
    assert abs(L - math.log(64)) < 1e-14
    # zero hidden activations: only the output biases receive gradient, mean(p - onehot)
    gb3 = g[-64:]
    assert np.allclose(g[:-64], 0.0)
    ref = np.full(64, 1 / 64)
    ref[np.arange(10)] -= 0.1
    np.testing.assert_allclose(gb3, ref, atol=1e-15)
