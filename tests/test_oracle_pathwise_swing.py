"""Pins of the oracle's Algorithm II (the path-wise estimator, also for an
Euler-scheme chain) and of its swing-option backward induction (eq. (stochCtrl)
and the bang-bang BDP of Sec. 2), against things other than themselves:
Algorithm III's own layer-0 pair, the exact Markov bookkeeping of a path, the
AR(1) and square-root-diffusion moment recursions, the 1-d transition law by
quadrature, the Bermudan backward induction, the strip of forward-propagated
expectations, and a hand-computed tree.  Citations are to Pages & Wilbertz,
arXiv:1101.3228.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
import qt_workloads as W


# --------------------------------------------------------------------------- Algorithm II

def test_pathwise_first_step_is_algorithm3_layer0():
    """X_0 and X_1 of every path are the pair Algorithm III draws for layer 0, so the
    layer-0 counts of both estimators coincide bit for bit (FP32 and FP64 samples)."""
    for model, prec in ((W.ou2(M=3000, n=3, N=64), oracle.PREC_F32), (W.bs1d(M=3000), oracle.PREC_F64)):
        g = W.layer_grids(model)
        c2, paths, cells = oracle.pathwise(model, g, model.M, model.seed, prec, want_paths=True)
        c3 = oracle.transitions(model, g, model.M, model.seed, prec)
        np.testing.assert_array_equal(c2[0], c3[0])
        X, Y = oracle.sample_pairs(model.d, prec, model.seed, 0, 0, model.M, model.m[0], model.L[0],
                                   model.A[0], model.b[0], model.T[0])
        np.testing.assert_array_equal(paths[0], X)
        np.testing.assert_array_equal(paths[1], Y)
        # later layers are not Algorithm III's independent pairs
        assert not np.array_equal(c2[1], c3[1])


def test_pathwise_counts_chain_exactly():
    """Each path is in one cell of every layer: the column sums of p^{k-1} are the row
    sums of p^k exactly (Algorithm II's p^{k+1}_j counter), and the cells are the
    nearest cells of the recorded states."""
    model = W.ou2(M=5000, n=6, N=100)
    g = W.layer_grids(model)
    c, paths, cells = oracle.pathwise(model, g, model.M, model.seed, oracle.PREC_F32, want_paths=True)
    off = model.offsets()
    for k in range(model.n):
        assert int(c[k].sum()) == model.M
        if k > 0:
            np.testing.assert_array_equal(c[k - 1].sum(axis=0), c[k].sum(axis=1))
    for k in (0, 3, 6):
        np.testing.assert_array_equal(cells[k], oracle.nearest(g[off[k]:off[k + 1]], paths[k]))
    # the counts are the histogram of consecutive cells
    h = np.zeros_like(c[2])
    np.add.at(h, (cells[2], cells[3]), 1)
    np.testing.assert_array_equal(h, c[2])


@pytest.mark.parametrize("prec", [oracle.PREC_F32, oracle.PREC_F64])
def test_pathwise_marginals_follow_the_ar1_moments(prec):
    """Along the paths X_k has the marginal law N(m_k, L_k L_k^T) of Prop. 1's chain
    (m and L come from the model's own moment recursion)."""
    model = W.ou2(M=200000, n=40, N=16)
    g = W.layer_grids(model)
    _, paths, _ = oracle.pathwise(model, g, model.M, model.seed, prec, want_paths=True)
    M = model.M
    for k in (1, 13, 40):
        X = paths[k]
        S = model.L[k] @ model.L[k].T
        mean_z = (X.mean(axis=0) - model.m[k]) / np.sqrt(np.diag(S) / M)
        assert np.all(np.abs(mean_z) < 5.0), (k, mean_z)
        C = np.cov(X.T)
        for a in range(2):
            for b in range(2):
                se = math.sqrt((S[a, a] * S[b, b] + S[a, b] ** 2) / M)
                assert abs(C[a, b] - S[a, b]) < 5.0 * se, (k, a, b, C[a, b], S[a, b])


def _bivariate_cell_prob(mu1, s1, b, tau, lo_i, hi_i, lo_j, hi_j):
    def f(x):
        return stats.norm.pdf(x, mu1, s1) * (special.ndtr((hi_j - x - b) / tau) - special.ndtr((lo_j - x - b) / tau))
    a = max(lo_i, mu1 - 12 * s1)
    c = min(hi_i, mu1 + 12 * s1)
    if a >= c:
        return 0.0
    return integrate.quad(f, a, c, epsabs=1e-13, epsrel=1e-10, limit=200)[0]


def test_pathwise_counts_follow_exact_transition_law_1d():
    """Algorithm II estimates the same p^k_ij as Algorithm III: at layer k the counts
    are Multinomial(M, P(X_k in C_i, X_{k+1} in C_j)) (eq. (defPi))."""
    m = W.bs1d()
    grids = W.layer_grids(m)
    off = m.offsets()
    M, k = 400000, 6
    c = oracle.pathwise(m, grids, M, seed=77, prec=oracle.PREC_F64)[k]
    gA = grids[off[k]:off[k + 1], 0]
    gB = grids[off[k + 1]:off[k + 2], 0]
    bA = np.concatenate([[-np.inf], 0.5 * (gA[1:] + gA[:-1]), [np.inf]])
    bB = np.concatenate([[-np.inf], 0.5 * (gB[1:] + gB[:-1]), [np.inf]])
    mu, s = m.m[k, 0], m.L[k, 0, 0]
    b, tau = m.b[k, 0], m.T[k, 0, 0]
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


def test_euler_chain_with_unit_scale_is_the_ar1_chain():
    """alpha = 1, beta = 0 scales no innovation: the same states and counts, bit for bit."""
    model = W.ou2(M=4000, n=5, N=81)
    g = W.layer_grids(model)
    ones, zeros = np.ones((model.n, model.d)), np.zeros((model.n, model.d))
    for prec in (oracle.PREC_F32, oracle.PREC_F64):
        a = oracle.pathwise(model, g, model.M, model.seed, prec, want_paths=True)
        e = oracle.pathwise(model, g, model.M, model.seed, prec, euler=(ones, zeros), want_paths=True)
        for k in range(model.n):
            np.testing.assert_array_equal(a[0][k], e[0][k])
        np.testing.assert_array_equal(a[1], e[1])


def _cir_model(M, n=50, dt=1.0 / 50):
    """Two square-root (CIR-type) factors, Euler scheme:
    X_{k+1} = X_k + kappa (theta - X_k) dt + sqrt(X_k) sigma sqrt(dt) (R^{1/2} eps)_l."""
    kappa = np.array([1.5, 3.0])
    theta = np.array([0.04, 0.09])
    sig = np.array([0.2, 0.3])
    rho = 0.4
    R = np.array([[1.0, rho], [rho, 1.0]])
    x0 = theta.copy()
    d = 2
    A = np.repeat(np.diag(1.0 - kappa * dt)[None], n, 0)
    b = np.repeat((kappa * theta * dt)[None], n, 0)
    T = np.repeat((np.diag(sig * math.sqrt(dt)) @ np.linalg.cholesky(R))[None], n, 0)
    m = np.repeat(x0[None], n + 1, 0)
    L = np.zeros((n + 1, d, d))
    L[1:] = np.diag(np.sqrt(theta) * 0.2)[None]          # grids only: a rough spread
    N = np.array([1] + [64] * n, dtype=np.int64)
    mdl = W.Model("cir2", d, n, N, A, b, T, m, L, np.arange(n + 1) * dt, 0.0, "max_call", 1.0, None, M,
                  0xC1A0, oracle.PREC_F64, "product")
    alpha = np.zeros((n, d))
    beta = np.ones((n, d))
    return mdl, alpha, beta, kappa, theta, sig, rho, dt, x0


def test_euler_square_root_chain_moments():
    """The Euler-scheme chain (not AR(1)): E X_{k+1} = b + A E X_k exactly, and
    Var X^l_{k+1} = A_ll^2 Var X^l_k + E[max(X^l_k, 0)] (T T^T)_ll, since the
    innovation of row l is scaled by sqrt(X^l_k) and independent of X_k.  The
    second recursion also fails if a column were scaled instead of a row."""
    mdl, alpha, beta, kappa, theta, sig, rho, dt, x0 = _cir_model(M=200000)
    g = W.layer_grids(mdl)
    _, paths, _ = oracle.pathwise(mdl, g, mdl.M, mdl.seed, oracle.PREC_F64, euler=(alpha, beta),
                                  want_paths=True)
    M = mdl.M
    Ad = np.diag(mdl.A[0])
    TT = np.diag(mdl.T[0] @ mdl.T[0].T)
    mean = x0.copy()
    var = np.zeros(2)
    for k in range(mdl.n):
        var = Ad ** 2 * var + TT * np.maximum(mean, 0.0)
        mean = mdl.b[k] + Ad * mean
        if k + 1 in (5, 25, 50):
            X = paths[k + 1]
            assert np.mean(X < 0) < 1e-4                     # the Feller condition keeps X positive
            se_m = np.sqrt(var / M)
            assert np.all(np.abs(X.mean(axis=0) - mean) < 5 * se_m), (k, X.mean(axis=0), mean)
            v = X.var(axis=0)
            se_v = var * math.sqrt(2.0 / M) * 1.5                # mild excess kurtosis
            assert np.all(np.abs(v - var) < 5 * se_v), (k, v, var)
    # the unscaled (AR(1)) chain has a variance about 1/theta larger
    _, p_ar, _ = oracle.pathwise(mdl, g, 20000, mdl.seed, oracle.PREC_F64, want_paths=True)
    assert np.all(p_ar[mdl.n].var(axis=0) > 5 * paths[mdl.n].var(axis=0))


# --------------------------------------------------------------------------- swing option

def _strip(N, counts, v, use_max=True):
    """sum_{k<n} E v_k(X^_k)^(+) under the tree's chain: the law of X^_k propagated
    forward with pi (empty rows pass no mass on, as in the backward induction)."""
    N = np.asarray(N)
    n = len(N) - 1
    off = np.concatenate([[0], np.cumsum(N)])
    c0 = np.asarray(counts[0], dtype=np.float64)
    law = np.ones(1) if N[0] == 1 else c0.sum(axis=1) / c0.sum()
    tot = 0.0
    for k in range(n):
        vk = v[off[k]:off[k + 1]]
        tot += float(law @ (np.maximum(vk, 0.0) if use_max else vk))
        c = np.asarray(counts[k], dtype=np.float64)
        row = c.sum(axis=1)
        pi = np.divide(c, row[:, None], where=row[:, None] > 0, out=np.zeros_like(c))
        law = law @ pi
    return tot


@pytest.fixture(scope="module")
def ou2_tree():
    model = W.ou2(M=200000, n=12, N=100)
    g = W.layer_grids(model)
    counts = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    return model, g, counts


def test_swing_with_one_right_is_the_bermudan(ou2_tree):
    """Qmax = 1, Qmin = 0: one exercise right at dates 0..n-1, i.e. the Bermudan of the
    BDP with V_n = 0 (bit for bit: the same continuation sums, the same max)."""
    model, g, counts = ou2_tree
    phi = W.payoff_values(model, g)                      # a put: v >= 0
    off = model.offsets()
    P, price = oracle.swing(model.N, counts, phi, 0, 1)
    phi0 = phi.copy()
    phi0[off[model.n]:] = 0.0
    V = oracle.backward(model.N, counts, phi0)
    blocks = oracle.swing_blocks(model.N, P, 1)
    for k in range(model.n + 1):
        np.testing.assert_array_equal(blocks[k][0], V[off[k]:off[k + 1]])
    assert price == oracle.price(model.N, counts, phi0)


def test_swing_without_constraint_is_the_strip(ou2_tree):
    """Qmin = 0, Qmax = n: every date is a free option, so the value is the strip
    sum_k E v_k^+ of forward-propagated expectations on the tree."""
    model, g, counts = ou2_tree
    v = W.payoff_values(model, g) - 0.004               # some negative values
    _, price = oracle.swing(model.N, counts, v, 0, model.n)
    ref = _strip(model.N, counts, v, use_max=True)
    assert abs(price - ref) <= 1e-12 * abs(ref)


def test_swing_forced_consumption_is_the_plain_strip(ou2_tree):
    """Qmin = Qmax = n: every date must be exercised, so the value is sum_k E v_k."""
    model, g, counts = ou2_tree
    v = W.payoff_values(model, g) - 0.004
    _, price = oracle.swing(model.N, counts, v, model.n, model.n)
    ref = _strip(model.N, counts, v, use_max=False)
    assert abs(price - ref) <= 1e-12 * max(1.0, abs(ref))


def test_swing_monotone_in_the_constraints(ou2_tree):
    model, g, counts = ou2_tree
    v = W.payoff_values(model, g) - 0.004
    n = model.n
    p = {(a, b): oracle.swing(model.N, counts, v, a, b)[1] for a in (0, 3, 6) for b in (6, 9, n)}
    for a in (0, 3, 6):
        assert p[(a, 6)] <= p[(a, 9)] <= p[(a, n)]
    for b in (6, 9, n):
        assert p[(0, b)] >= p[(3, b)] >= p[(6, b)]


def test_swing_hand_made_tree():
    """n = 2, N = (1, 2, 2), exactly one unit to take (Qmin = Qmax = 1)."""
    N = np.array([1, 2, 2])
    c0 = np.array([[3, 1]])
    c1 = np.array([[2, 2], [1, 3]])
    v = np.array([0.3, 0.5, -0.2, 9.0, 9.0])            # v_0 | v_1 | (v_2 unused)
    P, price = oracle.swing(N, [c0, c1], v, 1, 1)
    b = oracle.swing_blocks(N, P, 1)
    # date 1, nothing taken yet: the last date forces x = 1
    np.testing.assert_array_equal(b[1][0], [0.5, -0.2])
    np.testing.assert_array_equal(b[1][1], [0.0, 0.0])  # already taken: x = 0, nothing follows
    np.testing.assert_array_equal(b[2][1], [0.0, 0.0])
    assert np.all(np.isneginf(b[2][0]))                  # ending with nothing taken is infeasible
    # date 0: take now (0.3 + E P_1(., 1) = 0.3) or later (E P_1(., 0) = 0.75 * 0.5 + 0.25 * -0.2)
    assert b[0][0][0] == max(0.3, 0.75 * 0.5 + 0.25 * -0.2)
    assert price == b[0][0][0]
