"""GPU swing-option backward induction (eq. (stochCtrl) and the bang-bang BDP of
Sec. 2, Pages & Wilbertz, arXiv:1101.3228) through the C ABI against the CPU
oracle on the same counts.

Tolerance: both sides sum at most N_{k+1} products per continuation in binary64,
in different orders (the library in lanes j mod 32 then a fixed butterfly,
the oracle left to right with pi = p_ij / p_i), and the recursion takes maxima
and adds payoffs, which does not amplify the difference; so every finite value
agrees within 1e-12 of the layer's largest |P|, the infeasible states are -inf
on both sides, and the price agrees within 1e-12 relative.  The one-right swing
equals the library's own Bermudan backward induction bit for bit.
"""
import numpy as np
import pytest

import oracle
import qt_workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_1101_3228_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _compare(N, P_gpu, P_ref, Qmax):
    got = oracle.swing_blocks(N, P_gpu.cpu().numpy(), Qmax)
    ref = oracle.swing_blocks(N, P_ref, Qmax)
    for k, (a, b) in enumerate(zip(got, ref)):
        fin = np.isfinite(b)
        np.testing.assert_array_equal(np.isfinite(a), fin, err_msg=f"layer {k}")
        assert np.all(a[~fin] == b[~fin]), k
        if fin.any():
            scale = max(1.0, float(np.max(np.abs(b[fin]))))
            assert float(np.max(np.abs(a[fin] - b[fin]))) <= 1e-12 * scale, k


@pytest.fixture(scope="module")
def ou2_tree(ctx, B):
    model = W.ou2(M=200000, n=12, N=100)
    g = W.layer_grids(model)
    counts, _, _ = ctx.transitions(model, _dev(g), model.M, model.seed)
    return model, g, counts


@pytest.mark.parametrize("Qmin,Qmax", [(0, 1), (0, 12), (12, 12), (3, 7), (0, 5), (5, 20)])
def test_swing_matches_oracle(ctx, B, ou2_tree, Qmin, Qmax):
    model, g, counts = ou2_tree
    v = W.payoff_values(model, g) - 0.004          # negative and positive payoffs
    P, price = ctx.swing(model.N, counts, _dev(v), Qmin, Qmax)
    cl = B.split_counts(model.N, counts.cpu().numpy())
    Pref, pref = oracle.swing(model.N, cl, v, Qmin, Qmax)
    _compare(model.N, P, Pref, Qmax)
    assert abs(price - pref) <= 1e-12 * max(1.0, abs(pref))


def test_one_right_swing_is_the_bermudan_bit_for_bit(ctx, B, ou2_tree):
    model, g, counts = ou2_tree
    phi = W.payoff_values(model, g)
    off = model.offsets()
    phi0 = phi.copy()
    phi0[off[model.n]:] = 0.0
    P, price = ctx.swing(model.N, counts, _dev(phi0), 0, 1)
    V = ctx.backward(model.N, counts, _dev(phi0)).cpu().numpy()
    blocks = oracle.swing_blocks(model.N, P.cpu().numpy(), 1)
    for k in range(model.n + 1):
        np.testing.assert_array_equal(blocks[k][0], V[off[k]:off[k + 1]])
    p_b, _ = ctx.price(model, _dev(g), model.M, model.seed, _dev(phi0))
    assert price == p_b


def test_swing_paper_scenario_uint32_counts(ctx, B):
    """The paper's scenario for swing options (the 2-factor model, n = 365 daily dates,
    N = 100, M = 10^5) with v_k = spot - K, between 100 and 200 exercise dates."""
    model = W.paper(N=100)
    g = W.layer_grids(model)
    counts, _, _ = ctx.transitions(model, _dev(g), model.M, model.seed, B.options(counts_type=B.COUNTS_U32))
    off = model.offsets()
    v = np.empty(off[-1])
    for k in range(model.n + 1):
        x = g[off[k]:off[k + 1]]
        v[off[k]:off[k + 1]] = np.exp(x.sum(axis=1)) - 1.0
    P, price = ctx.swing(model.N, counts, _dev(v), 100, 200, counts_type=B.COUNTS_U32)
    cl = B.split_counts(model.N, counts.cpu().numpy().astype(np.int64))
    Pref, pref = oracle.swing(model.N, cl, v, 100, 200)
    _compare(model.N, P, Pref, 200)
    assert abs(price - pref) <= 1e-12 * max(1.0, abs(pref))


def test_swing_rejects_bad_constraints(ctx, B, ou2_tree):
    model, g, counts = ou2_tree
    v = _dev(W.payoff_values(model, g))
    for qmin, qmax in ((3, 2), (-1, 4), (model.n + 1, model.n + 3)):
        with pytest.raises(B.QtError) as e:
            ctx.swing(model.N, counts, v, qmin, qmax)
        assert e.value.status == B.QT_EINVAL
