"""The learned router with the Elkan certificate (form QT_FORM_ROUTER_CERT).

* Its forward/backward kernels give the loss and gradient of the FP64
  reference network (oracle/router_mlp.py) on the same parameters.
* Counts are bit-exact against the oracle with the trained router and with an
  untrained (random) one: a wrong start cell costs time, never exactness.
* The trained network evaluates fewer candidate distances per search than the
  same certificate without training, and far fewer than brute force.
"""
import numpy as np
import pytest

import oracle
from oracle import router_mlp as R
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


@pytest.fixture(scope="module")
def ar8_case(ctx, B):
    model = W.ar8(M=6007).restrict(n=3, N=1000)
    g = W.layer_grids(model, samples=20000, iters=4)
    gd = _dev(g)
    trained = ctx.router_train(model, gd, samples=200000, layers=3, epochs=10)
    untrained = ctx.router_train(model, gd, samples=4096, layers=1, epochs=1, untrained=True)
    yield model, g, gd, trained, untrained
    trained.close()
    untrained.close()


def test_router_gradient_matches_fp64_reference(ctx, B, ar8_case):
    model, g, gd, trained, _ = ar8_case
    rng = np.random.default_rng(3)
    P = trained.params().astype(np.float64)
    Z = rng.standard_normal((517, model.d)).astype(np.float32)
    y = rng.integers(0, 64, 517).astype(np.int32)
    loss, grad = trained.loss_grad(_dev(Z), _dev(y))
    L, G = R.loss_and_grad(P, Z.astype(np.float64), y)
    assert abs(loss - L) <= 1e-4 * max(1.0, abs(L))
    g = grad.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(G))
    assert np.max(np.abs(g - G)) <= 2e-4 * scale


@pytest.mark.parametrize("which", ["trained", "untrained"])
def test_router_counts_bit_exact(ctx, B, ar8_case, which):
    model, g, gd, trained, untrained = ar8_case
    rt = trained if which == "trained" else untrained
    counts, stats, _ = ctx.transitions(model, gd, model.M, model.seed,
                                       B.options(form=B.FORM_ROUTER_CERT, router=rt.handle))
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
    assert stats.form_used == B.FORM_ROUTER_CERT


def test_router_gains_over_untrained_and_brute_force(ctx, B, ar8_case):
    model, g, gd, trained, untrained = ar8_case
    info = trained.info()
    assert info.train_accuracy > 0.3, info.train_accuracy     # 64 classes: chance is 1/64
    cands = {}
    for name, rt in (("trained", trained), ("untrained", untrained)):
        _, stats, _ = ctx.transitions(model, gd, model.M, model.seed,
                                      B.options(form=B.FORM_ROUTER_CERT, router=rt.handle))
        # searches with more than one grid point: layer 0 has a single point
        searches = model.M * (2 * model.n - 1)
        cands[name] = stats.candidates / searches
    assert cands["trained"] < 0.8 * cands["untrained"], cands
    assert cands["trained"] < 0.5 * model.N[-1], cands


def test_router_rejects_other_grids(ctx, B, ar8_case):
    model, g, gd, trained, _ = ar8_case
    other = gd.clone()
    other[5, 0] += 1e-3
    with pytest.raises(B.QtError) as e:
        ctx.transitions(model, other, model.M, model.seed, B.options(form=B.FORM_ROUTER_CERT, router=trained.handle))
    assert e.value.status == B.QT_EINVAL


def test_router_fused_backward_price(ctx, B, ar8_case):
    """The fused reverse-order price with the router form: every layer pair in its own
    launch (the router finds its layer by the global index), the same price bits as the
    unfused path and the oracle's price within 1e-12."""
    model, g, gd, trained, _ = ar8_case
    phi = W.payoff_values(model, g)
    o = dict(form=B.FORM_ROUTER_CERT, router=trained.handle)
    p0, _ = ctx.price(model, gd, model.M, model.seed, _dev(phi), B.options(**o))
    p1, st = ctx.price(model, gd, model.M, model.seed, _dev(phi), B.options(flags=B.FLAG_FUSED_BACKWARD, **o))
    assert st.device_status == 0 and st.form_used == B.FORM_ROUTER_CERT
    assert p1 == p0
    ref = oracle.price(model.N, oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32), phi)
    assert abs(p1 - ref) <= 1e-12 * abs(ref)


def test_router_timeout_is_reported(ctx, B, ar8_case):
    """A wait for the router network's tensor-core layers that gives up is
    reported as a timeout, and the next call on the same context is exact."""
    model, g, gd, trained, _ = ar8_case
    with pytest.raises(B.QtError) as e:
        ctx.transitions(model, gd, model.M, model.seed,
                        B.options(form=B.FORM_ROUTER_CERT, router=trained.handle, spin_budget=-1))
    assert e.value.status == B.QT_ETIMEOUT
    counts, _, _ = ctx.transitions(model, gd, model.M, model.seed,
                                   B.options(form=B.FORM_ROUTER_CERT, router=trained.handle))
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")


@pytest.mark.parametrize("d", [2, 5, 16])
def test_router_counts_bit_exact_across_dimension_classes(ctx, B, d):
    """The tensor-core inference builds its first-layer rows from the whitened
    coordinates zero-padded to 16 columns: d = 2 and 5 leave padding in the
    dimension classes 2 and 6, d = 16 fills every column.  Counts bit-exact
    against the oracle in each case."""
    model = W._ar_model(f"ar{d}", d, 2, 256, 3001, "basket_put", 1.0, 9)
    g = W.layer_grids(model, samples=8000, iters=3)
    gd = _dev(g)
    rt = ctx.router_train(model, gd, samples=20000, layers=2, epochs=3)
    try:
        counts, stats, _ = ctx.transitions(model, gd, model.M, model.seed,
                                           B.options(form=B.FORM_ROUTER_CERT, router=rt.handle))
    finally:
        rt.close()
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"d={d} layer {k}")
    assert stats.form_used == B.FORM_ROUTER_CERT and stats.device_status == 0
