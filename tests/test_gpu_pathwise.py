"""GPU parity of Algorithm II (the path-wise estimator, Sec. 3 of Pages &
Wilbertz, arXiv:1101.3228) through the C ABI against the CPU oracle: counts bit
for bit, path states and cells of dumped paths bit for bit, for the AR(1)
chain of Prop. 1 and for the Euler-scheme (square-root) chain that is not
AR(1); FP32 and FP64 samples; grids streamed in segments; the full 2-factor
workload in the benchmark's launch configuration; the unsupported requests and
the timeout path.
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


def _check_counts(B, model, counts, ref):
    got = B.split_counts(model.N, counts.cpu().numpy().astype(np.int64))
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
        assert int(got[k].sum()) == model.M


def _cases():
    return [
        ("ou2", lambda: W.ou2(M=20011, n=7, N=500), oracle.PREC_F32),
        ("ou2-f64", lambda: W.ou2(M=5003, n=5, N=300), oracle.PREC_F64),
        ("bs1d-f64", lambda: W.bs1d(M=30011), oracle.PREC_F64),
        ("bs1d-f32", lambda: W.bs1d(M=30011), oracle.PREC_F32),
        ("basket4", lambda: W.basket4(M=9001).restrict(n=6), oracle.PREC_F32),
        ("ar8", lambda: W.ar8(M=4001).restrict(n=3, N=700), oracle.PREC_F32),
        ("ar8-f64", lambda: W.ar8(M=2001).restrict(n=2, N=300), oracle.PREC_F64),
        ("maxcall10", lambda: W.maxcall10(M=3001).restrict(n=3, N=600), oracle.PREC_F32),
    ]


@pytest.mark.parametrize("name,make,prec", _cases(), ids=[c[0] for c in _cases()])
def test_pathwise_counts_bit_exact(ctx, B, name, make, prec):
    model = make()
    g = W.layer_grids(model, samples=20000, iters=3) if model.grid_kind == "kmeans" else W.layer_grids(model)
    counts, stats, _ = ctx.transitions_pathwise(model, _dev(g), model.M, model.seed, B.options(prec=prec))
    assert stats.device_status == 0
    ref = oracle.pathwise(model, g, model.M, model.seed, prec)
    _check_counts(B, model, counts, ref)


def _cir(M, n=30):
    d = 2
    dt = 1.0 / 50
    kappa, theta, sig = np.array([1.5, 3.0]), np.array([0.04, 0.09]), np.array([0.2, 0.3])
    R = np.array([[1.0, 0.4], [0.4, 1.0]])
    A = np.repeat(np.diag(1.0 - kappa * dt)[None], n, 0)
    b = np.repeat((kappa * theta * dt)[None], n, 0)
    T = np.repeat((np.diag(sig * np.sqrt(dt)) @ np.linalg.cholesky(R))[None], n, 0)
    m = np.repeat(theta[None], n + 1, 0)
    L = np.zeros((n + 1, d, d))
    L[1:] = np.diag(np.sqrt(theta) * 0.2)[None]
    N = np.array([1] + [150] * n, dtype=np.int64)
    model = W.Model("cir2", d, n, N, A, b, T, m, L, np.arange(n + 1) * dt, 0.0, "max_call", 1.0, None, M,
                    0xC1A0, oracle.PREC_F32, "product")
    return model, (np.zeros((n, d)), np.ones((n, d)))


@pytest.mark.parametrize("prec", [oracle.PREC_F32, oracle.PREC_F64])
def test_euler_chain_counts_and_paths_bit_exact(ctx, B, prec):
    """The square-root (Euler-scheme) chain, which Algorithm III cannot sample:
    counts, and every state and cell of strided paths, against the oracle."""
    model, eu = _cir(M=12007)
    g = W.layer_grids(model)
    stride = 7
    cnt = (model.M + stride - 1) // stride
    counts, stats, dump = ctx.transitions_pathwise(model, _dev(g), model.M, model.seed, B.options(prec=prec),
                                                   euler=eu, dump_count=cnt, dump_stride=stride)
    assert stats.device_status == 0
    ref, paths, cells = oracle.pathwise(model, g, model.M, model.seed, prec, euler=eu, want_paths=True)
    _check_counts(B, model, counts, ref)
    for k in range(model.n):
        np.testing.assert_array_equal(dump["X"][k].cpu().numpy(), paths[k, ::stride])
        np.testing.assert_array_equal(dump["Y"][k].cpu().numpy(), paths[k + 1, ::stride])
        np.testing.assert_array_equal(dump["i"][k].cpu().numpy(), cells[k, ::stride])
        np.testing.assert_array_equal(dump["j"][k].cpu().numpy(), cells[k + 1, ::stride])
    # the unit scale (alpha = 1, beta = 0) reproduces the AR(1) chain on the GPU too
    ones = (np.ones_like(eu[0]), np.zeros_like(eu[1]))
    a, _, _ = ctx.transitions_pathwise(model, _dev(g), model.M, model.seed, B.options(prec=prec))
    e, _, _ = ctx.transitions_pathwise(model, _dev(g), model.M, model.seed, B.options(prec=prec), euler=ones)
    assert torch.equal(a, e)


def test_pathwise_first_layer_equals_algorithm3(ctx, B):
    model = W.ou2(M=50021, n=3, N=500)
    g = _dev(W.layer_grids(model))
    c2, _, _ = ctx.transitions_pathwise(model, g, model.M, model.seed)
    c3, _, _ = ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_F32_RECHECK))
    n0 = int(model.N[0] * model.N[1])
    assert torch.equal(c2[:n0], c3[:n0])
    assert not torch.equal(c2[n0:], c3[n0:])


def test_full_size_ou2_pathwise_bit_exact(ctx, B):
    """The 2-factor workload (n = 100 daily layers, N = 500) in the benchmark's launch,
    M = 2 x 10^6 paths: every count matrix against the oracle."""
    model = W.ou2(M=2 * 10**6)
    g = ctx.build_grids(model, B.GRID_PRODUCT)
    counts, stats, _ = ctx.transitions_pathwise(model, g, model.M, model.seed)
    assert stats.device_status == 0
    ref = oracle.pathwise(model, g.cpu().numpy(), model.M, model.seed, oracle.PREC_F32)
    _check_counts(B, model, counts, ref)
    got = B.split_counts(model.N, counts)
    for k in range(1, model.n):
        assert torch.equal(got[k - 1].sum(dim=0), got[k].sum(dim=1))


def test_pathwise_unsupported_requests(ctx, B):
    model = W.ou2(M=100, n=2, N=64)
    g = _dev(W.layer_grids(model))
    with pytest.raises(B.QtError) as e:
        ctx.transitions_pathwise(model, g, model.M, model.seed, B.options(form=B.FORM_TC_RECHECK))
    assert e.value.status == B.QT_EUNSUPPORTED


@pytest.mark.parametrize("name,n,N,M", [("ar8", 3, 4000, 4001), ("maxcall10", 2, 8000, 2001),
                                         ("basket4", 50, 0, 1501)])
def test_pathwise_streamed_grids_bit_exact(ctx, B, name, n, N, M):
    """Grids larger than half of the shared memory (8-d N = 4000, 10-d N = 8000) go
    through the two buffers in segments (layer 0's one-point grid in one); the 4-d
    basket's uneven grids (N_k up to 2000) fit whole.  Counts against the oracle."""
    full = W.get(name, M=M)
    model = full.restrict(n=n, N=N) if N else full.restrict(n=n)
    g = W.layer_grids(model, samples=3 * int(np.max(model.N)), iters=2)
    counts, stats, _ = ctx.transitions_pathwise(model, _dev(g), model.M, model.seed)
    assert stats.device_status == 0
    ref = oracle.pathwise(model, g, model.M, model.seed, oracle.PREC_F32)
    _check_counts(B, model, counts, ref)


def test_pathwise_timeout_is_reported_and_context_survives(ctx, B):
    model = W.ou2(M=3000, n=4, N=64)
    g = _dev(W.layer_grids(model))
    with pytest.raises(B.QtError) as e:
        ctx.transitions_pathwise(model, g, model.M, model.seed, B.options(spin_budget=-1))
    assert e.value.status == B.QT_ETIMEOUT
    counts, st, _ = ctx.transitions_pathwise(model, g, model.M, model.seed)
    assert st.device_status == 0
    ref = oracle.pathwise(model, g.cpu().numpy(), model.M, model.seed, oracle.PREC_F32)
    _check_counts(B, model, counts, ref)
