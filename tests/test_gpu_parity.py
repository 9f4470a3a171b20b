"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Counts and cells are compared bit for bit; values of the backward induction
(Sec. 2) and prices within 1e-12 relative.  The 1e-12 bound: both sides sum
at most N_{k+1} <= 8000 non-negative products per row in binary64 (relative
error below (N+2) 2^-53 < 1e-12 per layer for the order-independent part) and
the recursion does not amplify errors (V_k is a convex combination of V_{k+1}
and a max); the observed differences are ~1e-15.
"""
import os

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


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _model(name, **kw):
    if name == "bs1d":
        return W.bs1d(M=kw.get("M", 100000))
    if name == "ou2":
        return W.ou2(M=kw.get("M", 20011), n=kw.get("n", 6), N=kw.get("N", 500))
    if name == "basket4":
        m = W.basket4(M=kw.get("M", 7001)).restrict(n=kw.get("n", 3))
        return m
    if name == "ar8":
        return W.ar8(M=kw.get("M", 5003)).restrict(n=kw.get("n", 2), N=kw.get("N", 700))
    if name == "maxcall10":
        return W.maxcall10(M=kw.get("M", 3001)).restrict(n=kw.get("n", 2), N=kw.get("N", 500))
    raise ValueError(name)


def _grids(model):
    if model.grid_kind == "kmeans":
        return W.layer_grids(model, samples=20000, iters=5)
    return W.layer_grids(model)


CASES = [
    ("bs1d", "plain_f64", oracle.PREC_F64),
    ("bs1d", "f32_recheck", oracle.PREC_F64),
    ("ou2", "f32_recheck", oracle.PREC_F32),
    ("ou2", "plain_f64", oracle.PREC_F32),
    ("ou2", "f32_recheck", oracle.PREC_F64),
    ("basket4", "f32_recheck", oracle.PREC_F32),
    ("ar8", "f32_recheck", oracle.PREC_F32),
    ("maxcall10", "f32_recheck", oracle.PREC_F32),
]


@pytest.mark.parametrize("name,form,prec", CASES)
def test_counts_bit_exact(ctx, B, name, form, prec):
    model = _model(name)
    g = _grids(model)
    fcode = {"plain_f64": B.FORM_PLAIN_F64, "f32_recheck": B.FORM_F32_RECHECK}[form]
    counts, stats, _ = ctx.transitions(model, _dev(g), model.M, model.seed, B.options(form=fcode, prec=prec))
    ref = oracle.transitions(model, g, model.M, model.seed, prec)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
        assert int(got[k].sum()) == model.M
    assert stats.device_status == 0
    assert stats.form_used == fcode
    # backward induction and price on the same counts
    phi = W.payoff_values(model, g)
    V = ctx.backward(model.N, counts, _dev(phi)).cpu().numpy()
    Vref = oracle.backward(model.N, ref, phi)
    assert _rel(V, Vref) <= 1e-12


@pytest.mark.parametrize("name,N,M", [("ar8", 4000, 3001), ("maxcall10", 8000, 2003), ("basket4", 0, 5003)])
def test_counts_bit_exact_large_grids(ctx, B, name, N, M):
    """Grids too large for one CTA's shared memory: the streamed ring of bulk copies
    (d = 8, N = 4000 and d = 10, N = 8000), and the widest uneven layers (N_k up to 2000)."""
    if name == "basket4":
        full = W.basket4(M=M)
        keep = [0, full.n - 2, full.n - 1]
        model = W.Model("basket4", full.d, 2, full.N[[0, full.n - 1, full.n]].copy(), full.A[keep[1:]],
                        full.b[keep[1:]], full.T[keep[1:]], full.m[[0, full.n - 1, full.n]],
                        full.L[[0, full.n - 1, full.n]], full.t[[0, full.n - 1, full.n]], full.r, full.payoff, full.K,
                        full.weights, M, full.seed, full.prec, "kmeans")
    else:
        model = _model(name, M=M, n=2, N=N)
    g = W.layer_grids(model, samples=3 * int(model.N[-1]), iters=3)
    counts, stats, _ = ctx.transitions(model, _dev(g), model.M, model.seed, B.options(form=B.FORM_F32_RECHECK))
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
    assert stats.device_status == 0


def test_streamed_timeout_is_reported(ctx, B):
    model = _model("ar8", M=600, n=2, N=4000)
    g = _dev(W.layer_grids(model, samples=12000, iters=2))
    with pytest.raises(B.QtError) as e:
        ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_F32_RECHECK, spin_budget=-1))
    assert e.value.status == B.QT_ETIMEOUT
    counts, _, _ = ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_F32_RECHECK))
    assert int(counts.sum()) == model.n * model.M


TC_CASES = [("ou2", 500, 20011, 6), ("basket4", 0, 9001, 3), ("ar8", 700, 5003, 2), ("ar8", 4000, 3001, 2),
            ("maxcall10", 500, 3001, 2), ("maxcall10", 8000, 2003, 2)]


@pytest.mark.parametrize("draw", [1, 2], ids=["draw-pass", "draw-in-kernel"])
@pytest.mark.parametrize("name,N,M,n", TC_CASES)
def test_counts_bit_exact_tensor_core(ctx, B, name, N, M, n, draw):
    """tcgen05 screen: resident operand tiles (N <= a few thousand) and the
    streamed ring (d = 8, N = 4000; d = 10, N = 8000), against the oracle, with
    both sample-draw layouts."""
    model = _model(name, M=M, n=n, N=N) if N else _model(name, M=M, n=n)
    g = W.layer_grids(model, samples=max(20000, 3 * int(model.N[-1])), iters=3) if model.grid_kind == "kmeans" \
        else W.layer_grids(model)
    counts, stats, _ = ctx.transitions(model, _dev(g), model.M, model.seed,
                                       B.options(form=B.FORM_TC_RECHECK, tc_draw=draw))
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
    assert stats.device_status == 0 and stats.form_used == B.FORM_TC_RECHECK


@pytest.mark.parametrize("name,N", [("ar8", 4000), ("basket4", 0)])
def test_tensor_core_dump_samples_and_cells(ctx, B, name, N):
    """Tensor-core form (automatic choice for these d): strided samples of every layer and
    their cells against the oracle's sampler and exact search, one by one."""
    model = _model(name, M=40000, n=3, N=N) if N else _model(name, M=40000, n=3)
    g = W.layer_grids(model, samples=max(20000, 3 * int(model.N[-1])), iters=3)
    stride = 97
    cnt = (model.M + stride - 1) // stride
    counts, stats, dump = ctx.transitions(model, _dev(g), model.M, model.seed, B.options(), dump_count=cnt,
                                          dump_stride=stride)
    assert stats.form_used == B.FORM_TC_RECHECK and stats.device_status == 0
    off = model.offsets()
    for k in range(model.n):
        X, Y = oracle.sample_pairs(model.d, oracle.PREC_F32, model.seed, k, 0, model.M, model.m[k], model.L[k],
                                   model.A[k], model.b[k], model.T[k])
        X, Y = X[::stride], Y[::stride]
        np.testing.assert_array_equal(dump["X"][k].cpu().numpy(), X)
        np.testing.assert_array_equal(dump["Y"][k].cpu().numpy(), Y)
        np.testing.assert_array_equal(dump["i"][k].cpu().numpy(), oracle.nearest(g[off[k]:off[k + 1]], X))
        np.testing.assert_array_equal(dump["j"][k].cpu().numpy(), oracle.nearest(g[off[k + 1]:off[k + 2]], Y))


def test_tensor_core_adversarial_near_ties(ctx, B):
    rng = np.random.default_rng(12)
    for d, N in ((2, 300), (4, 600), (8, 900), (10, 700)):
        gA = rng.standard_normal((N, d))
        gB = rng.standard_normal((N + 37, d)) * 1.1
        X = np.concatenate([W.boundary_samples(gA, 2000, seed=5), W.boundary_samples(gA, 2000, seed=6, jitter=1e-6),
                            rng.standard_normal((2000, d)), rng.standard_normal((50, d)) * 40.0])
        Y = np.concatenate([W.boundary_samples(gB, 2000, seed=7), W.boundary_samples(gB, 2000, seed=8, jitter=1e-8),
                            rng.standard_normal((2050, d))])
        counts, stats, ii, jj = ctx.counts_from_samples(_dev(gA), _dev(gB), _dev(X), _dev(Y),
                                                        B.options(form=B.FORM_TC_RECHECK), want_cells=True)
        np.testing.assert_array_equal(ii.cpu().numpy(), oracle.nearest(gA, X))
        np.testing.assert_array_equal(jj.cpu().numpy(), oracle.nearest(gB, Y))
        assert stats.rechecks > 100


@pytest.mark.parametrize("d", [1, 3, 5, 7, 9])
def test_tensor_core_odd_dimensions(ctx, B, d):
    """Dimensions between the compiled classes (zero-padded operand columns): cells of
    near-tie, jittered and Gaussian samples against the oracle's exact search."""
    rng = np.random.default_rng(100 + d)
    N = 257 + 40 * d                      # a second, ragged operand tile
    gA = rng.standard_normal((N, d))
    gB = rng.standard_normal((N + 29, d)) * 0.8
    X = np.concatenate([W.boundary_samples(gA, 1500, seed=d), W.boundary_samples(gA, 500, seed=d + 50, jitter=1e-6),
                        rng.standard_normal((1003, d))])
    Y = np.concatenate([W.boundary_samples(gB, 1500, seed=d + 7), rng.standard_normal((1503, d)) * 1.3])
    counts, stats, ii, jj = ctx.counts_from_samples(_dev(gA), _dev(gB), _dev(X), _dev(Y),
                                                    B.options(form=B.FORM_TC_RECHECK), want_cells=True)
    np.testing.assert_array_equal(ii.cpu().numpy(), oracle.nearest(gA, X))
    np.testing.assert_array_equal(jj.cpu().numpy(), oracle.nearest(gB, Y))
    np.testing.assert_array_equal(counts.cpu().numpy(), oracle.counts_from_samples(gA, gB, X, Y))
    assert stats.form_used == B.FORM_TC_RECHECK


def test_tensor_core_fp64_samples_and_u32_counts(ctx, B):
    """Tensor-core form on FP64 samples (the draw pass centres FP64 pairs) with uint32
    counts, against the oracle's FP64 sampler and exact search."""
    model = _model("ar8", M=3001, n=2, N=700)
    g = W.layer_grids(model, samples=20000, iters=3)
    counts, stats, _ = ctx.transitions(model, _dev(g), model.M, model.seed,
                                       B.options(form=B.FORM_TC_RECHECK, prec=B.PREC_F64,
                                                 counts_type=B.COUNTS_U32))
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F64)
    got = B.split_counts(model.N, counts.cpu().numpy().astype(np.int64))
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
    assert stats.form_used == B.FORM_TC_RECHECK and stats.device_status == 0


@pytest.mark.parametrize("draw", [1, 2], ids=["draw-pass", "draw-in-kernel"])
def test_tensor_core_timeout_is_reported(ctx, B, draw):
    model = _model("ar8", M=600, n=2, N=4000)
    g = _dev(W.layer_grids(model, samples=12000, iters=2))
    with pytest.raises(B.QtError) as e:
        ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_TC_RECHECK, spin_budget=-1,
                                                                 tc_draw=draw))
    assert e.value.status == B.QT_ETIMEOUT
    counts, _, _ = ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_TC_RECHECK))
    assert int(counts.sum()) == model.n * model.M


def test_dump_samples_and_cells_bit_exact(ctx, B):
    """Every drawn (X_k, Y) and both cells, against the oracle's own sampler and search."""
    model = _model("ou2", M=5000, n=3, N=200)
    g = _grids(model)
    _, _, dump = ctx.transitions(model, _dev(g), model.M, model.seed, B.options(prec=B.PREC_F32),
                                 dump_count=model.M, dump_stride=1)
    off = model.offsets()
    for k in range(model.n):
        X, Y = oracle.sample_pairs(model.d, oracle.PREC_F32, model.seed, k, 0, model.M, model.m[k], model.L[k],
                                   model.A[k], model.b[k], model.T[k])
        np.testing.assert_array_equal(dump["X"][k].cpu().numpy(), X)
        np.testing.assert_array_equal(dump["Y"][k].cpu().numpy(), Y)
        np.testing.assert_array_equal(dump["i"][k].cpu().numpy(), oracle.nearest(g[off[k]:off[k + 1]], X))
        np.testing.assert_array_equal(dump["j"][k].cpu().numpy(), oracle.nearest(g[off[k + 1]:off[k + 2]], Y))


def test_dump_fp64_sampler_bit_exact(ctx, B):
    model = _model("bs1d", M=4000)
    g = _grids(model)
    _, _, dump = ctx.transitions(model, _dev(g), model.M, model.seed,
                                 B.options(form=B.FORM_PLAIN_F64, prec=B.PREC_F64), dump_count=1000, dump_stride=4)
    for k in (0, 5, 9):
        X, Y = oracle.sample_pairs(1, oracle.PREC_F64, model.seed, k, 0, model.M, model.m[k], model.L[k],
                                   model.A[k], model.b[k], model.T[k])
        np.testing.assert_array_equal(dump["X"][k].cpu().numpy(), X[::4])
        np.testing.assert_array_equal(dump["Y"][k].cpu().numpy(), Y[::4])


@pytest.mark.parametrize("flag", ["smem", "global"])
def test_histogram_modes_and_u32(ctx, B, flag):
    model = _model("bs1d", M=300007)
    g = _grids(model)
    f = B.FLAG_SMEM_HIST if flag == "smem" else B.FLAG_GLOBAL_HIST
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F64)
    for ct in (B.COUNTS_I64, B.COUNTS_U32):
        counts, _, _ = ctx.transitions(model, _dev(g), model.M, model.seed,
                                       B.options(form=B.FORM_F32_RECHECK, prec=B.PREC_F64, flags=f, counts_type=ct))
        got = B.split_counts(model.N, counts.cpu().numpy().astype(np.int64))
        for k in range(model.n):
            np.testing.assert_array_equal(got[k], ref[k])


def test_adversarial_near_ties_force_rechecks(ctx, B):
    """Samples on and next to Voronoi bisectors: the screen cannot certify them,
    the FP64 recheck must give the oracle's cells (ties to the lowest index)."""
    rng = np.random.default_rng(11)
    for d, N in ((1, 64), (2, 300), (4, 500), (10, 400)):
        gA = rng.standard_normal((N, d))
        gB = rng.standard_normal((N + 17, d)) * 1.2
        if d == 1:
            gA = np.sort(np.round(gA * 64) / 64, axis=0)   # dyadic points: exact midpoints, exact ties
        X = np.concatenate([W.boundary_samples(gA, 3000, seed=1),
                            W.boundary_samples(gA, 3000, seed=2, jitter=1e-7),
                            rng.standard_normal((2000, d))])
        Y = np.concatenate([W.boundary_samples(gB, 3000, seed=3),
                            W.boundary_samples(gB, 3000, seed=4, jitter=1e-9),
                            rng.standard_normal((2000, d))])
        counts, stats, ii, jj = ctx.counts_from_samples(_dev(gA), _dev(gB), _dev(X), _dev(Y),
                                                        B.options(form=B.FORM_F32_RECHECK), want_cells=True)
        np.testing.assert_array_equal(ii.cpu().numpy(), oracle.nearest(gA, X))
        np.testing.assert_array_equal(jj.cpu().numpy(), oracle.nearest(gB, Y))
        np.testing.assert_array_equal(counts.cpu().numpy(), oracle.counts_from_samples(gA, gB, X, Y))
        assert stats.rechecks > 100, (d, stats.rechecks)


def test_duplicate_grid_points_tie_to_lowest_index(ctx, B):
    gA = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0]])
    gB = np.array([[0.5, 0.5], [0.5, 0.5]])
    X = np.array([[0.1, 0.0], [0.9, 1.0], [0.5, 0.5], [0.0, 0.0]])
    Y = X.copy()
    counts, _, ii, jj = ctx.counts_from_samples(_dev(gA), _dev(gB), _dev(X), _dev(Y), want_cells=True)
    np.testing.assert_array_equal(ii.cpu().numpy(), [0, 1, 0, 0])
    np.testing.assert_array_equal(jj.cpu().numpy(), [0, 0, 0, 0])


def test_degenerate_sizes(ctx, B):
    """M = 1, single-point layers, a ragged tail smaller than one warp."""
    model = W.ou2(M=1, n=3, N=1)
    g = _grids(model)
    counts, _, _ = ctx.transitions(model, _dev(g), 1, model.seed)
    assert counts.cpu().numpy().tolist() == [1, 1, 1]
    model = W.ou2(M=19, n=2, N=37)
    g = _grids(model)
    counts, _, _ = ctx.transitions(model, _dev(g), model.M, model.seed)
    ref = oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k])


def test_max_dimension_16(ctx, B):
    rng = np.random.default_rng(3)
    d, n, N, M = 16, 2, 200, 2003
    A = np.repeat(np.eye(d)[None] * 0.95, n, 0)
    T = np.repeat(np.eye(d)[None] * 0.1, n, 0)
    L = np.concatenate([np.zeros((1, d, d)), np.repeat(np.eye(d)[None] * 0.3, n, 0)])
    model = W.Model("d16", d, n, np.array([1, N, N]), A, np.zeros((n, d)), T, np.zeros((n + 1, d)), L,
                    np.arange(n + 1.0), 0.0, "max_call", 1.0, None, M, 77, 1, "kmeans")
    g = np.concatenate([np.zeros((1, d)), rng.standard_normal((2 * N, d)) * 0.3])
    counts, _, _ = ctx.transitions(model, _dev(g), M, 77)
    ref = oracle.transitions(model, g, M, 77, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(n):
        np.testing.assert_array_equal(got[k], ref[k])


def test_graph_replay_and_direct_launch_agree(ctx, B):
    model = _model("ou2", M=40000, n=4)
    g = _dev(_grids(model))
    a, _, _ = ctx.transitions(model, g, model.M, model.seed)
    b, _, _ = ctx.transitions(model, g, model.M, model.seed)          # cached graph replay
    c, _, _ = ctx.transitions(model, g, model.M, model.seed, B.options(flags=B.FLAG_NO_GRAPH))
    d, _, _ = ctx.transitions(model, g, model.M, model.seed + 1)      # new key -> new graph
    assert torch.equal(a, b) and torch.equal(a, c)
    assert not torch.equal(a, d)


def test_price_matches_oracle_with_host_buffers(ctx, B):
    model = W.bs1d(M=200000)
    g = _grids(model)
    phi = W.payoff_values(model, g)
    p_host, _ = ctx.price(model, g, model.M, model.seed, phi, B.options(form=B.FORM_PLAIN_F64, prec=B.PREC_F64))
    p_dev, _ = ctx.price(model, _dev(g), model.M, model.seed, _dev(phi),
                         B.options(form=B.FORM_PLAIN_F64, prec=B.PREC_F64))
    ref = oracle.price(model.N, oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F64), phi)
    assert p_host == p_dev
    assert abs(p_dev - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("name,N,form,flags", [("ou2", 64, "f32", 0), ("ou2", 500, "f32", 0),
                                                ("basket4", 0, "tc", 0), ("ou2", 300, "f32", "graph")])
def test_fused_backward_price_is_bit_identical(ctx, B, name, N, form, flags):
    """Layer pairs in reverse order, each pair's counts folded into V at once (one pair's
    counts in memory): the same price bits as the unfused path, and the oracle's within 1e-12."""
    model = _model(name, M=20011, n=4, N=N) if N else _model(name, M=20011, n=4)
    g = W.layer_grids(model, samples=20000, iters=3) if model.grid_kind == "kmeans" else W.layer_grids(model)
    phi = W.payoff_values(model, g)
    f = B.FORM_F32_RECHECK if form == "f32" else B.FORM_TC_RECHECK
    base = 0 if flags == "graph" else B.FLAG_NO_GRAPH
    p0, _ = ctx.price(model, _dev(g), model.M, model.seed, _dev(phi), B.options(form=f, flags=base))
    p1, st = ctx.price(model, _dev(g), model.M, model.seed, _dev(phi),
                       B.options(form=f, flags=base | B.FLAG_FUSED_BACKWARD))
    assert st.device_status == 0
    assert p1 == p0
    ref = oracle.price(model.N, oracle.transitions(model, g, model.M, model.seed, oracle.PREC_F32), phi)
    assert abs(p1 - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("layer", [3, 1])
def test_fused_backward_reports_a_timeout_in_one_layer(ctx, B, layer):
    """A bounded wait that gives up in one layer pair k > 0 only (host-side injection:
    that layer's launch alone gets a negative wait budget) must reach the caller of the
    fused price, although the layers after it (k - 1 .. 0) run clean launches."""
    model = _model("ou2", M=20011, n=4, N=64)
    g = _dev(_grids(model))
    phi = _dev(W.payoff_values(model, _grids(model)))
    os.environ["QT_FAULT"] = f"timeout_layer:{layer}"
    try:
        with pytest.raises(B.QtError) as e:
            ctx.price(model, g, model.M, model.seed, phi, B.options(form=B.FORM_F32_RECHECK,
                                                                   flags=B.FLAG_FUSED_BACKWARD))
        assert e.value.status == B.QT_ETIMEOUT
    finally:
        del os.environ["QT_FAULT"]
    p, st = ctx.price(model, g, model.M, model.seed, phi, B.options(form=B.FORM_F32_RECHECK,
                                                                   flags=B.FLAG_FUSED_BACKWARD))
    assert st.device_status == 0


def test_build_grids_lloyd1d_and_product(ctx, B):
    model = W.bs1d()
    g = ctx.build_grids(model, B.GRID_LLOYD1D).cpu().numpy()
    ref = W.layer_grids(model)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-11)
    m2 = W.ou2(n=3, N=500)
    g2 = ctx.build_grids(m2, B.GRID_PRODUCT).cpu().numpy()
    np.testing.assert_allclose(g2, W.layer_grids(m2), rtol=0, atol=1e-11)


def test_build_grids_kmeans_is_lloyd_descent(ctx, B):
    """Sample Lloyd on the library's training draws (regenerated bit for bit by the
    oracle's sampler, stream 0xFFFF): the quadratic error of eq. (Qerr) on those
    draws never increases from the start (first N draws) through 1, 4, 15 steps."""
    d, N, S, seed = 8, 256, 60000, 5
    model = W.ar8(M=1000).restrict(n=2, N=N)
    kseed = (seed ^ (0x9E3779B97F4A7C15 * N)) & 0xFFFFFFFFFFFFFFFF
    Z = oracle.normals(oracle.PREC_F32, kseed, 0xFFFF, 0, S, d)
    off = model.offsets()
    dist = [float(np.mean(oracle.nearest_dist(Z[:N], Z)))]
    for it in (1, 4, 15):
        g = ctx.build_grids(model, B.GRID_KMEANS, samples=S, iters=it, seed=seed).cpu().numpy()
        base = np.linalg.solve(model.L[1], (g[off[1]:off[2]] - model.m[1]).T).T
        dist.append(float(np.mean(oracle.nearest_dist(base, Z))))
    assert all(b <= a * (1 + 1e-6) for a, b in zip(dist, dist[1:])), dist
    assert dist[-1] < 0.9 * dist[0], dist


# ------------------------------------------------------------------ full sizes, bench launch configuration

def test_full_size_bs1d_bit_exact(ctx, B):
    """1-d Black-Scholes Bermudan put, M = 10^6, n = 10, plain FP64 (the first workload)."""
    model = W.bs1d()
    g = ctx.build_grids(model, B.GRID_LLOYD1D)
    gn = g.cpu().numpy()
    opts = B.options(form=B.FORM_PLAIN_F64, prec=B.PREC_F64)
    counts, _, _ = ctx.transitions(model, g, model.M, model.seed, opts)
    ref = oracle.transitions(model, gn, model.M, model.seed, oracle.PREC_F64)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k])
    phi = W.payoff_values(model, gn)
    price, _ = ctx.price(model, g, model.M, model.seed, _dev(phi), opts)
    pref = oracle.price(model.N, ref, phi)
    assert abs(price - pref) <= 1e-12 * pref
    assert abs(price - 6.0335) < 0.02               # CRR Bermudan value (10 dates)


def test_full_size_ou2_sampled_outputs(ctx, B):
    """2-factor OU, n = 100, N = 500, M = 10^7 in the benchmark's launch: strided samples
    and their cells against the oracle one by one, plus the count invariants."""
    model = W.ou2()
    g = ctx.build_grids(model, B.GRID_PRODUCT)
    gn = g.cpu().numpy()
    stride = 9973
    cnt = (model.M + stride - 1) // stride
    counts, stats, dump = ctx.transitions(model, g, model.M, model.seed, B.options(), dump_count=cnt,
                                          dump_stride=stride)
    assert stats.device_status == 0
    off = model.offsets()
    got = B.split_counts(model.N, counts)
    for k in (0, 1, 37, 99):
        rows = got[k].sum(dim=1)
        assert int(rows.sum()) == model.M
        m = np.arange(cnt) * stride
        X = np.empty((cnt, 2))
        Y = np.empty((cnt, 2))
        for t, mm in enumerate(m):
            X[t], Y[t] = [a[0] for a in oracle.sample_pairs(2, oracle.PREC_F32, model.seed, k, int(mm), 1,
                                                             model.m[k], model.L[k], model.A[k], model.b[k],
                                                             model.T[k])]
        np.testing.assert_array_equal(dump["X"][k].cpu().numpy(), X)
        np.testing.assert_array_equal(dump["Y"][k].cpu().numpy(), Y)
        np.testing.assert_array_equal(dump["i"][k].cpu().numpy(), oracle.nearest(gn[off[k]:off[k + 1]], X))
        np.testing.assert_array_equal(dump["j"][k].cpu().numpy(), oracle.nearest(gn[off[k + 1]:off[k + 2]], Y))
    # column sums of layer k-1 and row sums of layer k both estimate the law of X_k
    c1 = got[1].sum(dim=1).double()
    c0 = got[0].sum(dim=0).double()
    z = (c1 - c0) / torch.sqrt(torch.clamp(c1 + c0, min=1.0))
    assert float(z.abs().max()) < 6.0


# ------------------------------------------------------------------ failure paths (host-made, no GPU fault)

def test_bounded_wait_timeout_is_reported_and_context_survives(ctx, B):
    """The plain FP64 form stages its grids by bulk copy and waits on an mbarrier
    (the resident FP32 screen stages them with plain loads and has no such wait)."""
    model = _model("ou2", M=3000, n=2, N=64)
    g = _dev(_grids(model))
    with pytest.raises(B.QtError) as e:
        ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_PLAIN_F64, spin_budget=-1))
    assert e.value.status == B.QT_ETIMEOUT
    counts, stats, _ = ctx.transitions(model, g, model.M, model.seed)
    ref = oracle.transitions(model, g.cpu().numpy(), model.M, model.seed, oracle.PREC_F32)
    got = B.split_counts(model.N, counts.cpu().numpy())
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k])


def test_invalid_arguments_are_rejected(ctx, B):
    model = _model("ou2", M=100, n=2, N=16)
    g = _dev(_grids(model))
    for M in (0, 1 << 32):
        with pytest.raises(B.QtError) as e:
            ctx.transitions(model, g, M, 1)
        assert e.value.status == B.QT_EINVAL
    with pytest.raises(B.QtError) as e:
        ctx.transitions(model, g, 100, 1, B.options(form=17))
    assert e.value.status == B.QT_EINVAL
    bad = W.ou2(M=100, n=2, N=16)
    bad.N[1] = 0
    with pytest.raises(B.QtError) as e:
        ctx.transitions(bad, g, 100, 1)
    assert e.value.status == B.QT_EINVAL


def test_injected_allocation_failure(B):
    c = B.Context(0)
    try:
        model = _model("ou2", M=100, n=2, N=16)
        g = _dev(_grids(model))
        os.environ["QT_FAULT"] = "alloc"
        try:
            with pytest.raises(B.QtError) as e:
                c.transitions(model, g, 100, 1)
            assert e.value.status == B.QT_ENOMEM
        finally:
            del os.environ["QT_FAULT"]
        counts, _, _ = c.transitions(model, g, 100, 1)
        assert int(counts.sum()) == 2 * 100
    finally:
        c.close()
