"""GPU parity at the workloads' full grid sizes, in the launch configuration the
benchmark times, against the CPU oracle (Algorithm III of Pages & Wilbertz,
arXiv:1101.3228, Sec. 4: the counts p^k_ij are the definition, so every count
matrix compared is compared bit for bit).

* 2-factor OU (d = 2, N = 500): M = 10^7, five whole layers;
* 4-d basket (N_k from 200 to 2000): M = 10^6, all 50 layers;
* 8-d AR(1) (N = 4000): M = 10^6, four layers;
* 10-d AR(1) max-call (N = 8000): M = 10^6 (the parity subsample of the
  full-size workload), two layers, uint32 counts as in the benchmark;
* the tensor-core form forced through several draw/forward passes with a
  ragged last pass (the chunk loop the full-size runs take);
* prices of the fused reverse-order mode at the 8-d size within 1e-12.

Grids are built by the library (qt_build_grids) with the benchmark's recipe and
copied to the host for the oracle.  Each case takes seconds to about a minute
of oracle time on the host cores.
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


def _bench_grids(ctx, B, model):
    """The benchmark's grids: product grids for the 2-factor model, sample Lloyd otherwise."""
    method = {"lloyd1d": B.GRID_LLOYD1D, "product": B.GRID_PRODUCT, "kmeans": B.GRID_KMEANS}[model.grid_kind]
    return ctx.build_grids(model, method, samples=max(20 * int(np.max(model.N)), 200000), iters=20,
                           seed=W.GRID_SEED_BASE + W.CONFIG_INDEX[model.name])


def _compare(B, model, counts, ref):
    got = B.split_counts(model.N, counts.cpu().numpy().astype(np.int64))
    for k in range(model.n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"layer {k}")
        assert int(got[k].sum()) == model.M


@pytest.mark.parametrize("name,n,M,ctype", [
    ("ou2", 5, 10**7, "i64"),
    ("basket4", 50, 10**6, "i64"),
    ("ar8", 4, 10**6, "i64"),
    ("maxcall10", 2, 10**6, "u32"),
])
def test_full_grid_sizes_bit_exact(ctx, B, name, n, M, ctype):
    model = W.get(name, M=M).restrict(n=n)
    g = _bench_grids(ctx, B, model)
    ct = B.COUNTS_I64 if ctype == "i64" else B.COUNTS_U32
    counts, stats, _ = ctx.transitions(model, g, model.M, model.seed, B.options(counts_type=ct))
    assert stats.device_status == 0
    # the automatic form is the one the benchmark times at these sizes
    assert stats.form_used == (B.FORM_TC_RECHECK if 3 <= model.d <= 10 else B.FORM_F32_RECHECK)
    ref = oracle.transitions(model, g.cpu().numpy(), model.M, model.seed, oracle.PREC_F32)
    _compare(B, model, counts, ref)


@pytest.mark.parametrize("draw", [1, 2], ids=["draw-pass", "draw-in-kernel"])
@pytest.mark.parametrize("name,n,N,M,chunk", [
    ("basket4", 50, 0, 4999, 7),          # uneven N_k up to 2000, resident operand tiles
    ("ar8", 3, 4000, 40111, 29),         # streamed operand-tile ring
    ("maxcall10", 2, 8000, 9001, 40),    # streamed ring, K = 32
])
def test_tensor_core_many_passes_bit_exact(ctx, B, name, n, N, M, chunk, draw):
    """Several launches, each over its own window of work items, the last one ragged,
    counts accumulated: with the draw pass (a reused sample buffer in device memory)
    and with the screen kernel drawing its own samples."""
    full = W.get(name, M=M)
    model = full.restrict(n=n, N=N) if N else full.restrict(n=n)
    g = _bench_grids(ctx, B, model)
    items = model.n * ((model.M + 127) // 128)
    assert items // chunk >= 3 and items % chunk != 0
    counts, stats, _ = ctx.transitions(model, g, model.M, model.seed,
                                       B.options(form=B.FORM_TC_RECHECK, tc_chunk_items=chunk, tc_draw=draw))
    assert stats.device_status == 0 and stats.form_used == B.FORM_TC_RECHECK
    ref = oracle.transitions(model, g.cpu().numpy(), model.M, model.seed, oracle.PREC_F32)
    _compare(B, model, counts, ref)
    # the same counts in one launch, in the other layout
    one, _, _ = ctx.transitions(model, g, model.M, model.seed, B.options(form=B.FORM_TC_RECHECK, tc_draw=3 - draw))
    assert torch.equal(one, counts)


def test_full_size_ar8_fused_price(ctx, B):
    """The fused reverse-order price at the 8-d grid size (N = 4000, M = 10^6, four
    layers) against the oracle's backward induction on its own counts."""
    model = W.ar8(M=10**6).restrict(n=4)
    g = _bench_grids(ctx, B, model)
    gn = g.cpu().numpy()
    phi = W.payoff_values(model, gn)
    price, st = ctx.price(model, g, model.M, model.seed, torch.from_numpy(phi).cuda(),
                          B.options(flags=B.FLAG_FUSED_BACKWARD))
    assert st.device_status == 0
    ref = oracle.price(model.N, oracle.transitions(model, gn, model.M, model.seed, oracle.PREC_F32), phi)
    assert abs(price - ref) <= 1e-12 * abs(ref)
