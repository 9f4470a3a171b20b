"""The allocation-free counting entry point, called through the C ABI.

qt_counts_from_samples_noalloc serves callers that cannot allocate device
memory (an application whose allocator already owns the device memory, a
plug-in that may not own any, a loop that cannot afford cudaMalloc's implicit
synchronisation).  Its scratch is a fixed array inside the library, shared by
every call on a device.  This file is collected last so that a failure here
leaves every other test already run.  Two calls in a row, with different
sizes, must each equal qt_counts_from_samples on the same inputs (counts and
cells bit for bit, the tolerance of every count test), which also shows that
the shared scratch keeps nothing from the previous call.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(lib, gA, gB, X, Y, counts_type=0, stream=None):
    import torch
    dt = torch.int64 if counts_type == 0 else torch.int32
    counts = torch.full((gA.shape[0], gB.shape[0]), 7, dtype=dt, device="cuda")   # overwritten
    ii = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    jj = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    st = lib.qt_counts_from_samples_noalloc(
        int(gA.shape[1]), gA.data_ptr(), gA.shape[0], gB.data_ptr(), gB.shape[0], X.data_ptr(), Y.data_ptr(),
        X.shape[0], counts_type, counts.data_ptr(), ii.data_ptr(), jj.data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    return st, counts, ii, jj


def _case(rng, d, NA, NB, M):
    gA = torch.from_numpy(rng.standard_normal((NA, d))).cuda()
    gB = torch.from_numpy(rng.standard_normal((NB, d)) * 1.3).cuda()
    X = torch.from_numpy(rng.standard_normal((M, d))).cuda()
    Y = torch.from_numpy(rng.standard_normal((M, d)) * 1.2).cuda()
    return gA, gB, X, Y


def test_noalloc_matches_counts_from_samples_twice(gpu_lib):
    from paper_1101_3228_gb300 import binding as B
    lib = B.load()
    ctx = B.Context(0)
    try:
        rng = np.random.default_rng(2024)
        for (d, NA, NB, M, ct) in ((2, 500, 480, 200003, 0), (8, 700, 900, 50021, 1)):
            gA, gB, X, Y = _case(rng, d, NA, NB, M)
            st, counts, ii, jj = _noalloc(lib, gA, gB, X, Y, ct)
            assert st == B.QT_OK
            ref, _, rii, rjj = ctx.counts_from_samples(gA, gB, X, Y, B.options(form=B.FORM_F32_RECHECK,
                                                                               counts_type=ct), want_cells=True)
            assert torch.equal(counts, ref)
            assert torch.equal(ii, rii) and torch.equal(jj, rjj)
            assert int(counts.sum()) == M
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    from paper_1101_3228_gb300 import binding as B
    lib = B.load()
    rng = np.random.default_rng(1)
    gA, gB, X, Y = _case(rng, 2, 3000, 2000, 100)     # NA + NB > QT_NOALLOC_MAX_POINTS
    st, _, _, _ = _noalloc(lib, gA, gB, X, Y)
    assert st == B.QT_EINVAL


def test_noalloc_rejects_records_beyond_shared_memory(gpu_lib):
    """d = 16 with 4096 points fits the scratch array but not one CTA's shared memory
    (about 330 KB of screened records): rejected before any work is enqueued."""
    from paper_1101_3228_gb300 import binding as B
    lib = B.load()
    rng = np.random.default_rng(5)
    gA, gB, X, Y = _case(rng, 16, 2048, 2048, 64)
    st, _, _, _ = _noalloc(lib, gA, gB, X, Y)
    assert st == B.QT_EINVAL


@pytest.mark.parametrize("d,NA,NB,M", [(1, 100, 37, 5003), (3, 300, 211, 2011), (16, 200, 150, 1999)])
def test_noalloc_matches_the_oracle(gpu_lib, d, NA, NB, M):
    """Small cases at the dimension bounds against the FP64 oracle's brute-force
    cells and counts, with near-tie samples on the grids' bisectors."""
    import qt_workloads as W
    from paper_1101_3228_gb300 import binding as B
    lib = B.load()
    rng = np.random.default_rng(40 + d)
    ga = rng.standard_normal((NA, d))
    gb = rng.standard_normal((NB, d)) * 1.2
    half = M // 2
    x = np.concatenate([W.boundary_samples(ga, half, seed=d), rng.standard_normal((M - half, d))])
    y = np.concatenate([rng.standard_normal((M - half, d)), W.boundary_samples(gb, half, seed=d + 1)])
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ga, gb, x, y)]
    for _ in range(2):
        st, counts, ii, jj = _noalloc(lib, *dev)
        assert st == B.QT_OK
        np.testing.assert_array_equal(ii.cpu().numpy(), oracle.nearest(ga, x))
        np.testing.assert_array_equal(jj.cpu().numpy(), oracle.nearest(gb, y))
        np.testing.assert_array_equal(counts.cpu().numpy(), oracle.counts_from_samples(ga, gb, x, y))
