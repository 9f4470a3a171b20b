"""Thin Python binding of libqt (include/qt.h): argument marshalling only.

Every step of the quantization-tree path runs in the library's CUDA kernels.
PyTorch supplies device memory and streams; numpy arrays carry the host-side
model description.  Loading fails loudly when libqt.so is missing or no GPU is
present: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqt.so")

QT_OK, QT_EINVAL, QT_ENOMEM, QT_ECUDA, QT_ETIMEOUT, QT_EUNSUPPORTED, QT_EDEVICE = range(7)
FORM_AUTO, FORM_PLAIN_F64, FORM_F32_RECHECK, FORM_TC_RECHECK, FORM_ROUTER_CERT = range(5)
PREC_F64, PREC_F32 = 0, 1
COUNTS_I64, COUNTS_U32 = 0, 1
FLAG_NO_GRAPH, FLAG_NO_TUNE, FLAG_SMEM_HIST, FLAG_GLOBAL_HIST, FLAG_FUSED_BACKWARD = 1, 2, 4, 8, 16
GRID_LLOYD1D, GRID_PRODUCT, GRID_KMEANS = 1, 2, 3

FORM_NAMES = {FORM_AUTO: "auto", FORM_PLAIN_F64: "plain_f64", FORM_F32_RECHECK: "f32_recheck",
              FORM_TC_RECHECK: "tc_recheck", FORM_ROUTER_CERT: "router_cert"}

# every symbol include/qt.h declares (checked by the CPU test of the ABI)
EXPORTS = ["qt_create", "qt_destroy", "qt_last_error", "qt_status_string", "qt_default_options",
           "qt_build_grids", "qt_transitions", "qt_transitions_pathwise", "qt_counts_from_samples",
           "qt_backward", "qt_swing", "qt_price",
           "qt_get_status", "qt_transitions_workspace", "qt_counts_from_samples_noalloc",
           "qt_router_train", "qt_router_destroy", "qt_router_get_info", "qt_router_get_params",
           "qt_router_set_params", "qt_router_loss_grad"]

P = ctypes.c_void_p
i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64


class QtModel(ctypes.Structure):
    _fields_ = [("d", i32), ("n", i32), ("N", P), ("A", P), ("b", P), ("T", P), ("m", P), ("L", P)]


class QtOptions(ctypes.Structure):
    _fields_ = [("form", i32), ("sample_prec", i32), ("counts_type", i32), ("flags", u32),
                ("spin_budget", i64), ("router", P), ("tile_samples_per_thread", i32), ("tc_chunk_items", i32), ("tc_draw", i32),
                ("reserved", i32 * 1)]


class QtDump(ctypes.Structure):
    _fields_ = [("count", i64), ("stride", i64), ("X", P), ("Y", P), ("i", P), ("j", P)]


class QtEuler(ctypes.Structure):
    _fields_ = [("alpha", P), ("beta", P)]


class QtStats(ctypes.Structure):
    _fields_ = [("samples", i64), ("rechecks", i64), ("searches", i64), ("candidates", i64),
                ("form_used", i32), ("device_status", i32), ("ms", ctypes.c_double), ("diag", i64 * 3),
                ("launches", i32), ("tc_draw", i32)]


class QtRouterConfig(ctypes.Structure):
    _fields_ = [("train_samples", i64), ("train_layers", i32), ("epochs", i32), ("batch", i32),
                ("neighbours", i32), ("lr", ctypes.c_float), ("untrained", i32), ("reserved", i32 * 3)]


class QtRouterInfo(ctypes.Structure):
    _fields_ = [("params", i64), ("d", i32), ("buckets", i32), ("hidden", i32), ("neighbours", i32),
                ("train_loss", ctypes.c_double), ("train_accuracy", ctypes.c_double), ("build_ms", ctypes.c_double)]


class QtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libqt status {status}: {msg}")
        self.status = status


_lib = None

_SIGS = {
    "qt_create": (i32, [P, i32]),
    "qt_destroy": (i32, [P]),
    "qt_last_error": (ctypes.c_char_p, [P]),
    "qt_status_string": (ctypes.c_char_p, [i32]),
    "qt_default_options": (None, [P]),
    "qt_build_grids": (i32, [P, P, i32, i64, i32, ctypes.c_double, u64, P, P]),
    "qt_transitions": (i32, [P, P, P, i64, u64, P, P, P, P, P]),
    "qt_transitions_pathwise": (i32, [P, P, P, P, i64, u64, P, P, P, P, P]),
    "qt_counts_from_samples": (i32, [P, i32, P, i64, P, i64, P, P, i64, P, P, P, P, P, P]),
    "qt_backward": (i32, [P, i32, P, P, i32, P, P, P]),
    "qt_price": (i32, [P, P, P, i64, u64, P, P, P, P, P]),
    "qt_swing": (i32, [P, i32, P, P, i32, P, i32, i32, P, P, P]),
    "qt_get_status": (i32, [P, P, P]),
    "qt_transitions_workspace": (i32, [P, P, P]),
    "qt_counts_from_samples_noalloc": (i32, [i32, P, i64, P, i64, P, P, i64, i32, P, P, P, P]),
    "qt_router_train": (i32, [P, P, P, P, u64, P, P]),
    "qt_router_destroy": (i32, [P]),
    "qt_router_get_info": (i32, [P, P]),
    "qt_router_get_params": (i32, [P, P, i64]),
    "qt_router_set_params": (i32, [P, P, i64]),
    "qt_router_loss_grad": (i32, [P, P, P, P, i64, P, P, P]),
}


def load(path: Optional[str] = None):
    """Load libqt.so (built by paper_1101_3228_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libqt.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(t) -> int:
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class HostModel:
    """Keeps the contiguous FP64 host arrays of a model alive for a call."""

    def __init__(self, model):
        self.d = int(model.d)
        self.n = int(model.n)
        self.N = np.ascontiguousarray(model.N, dtype=np.int64)
        self.A = np.ascontiguousarray(model.A, dtype=np.float64)
        self.b = np.ascontiguousarray(model.b, dtype=np.float64)
        self.T = np.ascontiguousarray(model.T, dtype=np.float64)
        self.m = np.ascontiguousarray(model.m, dtype=np.float64)
        self.L = np.ascontiguousarray(model.L, dtype=np.float64)
        assert self.N.shape == (self.n + 1,)
        assert self.A.shape == (self.n, self.d, self.d) and self.T.shape == (self.n, self.d, self.d)
        assert self.m.shape == (self.n + 1, self.d) and self.L.shape == (self.n + 1, self.d, self.d)
        self.c = QtModel(self.d, self.n, self.N.ctypes.data, self.A.ctypes.data, self.b.ctypes.data,
                         self.T.ctypes.data, self.m.ctypes.data, self.L.ctypes.data)

    @property
    def count_entries(self) -> int:
        return int(np.sum(self.N[:-1] * self.N[1:]))

    @property
    def total_points(self) -> int:
        return int(np.sum(self.N))


def options(form=FORM_AUTO, prec=PREC_F32, counts_type=COUNTS_I64, flags=0, spin_budget=0, router=None,
            samples_per_thread=0, tc_chunk_items=0, tc_draw=0) -> QtOptions:
    o = QtOptions()
    o.form, o.sample_prec, o.counts_type, o.flags = form, prec, counts_type, flags
    o.spin_budget = spin_budget
    o.router = router
    o.tile_samples_per_thread = samples_per_thread
    o.tc_chunk_items = tc_chunk_items
    o.tc_draw = tc_draw
    return o


class Context:
    """One libqt context on one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libqt needs a CUDA device; none is available")
        self.lib = load()
        self.device = device
        torch.cuda.init()
        h = P()
        st = self.lib.qt_create(ctypes.byref(h), device)
        if st != QT_OK:
            raise QtError(st, self.lib.qt_status_string(st).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.qt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != QT_OK:
            raise QtError(st, self.lib.qt_last_error(self.h).decode())

    # ----------------------------------------------------------------- calls

    def build_grids(self, model, method: int, samples: int = 0, iters: int = 0, tol: float = 1e-14,
                    seed: int = 0, stream=None):
        import torch
        hm = HostModel(model)
        grids = torch.empty((hm.total_points, hm.d), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self.lib.qt_build_grids(self.h, ctypes.byref(hm.c), method, samples, iters, tol, seed,
                                            _ptr(grids), _stream_ptr(stream)))
        return grids

    def transitions(self, model, grids, M: int, seed: int, opts: Optional[QtOptions] = None, counts=None,
                    dump_count: int = 0, dump_stride: int = 1, want_stats: bool = True, stream=None):
        """Algorithm III counts (flat tensor, concatenated [N_k][N_{k+1}] blocks), stats, dump."""
        import torch
        hm = HostModel(model)
        opts = opts or options()
        dt = torch.int64 if opts.counts_type == COUNTS_I64 else torch.int32
        dev = grids.device
        if counts is None:
            counts = torch.empty(hm.count_entries, dtype=dt, device=dev)
        dump = None
        dump_t = None
        if dump_count > 0:
            dump_t = dict(X=torch.empty((hm.n, dump_count, hm.d), dtype=torch.float64, device=dev),
                          Y=torch.empty((hm.n, dump_count, hm.d), dtype=torch.float64, device=dev),
                          i=torch.empty((hm.n, dump_count), dtype=torch.int32, device=dev),
                          j=torch.empty((hm.n, dump_count), dtype=torch.int32, device=dev))
            dump = QtDump(dump_count, dump_stride, _ptr(dump_t["X"]), _ptr(dump_t["Y"]), _ptr(dump_t["i"]),
                          _ptr(dump_t["j"]))
        stats = QtStats() if want_stats else None
        self._check(self.lib.qt_transitions(self.h, ctypes.byref(hm.c), _ptr(grids), int(M), int(seed),
                                            ctypes.byref(opts), _ptr(counts),
                                            ctypes.byref(dump) if dump is not None else None,
                                            ctypes.byref(stats) if stats is not None else None,
                                            _stream_ptr(stream)))
        return counts, stats, dump_t

    def transitions_pathwise(self, model, grids, M: int, seed: int, opts: Optional[QtOptions] = None, euler=None,
                             counts=None, dump_count: int = 0, dump_stride: int = 1, want_stats: bool = True,
                             stream=None):
        """Algorithm II counts (same layout as transitions), stats, dump.  euler: None (AR(1)
        chain) or (alpha, beta) host arrays [n, d] of the Euler-scheme chain."""
        import torch
        hm = HostModel(model)
        opts = opts or options()
        dt = torch.int64 if opts.counts_type == COUNTS_I64 else torch.int32
        dev = grids.device
        if counts is None:
            counts = torch.empty(hm.count_entries, dtype=dt, device=dev)
        eu = None
        keep = None
        if euler is not None:
            keep = [np.ascontiguousarray(euler[0], dtype=np.float64).reshape(hm.n, hm.d),
                    np.ascontiguousarray(euler[1], dtype=np.float64).reshape(hm.n, hm.d)]
            eu = QtEuler(keep[0].ctypes.data, keep[1].ctypes.data)
        dump = None
        dump_t = None
        if dump_count > 0:
            dump_t = dict(X=torch.empty((hm.n, dump_count, hm.d), dtype=torch.float64, device=dev),
                          Y=torch.empty((hm.n, dump_count, hm.d), dtype=torch.float64, device=dev),
                          i=torch.empty((hm.n, dump_count), dtype=torch.int32, device=dev),
                          j=torch.empty((hm.n, dump_count), dtype=torch.int32, device=dev))
            dump = QtDump(dump_count, dump_stride, _ptr(dump_t["X"]), _ptr(dump_t["Y"]), _ptr(dump_t["i"]),
                          _ptr(dump_t["j"]))
        stats = QtStats() if want_stats else None
        self._check(self.lib.qt_transitions_pathwise(self.h, ctypes.byref(hm.c),
                                                     ctypes.byref(eu) if eu is not None else None, _ptr(grids),
                                                     int(M), int(seed), ctypes.byref(opts), _ptr(counts),
                                                     ctypes.byref(dump) if dump is not None else None,
                                                     ctypes.byref(stats) if stats is not None else None,
                                                     _stream_ptr(stream)))
        del keep
        return counts, stats, dump_t

    def counts_from_samples(self, gA, gB, X, Y, opts: Optional[QtOptions] = None, want_cells: bool = False,
                            stream=None):
        import torch
        opts = opts or options()
        d = int(gA.shape[1])
        dt = torch.int64 if opts.counts_type == COUNTS_I64 else torch.int32
        counts = torch.empty((gA.shape[0], gB.shape[0]), dtype=dt, device=gA.device)
        ii = jj = None
        if want_cells:
            ii = torch.empty(X.shape[0], dtype=torch.int32, device=gA.device)
            jj = torch.empty(X.shape[0], dtype=torch.int32, device=gA.device)
        stats = QtStats()
        self._check(self.lib.qt_counts_from_samples(self.h, d, _ptr(gA), gA.shape[0], _ptr(gB), gB.shape[0],
                                                    _ptr(X), _ptr(Y), X.shape[0], ctypes.byref(opts),
                                                    _ptr(counts), _ptr(ii), _ptr(jj), ctypes.byref(stats),
                                                    _stream_ptr(stream)))
        return counts, stats, ii, jj

    def backward(self, N, counts, phi, counts_type: int = COUNTS_I64, stream=None):
        import torch
        Nh = np.ascontiguousarray(N, dtype=np.int64)
        V = torch.empty_like(phi)
        self._check(self.lib.qt_backward(self.h, len(Nh) - 1, Nh.ctypes.data, _ptr(counts), counts_type,
                                         _ptr(phi), _ptr(V), _stream_ptr(stream)))
        return V

    def swing(self, N, counts, v, Qmin: int, Qmax: int, counts_type: int = COUNTS_I64, stream=None):
        """Swing values P (flat, Q-major blocks [Qmax+1, N_k] per layer) and the price."""
        import torch
        Nh = np.ascontiguousarray(N, dtype=np.int64)
        P_ = torch.empty(int(np.sum(Nh)) * (Qmax + 1), dtype=torch.float64, device=v.device)
        out = ctypes.c_double(0.0)
        self._check(self.lib.qt_swing(self.h, len(Nh) - 1, Nh.ctypes.data, _ptr(counts), counts_type, _ptr(v),
                                      int(Qmin), int(Qmax), _ptr(P_), ctypes.byref(out), _stream_ptr(stream)))
        return P_, out.value

    def price(self, model, grids, M: int, seed: int, phi, opts: Optional[QtOptions] = None, stream=None):
        """grids / phi may be torch CUDA tensors or host numpy arrays (copied in by the library)."""
        hm = HostModel(model)
        opts = opts or options()
        out = ctypes.c_double(0.0)
        stats = QtStats()
        if isinstance(grids, np.ndarray):
            grids = np.ascontiguousarray(grids, dtype=np.float64)
        if isinstance(phi, np.ndarray):
            phi = np.ascontiguousarray(phi, dtype=np.float64)
        self._check(self.lib.qt_price(self.h, ctypes.byref(hm.c), _ptr(grids), int(M), int(seed),
                                      ctypes.byref(opts), _ptr(phi), ctypes.byref(out), ctypes.byref(stats),
                                      _stream_ptr(stream)))
        return out.value, stats

    def router_train(self, model, grids, samples: int = 200000, layers: int = 4, epochs: int = 0,
                     batch: int = 4096, neighbours: int = 0, lr: float = 0.0, untrained: bool = False,
                     seed: int = 7, stream=None) -> "Router":
        hm = HostModel(model)
        cfg = QtRouterConfig(samples, layers, epochs, batch, neighbours, lr, 1 if untrained else 0)
        h = P()
        self._check(self.lib.qt_router_train(self.h, ctypes.byref(hm.c), _ptr(grids), ctypes.byref(cfg), seed,
                                             ctypes.byref(h), _stream_ptr(stream)))
        return Router(self, h)

    def status(self, stream=None):
        stats = QtStats()
        st = self.lib.qt_get_status(self.h, _stream_ptr(stream), ctypes.byref(stats))
        return st, stats

    def workspace_bytes(self, model, opts: Optional[QtOptions] = None) -> int:
        hm = HostModel(model)
        opts = opts or options()
        out = ctypes.c_size_t(0)
        self._check(self.lib.qt_transitions_workspace(ctypes.byref(hm.c), ctypes.byref(opts), ctypes.byref(out)))
        return out.value


class Router:
    """A trained router (qt_router*), usable as options(form=FORM_ROUTER_CERT, router=r.handle)."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.lib = ctx.lib
        self.h = h

    @property
    def handle(self):
        return self.h.value

    def info(self) -> QtRouterInfo:
        out = QtRouterInfo()
        self.ctx._check(self.lib.qt_router_get_info(self.h, ctypes.byref(out)))
        return out

    def params(self) -> np.ndarray:
        n = self.info().params
        out = np.empty(n, dtype=np.float32)
        self.ctx._check(self.lib.qt_router_get_params(self.h, out.ctypes.data, n))
        return out

    def set_params(self, values) -> None:
        v = np.ascontiguousarray(values, dtype=np.float32)
        self.ctx._check(self.lib.qt_router_set_params(self.h, v.ctypes.data, v.size))

    def loss_grad(self, z, labels, stream=None):
        import torch
        grad = torch.empty(self.info().params, dtype=torch.float32, device=z.device)
        loss = ctypes.c_double(0.0)
        self.ctx._check(self.lib.qt_router_loss_grad(self.ctx.h, self.h, _ptr(z), _ptr(labels), z.shape[0],
                                                     _ptr(grad), ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value, grad

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.qt_router_destroy(self.h)
            self.h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split_counts(N, flat):
    """Flat concatenated counts -> list of [N_k, N_{k+1}] views."""
    N = np.asarray(N, dtype=np.int64)
    out, off = [], 0
    for k in range(len(N) - 1):
        sz = int(N[k] * N[k + 1])
        out.append(flat[off:off + sz].reshape(int(N[k]), int(N[k + 1])))
        off += sz
    return out
