"""FP64 CPU oracle for the Quantization Tree forward step and backward induction.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package, and this package never imports the product library.

The arithmetic lives in ``qt_oracle.c`` (plain C, compiled with
``-ffp-contract=off``, no fast-math).  This module only compiles it, loads it
with ctypes and converts numpy arrays.  Citations (Pages & Wilbertz,
arXiv:1101.3228):

* ``sample_pairs``  -- Prop. 1 (AR(1) form) and the pair draw that precedes
  Algorithm III, with the sampler defined in ``qt_oracle.c``;
* ``nearest``       -- the nearest-neighbour projection of Sec. 2, exact under
  the FP64 distance, ties to the lowest index;
* ``counts_from_samples`` / ``transitions`` -- Algorithm III's counters p^k_ij;
* ``backward`` / ``price`` -- the BDP recursion on the tree of Sec. 2 with
  pi^k_ij = p^k_ij / p^k_i;
* ``pathwise``      -- Algorithm II: every path simulated through all layers
  (one search per layer), for the AR(1) chain or an Euler-scheme chain;
* ``swing``         -- eq. (stochCtrl): the swing option's bang-bang BDP over
  consumption states on the tree.

Parity status of each function is recorded by the pin tests in
``tests/test_oracle_pins.py``; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PREC_F64 = 0
PREC_F32 = 1


def build(force: bool = False) -> str:
    """Compile qt_oracle.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "qto_philox": (None, [P, P, P, i64]),
            "qto_ln_f32": (ctypes.c_float, [ctypes.c_float]),
            "qto_ln_f64": (ctypes.c_double, [ctypes.c_double]),
            "qto_sincos2pi_f32": (None, [ctypes.c_float, P, P]),
            "qto_sincos2pi_f64": (None, [ctypes.c_double, P, P]),
            "qto_normals": (ctypes.c_int, [i32, u64, i32, i64, i64, i32, P]),
            "qto_uniforms_f32": (ctypes.c_int, [u64, i32, ctypes.c_uint32, i64, i64, P]),
            "qto_sample_pairs": (ctypes.c_int, [i32, i32, u64, i32, i64, i64, P, P, P, P, P, P, P]),
            "qto_nearest": (ctypes.c_int, [i32, P, i64, P, i64, P]),
            "qto_nearest_dist": (ctypes.c_int, [i32, P, i64, P, i64, P]),
            "qto_counts_from_samples": (ctypes.c_int, [i32, P, i64, P, i64, P, P, i64, P]),
            "qto_transitions": (ctypes.c_int, [i32, i32, P, P, P, P, P, P, P, i64, i64, u64, i32, P, P, P]),
            "qto_backward": (ctypes.c_int, [i32, P, P, P, P]),
            "qto_price_from_V": (ctypes.c_double, [P, P, P]),
            "qto_num_threads": (ctypes.c_int, []),
            "qto_pathwise": (ctypes.c_int, [i32, i32, P, P, P, P, P, P, P, P, P, i64, i64, u64, i32, P, P, P]),
            "qto_swing": (ctypes.c_int, [i32, P, P, P, i32, i32, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return int(_load().qto_num_threads())


# --------------------------------------------------------------------------- sampler

def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 blocks: ctr [count,4] uint32, key (k0, k1) -> [count,4] uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    _load().qto_philox(_p(ctr), _p(k), _p(out), ctr.shape[0])
    return out


def ln_f32(u: float) -> float:
    return float(_load().qto_ln_f32(u))


def ln_f64(u: float) -> float:
    return float(_load().qto_ln_f64(u))


def sincos2pi_f32(u: float):
    s, c = ctypes.c_float(), ctypes.c_float()
    _load().qto_sincos2pi_f32(u, ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sincos2pi_f64(u: float):
    s, c = ctypes.c_double(), ctypes.c_double()
    _load().qto_sincos2pi_f64(u, ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def normals(prec: int, seed: int, k: int, m0: int, M: int, count: int) -> np.ndarray:
    g = np.empty((M, count), dtype=np.float64)
    _check(_load().qto_normals(prec, seed, k, m0, M, count, _p(g)), "normals")
    return g


def uniforms_f32(seed: int, k: int, r: int, m0: int, M: int) -> np.ndarray:
    u = np.empty((M, 4), dtype=np.float32)
    _check(_load().qto_uniforms_f32(seed, k, r, m0, M, _p(u)), "uniforms")
    return u


def sample_pairs(d, prec, seed, k, m0, M, mk, Lk, Ak, bk, Tk):
    """(X_k, Y) of samples m0..m0+M-1 at layer k, each [M, d] FP64."""
    X = np.empty((M, d), dtype=np.float64)
    Y = np.empty((M, d), dtype=np.float64)
    args = [_f64(a) for a in (mk, Lk, Ak, bk, Tk)]
    _check(_load().qto_sample_pairs(d, prec, seed, k, m0, M, *[_p(a) for a in args], _p(X), _p(Y)),
           "sample_pairs")
    return X, Y


# --------------------------------------------------------------------------- search / counts

def nearest(grid: np.ndarray, Z: np.ndarray) -> np.ndarray:
    grid = _f64(grid)
    Z = _f64(Z)
    d = grid.shape[1]
    idx = np.empty(Z.shape[0], dtype=np.int32)
    _check(_load().qto_nearest(d, _p(grid), grid.shape[0], _p(Z), Z.shape[0], _p(idx)), "nearest")
    return idx


def nearest_dist(grid: np.ndarray, Z: np.ndarray) -> np.ndarray:
    grid = _f64(grid)
    Z = _f64(Z)
    out = np.empty(Z.shape[0], dtype=np.float64)
    _check(_load().qto_nearest_dist(grid.shape[1], _p(grid), grid.shape[0], _p(Z), Z.shape[0], _p(out)),
           "nearest_dist")
    return out


def counts_from_samples(gA, gB, X, Y) -> np.ndarray:
    gA, gB, X, Y = _f64(gA), _f64(gB), _f64(X), _f64(Y)
    c = np.zeros((gA.shape[0], gB.shape[0]), dtype=np.int64)
    _check(_load().qto_counts_from_samples(gA.shape[1], _p(gA), gA.shape[0], _p(gB), gB.shape[0],
                                           _p(X), _p(Y), X.shape[0], _p(c)), "counts_from_samples")
    return c


def transitions(model, grids: np.ndarray, M: int, seed: int, prec: int, m0: int = 0,
                want_cells: bool = False):
    """Algorithm III over all layers.  model needs d, n, N, A, b, T, m, L.

    Returns the list of per-layer count matrices (int64 [N_k, N_{k+1}]), and
    with want_cells the per-sample cells ii, jj ([n, M] int32)."""
    N = np.ascontiguousarray(model.N, dtype=np.int64)
    total = int(sum(int(N[k]) * int(N[k + 1]) for k in range(model.n)))
    flat = np.zeros(total, dtype=np.int64)
    ii = jj = None
    pii = pjj = None
    if want_cells:
        ii = np.empty((model.n, M), dtype=np.int32)
        jj = np.empty((model.n, M), dtype=np.int32)
        pii, pjj = _p(ii), _p(jj)
    arrs = [_f64(a) for a in (model.A, model.b, model.T, model.m, model.L)]
    g = _f64(grids)
    _check(_load().qto_transitions(model.d, model.n, _p(N), *[_p(a) for a in arrs], _p(g), m0, M,
                                   seed, prec, _p(flat), pii, pjj), "transitions")
    out, off = [], 0
    for k in range(model.n):
        sz = int(N[k]) * int(N[k + 1])
        out.append(flat[off:off + sz].reshape(int(N[k]), int(N[k + 1])))
        off += sz
    if want_cells:
        return out, ii, jj
    return out


def _flat_counts(counts_list) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int64).ravel() for c in counts_list]))


def backward(N, counts_list, phi: np.ndarray) -> np.ndarray:
    """V (concatenated [sum N_k]) from counts and phi on the grid points."""
    N = np.ascontiguousarray(N, dtype=np.int64)
    n = len(N) - 1
    flat = _flat_counts(counts_list)
    phi = _f64(phi)
    V = np.empty_like(phi)
    _check(_load().qto_backward(n, _p(N), _p(flat), _p(phi), _p(V)), "backward")
    return V


def price(N, counts_list, phi: np.ndarray) -> float:
    N = np.ascontiguousarray(N, dtype=np.int64)
    V = backward(N, counts_list, phi)
    c0 = np.ascontiguousarray(counts_list[0], dtype=np.int64)
    return float(_load().qto_price_from_V(_p(N), _p(c0), _p(V)))


# --------------------------------------------------------------------------- Algorithm II and the swing option

def pathwise(model, grids: np.ndarray, M: int, seed: int, prec: int, euler=None, m0: int = 0,
             want_paths: bool = False):
    """Algorithm II over all layers: list of per-layer counts (int64 [N_k, N_{k+1}]).

    euler: None (the AR(1) chain) or (alpha, beta), each [n, d]: the innovation of
    row l scaled by sqrt(max(alpha_l + beta_l x_l, 0)).  With want_paths the states
    X [n+1, M, d] and cells [n+1, M] are returned too."""
    N = np.ascontiguousarray(model.N, dtype=np.int64)
    total = int(sum(int(N[k]) * int(N[k + 1]) for k in range(model.n)))
    flat = np.zeros(total, dtype=np.int64)
    arrs = [_f64(a) for a in (model.A, model.b, model.T, model.m, model.L)]
    al = be = None
    if euler is not None:
        al = _f64(euler[0]).reshape(model.n, model.d)
        be = _f64(euler[1]).reshape(model.n, model.d)
    paths = cells = None
    if want_paths:
        paths = np.empty((model.n + 1, M, model.d), dtype=np.float64)
        cells = np.empty((model.n + 1, M), dtype=np.int32)
    g = _f64(grids)
    _check(_load().qto_pathwise(model.d, model.n, _p(N), *[_p(a) for a in arrs],
                                _p(al) if al is not None else None, _p(be) if be is not None else None,
                                _p(g), m0, M, seed, prec, _p(flat),
                                _p(paths) if want_paths else None, _p(cells) if want_paths else None),
           "pathwise")
    out, off = [], 0
    for k in range(model.n):
        sz = int(N[k]) * int(N[k + 1])
        out.append(flat[off:off + sz].reshape(int(N[k]), int(N[k + 1])))
        off += sz
    if want_paths:
        return out, paths, cells
    return out


def swing(N, counts_list, v: np.ndarray, Qmin: int, Qmax: int):
    """Swing values P (concatenated Q-major blocks [Qmax+1, N_k]) and the price."""
    N = np.ascontiguousarray(N, dtype=np.int64)
    n = len(N) - 1
    flat = _flat_counts(counts_list)
    v = _f64(v)
    P = np.empty(int(np.sum(N)) * (Qmax + 1), dtype=np.float64)
    _check(_load().qto_swing(n, _p(N), _p(flat), _p(v), int(Qmin), int(Qmax), _p(P)), "swing")
    c0 = np.ascontiguousarray(counts_list[0], dtype=np.int64)
    price = float(_load().qto_price_from_V(_p(N), _p(c0), _p(np.ascontiguousarray(P[: int(N[0])]))))
    return P, price


def swing_blocks(N, P: np.ndarray, Qmax: int):
    """Split the concatenated swing values into per-layer [Qmax+1, N_k] arrays."""
    out, off = [], 0
    for Nk in np.asarray(N, dtype=np.int64):
        sz = int(Nk) * (Qmax + 1)
        out.append(P[off:off + sz].reshape(Qmax + 1, int(Nk)))
        off += sz
    return out
