"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds model set-up only: the AR(1) coefficients of each workload
(Prop. 1 of Pages & Wilbertz, arXiv:1101.3228), the marginal mean and Cholesky
factor of every X_k, host-built quantization grids (Sec. 2) and the payoff
values phi_k on the grid points.  It contains none of the method's arithmetic
(no sampling, no nearest-cell search, no counting, no backward induction), and
it imports neither the oracle nor the CUDA library.

Workloads (sizes as named by the five configurations of this project plus the
paper's own scenario of Sec. 3):

* ``bs1d``      d=1 Black-Scholes log-price, n=10, N_k=100, M=10^6, FP64 samples
* ``ou2``       d=2 Gaussian 2-factor OU model (Sec. 3, eq. (ou)), n=100 daily
                layers, N_k=500 product grids, M=10^7, FP32 samples
* ``basket4``   d=4 correlated log-prices, n=50, N_k rising 200 -> 2000, M=10^8
* ``ar8``       d=8 AR(1), n=50, N_k=4000, M=10^8
* ``maxcall10`` d=10 AR(1), n=365, N_k=8000, M=10^8
* ``paper``     the paper's scenario: ou2 model with n=365, M=10^5, N=100/250/500
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
from scipy import linalg as sla
from scipy import special

PREC_F64 = 0
PREC_F32 = 1

SEED_BASE = 0x0000C0FFEE000001
GRID_SEED_BASE = 20110115
CONFIG_INDEX = {"bs1d": 0, "ou2": 1, "basket4": 2, "ar8": 3, "maxcall10": 4, "paper": 5}


@dataclasses.dataclass
class Model:
    name: str
    d: int
    n: int
    N: np.ndarray            # int64 [n+1]
    A: np.ndarray            # [n, d, d]
    b: np.ndarray            # [n, d]
    T: np.ndarray            # [n, d, d] lower triangular
    m: np.ndarray            # [n+1, d] mean of X_k
    L: np.ndarray            # [n+1, d, d] lower Cholesky factor of Cov(X_k)
    t: np.ndarray            # [n+1] times t_k
    r: float                 # discount rate
    payoff: str              # "put_exp1d", "put_expsum", "basket_put", "max_call"
    K: float
    weights: Optional[np.ndarray]
    M: int                   # samples per layer of the full workload
    seed: int
    prec: int                # sample precision (PREC_F64 / PREC_F32)
    grid_kind: str           # "lloyd1d", "product", "kmeans"
    grid_base: dict = dataclasses.field(default_factory=dict)  # N -> base grid of N(0, I_d)

    @property
    def total_points(self) -> int:
        return int(np.sum(self.N))

    @property
    def count_entries(self) -> int:
        return int(sum(int(self.N[k]) * int(self.N[k + 1]) for k in range(self.n)))

    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N)]).astype(np.int64)

    def restrict(self, n: Optional[int] = None, M: Optional[int] = None, N: Optional[int] = None) -> "Model":
        """Same model on the first n layers, with M samples and (optionally) N points per layer k >= 1."""
        n = self.n if n is None else int(n)
        Nv = self.N[: n + 1].copy()
        if N is not None:
            Nv[1:] = int(N)
        return dataclasses.replace(self, n=n, N=Nv, A=self.A[:n], b=self.b[:n], T=self.T[:n],
                                   m=self.m[: n + 1], L=self.L[: n + 1], t=self.t[: n + 1],
                                   M=self.M if M is None else int(M), grid_base={})


def _chol(S: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor; the zero matrix (deterministic X_0) maps to zero."""
    if not np.any(S):
        return np.zeros_like(S)
    return np.linalg.cholesky(0.5 * (S + S.T))


# --------------------------------------------------------------------------- models

def bs1d(M: int = 10**6) -> Model:
    """Black-Scholes put, X_k = log S_{t_k}: A = 1, b = (r - s^2/2) dt, T = s sqrt(dt)."""
    S0, K, r, sig, Tm, n = 100.0, 100.0, 0.05, 0.2, 1.0, 10
    dt = Tm / n
    t = np.arange(n + 1) * dt
    A = np.ones((n, 1, 1))
    b = np.full((n, 1), (r - 0.5 * sig * sig) * dt)
    T = np.full((n, 1, 1), sig * math.sqrt(dt))
    m = (math.log(S0) + (r - 0.5 * sig * sig) * t)[:, None]
    L = (sig * np.sqrt(t))[:, None, None]
    N = np.array([1] + [100] * n, dtype=np.int64)
    return Model("bs1d", 1, n, N, A, b, T, m, L, t, r, "put_exp1d", K, None, M,
                 SEED_BASE + 0, PREC_F64, "lloyd1d")


def _ou_moments(alpha, sig, rho, dt):
    a = np.asarray(alpha, float)
    s = np.asarray(sig, float)
    R = np.asarray(rho, float)
    ssum = a[:, None] + a[None, :]
    Q = s[:, None] * s[None, :] * R * (1.0 - np.exp(-ssum * dt)) / ssum
    return np.diag(np.exp(-a * dt)), Q


def ou2(M: int = 10**7, n: int = 100, N: int = 500) -> Model:
    """Gaussian 2-factor model of Sec. 3: X = (OU_1, OU_2), spot = exp(X1 + X2)."""
    alpha, sig, rho = (0.5, 5.0), (0.3, 0.6), -0.3
    R = np.array([[1.0, rho], [rho, 1.0]])
    dt = 1.0 / 365.0
    t = np.arange(n + 1) * dt
    Ak, Qk = _ou_moments(alpha, sig, R, dt)
    A = np.repeat(Ak[None], n, axis=0)
    b = np.zeros((n, 2))
    T = np.repeat(_chol(Qk)[None], n, axis=0)
    m = np.zeros((n + 1, 2))
    L = np.stack([_chol(_ou_moments(alpha, sig, R, tk)[1]) for tk in t])
    Nv = np.array([1] + [N] * n, dtype=np.int64)
    return Model("ou2", 2, n, Nv, A, b, T, m, L, t, 0.0, "put_expsum", 1.0, None, M,
                 SEED_BASE + 1, PREC_F32, "product")


def basket4(M: int = 10**8) -> Model:
    """4 correlated log-prices (vols 0.2..0.4, correlation 0.5), N_k from 200 to 2000."""
    d, n, S0, K, r, Tm = 4, 50, 100.0, 100.0, 0.05, 1.0
    sig = np.linspace(0.2, 0.4, d)
    R = np.full((d, d), 0.5) + 0.5 * np.eye(d)
    S = sig[:, None] * sig[None, :] * R
    dt = Tm / n
    t = np.arange(n + 1) * dt
    A = np.repeat(np.eye(d)[None], n, axis=0)
    b = np.repeat(((r - 0.5 * sig * sig) * dt)[None], n, axis=0)
    T = np.repeat(_chol(S * dt)[None], n, axis=0)
    m = math.log(S0) + (r - 0.5 * sig * sig)[None, :] * t[:, None]
    L = np.stack([_chol(S * tk) for tk in t])
    Nv = np.array([1] + [int(round(200 + 1800 * (k - 1) / (n - 1))) for k in range(1, n + 1)], dtype=np.int64)
    return Model("basket4", d, n, Nv, A, b, T, m, L, t, r, "basket_put", K, np.full(d, 1.0 / d), M,
                 SEED_BASE + 2, PREC_F32, "kmeans")


def _ar_model(name, d, n, N, M, payoff, K, cfg_index) -> Model:
    """X_{k+1} = diag(a) X_k + T eps, a = 0.9..0.99, Cov(T eps) = Q diag(lam) Q^T, lam in [1e-4, 1e-2]."""
    rng = np.random.default_rng(GRID_SEED_BASE + 1000 + cfg_index)
    Qm, _ = np.linalg.qr(rng.standard_normal((d, d)))
    lam = np.logspace(-4.0, -2.0, d)              # condition number 100
    C = Qm @ np.diag(lam) @ Qm.T
    C = 0.5 * (C + C.T)
    Ak = np.diag(np.linspace(0.9, 0.99, d))
    A = np.repeat(Ak[None], n, axis=0)
    b = np.zeros((n, d))
    T = np.repeat(_chol(C)[None], n, axis=0)
    m = np.zeros((n + 1, d))
    covs = [np.zeros((d, d))]
    for _ in range(n):
        covs.append(Ak @ covs[-1] @ Ak.T + C)
    L = np.stack([_chol(S) for S in covs])
    t = np.arange(n + 1) / 365.0 if n == 365 else np.arange(n + 1) / n
    Nv = np.array([1] + [N] * n, dtype=np.int64)
    return Model(name, d, n, Nv, A, b, T, m, L, t, 0.0, payoff, K, np.full(d, 1.0 / d), M,
                 SEED_BASE + cfg_index, PREC_F32, "kmeans")


def ar8(M: int = 10**8) -> Model:
    return _ar_model("ar8", 8, 50, 4000, M, "basket_put", 1.0, 3)


def maxcall10(M: int = 10**8) -> Model:
    return _ar_model("maxcall10", 10, 365, 8000, M, "max_call", 1.0, 4)


def paper(N: int = 500, M: int = 10**5) -> Model:
    mdl = ou2(M=M, n=365, N=N)
    return dataclasses.replace(mdl, name="paper", seed=SEED_BASE + 5)


BUILDERS = {"bs1d": bs1d, "ou2": ou2, "basket4": basket4, "ar8": ar8, "maxcall10": maxcall10, "paper": paper}


def get(name: str, **kw) -> Model:
    return BUILDERS[name](**kw)


# --------------------------------------------------------------------------- 1-d optimal quantizer of N(0,1)

def _cells(x):
    bnd = 0.5 * (x[1:] + x[:-1])
    lo = np.concatenate([[-np.inf], bnd])
    hi = np.concatenate([bnd, [np.inf]])
    return lo, hi


def _mass(lo, hi):
    # P(lo < Z < hi) without cancellation in either tail
    return np.where(hi <= 0, special.ndtr(hi) - special.ndtr(lo), special.ndtr(-lo) - special.ndtr(-hi))


def _pdf(z):
    return np.where(np.isfinite(z), np.exp(-0.5 * np.square(np.where(np.isfinite(z), z, 0.0))) / math.sqrt(2 * math.pi), 0.0)


def lloyd_gaussian_1d(N: int, tol: float = 1e-14, max_newton: int = 100) -> np.ndarray:
    """Stationary N-point quantizer of N(0,1): x_i = E[Z | Z in C_i] (Sec. 2, the grids of eq. (Qerr)).

    Lloyd's fixed point on closed-form cell means, finished by Newton's method on
    G_i(x) = x_i P_i - (pdf(b_{i-1}) - pdf(b_i)) with its tridiagonal Jacobian; stops
    when the Newton step is below tol."""
    if N == 1:
        return np.zeros(1)
    x = special.ndtri((np.arange(N) + 0.5) / N)
    for _ in range(200):                           # Lloyd warm start
        lo, hi = _cells(x)
        x = (_pdf(lo) - _pdf(hi)) / _mass(lo, hi)
    for _ in range(max_newton):
        lo, hi = _cells(x)
        P = _mass(lo, hi)
        Qm = _pdf(lo) - _pdf(hi)
        G = x * P - Qm
        plo, phi_ = _pdf(lo), _pdf(hi)
        lo_f = np.where(np.isfinite(lo), lo, 0.0)
        hi_f = np.where(np.isfinite(hi), hi, 0.0)
        diag = P + 0.5 * (x - hi_f) * phi_ + 0.5 * (lo_f - x) * plo
        upper = 0.5 * (x[:-1] - hi_f[:-1]) * phi_[:-1]     # dG_i / dx_{i+1}
        lower = 0.5 * (lo_f[1:] - x[1:]) * plo[1:]          # dG_i / dx_{i-1}
        ab = np.zeros((3, N))
        ab[0, 1:] = upper
        ab[1] = diag
        ab[2, :-1] = lower
        step = sla.solve_banded((1, 1), ab, G)
        x = x - step
        x = 0.5 * (x - x[::-1])                      # exact symmetry of the optimum
        if np.max(np.abs(step)) < tol:
            break
    return x


def distortion_1d(x: np.ndarray) -> float:
    """E min_i (Z - x_i)^2 for Z ~ N(0,1) in closed form (eq. (Qerr))."""
    lo, hi = _cells(x)
    P = _mass(lo, hi)
    m1 = _pdf(lo) - _pdf(hi)
    lo_f = np.where(np.isfinite(lo), lo, 0.0)
    hi_f = np.where(np.isfinite(hi), hi, 0.0)
    m2 = P + lo_f * _pdf(lo) - hi_f * _pdf(hi)       # E[Z^2 ; C_i]
    return float(np.sum(m2 - 2 * x * m1 + x * x * P))


def product_grid(sizes) -> np.ndarray:
    axes = [lloyd_gaussian_1d(int(s)) for s in sizes]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in mesh], axis=1)


def product_sizes(N: int, d: int):
    """Factor N into d near-equal sizes, largest last (N = 500, d = 2 -> (20, 25))."""
    if d == 1:
        return (N,)
    best = None
    for a in range(1, N + 1):
        if N % a:
            continue
        rest = product_sizes(N // a, d - 1)
        cand = tuple(sorted((a,) + tuple(rest)))
        score = max(cand) / min(cand)
        if best is None or score < best[0]:
            best = (score, cand)
    return best[1]


def kmeans_gaussian(N: int, d: int, samples: int, iters: int, seed: int) -> np.ndarray:
    """Sample Lloyd (k-means) on `samples` seeded N(0, I_d) draws; an input recipe, not exact."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((samples, d))
    G = Z[:N].copy()
    zz = np.einsum("ij,ij->i", Z, Z)
    for _ in range(iters):
        idx = np.empty(samples, dtype=np.int64)
        gg = np.einsum("ij,ij->i", G, G)
        for s in range(0, samples, 65536):
            blk = Z[s:s + 65536]
            D = zz[s:s + 65536, None] - 2.0 * blk @ G.T + gg[None, :]
            idx[s:s + 65536] = np.argmin(D, axis=1)
        cnt = np.bincount(idx, minlength=N).astype(float)
        sums = np.zeros((N, d))
        np.add.at(sums, idx, Z)
        keep = cnt > 0
        G[keep] = sums[keep] / cnt[keep, None]
    return G


def base_grid(model: Model, N: int, samples: Optional[int] = None, iters: Optional[int] = None) -> np.ndarray:
    """Grid of N(0, I_d) with N points, cached on the model."""
    key = (int(N), samples, iters)
    if key in model.grid_base:
        return model.grid_base[key]
    if N == 1:
        g = np.zeros((1, model.d))
    elif model.grid_kind == "lloyd1d":
        g = lloyd_gaussian_1d(N)[:, None]
    elif model.grid_kind == "product":
        g = product_grid(product_sizes(N, model.d))
    else:
        s = samples if samples is not None else max(20 * N, 20000)
        it = iters if iters is not None else 10
        g = kmeans_gaussian(N, model.d, s, it, GRID_SEED_BASE + CONFIG_INDEX.get(model.name, 9) * 7919 + N)
    model.grid_base[key] = g
    return g


def layer_grids(model: Model, samples: Optional[int] = None, iters: Optional[int] = None) -> np.ndarray:
    """Concatenated grids [sum_k N_k, d]: Gamma_k = m_k + L_k g for the base grid g of size N_k."""
    out = []
    for k in range(model.n + 1):
        Nk = int(model.N[k])
        g = base_grid(model, Nk, samples, iters)
        out.append(model.m[k][None, :] + g @ model.L[k].T)
    return np.ascontiguousarray(np.concatenate(out, axis=0))


def payoff_values(model: Model, grids: np.ndarray) -> np.ndarray:
    """phi_k(x) = exp(-r t_k) * payoff(x) on every grid point (discounted obstacle)."""
    off = model.offsets()
    phi = np.empty(off[-1])
    for k in range(model.n + 1):
        x = grids[off[k]:off[k + 1]]
        if model.payoff == "put_exp1d":
            v = np.maximum(model.K - np.exp(x[:, 0]), 0.0)
        elif model.payoff == "put_expsum":
            v = np.maximum(model.K - np.exp(np.sum(x, axis=1)), 0.0)
        elif model.payoff == "basket_put":
            v = np.maximum(model.K - np.exp(x) @ model.weights, 0.0)
        elif model.payoff == "max_call":
            v = np.maximum(np.max(np.exp(x), axis=1) - model.K, 0.0)
        else:
            raise ValueError(model.payoff)
        phi[off[k]:off[k + 1]] = math.exp(-model.r * model.t[k]) * v
    return phi


def european_phi(model: Model, phi: np.ndarray) -> np.ndarray:
    """Obstacle that only pays at t_n (the European special case)."""
    off = model.offsets()
    out = np.zeros_like(phi)
    out[off[model.n]:] = phi[off[model.n]:]
    return out


# --------------------------------------------------------------------------- adversarial samples

def boundary_samples(grid: np.ndarray, count: int, seed: int, jitter: float = 0.0) -> np.ndarray:
    """Points on (or within `jitter` relative of) the bisector of random pairs of
    nearby grid points: the inputs where a screened distance is least certain."""
    rng = np.random.default_rng(seed)
    N, d = grid.shape
    out = np.empty((count, d))
    for t in range(count):
        i = int(rng.integers(N))
        dd = np.sum((grid - grid[i]) ** 2, axis=1)
        dd[i] = np.inf
        j = int(np.argsort(dd)[int(rng.integers(min(3, N - 1)))])
        mid = 0.5 * (grid[i] + grid[j])
        if d > 1:
            nrm = grid[j] - grid[i]
            tang = rng.standard_normal(d)
            tang -= nrm * (tang @ nrm) / max(nrm @ nrm, 1e-300)
            mid = mid + tang * 0.1 * math.sqrt(dd[j])
        out[t] = mid * (1.0 + jitter * rng.standard_normal(d)) if jitter else mid
    return out
