"""Seeded synthetic inputs shaped like the paper's synthetic workloads (Sec. 5.1).

This module is the only one shared by the CUDA path's tests/bench and by the
FP64 oracle's tests.  It draws random numbers and assembles input tensors; it
holds none of the decomposition's arithmetic (no MTTKRP, no solve, no
fitness).  The random numbers the method itself would draw (the initial
factors that Algorithm 1 draws at its start) are drawn here and passed to both sides as
inputs.

Recipes (one per workload; sizes and distributions as the paper describes its
synthetic tensors, Sec. 5.1 items 1-2):

* factors with a prescribed column collinearity C (item 1): for s >= R,
  A = Q chol(K)^T with K = (1-C) I + C 11^T and Q an s x R orthonormal basis
  (QR of a Gaussian matrix), so every pair of columns has cosine exactly C;
  for s < R that K cannot be realised, and a_r = sqrt(C) u + sqrt(1-C) w_r
  with random unit vectors u, w_r gives cosine C in expectation;
* factors with i.i.d. N(0,1) or U[0,1] entries (item 2);
* X = [[A^(1), ..., A^(N)]] plus Gaussian noise E, either absolute
  (X + sigma E) or relative (X + eta ||X|| / ||E|| E).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream)]))


def factors_normal(dims, R, seed, stream=1):
    g = _rng(seed, stream)
    return [g.standard_normal((s, R)) for s in dims]


def factors_uniform(dims, R, seed, stream=2):
    g = _rng(seed, stream)
    return [g.random((s, R)) for s in dims]


def factors_collinear(dims, R, C, seed, stream=3):
    g = _rng(seed, stream)
    out = []
    for s in dims:
        if s >= R:
            Q, _ = np.linalg.qr(g.standard_normal((s, R)))
            K = (1.0 - C) * np.eye(R) + C * np.ones((R, R))
            L = np.linalg.cholesky(K)
            out.append(Q @ L.T)
        else:
            u = g.standard_normal(s)
            u /= np.linalg.norm(u)
            W = g.standard_normal((s, R))
            W /= np.linalg.norm(W, axis=0, keepdims=True)
            out.append(np.sqrt(C) * u[:, None] + np.sqrt(1.0 - C) * W)
    return out


def _kr_rows(mats):
    """Row-wise expansion of a list of factors into their column-wise
    Kronecker product (input assembly only)."""
    R = mats[0].shape[1]
    out = np.ones((1, R))
    for A in mats:
        out = (out[:, None, :] * A[None, :, :]).reshape(-1, R)
    return out


def low_rank_tensor(factors) -> np.ndarray:
    """Dense sum_r a_r^(1) o ... o a_r^(N), row-major, last mode fastest."""
    dims = [a.shape[0] for a in factors]
    return (factors[0] @ _kr_rows(factors[1:]).T).reshape(dims)


def add_noise(X, level, seed, relative=True, stream=4):
    g = _rng(seed, stream)
    E = g.standard_normal(X.shape)
    if relative:
        return X + level * (np.linalg.norm(X) / np.linalg.norm(E)) * E
    return X + level * E


@dataclass
class Problem:
    """One decomposition problem: tensor, initial factors and run settings."""
    name: str
    X: np.ndarray                      # storage precision (float64 or float32)
    A0: list                           # float64 initial factors
    R: int
    eps: float
    sweeps: int
    storage: str                       # "f64" | "f32"
    meta: dict = field(default_factory=dict)

    @property
    def dims(self):
        return list(self.X.shape)


def make_problem(kind: str, dims, R, *, seed=0, noise=1e-2, relative=True,
                 collinearity=None, init="uniform", storage="f32", eps=0.1,
                 sweeps=100, name=None) -> Problem:
    """Assemble X = [[A_true]] + noise and an initial guess.

    kind: "normal" | "uniform" | "collinear" (true factors' distribution).
    init: "uniform" (U[0,1], the initial guess of Algorithm 1) | "normal".
    """
    dims = [int(d) for d in dims]
    meta = {}
    if kind == "normal":
        At = factors_normal(dims, R, seed)
    elif kind == "uniform":
        At = factors_uniform(dims, R, seed)
    elif kind == "collinear":
        if collinearity is None:
            C = float(_rng(seed, 5).uniform(0.5, 0.9))
        else:
            C = float(collinearity)
        meta["collinearity"] = C
        At = factors_collinear(dims, R, C, seed)
    else:
        raise ValueError(kind)
    X = low_rank_tensor(At)
    if noise:
        X = add_noise(X, noise, seed, relative=relative)
    if init == "uniform":
        A0 = factors_uniform(dims, R, seed, stream=6)
    else:
        A0 = factors_normal(dims, R, seed, stream=6)
    Xs = X.astype(np.float32) if storage == "f32" else X
    return Problem(name or kind, np.ascontiguousarray(Xs), A0, R, eps, sweeps,
                   storage, meta)


# The five workloads (sizes from the paper's synthetic experiments, Sec. 5.1).
def order3_60_rank10(seed=0) -> Problem:
    """60x60x60 FP64, exact rank 10 from N(0,1) factors + 1e-3 N(0,1) absolute
    noise, N(0,1) init, eps 0.2, 50 sweeps."""
    return make_problem("normal", [60, 60, 60], 10, seed=seed, noise=1e-3,
                        relative=False, init="normal", storage="f64", eps=0.2,
                        sweeps=50, name="order3_60_rank10_f64")


def order3_400_rank100(seed=0) -> Problem:
    """400^3 FP32 storage, rank 100, collinearity C ~ U[0.5,0.9), 1e-2
    relative noise, U[0,1] init, eps 0.1, 200 sweeps."""
    return make_problem("collinear", [400, 400, 400], 100, seed=seed,
                        noise=1e-2, init="uniform", storage="f32", eps=0.1,
                        sweeps=200, name="order3_400_rank100_f32")


def order4_120_rank64(seed=0) -> Problem:
    """120^4 FP32 storage, rank 64, N(0,1) factors, 1e-2 relative noise."""
    return make_problem("normal", [120] * 4, 64, seed=seed, noise=1e-2,
                        init="uniform", storage="f32", eps=0.1, sweeps=100,
                        name="order4_120_rank64_f32")


def order6_24_rank50(seed=0) -> Problem:
    """24^6 FP32 storage, rank 50, collinearity 0.7 (approximate: s < R),
    1e-2 relative noise, 300 sweeps."""
    return make_problem("collinear", [24] * 6, 50, seed=seed, noise=1e-2,
                        collinearity=0.7, init="uniform", storage="f32",
                        eps=0.1, sweeps=300, name="order6_24_rank50_f32")


def symmetric_order3(sa, sb, R, *, seed=0, noise=1e-2, collinearity=None, storage="f32",
                     eps=0.1, sweeps=100, name=None) -> Problem:
    """Order-3 tensor symmetric in modes 1 and 2, X = [[A, B, B]] + noise
    (the structure of Sec. 5.1's symmetric decomposition), noise symmetrised
    over modes 1 and 2 and scaled relative to ||X||.  True factors N(0,1), or
    collinear with cosine C per factor when ``collinearity`` is given (C10
    construction).  Initial factors U[0,1] with A0[2] = A0[1]."""
    if collinearity is None:
        At, Bt = factors_normal([sa, sb], R, seed)
    else:
        At, Bt = factors_collinear([sa, sb], R, float(collinearity), seed)
    X = low_rank_tensor([At, Bt, Bt])
    if noise:
        E = _rng(seed, 4).standard_normal(X.shape)
        E = E + E.transpose(0, 2, 1)
        X = X + noise * (np.linalg.norm(X) / np.linalg.norm(E)) * E
    A0 = factors_uniform([sa, sb], R, seed, stream=6)
    A0 = [A0[0], A0[1], A0[1].copy()]
    Xs = X.astype(np.float32) if storage == "f32" else X
    meta = {} if collinearity is None else {"collinearity": float(collinearity)}
    return Problem(name or f"symmetric_order3_{sa}x{sb}x{sb}_rank{R}", np.ascontiguousarray(Xs),
                   A0, R, eps, sweeps, storage, meta)


def orthonormal(s, R, seed, stream):
    """An s x R matrix with orthonormal columns (QR of a Gaussian matrix)."""
    Q, _ = np.linalg.qr(_rng(seed, stream).standard_normal((s, R)))
    return Q


def tucker_problem(dims, ranks, *, seed=0, noise=1e-2, storage="f64", eps=0.3, sweeps=20,
                   name=None) -> Problem:
    """X = [[G; A^(1), ..., A^(N)]] + noise (Sec. 2.4): core G N(0,1), factors
    with orthonormal columns, noise relative to ||X||.  A0: random
    orthonormal factors (the paper starts from HOSVD, which the tests compute
    with the oracle).  Problem.R holds the ranks."""
    dims = [int(d) for d in dims]
    G = _rng(seed, 8).standard_normal(tuple(int(r) for r in ranks))
    At = [orthonormal(s, r, seed, 20 + k) for k, (s, r) in enumerate(zip(dims, ranks))]
    X = G
    for k, A in enumerate(At):
        X = np.moveaxis(np.tensordot(X, A, axes=([k], [1])), -1, k)
    if noise:
        X = add_noise(X, noise, seed)
    A0 = [orthonormal(s, r, seed, 40 + k) for k, (s, r) in enumerate(zip(dims, ranks))]
    Xs = X.astype(np.float32) if storage == "f32" else X
    return Problem(name or "tucker", np.ascontiguousarray(Xs), A0, list(ranks), eps, sweeps, storage,
                   {"ranks": list(ranks)})


def batch_order3(count=256, seed=0, smin=32, smax=160, rmin=8, rmax=64):
    """Many small order-3 problems with per-mode sizes U{smin..smax} and ranks
    U{rmin..rmax}, FP32, 1e-2 relative noise, 100 sweeps each."""
    g = _rng(seed, 7)
    out = []
    for b in range(count):
        dims = [int(v) for v in g.integers(smin, smax + 1, size=3)]
        R = int(g.integers(rmin, rmax + 1))
        out.append(make_problem("normal", dims, R, seed=seed * 100003 + b,
                                noise=1e-2, init="uniform", storage="f32",
                                eps=0.1, sweeps=100, name=f"batch{b}"))
    return out


def scaled(kind: str, s: int, N: int, R: int, seed=0, **kw) -> Problem:
    """Scaled-down copy of a workload for fast CPU checks."""
    return make_problem(kind, [s] * N, R, seed=seed, **kw)
