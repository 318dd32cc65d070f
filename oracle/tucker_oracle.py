"""FP64 CPU oracle for Tucker-ALS (HOOI) and pairwise-perturbation Tucker-ALS.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s oracle legs
may call it.  It shares no code with the CUDA library; the only module both
sides use is the seeded input generator ``paper_1811_10573_gb300.synth``.

Source: Ma & Solomonik, arXiv 1811.10573, Sec. 2.4 (Tucker-ALS, Algorithm 2),
Sec. 3.1.2 and Sec. 3.2.2 (pairwise perturbation for Tucker-ALS,
Algorithm 4).  Modes are 0-based; a factor A^(n) is an s_n x R_n matrix with
orthonormal columns; X x_n A^T contracts mode n of X with the rows of A.
Everything is float64; contractions use numpy tensordot on the definitions.

Readings (where the paper leaves room):
* The R_n leading left singular vectors of Y^(n)_(n) are taken, as the paper
  does, as the leading eigenvectors of the Gram matrix W = Y_(n) Y_(n)^T
  (numpy eigh), in decreasing eigenvalue order.
* Signs: an eigenvector is only defined up to sign, and PP needs
  dA = A - A_p small, so each new column is flipped to have a non-negative
  inner product with the same column of the factor it replaces (for HOSVD,
  which has no previous factor, the entry of largest magnitude is made
  positive).
* Algorithm 4's inner loop is run on the same test as Algorithm 3 (every
  ||dA^(i)|| < eps ||A^(i)||, checked at the head of each PP sweep); the
  core-change criterion on F is not used (fixed sweep budgets).

Pinned by ``tests/test_oracle_pins.py`` (brute-force TTMc, exact recovery
of a tensor of exact multilinear rank, the non-decreasing core norm of HOOI,
agreement of the Gram eigenvectors with the SVD, exactness of PP at dA = 0
and its second-order error, and the core estimate a PP sweep returns against
the exact core minus the order-3 product term of Sec. 3.1.2's expansion;
at order 4: brute-force TTMc, the full multilinear expansion of Y^(n) around
A_p against the PP right-hand side, exact recovery, PP tracking HOOI).
Every function is written for any order N.
"""
from __future__ import annotations

import numpy as np


def ttm(X: np.ndarray, A: np.ndarray, n: int) -> np.ndarray:
    """X x_n A^T: mode n (size s_n) replaced by a mode of size R = A.shape[1]."""
    return np.moveaxis(np.tensordot(X, A, axes=([n], [0])), -1, n)


def ttmc(X: np.ndarray, A, n: int) -> np.ndarray:
    """Y^(n) = X x_k A^(k)T for every k != n (Sec. 2.4), modes in order."""
    Y = X
    for k in range(X.ndim):
        if k != n:
            Y = ttm(Y, A[k], k)
    return Y


def unfold(Y: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding Y_(n): rows indexed by mode n, the other modes in order."""
    return np.moveaxis(Y, n, 0).reshape(Y.shape[n], -1)


def _signs(V: np.ndarray, ref: np.ndarray | None) -> np.ndarray:
    V = V.copy()
    for r in range(V.shape[1]):
        if ref is not None:
            flip = float(V[:, r] @ ref[:, r]) < 0.0
        else:
            k = int(np.argmax(np.abs(V[:, r])))
            flip = V[k, r] < 0.0
        if flip:
            V[:, r] = -V[:, r]
    return V


def leading_eigvecs(W: np.ndarray, R: int, ref: np.ndarray | None = None) -> np.ndarray:
    """The R leading eigenvectors of the symmetric W (eigenvalues in
    decreasing order), signs as described in the module docstring."""
    w, V = np.linalg.eigh(W)
    order = np.argsort(-w, kind="stable")[:R]
    return _signs(V[:, order], ref)


def hosvd(X: np.ndarray, ranks) -> list:
    """Classical HOSVD (Sec. 2.4): A^(n) = leading left singular vectors of X_(n)."""
    A = []
    for n in range(X.ndim):
        Xn = unfold(X, n)
        A.append(leading_eigvecs(Xn @ Xn.T, ranks[n]))
    return A


def core(X: np.ndarray, A) -> np.ndarray:
    """G = X x_1 A^(1)T ... x_N A^(N)T."""
    G = X
    for k in range(X.ndim):
        G = ttm(G, A[k], k)
    return G


def reconstruct(G: np.ndarray, A) -> np.ndarray:
    """[[G; A^(1), ..., A^(N)]] = G x_1 A^(1) ... x_N A^(N)."""
    T = G
    for k in range(G.ndim):
        T = np.moveaxis(np.tensordot(T, A[k], axes=([k], [1])), -1, k)
    return T


def fitness(normX: float, G: np.ndarray) -> float:
    """1 - ||X - [[G; A]]|| / ||X|| for orthonormal factors and G = X x A^T:
    ||X - [[G; A]]||^2 = ||X||^2 - ||G||^2."""
    res2 = normX * normX - float(np.sum(G * G))
    return 1.0 - np.sqrt(max(res2, 0.0)) / normX


def als_sweep(X: np.ndarray, A) -> tuple:
    """One sweep of Algorithm 2 (HOOI); A is updated in place.  Returns
    (dA, G): dA[n] = A^(n)_new - A^(n)_old and the new core."""
    N = X.ndim
    dA = [None] * N
    Y = None
    for n in range(N):
        Y = ttmc(X, A, n)
        Yn = unfold(Y, n)
        Anew = leading_eigvecs(Yn @ Yn.T, A[n].shape[1], ref=A[n])
        dA[n] = Anew - A[n]
        A[n] = Anew
    return dA, ttm(Y, A[N - 1], N - 1)


def pp_operators(X: np.ndarray, Ap) -> tuple:
    """PP operators of Sec. 3.2.2: ops[(i, n)] (i < n) = X x_k A_p^(k)T for
    every k not in {i, n} (modes in order, i and n keep their sizes), and
    Mp[n] = Y_p^(n) = X x_k A_p^(k)T for every k != n."""
    N = X.ndim
    ops = {}
    for i in range(N):
        for n in range(i + 1, N):
            T = X
            for k in range(N):
                if k not in (i, n):
                    T = ttm(T, Ap[k], k)
            ops[(i, n)] = T
    Mp = [ttmc(X, Ap, n) for n in range(N)]
    return ops, Mp


def pp_ttmc(ops, Mp, dA, n: int) -> np.ndarray:
    """Y~^(n) = Y_p^(n) + sum_{i != n} Y_p^(i,n) x_i dA^(i)T (Sec. 3.2.2)."""
    out = Mp[n].copy()
    for i in range(len(Mp)):
        if i == n:
            continue
        T = ops[(min(i, n), max(i, n))]
        out = out + ttm(T, dA[i], i)
    return out


def pp_sweep(ops, Mp, A, Ap, dA) -> np.ndarray:
    """One PP approximated sweep of Algorithm 4 (lists updated in place);
    returns the core estimate from Y~^(N)."""
    N = len(A)
    Y = None
    for n in range(N):
        Y = pp_ttmc(ops, Mp, dA, n)
        Yn = unfold(Y, n)
        Anew = leading_eigvecs(Yn @ Yn.T, A[n].shape[1], ref=A[n])
        A[n] = Anew
        dA[n] = Anew - Ap[n]
    return ttm(Y, A[N - 1], N - 1)


def _small(dA, A, eps: float) -> bool:
    return all(np.linalg.norm(d) < eps * np.linalg.norm(a) for d, a in zip(dA, A))


def pp_tucker_als(X: np.ndarray, A0, n_sweeps: int, eps: float):
    """Algorithm 4 for a budget of sweeps (each of ALS, PP-init and
    PP-approx counts as one).  Returns (A, kinds, fitness) with the exact
    fitness after every sweep."""
    A = [a.copy() for a in A0]
    dA = [a.copy() for a in A]            # Algorithm 4 starts from dA <- A
    normX = float(np.linalg.norm(X))
    kinds, fit = [], []
    t = 0
    while t < n_sweeps:
        if _small(dA, A, eps):
            Ap = [a.copy() for a in A]
            ops, Mp = pp_operators(X, Ap)
            dA = [np.zeros_like(a) for a in A]
            first = True
            while t < n_sweeps and _small(dA, A, eps):
                pp_sweep(ops, Mp, A, Ap, dA)
                t += 1
                kinds.append("pp_init" if first else "pp_approx")
                fit.append(fitness(normX, core(X, A)))
                first = False
            if t >= n_sweeps:
                break
        dA, G = als_sweep(X, A)
        t += 1
        kinds.append("als")
        fit.append(fitness(normX, G))
    return A, kinds, fit
