"""FP64 CPU oracle for CP-ALS and pairwise-perturbation CP-ALS (PP-CP-ALS).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code with
the CUDA library (``paper_1811_10573_gb300``); the only module both sides use
is the seeded input generator ``paper_1811_10573_gb300.synth``, which holds
none of the method's arithmetic.

Source: Ma & Solomonik, "Accelerating Alternating Least Squares for Tensor
Decomposition by Pairwise Perturbation" (arXiv 1811.10573).  Citations name
the paper's sections, equations (numbered in order of appearance: Eq. 1 =
partially contracted MTTKRP intermediates, Eq. 2 = order-3 expansion of
M^(1), Eq. 3 = PP update), algorithms (Algorithm 1 = CP-ALS, Algorithm 3 =
PP-CP-ALS, Algorithm 5 = reinterpreted pairwise-update ALS) and tables.

Conventions (Sec. 2.1): tensors are dense numpy arrays, row-major, last mode
fastest; a factor A^(n) is an s_n x R matrix; modes are 0-based here
(the paper's mode n is index n-1).  Everything is float64; contractions use
numpy matmul (a library primitive) on the matricized forms the paper writes,
with no blocking, fusion or reordering beyond those definitions.

Pinned by the tests in ``tests/test_oracle_pins.py`` (brute-force MTTKRP,
closed forms, invariants, Hurwitz unit-condition tensors from the appendix,
exact low-rank recovery, the t^2 scaling of the PP error, and the sweep
sequence of ``pp_cp_als`` against eps crossings fixed by a plain ALS trace and
the Algorithm 3 rule re-derived from the factor history).  Parity unpinned:
the long-run fitness trajectory of ``pp_cp_als`` against the paper's own
experiments (its figures are not recoverable and its seeds are unknown); only
its parts are pinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Sec. 2.1 notation: matricization, Khatri-Rao product
# ---------------------------------------------------------------------------


def unfold(X: np.ndarray, modes) -> np.ndarray:
    """Generalised unfolding X_(i1..iM) of Sec. 2.1.

    Returns an array of shape (s_i1, ..., s_iM, K) where the last axis runs
    over the remaining modes in increasing order with the last mode fastest
    (the row-major counterpart of the paper's column ordering).
    """
    modes = list(modes)
    rest = [k for k in range(X.ndim) if k not in modes]
    Y = np.transpose(X, modes + rest)
    return Y.reshape([X.shape[m] for m in modes] + [-1])


def khatri_rao(mats) -> np.ndarray:
    """Column-wise Kronecker product A (.) B (.) ... (Sec. 2.1).

    Row index of the result is (i_1, i_2, ...) with the last factor fastest,
    matching ``unfold``'s ordering of the contracted modes.
    """
    mats = list(mats)
    R = mats[0].shape[1]
    out = np.ones((1, R))
    for A in mats:
        out = (out[:, None, :] * A[None, :, :]).reshape(-1, R)
    return out


# ---------------------------------------------------------------------------
# MTTKRP and the partially contracted intermediates (Sec. 2.3, Sec. 2.5 Eq. 1)
# ---------------------------------------------------------------------------


def mttkrp(X: np.ndarray, A, n: int) -> np.ndarray:
    """M^(n) = X_(n) P^(n), P^(n) = Khatri-Rao of all A^(k), k != n (Sec. 2.3)."""
    others = [A[k] for k in range(X.ndim) if k != n]
    return unfold(X, [n]) @ khatri_rao(others)


def partial_mttkrp(X: np.ndarray, A, modes) -> np.ndarray:
    """M^(i1..im) of Eq. 1: X_(i1..im) times the Khatri-Rao product of the
    factors of every mode not in ``modes``.  Shape (s_i1, ..., s_im, R)."""
    modes = list(modes)
    others = [A[k] for k in range(X.ndim) if k not in modes]
    return unfold(X, modes) @ khatri_rao(others)


def partial_row(X: np.ndarray, A, fixed) -> np.ndarray:
    """One length-R vector of Eq. 1: M^(I)(x_I, :) for the modes I of
    ``fixed`` (a dict mode -> index), i.e. X with those modes fixed,
    contracted with A^(k)(x_k, r) over every other mode k.  The modes are
    contracted one at a time (last first), so a row of a large tensor costs
    one pass over its slice; M^(n)[y] = partial_row(X, A, {n: y}) and
    M_p^(i,n)[x_i, x_n] = partial_row(X, A_p, {i: x_i, n: x_n})."""
    sub = X
    for k in sorted(fixed, reverse=True):
        sub = np.take(sub, fixed[k], axis=k)
    others = [A[k] for k in range(X.ndim) if k not in fixed]
    t = np.asarray(sub, dtype=np.float64)
    if not others:
        raise ValueError("at least one mode must be contracted")
    t = t @ others[-1]                                   # (..., R)
    for a in reversed(others[:-1]):
        t = np.einsum("...ir,ir->...r", t, a)
    return t


# ---------------------------------------------------------------------------
# Normal equations (Sec. 2.3)
# ---------------------------------------------------------------------------


def gram(A: np.ndarray) -> np.ndarray:
    """S = A^T A (Sec. 2.3)."""
    return A.T @ A


def gamma(S, n: int) -> np.ndarray:
    """Gamma^(n) = Hadamard product of all S^(k), k != n (Algorithm 1)."""
    G = np.ones_like(S[0])
    for k, Sk in enumerate(S):
        if k != n:
            G = G * Sk
    return G


class SolveInfo:
    """Records whether the Cholesky solve fell back to the pseudo-inverse."""

    def __init__(self):
        self.singular = False


def solve_normal(M: np.ndarray, G: np.ndarray, info: SolveInfo | None = None) -> np.ndarray:
    """A_new = M Gamma^dagger (Algorithm 1).

    Gamma is symmetric positive (semi)definite.  The paper writes the
    pseudo-inverse and implements an SPD solve; this oracle takes the reading
    used throughout the project: a Cholesky factorisation Gamma = L L^T with
    two triangular solves per row; if a pivot is not positive the
    pseudo-inverse from the symmetric eigendecomposition (relative cut-off
    1e-13 of the largest eigenvalue) is used instead and ``info.singular`` is
    set.
    """
    R = G.shape[0]
    L = np.zeros_like(G)
    ok = True
    # Column-by-column Cholesky (textbook form, no library call).
    for j in range(R):
        d = G[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (d > 0.0) or not math.isfinite(d):
            ok = False
            break
        L[j, j] = math.sqrt(d)
        L[j + 1:, j] = (G[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    if ok:
        # Solve X L L^T = M row-wise: first Z L^T ... written as L Z^T = M^T.
        Zt = _forward(L, M.T)
        return _backward(L.T, Zt).T
    if info is not None:
        info.singular = True
    w, V = np.linalg.eigh(G)
    cut = 1e-13 * max(w.max(), 0.0)
    winv = np.where(w > cut, 1.0 / np.where(w > cut, w, 1.0), 0.0)
    return M @ (V * winv) @ V.T


def _forward(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve L Y = B for lower-triangular L (forward substitution)."""
    Y = np.zeros_like(B)
    for i in range(L.shape[0]):
        Y[i] = (B[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def _backward(U: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve U Y = B for upper-triangular U (back substitution)."""
    n = U.shape[0]
    Y = np.zeros_like(B)
    for i in range(n - 1, -1, -1):
        Y[i] = (B[i] - U[i, i + 1:] @ Y[i + 1:]) / U[i, i]
    return Y


# ---------------------------------------------------------------------------
# Fitness (Sec. 5)
# ---------------------------------------------------------------------------


def reconstruct(A) -> np.ndarray:
    """[[A^(1), ..., A^(N)]] = sum_r a_r^(1) o ... o a_r^(N) (Sec. 2.3)."""
    dims = [a.shape[0] for a in A]
    X = A[0] @ khatri_rao(A[1:]).T
    return X.reshape(dims)


def norm_model_sq(A) -> float:
    """||[[A]]||_F^2 = sum of the Hadamard product of all Grams."""
    H = np.ones((A[0].shape[1], A[0].shape[1]))
    for a in A:
        H = H * gram(a)
    return float(H.sum())


def fitness(X: np.ndarray, A, normX: float | None = None) -> float:
    """f = 1 - ||X - [[A]]||_F / ||X||_F (Sec. 5), evaluated through
    ||X||^2 - 2<X,[[A]]> + ||[[A]]||^2 with the exact inner product
    <X,[[A]]> = sum(M^(N) * A^(N)) for the last mode."""
    if normX is None:
        normX = float(np.linalg.norm(X))
    N = X.ndim
    inner = float(np.sum(mttkrp(X, A, N - 1) * A[N - 1]))
    res2 = normX * normX - 2.0 * inner + norm_model_sq(A)
    return 1.0 - math.sqrt(max(res2, 0.0)) / normX


def fitness_explicit(X: np.ndarray, A) -> float:
    """Same quantity from an explicit reconstruction (small tensors only)."""
    return 1.0 - float(np.linalg.norm(X - reconstruct(A)) / np.linalg.norm(X))


# ---------------------------------------------------------------------------
# CP-ALS (Algorithm 1)
# ---------------------------------------------------------------------------


def _lam(lam, n: int) -> float:
    """Step size of mode n: None means 1 (plain ALS), a scalar applies to
    every mode, a sequence gives one value per mode."""
    if lam is None:
        return 1.0
    if np.ndim(lam) == 0:
        return float(lam)
    return float(lam[n])


def step(A_old: np.ndarray, A_ls: np.ndarray, lam: float) -> np.ndarray:
    """ALS variant with an update step size (Sec. 5.1, chemistry tensor):
    A_new = (1 - lambda) A^(n) + lambda M^(n) Gamma^(n)+, where A_ls is the
    least-squares update M^(n) Gamma^(n)+ and A_old the current factor."""
    if lam == 1.0:
        return A_ls
    return (1.0 - lam) * A_old + lam * A_ls


def _tie_copy(A, S, dA, n: int, tie):
    """Symmetry constraint (Sec. 5.1, X = [[A, B, B]]): every mode tied to
    mode n takes mode n's new factor, Gram and change."""
    if not tie:
        return
    for m2, m1 in tie.items():
        if m1 == n:
            A[m2] = A[n].copy()
            S[m2] = S[n].copy()
            dA[m2] = dA[n].copy()


def als_sweep(X: np.ndarray, A, S, info: SolveInfo | None = None, lam=None, tie=None):
    """One sweep of Algorithm 1, Gauss-Seidel over the modes.

    ``A`` and ``S`` are lists updated in place.  Returns (dA, gnorm) where
    dA[n] = A^(n)_new - A^(n)_old (the per-sweep change used by Algorithm 3's
    regular sweep) and gnorm[n] = ||G^(n)||_F.

    Variants of Sec. 5.1: ``lam`` is the update step size (see ``step``);
    ``tie`` maps a mode m2 to a mode m1 < m2 whose factor it shares (the
    symmetric decomposition [[A, B, B]] is tie = {2: 1}): mode m2 is not
    solved for, it takes mode m1's factor as soon as that is updated.
    """
    N = X.ndim
    dA = [None] * N
    gnorm = [0.0] * N
    for n in range(N):
        if tie and n in tie:
            continue
        G = gamma(S, n)
        M = mttkrp(X, A, n)
        Anew = step(A[n], solve_normal(M, G, info), _lam(lam, n))
        dA[n] = Anew - A[n]
        gnorm[n] = float(np.linalg.norm((A[n] - Anew) @ G))
        A[n] = Anew
        S[n] = gram(Anew)
        _tie_copy(A, S, dA, n, tie)
    return dA, gnorm


def cp_als(X: np.ndarray, A0, n_sweeps: int, lam=None, tie=None):
    """Algorithm 1 for a fixed number of sweeps; returns (A, fitness trace).
    ``lam`` and ``tie`` select the variants of Sec. 5.1 (see ``als_sweep``)."""
    A = [a.copy() for a in A0]
    for m2, m1 in (tie or {}).items():
        A[m2] = A[m1].copy()              # tied factors start equal
    S = [gram(a) for a in A]
    normX = float(np.linalg.norm(X))
    trace = []
    for _ in range(n_sweeps):
        als_sweep(X, A, S, lam=lam, tie=tie)
        trace.append(fitness(X, A, normX))
    return A, trace


# ---------------------------------------------------------------------------
# Pairwise perturbation (Sec. 3.2.1, Eq. 3, Algorithm 3)
# ---------------------------------------------------------------------------


def pp_operators(X: np.ndarray, Ap):
    """PP operators built directly from their definitions (Sec. 3.2.1).

    Returns (ops, Mp): ops[(i, n)] for i < n is M_p^(i,n) with axes
    (x_i, x_n, r) = X_(i,n) times the Khatri-Rao product of A_p^(k),
    k not in {i, n}; Mp[n] = M_p^(n) = X_(n) P_p^(n).
    """
    N = X.ndim
    ops = {}
    for i in range(N):
        for n in range(i + 1, N):
            ops[(i, n)] = partial_mttkrp(X, Ap, [i, n])
    Mp = [mttkrp(X, Ap, n) for n in range(N)]
    return ops, Mp


def pp_first_order(ops, Mp, dA, n: int) -> np.ndarray:
    """M_p^(n) + sum_{i != n} sum_x M_p^(i,n)(x, y, r) dA^(i)(x, r) (Eq. 3,
    first two terms).  For i > n the stored operator is M_p^(n,i) with axes
    (x_n, x_i, r), i.e. the same tensor with the two modes swapped."""
    out = Mp[n].copy()
    N = len(Mp)
    for i in range(N):
        if i == n:
            continue
        if i < n:
            T = ops[(i, n)]                      # (x_i, y, r)
            out += np.einsum("xyr,xr->yr", T, dA[i])
        else:
            T = ops[(n, i)]                      # (y, x_i, r)
            out += np.einsum("yxr,xr->yr", T, dA[i])
    return out


def pp_second_order(A, dA, n: int) -> np.ndarray:
    """sum over unordered pairs {i, j}, i, j != n, of
    V^(n,i,j) = A^(n) ((A^(i)T dA^(i)) * (A^(j)T dA^(j)) * (*_{k != i,j,n} A^(k)T A^(k)))
    (Eq. 3).  Each unordered pair is counted once (the order-3 derivation,
    Eq. 2, has exactly one such term); A^(k) are the current factors."""
    N = len(A)
    R = A[0].shape[1]
    Z = np.zeros((R, R))
    for i in range(N):
        for j in range(i + 1, N):
            if i == n or j == n:
                continue
            H = (A[i].T @ dA[i]) * (A[j].T @ dA[j])
            for k in range(N):
                if k not in (i, j, n):
                    H = H * (A[k].T @ A[k])
            Z += H
    return A[n] @ Z


def pp_mttkrp(ops, Mp, A, dA, n: int, use_V: bool = True) -> np.ndarray:
    """Approximated MTTKRP M~^(n) of Eq. 3."""
    out = pp_first_order(ops, Mp, dA, n)
    if use_V:
        out = out + pp_second_order(A, dA, n)
    return out


def pp_sweep(ops, Mp, A, Ap, dA, S, use_V: bool = True, info: SolveInfo | None = None,
             lam=None, tie=None, last_rhs=None):
    """One PP approximated sweep (the PP sweep of Algorithm 3); lists updated in
    place.  ``lam`` and ``tie`` as in ``als_sweep``: the step size blends the
    current factor with the solution of the approximated normal equations, and
    a tied mode takes its partner's factor, Gram and dA = A - A_p.  A list
    passed as ``last_rhs`` receives the last mode's M~^(N) (Eq. 3; for a
    tied last mode, which is not solved for, its first-order part)."""
    N = len(A)
    gnorm = [0.0] * N
    for n in range(N):
        if tie and n in tie:
            if last_rhs is not None and n == N - 1:
                last_rhs.append(pp_first_order(ops, Mp, dA, n))
            continue
        G = gamma(S, n)
        Mt = pp_mttkrp(ops, Mp, A, dA, n, use_V)
        if last_rhs is not None and n == N - 1:
            last_rhs.append(Mt)
        Anew = step(A[n], solve_normal(Mt, G, info), _lam(lam, n))
        gnorm[n] = float(np.linalg.norm((A[n] - Anew) @ G))
        A[n] = Anew
        S[n] = gram(Anew)
        dA[n] = Anew - Ap[n]
        _tie_copy(A, S, dA, n, tie)
    return gnorm


def pp_fitness_estimate(Mt, A, normX: float) -> float:
    """The fitness a PP sweep reports without touching X: the fitness formula
    of Sec. 5 with the inner product <X, [[A]]> taken from the last mode's
    approximated right-hand side Mt = M~^(N) of that sweep (Eq. 3, formed
    before the last mode's update) and the factors after the sweep."""
    N = len(A)
    inner = float(np.sum(Mt * A[N - 1]))
    res2 = normX * normX - 2.0 * inner + norm_model_sq(A)
    return 1.0 - math.sqrt(max(res2, 0.0)) / normX


@dataclass
class PPTrace:
    """Per-sweep log of Algorithm 3: type, exact fitness, dA ratios, and the
    fitness the algorithm itself sees (exact after ALS sweeps, the estimate
    of ``pp_fitness_estimate`` after PP sweeps)."""
    kinds: list = field(default_factory=list)      # "als" | "pp_init" | "pp_approx"
    fitness: list = field(default_factory=list)
    ratios: list = field(default_factory=list)     # ||dA^(i)|| / ||A^(i)|| after the sweep
    seen: list = field(default_factory=list)
    singular: int = 0


def _small(dA, A, eps: float) -> bool:
    """Algorithm 3 test: ||dA^(i)||_F < eps ||A^(i)||_F for every mode."""
    return all(np.linalg.norm(d) < eps * np.linalg.norm(a) for d, a in zip(dA, A))


def pp_cp_als(X: np.ndarray, A0, n_sweeps: int, eps: float, use_V: bool = True,
              on_sweep=None, lam=None, tie=None, pp_stop_tol: float = 0.0):
    """Algorithm 3 (PP-CP-ALS) for a budget of ``n_sweeps`` sweeps.

    Readings where the paper leaves room: the eps test is taken at the head
    of each PP sweep (whole-matrix Frobenius norms, as written); a PP
    initialisation sweep (operator build plus one PP pass), a PP approximated
    sweep and a regular ALS sweep each count as one sweep; the reported
    fitness is always the exact one.  The stopping test Delta of Algorithm 3
    is not used to end the run (fixed budgets); with ``pp_stop_tol`` > 0 it
    is taken inside the PP loop in the form of the paper's experiments
    (Sec. 5.1: the fitness difference of two neighbouring sweeps), between
    the two last sweeps of the PP run: at the head of every PP sweep after
    the second of a run, the run goes on only if the last PP sweep raised
    the fitness estimate (``pp_fitness_estimate``, ``PPTrace.seen``) over
    the one before it by at least ``pp_stop_tol``; otherwise the regular ALS
    sweep follows, as when the eps test fails.  (Both values are estimates
    from the same operators, so their difference follows the run's progress;
    the estimate against the exact fitness of the ALS sweep before the run
    would carry the estimate's own second-order error.)  ``on_sweep(kind, A)`` is called after every
    sweep.  ``lam`` and ``tie`` select the ALS variants of Sec. 5.1 for both
    sweep kinds (see ``als_sweep``).
    """
    A = [a.copy() for a in A0]
    for m2, m1 in (tie or {}).items():
        A[m2] = A[m1].copy()              # tied factors start equal
    N = len(A)
    S = [gram(a) for a in A]
    dA = [a.copy() for a in A]            # Algorithm 3 starts from dA <- A
    normX = float(np.linalg.norm(X))
    tr = PPTrace()
    info = SolveInfo()

    def log(kind, seen):
        tr.kinds.append(kind)
        tr.fitness.append(fitness(X, A, normX))
        tr.ratios.append([float(np.linalg.norm(d) / np.linalg.norm(a)) for d, a in zip(dA, A)])
        tr.seen.append(seen)
        if on_sweep is not None:
            on_sweep(kind, A)

    def gained(run):
        if pp_stop_tol <= 0.0 or run < 2:
            return True
        return tr.seen[-1] - tr.seen[-2] >= pp_stop_tol

    t = 0
    while t < n_sweeps:
        if _small(dA, A, eps):
            Ap = [a.copy() for a in A]
            ops, Mp = pp_operators(X, Ap)
            dA = [np.zeros_like(a) for a in A]
            first = True
            run = 0                       # PP sweeps of this run so far
            while t < n_sweeps and _small(dA, A, eps) and gained(run):
                last = []
                pp_sweep(ops, Mp, A, Ap, dA, S, use_V, info, lam=lam, tie=tie, last_rhs=last)
                t += 1
                run += 1
                log("pp_init" if first else "pp_approx", pp_fitness_estimate(last[0], A, normX))
                first = False
            if t >= n_sweeps:
                break
        dA, _ = als_sweep(X, A, S, info, lam=lam, tie=tie)
        t += 1
        log("als", None)
        tr.seen[-1] = tr.fitness[-1]
    tr.singular = int(info.singular)
    return A, tr


# ---------------------------------------------------------------------------
# Reinterpreted ALS (Algorithm 5): pairwise updates with exact M^(m,n)
# ---------------------------------------------------------------------------


def pairwise_update_als_sweep(X: np.ndarray, A, S, M):
    """One sweep of Algorithm 5.  ``M`` holds the current right-hand sides
    M^(m) and is updated by H^(m,n) = sum_y M^(m,n)(x, y, k) dA^(n)(y, k)
    after every mode update, with M^(m,n) recomputed from the current
    factors (the 'oracle-like' use the paper describes)."""
    N = X.ndim
    for n in range(N):
        G = gamma(S, n)
        Anew = solve_normal(M[n], G)
        dlt = Anew - A[n]
        for m in range(N):
            if m == n:
                continue
            a, b = min(m, n), max(m, n)
            T = partial_mttkrp(X, A, [a, b])          # M^(a,b) at the factors before A^(n) moves
            if m < n:
                M[m] = M[m] + np.einsum("xyr,yr->xr", T, dlt)
            else:
                M[m] = M[m] + np.einsum("yxr,yr->xr", T, dlt)
        A[n] = Anew
        S[n] = gram(Anew)


# ---------------------------------------------------------------------------
# Cost model (Table 1, Sec. 3.2.3)
# ---------------------------------------------------------------------------


def pp_operator_build_cost(s: int, N: int, R: int) -> int:
    """2 R sum_{l=2}^{N-1} C(l+1, 2) s^(N-l+2): flops of the PP operator
    dimension tree for an equidimensional tensor (Sec. 3.2.3)."""
    return 2 * R * sum(math.comb(l + 1, 2) * s ** (N - l + 2) for l in range(2, N))


def table1_cp(s: int, N: int, R: int) -> dict:
    """Leading-order CP costs of Table 1."""
    return {"als": 4 * s ** N * R, "pp_init": 6 * s ** N * R,
            "pp_approx": 2 * N * N * (s * s * R + s * R * R)}
