"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of these retypes the oracle's
own formula: they use brute-force loops, closed forms, invariants, library
routines for special cases, or the paper's printed unit-condition tensors.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_factors(dims, R, seed):
    g = np.random.default_rng(seed)
    return [g.standard_normal((s, R)) for s in dims]


def _brute_partial(X, A, keep):
    """Element-wise Eq. 1 by nested Python loops (tiny tensors only)."""
    N = X.ndim
    R = A[0].shape[1]
    out = np.zeros([X.shape[k] for k in keep] + [R])
    for idx in itertools.product(*[range(s) for s in X.shape]):
        for r in range(R):
            w = X[idx]
            for k in range(N):
                if k not in keep:
                    w *= A[k][idx[k], r]
            out[tuple(idx[k] for k in keep) + (r,)] += w
    return out


# --- T1: MTTKRP equals its element-wise definition (Sec. 2.3, Eq. 1) -------

@pytest.mark.parametrize("dims,R", [((3, 4, 5), 1), ((3, 4, 5), 3),
                                    ((2, 3, 2, 3), 2), ((2, 2, 3, 2, 2), 2)])
def test_mttkrp_brute_force(dims, R):
    g = np.random.default_rng(1)
    X = g.standard_normal(dims)
    A = _rand_factors(dims, R, 2)
    for n in range(len(dims)):
        np.testing.assert_allclose(O.mttkrp(X, A, n), _brute_partial(X, A, [n]),
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims,keep", [((3, 4, 5), [0, 2]), ((2, 3, 2, 3), [1, 3]),
                                       ((2, 3, 2, 3), [0, 1, 3])])
def test_partial_mttkrp_brute_force(dims, keep):
    g = np.random.default_rng(3)
    X = g.standard_normal(dims)
    A = _rand_factors(dims, 2, 4)
    np.testing.assert_allclose(O.partial_mttkrp(X, A, keep), _brute_partial(X, A, keep),
                               rtol=1e-12, atol=1e-12)


def test_khatri_rao_is_columnwise_kron():
    g = np.random.default_rng(5)
    A, B, C = g.standard_normal((3, 2)), g.standard_normal((4, 2)), g.standard_normal((2, 2))
    K = O.khatri_rao([A, B, C])
    for r in range(2):
        np.testing.assert_allclose(K[:, r], np.kron(np.kron(A[:, r], B[:, r]), C[:, r]))


# --- dimension-tree consistency: contracting an intermediate further gives
# the lower intermediate (Sec. 2.5); pins the mode bookkeeping of Eq. 1 -------

def test_intermediate_chain():
    dims = (3, 4, 2, 5)
    g = np.random.default_rng(6)
    X = g.standard_normal(dims)
    A = _rand_factors(dims, 3, 7)
    M123 = O.partial_mttkrp(X, A, [0, 1, 2])        # contract mode 3
    M13 = np.einsum("ijkr,jr->ikr", M123, A[1])      # then mode 1
    np.testing.assert_allclose(M13, O.partial_mttkrp(X, A, [0, 2]), rtol=1e-12)
    M1 = np.einsum("ikr,kr->ir", M13, A[2])
    np.testing.assert_allclose(M1, O.mttkrp(X, A, 0), rtol=1e-12)


# --- T9: Hurwitz unit-condition tensors (appendix) --------------------------

def _load_hurwitz(s):
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLD, f"hurwitz_s{s}.txt"))
            if l.strip() and not l.startswith("#")]
    if s in (2, 4):
        return np.array(rows).reshape(s, s, s)
    M, Nn = np.array(rows[:8], dtype=int), np.array(rows[8:])
    T = np.zeros((8, 8, 8))
    for i in range(8):
        for j in range(8):
            T[i, j, M[i, j] - 1] = Nn[i, j]
    return T


@pytest.mark.parametrize("s", [2, 4, 8])
def test_hurwitz_norm_preserving(s):
    T = _load_hurwitz(s)
    g = np.random.default_rng(s)
    for n in range(3):
        for _ in range(10):
            A = [g.standard_normal((s, 1)) for _ in range(3)]
            z = O.mttkrp(T, A, n)[:, 0]
            others = [k for k in range(3) if k != n]
            expect = np.linalg.norm(A[others[0]]) * np.linalg.norm(A[others[1]])
            assert abs(np.linalg.norm(z) - expect) < 1e-12 * max(1.0, expect)
    # the property is sharp: flipping one sign breaks it
    T2 = T.copy()
    T2[0, 0, 0] *= -1.0
    A = [np.ones((s, 1)) for _ in range(3)]
    z = O.mttkrp(T2, A, 0)[:, 0]
    assert abs(np.linalg.norm(z) - s) > 1e-6


# --- normal-equation solve (Sec. 2.3, Algorithm 1) --------------------

def test_solve_matches_library_spd():
    g = np.random.default_rng(8)
    B = g.standard_normal((12, 7))
    G = B.T @ B + 0.1 * np.eye(7)
    M = g.standard_normal((9, 7))
    X = O.solve_normal(M, G)
    np.testing.assert_allclose(X, np.linalg.solve(G, M.T).T, rtol=1e-11, atol=1e-12)


def test_solve_orthonormal_factors_identity():
    """T11: orthonormal columns give S = I, Gamma = I, so A_new = M."""
    g = np.random.default_rng(9)
    A = [np.linalg.qr(g.standard_normal((s, 4)))[0] for s in (6, 7, 8)]
    S = [O.gram(a) for a in A]
    for n in range(3):
        np.testing.assert_allclose(O.gamma(S, n), np.eye(4), atol=1e-14)
    M = g.standard_normal((6, 4))
    np.testing.assert_allclose(O.solve_normal(M, O.gamma(S, 0)), M, atol=1e-14)


def test_solve_singular_falls_back_to_pinv():
    g = np.random.default_rng(10)
    B = g.standard_normal((3, 6))           # rank 3 Gram of size 6
    G = B.T @ B
    M = g.standard_normal((5, 6)) @ G       # consistent right-hand sides
    info = O.SolveInfo()
    X = O.solve_normal(M, G, info)
    assert info.singular
    np.testing.assert_allclose(X, M @ np.linalg.pinv(G, rcond=1e-13), rtol=1e-8, atol=1e-9)


# --- T10: fitness formula equals explicit reconstruction (Sec. 5) -------------

def test_fitness_formula_vs_reconstruction():
    g = np.random.default_rng(11)
    dims = (5, 6, 7)
    X = g.standard_normal(dims)
    A = _rand_factors(dims, 3, 12)
    assert abs(O.fitness(X, A) - O.fitness_explicit(X, A)) < 1e-12


def test_norm_model_sq_is_reconstruction_norm():
    A = _rand_factors((4, 5, 3, 2), 3, 13)
    assert abs(O.norm_model_sq(A) - np.linalg.norm(O.reconstruct(A)) ** 2) < 1e-10


# --- T8: exact low-rank recovery and the noise floor (Sec. 5.1) -------------

def test_als_recovers_exact_low_rank():
    At = _rand_factors((8, 9, 10), 3, 14)
    X = O.reconstruct(At)
    g = np.random.default_rng(15)
    A0 = [a + 1e-2 * g.standard_normal(a.shape) for a in At]
    _, tr = O.cp_als(X, A0, 60)
    assert tr[-1] > 1.0 - 1e-9
    # ALS never increases the residual (checked on explicit reconstructions:
    # the formula saturates once the residual falls below sqrt(eps) ||X||)
    A = [a.copy() for a in A0]
    S = [O.gram(a) for a in A]
    res = []
    for _ in range(20):
        O.als_sweep(X, A, S)
        res.append(np.linalg.norm(X - O.reconstruct(A)))
    assert all(b <= a * (1 + 1e-9) + 1e-13 for a, b in zip(res, res[1:]))


def test_als_noise_floor():
    """At the least-squares optimum the residual is the noise projected off
    the model's tangent space: ||E|| sqrt(1 - dof / entries), dof = R(sum s - N + 1)."""
    dims, R = (20, 20, 20), 3
    At = _rand_factors(dims, R, 16)
    X0 = O.reconstruct(At)
    E = np.random.default_rng(17).standard_normal(dims) * 1e-3
    X = X0 + E
    _, tr = O.cp_als(X, [a.copy() for a in At], 30)
    res = (1.0 - tr[-1]) * np.linalg.norm(X)
    dof = R * (sum(dims) - len(dims) + 1)
    expect = np.linalg.norm(E) * math.sqrt(1.0 - dof / np.prod(dims))
    assert abs(res / expect - 1.0) < 0.03


# --- T3, T4, T5, T6: pairwise perturbation (Sec. 3.1.1, 3.2.1, Eq. 2-3) ------

def _pp_setup(dims, R, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal(dims)
    Ap = _rand_factors(dims, R, seed + 1)
    ops, Mp = O.pp_operators(X, Ap)
    return g, X, Ap, ops, Mp


@pytest.mark.parametrize("dims", [(4, 5, 6), (3, 4, 3, 5), (2, 3, 2, 3, 2)])
def test_pp_zero_perturbation_is_exact(dims):
    """T3: with dA = 0, M~^(n) = M_p^(n) = exact MTTKRP at A_p."""
    _, X, Ap, ops, Mp = _pp_setup(dims, 3, 20)
    dA = [np.zeros_like(a) for a in Ap]
    for n in range(len(dims)):
        exact = O.mttkrp(X, Ap, n)
        np.testing.assert_allclose(O.pp_mttkrp(ops, Mp, Ap, dA, n, True), exact, rtol=1e-12)
        np.testing.assert_allclose(Mp[n], exact, rtol=1e-12)


@pytest.mark.parametrize("dims", [(4, 5, 6), (3, 4, 3, 5)])
def test_pp_single_perturbation_is_exact(dims):
    """T4a: the MTTKRP is linear in each factor, so with one dA^(i) != 0 the
    first-order terms of Eq. 3 are exact."""
    g, X, Ap, ops, Mp = _pp_setup(dims, 3, 21)
    N = len(dims)
    for i in range(N):
        dA = [np.zeros_like(a) for a in Ap]
        dA[i] = g.standard_normal(Ap[i].shape)
        A = [a + d for a, d in zip(Ap, dA)]
        for n in range(N):
            np.testing.assert_allclose(O.pp_first_order(ops, Mp, dA, n), O.mttkrp(X, A, n),
                                       rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 3, 5, 4)])
def test_pp_error_scales_quadratically(dims):
    """T4b: the dropped terms carry >= 2 factors dA, so scaling every dA by t
    scales the error by t^2 (Sec. 3.2.1)."""
    g, X, Ap, ops, Mp = _pp_setup(dims, 3, 22)
    D = [g.standard_normal(a.shape) for a in Ap]
    N = len(dims)
    for n in range(N):
        errs = []
        ts = [1e-1, 1e-2, 1e-3]
        for t in ts:
            dA = [t * d for d in D]
            A = [a + d for a, d in zip(Ap, dA)]
            errs.append(np.linalg.norm(O.pp_first_order(ops, Mp, dA, n) - O.mttkrp(X, A, n)))
        slopes = np.diff(np.log(errs)) / np.diff(np.log(ts))
        assert np.all(np.abs(slopes - 2.0) < 0.05), slopes


def test_pp_order3_with_V_exact_on_cp_tensor():
    """T5: for N = 3 and X = [[A]] (A the current factors), Eq. 2's dropped
    term is exactly V^(1); PP with V reproduces the exact MTTKRP for every
    mode, whatever A_p.  Counting each pair twice would not."""
    g = np.random.default_rng(23)
    dims, R = (5, 6, 7), 3
    A = _rand_factors(dims, R, 24)
    X = O.reconstruct(A)
    Ap = [a + 0.3 * g.standard_normal(a.shape) for a in A]
    ops, Mp = O.pp_operators(X, Ap)
    dA = [a - b for a, b in zip(A, Ap)]
    for n in range(3):
        exact = O.mttkrp(X, A, n)
        np.testing.assert_allclose(O.pp_mttkrp(ops, Mp, A, dA, n, True), exact,
                                   rtol=1e-10, atol=1e-10)
        doubled = O.pp_first_order(ops, Mp, dA, n) + 2 * O.pp_second_order(A, dA, n)
        assert np.linalg.norm(doubled - exact) > 1e-3 * np.linalg.norm(exact)


@pytest.mark.parametrize("dims", [(4, 3, 5, 4), (3, 4, 3, 2, 3)])
def test_pp_with_V_third_order_on_cp_tensor(dims):
    """For N >= 4 and X = [[A]], the second-order terms of the expansion in
    Sec. 3.2.1 equal V^(n,i,j) up to one more factor dA (V takes A^(k)T A^(k)
    where the expansion has A^(k)T A_p^(k)), so PP with V is exact to second
    order: scaling dA by t scales its error by t^3 (and without V by t^2)."""
    g = np.random.default_rng(31)
    R = 2
    Ap = _rand_factors(dims, R, 32)
    D = [g.standard_normal(a.shape) for a in Ap]
    ts = [1e-2, 5e-3, 2.5e-3]
    for n in range(len(dims)):
        ev, e0 = [], []
        for t in ts:
            dA = [t * d for d in D]
            A = [a + d for a, d in zip(Ap, dA)]
            X = O.reconstruct(A)
            ops, Mp = O.pp_operators(X, Ap)
            exact = O.mttkrp(X, A, n)
            ev.append(np.linalg.norm(O.pp_mttkrp(ops, Mp, A, dA, n, True) - exact))
            e0.append(np.linalg.norm(O.pp_mttkrp(ops, Mp, A, dA, n, False) - exact))
        sv = np.diff(np.log(ev)) / np.diff(np.log(ts))
        s0 = np.diff(np.log(e0)) / np.diff(np.log(ts))
        assert np.all(np.abs(sv - 3.0) < 0.15), sv
        assert np.all(np.abs(s0 - 2.0) < 0.15), s0


@pytest.mark.parametrize("dims", [(4, 5, 6), (3, 4, 3, 5)])
def test_pp_operators_consistent(dims):
    """T6: M_p^(n) = M_p^(i,n) x_i A_p^(i) for every i != n (Sec. 3.2.3)."""
    _, X, Ap, ops, Mp = _pp_setup(dims, 2, 25)
    N = len(dims)
    for n in range(N):
        for i in range(N):
            if i == n:
                continue
            if i < n:
                v = np.einsum("xyr,xr->yr", ops[(i, n)], Ap[i])
            else:
                v = np.einsum("yxr,xr->yr", ops[(n, i)], Ap[i])
            np.testing.assert_allclose(v, Mp[n], rtol=1e-12, atol=1e-12)


def test_pp_operator_matches_brute_force():
    g = np.random.default_rng(26)
    dims = (3, 2, 4, 2)
    X = g.standard_normal(dims)
    Ap = _rand_factors(dims, 2, 27)
    ops, _ = O.pp_operators(X, Ap)
    for (i, n), T in ops.items():
        np.testing.assert_allclose(T, _brute_partial(X, Ap, [i, n]), rtol=1e-12, atol=1e-12)


# --- T7: pairwise-update ALS (Algorithm 5) equals ALS (Algorithm 1) --------

@pytest.mark.parametrize("dims", [(5, 6, 7), (3, 4, 3, 5)])
def test_pairwise_update_als_equals_als(dims):
    g = np.random.default_rng(28)
    X = g.standard_normal(dims)
    A0 = [g.random((s, 3)) for s in dims]
    A1 = [a.copy() for a in A0]
    S1 = [O.gram(a) for a in A1]
    A2 = [a.copy() for a in A0]
    S2 = [O.gram(a) for a in A2]
    M = [O.mttkrp(X, A2, n) for n in range(len(dims))]
    for _ in range(3):
        O.als_sweep(X, A1, S1)
        O.pairwise_update_als_sweep(X, A2, S2, M)
    for a, b in zip(A1, A2):
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)


# --- Algorithm 3 controller special cases ------------------------------------

def test_pp_als_eps_zero_is_als():
    p = synth.scaled("normal", 8, 3, 3, seed=3, noise=1e-2, storage="f64")
    X = p.X
    A_als, tr_als = O.cp_als(X, p.A0, 12)
    A_pp, tr = O.pp_cp_als(X, p.A0, 12, eps=0.0)
    assert tr.kinds == ["als"] * 12
    np.testing.assert_allclose(tr.fitness, tr_als, rtol=0, atol=1e-13)


def test_pp_init_first_mode_equals_als():
    """With eps > 1 the operators are built at once (dA = A initially); the
    first PP sweep starts from dA = 0, so its first mode update is exactly
    the ALS update."""
    p = synth.scaled("normal", 7, 3, 2, seed=4, noise=1e-2, storage="f64")
    A_pp, tr = O.pp_cp_als(p.X, p.A0, 1, eps=2.0)
    assert tr.kinds == ["pp_init"]
    A = [a.copy() for a in p.A0]
    S = [O.gram(a) for a in A]
    G = O.gamma(S, 0)
    a0 = O.solve_normal(O.mttkrp(p.X, A, 0), G)
    np.testing.assert_allclose(A_pp[0], a0, rtol=1e-11, atol=1e-12)


def test_pp_als_converges_on_exact_tensor():
    """On an exactly low-rank tensor the PP-ALS trajectory tracks ALS (the
    PP error is second order in dA, Sec. 4.1) and reaches the exact fit."""
    At = _rand_factors((9, 10, 11), 3, 29)
    X = O.reconstruct(At)
    g = np.random.default_rng(30)
    A0 = [a + 5e-2 * g.standard_normal(a.shape) for a in At]
    _, tr = O.pp_cp_als(X, A0, 80, eps=0.1)
    _, ta = O.cp_als(X, A0, 80)
    assert "pp_approx" in tr.kinds
    assert max(abs(a - b) for a, b in zip(tr.fitness, ta)) < 1e-5
    assert tr.fitness[-1] > 1.0 - 1e-7


# --- Table 1 / Sec. 3.2.3 cost formulas ---------------------------------------

@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_operator_build_cost_expansion(N):
    """2R sum_{l=2}^{N-1} C(l+1,2) s^{N-l+2} = 6 s^N R + 12 s^{N-1} R + O(s^{N-2})."""
    R = 7
    for s in (10, 100, 1000):
        c = O.pp_operator_build_cost(s, N, R)
        if N == 3:                       # a single level: three first-level contractions
            assert c == 6 * s ** 3 * R
            continue
        lead = 6 * s ** N * R + 12 * s ** (N - 1) * R
        rest = c - lead
        assert rest >= 0
        assert rest <= 2 * R * math.comb(N, 2) * N * s ** (N - 2)
    assert O.table1_cp(10, N, R)["pp_init"] == 6 * 10 ** N * R


@pytest.mark.parametrize("dims", [[5, 6, 7], [4, 3, 5, 6], [3, 4, 2, 3, 4]])
def test_partial_row_matches_definitions(dims):
    """The row-at-a-time contraction used for full-size samples equals the
    unfolded definitions: MTTKRP rows (Sec. 2.3) and PP operator entries
    (Eq. 1 with two fixed modes), against a brute-force loop as well."""
    rng = np.random.default_rng(11)
    R = 3
    X = rng.standard_normal(dims)
    A = [rng.standard_normal((d, R)) for d in dims]
    N = len(dims)
    for n in range(N):
        M = O.mttkrp(X, A, n)
        for y in range(dims[n]):
            assert np.allclose(O.partial_row(X, A, {n: y}), M[y], rtol=1e-12, atol=1e-12)
    for i in range(N):
        for n in range(i + 1, N):
            P = O.partial_mttkrp(X, A, [i, n])
            for xi in range(dims[i]):
                for xn in range(dims[n]):
                    assert np.allclose(O.partial_row(X, A, {i: xi, n: xn}), P[xi, xn], rtol=1e-12, atol=1e-12)
    # brute force for one entry
    idx = [rng.integers(d) for d in dims]
    fixed = {0: idx[0], N - 1: idx[-1]}
    brute = np.zeros(R)
    for x in np.ndindex(*dims):
        if x[0] != idx[0] or x[-1] != idx[-1]:
            continue
        w = X[x]
        prod = np.ones(R)
        for k in range(1, N - 1):
            prod = prod * A[k][x[k]]
        brute += w * prod
    assert np.allclose(O.partial_row(X, A, fixed), brute, rtol=1e-12, atol=1e-12)


# --- Sec. 5.1 ALS variants: update step size and the symmetry constraint -------

def _residual_sq(X, A):
    return float(np.sum((X - O.reconstruct(A)) ** 2))


@pytest.mark.parametrize("lam", [0.3, 0.7, 1.4])
def test_step_size_residual_is_quadratic_in_lambda(lam):
    """With the other factors fixed the residual is a convex quadratic in
    A^(n) whose minimiser is the least-squares update, so along
    A + lam (A_ls - A): r(lam) - r(1) = (1 - lam)^2 (r(0) - r(1)).  Only mode 0
    moves (step size 0 leaves a factor exactly unchanged)."""
    g = np.random.default_rng(11)
    X = g.standard_normal((7, 6, 5))
    A0 = _rand_factors((7, 6, 5), 3, 12)
    def upd(l):
        A = [a.copy() for a in A0]
        S = [O.gram(a) for a in A]
        O.als_sweep(X, A, S, lam=[l, 0.0, 0.0])
        for k in (1, 2):
            np.testing.assert_array_equal(A[k], A0[k])
        return A
    r0, r1, rl = (_residual_sq(X, upd(l)) for l in (0.0, 1.0, lam))
    assert r0 > r1
    np.testing.assert_allclose(rl - r1, (1 - lam) ** 2 * (r0 - r1), rtol=1e-9)


def _lstsq_mode(X, A, n):
    """min_B ||X_(n) - B K^T|| by numpy lstsq on the explicit unfolding, with
    K[(x_other), r] = prod_{k != n} A^(k)(x_k, r) written out by einsum."""
    N = X.ndim
    other = [k for k in range(N) if k != n]
    letters = "abcdefg"
    spec = ",".join(letters[k] + "r" for k in other) + "->" + "".join(letters[k] for k in other) + "r"
    R = A[other[0]].shape[1]
    K = np.einsum(spec, *[A[k] for k in other]).reshape(-1, R)
    Xn = np.moveaxis(X, n, 0).reshape(X.shape[n], -1)
    return np.linalg.lstsq(K, Xn.T, rcond=None)[0].T


def test_symmetric_sweep_matches_least_squares():
    """[[A, B, B]] (Sec. 5.1): A takes the plain least-squares update with
    (B, B); B the step-size-0.8 blend of its least-squares update with
    (A_new, B_old) in the other two modes; mode 2 then carries B."""
    g = np.random.default_rng(21)
    At, Bt = g.standard_normal((9, 3)), g.standard_normal((6, 3))
    X = O.reconstruct([At, Bt, Bt])
    E = g.standard_normal(X.shape)
    X = X + 1e-2 * (E + E.transpose(0, 2, 1))            # noise symmetric in modes 1, 2
    A0 = _rand_factors((9, 6, 6), 3, 22)
    A = [a.copy() for a in A0]
    A[2] = A[1].copy()
    S = [O.gram(a) for a in A]
    O.als_sweep(X, A, S, lam=[1.0, 0.8, 1.0], tie={2: 1})
    a_new = _lstsq_mode(X, [None, A0[1], A0[1]], 0)
    b_ls = _lstsq_mode(X, [a_new, None, A0[1]], 1)
    b_new = 0.2 * A0[1] + 0.8 * b_ls
    np.testing.assert_allclose(A[0], a_new, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(A[1], b_new, rtol=1e-9, atol=1e-10)
    np.testing.assert_array_equal(A[2], A[1])
    np.testing.assert_allclose(S[2], b_new.T @ b_new, rtol=1e-9, atol=1e-10)


def test_symmetric_als_and_pp_recover_exact_symmetric_tensor():
    """An exactly symmetric rank-3 tensor [[A, B, B]] is approached from a
    nearby start by the symmetric ALS (B step 0.8) and by symmetric PP-ALS;
    the two trajectories agree to second order in dA."""
    g = np.random.default_rng(31)
    At, Bt = g.standard_normal((10, 3)), g.standard_normal((8, 3))
    X = O.reconstruct([At, Bt, Bt])
    A0 = [At + 3e-2 * g.standard_normal(At.shape), Bt + 3e-2 * g.standard_normal(Bt.shape), None]
    A0[2] = A0[1].copy()
    lam, tie = [1.0, 0.8, 1.0], {2: 1}
    Aa, ta = O.cp_als(X, A0, 150, lam=lam, tie=tie)
    Ap, tp = O.pp_cp_als(X, A0, 150, eps=0.1, lam=lam, tie=tie)
    assert ta[-1] > 1 - 1e-5 and tp.fitness[-1] > 1 - 1e-5          # from 0.990 at sweep 1
    assert "pp_approx" in tp.kinds
    np.testing.assert_array_equal(Aa[2], Aa[1])
    np.testing.assert_array_equal(Ap[2], Ap[1])
    assert max(abs(a - b) for a, b in zip(tp.fitness, ta)) < 1e-6


def test_pp_init_first_mode_equals_als_with_step_size():
    """As test_pp_init_first_mode_equals_als, with step size 0.7: the first
    PP mode update (all dA = 0) is the ALS update blended with the current
    factor."""
    p = synth.scaled("normal", 7, 3, 2, seed=4, noise=1e-2, storage="f64")
    A_pp, tr = O.pp_cp_als(p.X, p.A0, 1, eps=2.0, lam=0.7)
    A = [a.copy() for a in p.A0]
    S = [O.gram(a) for a in A]
    O.als_sweep(p.X, A, S, lam=[0.7, 0.0, 0.0])
    np.testing.assert_allclose(A_pp[0], A[0], rtol=1e-11, atol=1e-12)
    assert not np.allclose(A_pp[0], O.solve_normal(O.mttkrp(p.X, p.A0, 0),
                                                   O.gamma([O.gram(a) for a in p.A0], 0)))


# --- Tucker-ALS and PP-Tucker-ALS (Sec. 2.4, Sec. 3.1.2, Sec. 3.2.2) ----------

from oracle import tucker_oracle as TO  # noqa: E402


def test_tucker_ttmc_brute_force():
    g = np.random.default_rng(61)
    X = g.standard_normal((3, 4, 5))
    A = [g.standard_normal((3, 2)), g.standard_normal((4, 2)), g.standard_normal((5, 3))]
    for n in range(3):
        Y = TO.ttmc(X, A, n)
        ref = np.zeros(Y.shape)
        for idx in itertools.product(*[range(s) for s in X.shape]):
            for out in itertools.product(*[range(d) for d in Y.shape]):
                if out[n] != idx[n]:
                    continue
                w = X[idx]
                for k in range(3):
                    if k != n:
                        w *= A[k][idx[k], out[k]]
                ref[out] += w
        np.testing.assert_allclose(Y, ref, rtol=1e-12, atol=1e-12)


def test_tucker_hosvd_recovers_exact_multilinear_rank():
    p = synth.tucker_problem([12, 10, 9], [3, 4, 2], seed=3, noise=0.0)
    A = TO.hosvd(p.X, p.R)
    G = TO.core(p.X, A)
    normX = float(np.linalg.norm(p.X))
    assert TO.fitness(normX, G) > 1 - 1e-7
    np.testing.assert_allclose(TO.reconstruct(G, A), p.X, rtol=0, atol=1e-10 * normX)
    for a in A:
        np.testing.assert_allclose(a.T @ a, np.eye(a.shape[1]), atol=1e-12)


def test_tucker_hooi_core_norm_nondecreasing_and_fitness_identity():
    """HOOI never decreases ||G|| (Sec. 4.2), and with orthonormal factors the
    fitness from ||G|| equals the explicit residual."""
    p = synth.tucker_problem([14, 12, 10], [3, 3, 2], seed=4, noise=0.3)
    A = [a.copy() for a in p.A0]
    normX = float(np.linalg.norm(p.X))
    last = -1.0
    for _ in range(6):
        _, G = TO.als_sweep(p.X, A)
        gn = float(np.linalg.norm(G))
        assert gn >= last - 1e-12
        last = gn
        explicit = 1 - np.linalg.norm(p.X - TO.reconstruct(G, A)) / normX
        assert abs(TO.fitness(normX, G) - explicit) < 1e-12


def test_tucker_gram_eigvecs_span_the_svd_subspace():
    g = np.random.default_rng(62)
    Y = g.standard_normal((15, 40))
    V = TO.leading_eigvecs(Y @ Y.T, 4)
    U = np.linalg.svd(Y, full_matrices=False)[0][:, :4]
    np.testing.assert_allclose(V @ V.T, U @ U.T, atol=1e-12)
    np.testing.assert_allclose(np.abs(V.T @ U), np.eye(4), atol=1e-10)


def test_pp_tucker_exact_at_zero_and_second_order():
    """Order 3: Y^(n)(A_p + dA) = Y~^(n) + X x_i dA^(i)T x_j dA^(j)T exactly
    (the expansion of Sec. 3.1.2 has four terms), so Y~ is exact at dA = 0
    and its error is the product term."""
    g = np.random.default_rng(63)
    X = g.standard_normal((7, 6, 5))
    Ap = [np.linalg.qr(g.standard_normal((s, r)))[0] for s, r in zip(X.shape, (3, 2, 2))]
    ops, Mp = TO.pp_operators(X, Ap)
    D = [g.standard_normal(a.shape) for a in Ap]
    for n in range(3):
        zero = [np.zeros_like(a) for a in Ap]
        np.testing.assert_allclose(TO.pp_ttmc(ops, Mp, zero, n), TO.ttmc(X, Ap, n), atol=1e-12)
        for t in (1e-2, 0.3):
            dA = [t * d for d in D]
            A = [a + d for a, d in zip(Ap, dA)]
            i, j = [k for k in range(3) if k != n]
            product = TO.ttm(TO.ttm(X, dA[i], i), dA[j], j)
            np.testing.assert_allclose(TO.ttmc(X, A, n) - TO.pp_ttmc(ops, Mp, dA, n), product,
                                       rtol=1e-10, atol=1e-12)


def test_pp_tucker_als_tracks_hooi():
    p = synth.tucker_problem([16, 14, 12], [3, 3, 2], seed=5, noise=0.05)
    A0 = TO.hosvd(p.X, p.R)
    _, kinds, fit = TO.pp_tucker_als(p.X, A0, 20, eps=0.3)
    A = [a.copy() for a in A0]
    normX = float(np.linalg.norm(p.X))
    als = []
    for _ in range(20):
        _, G = TO.als_sweep(p.X, A)
        als.append(TO.fitness(normX, G))
    assert "pp_approx" in kinds
    assert max(abs(a - b) for a, b in zip(fit, als)) < 1e-6


# --- Algorithm 3 sequencing (the PP-CP-ALS algorithm, Sec. 3.2) -----------------

def _max_ratio(new, old):
    return max(float(np.linalg.norm(a - b) / np.linalg.norm(a)) for a, b in zip(new, old))


def test_pp_cp_als_schedule_follows_eps_crossings(monkeypatch):
    """Algorithm 3's control flow, checked against a schedule the test derives
    on its own.

    (i) eps is placed between two ratios of a plain ALS trace (als_sweep
    alone), so the first operator build must come right after the first ALS
    sweep whose ratio falls below eps.  (ii) From the factors after every
    sweep, the test recomputes ||dA^(i)|| / ||A^(i)|| by the paper's
    definitions (A_new - A_old after an ALS sweep, A_new - A_p after a PP
    sweep, A_p = the factors at the head of the PP initialisation sweep) and
    checks that each sweep's kind follows the rule taken at the head of that
    sweep: after an ALS sweep a build and PP initialisation sweep iff every
    ratio is below eps; inside a PP run another PP approximated sweep iff
    every ratio is below eps, and otherwise exactly one ALS sweep.  (iii) The
    eps test is evaluated only between sweeps, once per sweep head (twice at
    a build: the outer test and the PP loop's own test with dA = 0)."""
    p = synth.make_problem("collinear", [14, 13, 12], 4, seed=11, noise=1e-2, collinearity=0.8,
                           storage="f64")
    X = p.X
    A = [a.copy() for a in p.A0]
    S = [O.gram(a) for a in A]
    hist = [[a.copy() for a in A]]
    ratios = []
    for _ in range(20):
        O.als_sweep(X, A, S)
        hist.append([a.copy() for a in A])
        ratios.append(_max_ratio(hist[-1], hist[-2]))
    # first sweep t0 >= 3 whose ratio is below every earlier one
    t0 = next(t for t in range(3, 20) if ratios[t] < min(ratios[:t]))
    eps = float(np.sqrt(ratios[t0] * min(ratios[:t0])))

    state = {"done": 0, "inside": False}
    calls = []
    real_small, real_als, real_pp = O._small, O.als_sweep, O.pp_sweep

    def spy_small(dA, A, e):
        assert not state["inside"], "eps test taken inside a sweep"
        res = real_small(dA, A, e)
        calls.append((state["done"], res))
        return res

    def wrap(fn):
        def inner(*a, **k):
            state["inside"] = True
            try:
                return fn(*a, **k)
            finally:
                state["inside"] = False
        return inner

    monkeypatch.setattr(O, "_small", spy_small)
    monkeypatch.setattr(O, "als_sweep", wrap(real_als))
    monkeypatch.setattr(O, "pp_sweep", wrap(real_pp))
    after = []

    def on_sweep(kind, A):
        state["done"] += 1
        after.append([a.copy() for a in A])

    n = 45
    _, tr = O.pp_cp_als(X, p.A0, n, eps, use_V=True, on_sweep=on_sweep)
    kinds = tr.kinds
    assert len(kinds) == n
    # (i) the crossing fixed by the ALS-only trace
    assert kinds[: t0 + 2] == ["als"] * (t0 + 1) + ["pp_init"]
    for t in range(t0 + 1):
        for a, b in zip(after[t], hist[t + 1]):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    # (ii) every later kind follows the rule at its head
    prev_f = [a.copy() for a in p.A0]
    Ap = None
    r = []
    for t, k in enumerate(kinds):
        if k == "pp_init":
            Ap = prev_f
        r.append(_max_ratio(after[t], Ap if k != "als" else prev_f))
        prev_f = after[t]
    assert kinds[0] == "als"
    for t in range(1, n):
        small = r[t - 1] < eps
        if kinds[t - 1] == "als":
            assert kinds[t] == ("pp_init" if small else "als"), t
        else:
            assert kinds[t] == ("pp_approx" if small else "als"), t
    assert "pp_approx" in kinds and any(
        kinds[t - 1] in ("pp_init", "pp_approx") and kinds[t] == "als" for t in range(1, n)), kinds
    # the oracle's own ratio log agrees with the definitions
    np.testing.assert_allclose([max(x) for x in tr.ratios], r, rtol=1e-12, atol=0)
    # (iii) one test per sweep head, two at a build head, none at the budget's end
    per_head = {}
    for head, _ in calls:
        per_head[head] = per_head.get(head, 0) + 1
    for t in range(n):
        assert per_head.get(t, 0) == (2 if kinds[t] == "pp_init" else 1), (t, kinds[t], per_head.get(t))
    assert n not in per_head


def test_pp_tucker_core_estimate():
    """The core estimate a PP-Tucker sweep returns (Algorithm 4) is Y~^(3)
    contracted with the new A^(3).  Order 3 has the exact four-term expansion
    of Sec. 3.1.2, Y^(3)(A_p + dA) = Y~^(3) + X x_1 dA^(1)T x_2 dA^(2)T, so the
    exact core at the new factors minus the estimate must be
    X x_1 dA^(1)T x_2 dA^(2)T x_3 A^(3)T with the sweep's final changes
    dA = A - A_p (loop sums here, not the oracle's contractions); at dA = 0
    the two cores coincide."""
    def core_loops(X, U, V, W):
        return np.einsum("abc,ai,bj,ck->ijk", X, U, V, W, optimize=False)

    g = np.random.default_rng(64)
    X = g.standard_normal((9, 8, 7))
    ranks = (3, 2, 4)
    Ap = [np.linalg.qr(g.standard_normal((s, r)))[0] for s, r in zip(X.shape, ranks)]
    ops, Mp = TO.pp_operators(X, Ap)
    A = [a.copy() for a in Ap]
    dA = [np.zeros_like(a) for a in Ap]
    est = TO.pp_sweep(ops, Mp, A, Ap, dA)
    assert est.shape == ranks
    assert max(float(np.linalg.norm(d)) for d in dA) > 1e-3        # the sweep moved the factors
    for n in range(3):
        np.testing.assert_allclose(dA[n], A[n] - Ap[n], atol=1e-15)
    exact = core_loops(X, A[0], A[1], A[2])
    product = core_loops(X, dA[0], dA[1], A[2])
    np.testing.assert_allclose(exact - est, product, rtol=1e-10, atol=1e-12)
    # dA = 0: an exact multilinear-rank tensor at its HOSVD factors is a fixed point
    q = synth.tucker_problem([10, 9, 8], [3, 2, 4], seed=6, noise=0.0)
    H = TO.hosvd(q.X, q.R)
    ops, Mp = TO.pp_operators(q.X, H)
    A = [a.copy() for a in H]
    dA = [np.zeros_like(a) for a in H]
    est = TO.pp_sweep(ops, Mp, A, H, dA)
    assert max(float(np.max(np.abs(d))) for d in dA) < 1e-10
    exact = core_loops(q.X, A[0], A[1], A[2])
    np.testing.assert_allclose(est, exact, rtol=0, atol=1e-10 * float(np.linalg.norm(q.X)))


def test_pp_fitness_estimate_is_the_order3_expansion_with_V():
    """The fitness a PP sweep reports takes <X, [[A]]> from the last mode's
    M~^(N) (Eq. 3, formed before that mode's update) and the new factors.
    For order 3 the expansion of Sec. 3.1.1 has exactly one term beyond first
    order, X contracted with dA^(1) and dA^(2); Eq. 3 replaces it by the V
    term A^(3)_old ((A^(1)T dA^(1)) * (A^(2)T dA^(2))).  So the estimate's
    inner product is the exact one minus that term plus the V term, all
    summed here straight from X and the factors; at dA = 0 the estimate is
    the exact fitness."""
    g = np.random.default_rng(71)
    X = g.standard_normal((7, 6, 5))
    Ap = [g.standard_normal((s, 3)) for s in X.shape]
    ops, Mp = O.pp_operators(X, Ap)
    normX = float(np.linalg.norm(X))
    zero = [np.zeros_like(a) for a in Ap]
    Mt0 = O.pp_mttkrp(ops, Mp, Ap, zero, 2, True)
    assert abs(O.pp_fitness_estimate(Mt0, Ap, normX) - O.fitness(X, Ap)) < 1e-13
    dA = [0.05 * g.standard_normal(a.shape) for a in Ap]
    A_old = [Ap[0] + dA[0], Ap[1] + dA[1], Ap[2]]          # modes 1 and 2 updated, mode 3 not yet
    Mt = O.pp_mttkrp(ops, Mp, A_old, dA, 2, True)
    A_new = [A_old[0], A_old[1], Ap[2] + 0.05 * g.standard_normal(Ap[2].shape)]
    inner = float(np.einsum("abc,ar,br,cr->", X, A_new[0], A_new[1], A_new[2], optimize=False))
    second = float(np.einsum("abc,ar,br,cr->", X, dA[0], dA[1], A_new[2], optimize=False))
    H = (A_new[0].T @ dA[0]) * (A_new[1].T @ dA[1])
    vterm = float(np.sum((A_old[2] @ H) * A_new[2]))
    model = float(np.sum(reduce_hadamard([a.T @ a for a in A_new])))
    want = 1.0 - np.sqrt(max(normX ** 2 - 2.0 * (inner - second + vterm) + model, 0.0)) / normX
    got = O.pp_fitness_estimate(Mt, A_new, normX)
    assert abs(got - want) < 1e-12, (got, want)
    assert abs(got - O.fitness(X, A_new)) > 1e-8          # the terms beyond first order matter here
    # pp_sweep hands out the M~^(N) it formed for the last mode
    A = [a.copy() for a in Ap]
    dd = [np.zeros_like(a) for a in Ap]
    S = [O.gram(a) for a in A]
    last = []
    O.pp_sweep(ops, Mp, A, [a.copy() for a in Ap], dd, S, True, last_rhs=last)
    A_mid = [A[0], A[1], Ap[2]]
    np.testing.assert_allclose(last[0], O.pp_mttkrp(ops, Mp, A_mid, dd, 2, True), rtol=1e-12, atol=1e-12)


def reduce_hadamard(mats):
    out = np.ones_like(mats[0])
    for m in mats:
        out = out * m
    return out


def test_pp_stop_tolerance_sequence():
    """Algorithm 3's stopping test inside the PP loop, in the fitness-difference
    form of Sec. 5.1 (pp_stop_tol), between the two last PP sweeps of a run:
    at the head of each PP sweep after the second of a run, the run goes on
    only if the eps test holds and the last PP sweep raised the fitness
    estimate over the one before it by at least the tolerance; otherwise an
    ALS sweep follows.  Checked from the trace's own estimates and ratios
    recomputed from the factor history; a tolerance no sweep can meet ends
    every PP run after two sweeps; a zero tolerance is the run without the
    test."""
    p = synth.make_problem("collinear", [14, 13, 12], 4, seed=11, noise=1e-2, collinearity=0.8,
                           storage="f64")
    eps = 0.0993
    _, tr = O.pp_cp_als(p.X, p.A0, 45, eps)
    _, tr0 = O.pp_cp_als(p.X, p.A0, 45, eps, pp_stop_tol=0.0)
    assert tr0.kinds == tr.kinds
    _, big = O.pp_cp_als(p.X, p.A0, 45, eps, pp_stop_tol=1.0)
    runs, run = [], 0
    for k in big.kinds:
        if k == "pp_init":
            run = 1
        elif k == "pp_approx":
            run += 1
        else:
            if run:
                runs.append(run)
            run = 0
    assert runs and max(runs) <= 2 and 2 in runs
    tol = 1e-3
    after = []
    _, tt = O.pp_cp_als(p.X, p.A0, 45, eps, pp_stop_tol=tol,
                        on_sweep=lambda k, A: after.append([a.copy() for a in A]))
    kinds, seen = tt.kinds, tt.seen
    prev_f = [a.copy() for a in p.A0]
    Ap, r = None, []
    for t, k in enumerate(kinds):
        if k == "pp_init":
            Ap = prev_f
        r.append(_max_ratio(after[t], Ap if k != "als" else prev_f))
        prev_f = after[t]
    stops = 0
    run = 0
    for t in range(1, len(kinds)):
        run = run + 1 if kinds[t - 1] == "pp_approx" else (1 if kinds[t - 1] == "pp_init" else 0)
        if run:
            gain_ok = run < 2 or seen[t - 1] - seen[t - 2] >= tol
            go = r[t - 1] < eps and gain_ok
            assert kinds[t] == ("pp_approx" if go else "als"), t
            stops += r[t - 1] < eps and not gain_ok
    assert stops >= 1, "no PP run ended on the stopping test"
    assert kinds != tr.kinds


# --- Tucker at order N > 3 (Sec. 2.4, Sec. 3.1.2, Sec. 3.2.2 for any N) -------

def test_tucker_ttmc_brute_force_order4():
    g = np.random.default_rng(71)
    X = g.standard_normal((3, 2, 4, 3))
    A = [g.standard_normal((s, r)) for s, r in zip(X.shape, (2, 2, 3, 2))]
    for n in range(4):
        Y = TO.ttmc(X, A, n)
        ref = np.zeros(Y.shape)
        for idx in itertools.product(*[range(s) for s in X.shape]):
            for out in itertools.product(*[range(d) for d in Y.shape]):
                if out[n] != idx[n]:
                    continue
                w = X[idx]
                for k in range(4):
                    if k != n:
                        w *= A[k][idx[k], out[k]]
                ref[out] += w
        np.testing.assert_allclose(Y, ref, rtol=1e-12, atol=1e-12)


def test_pp_tucker_expansion_order4():
    """Order 4: Y^(n)(A_p + dA) is the sum over every subset S of the other
    modes of X x_{k in S} dA^(k)T x_{k not in S} A_p^(k)T (multilinearity);
    Y~^(n) holds the terms with |S| <= 1 (Sec. 3.2.2), so the difference is
    the sum of the terms with |S| >= 2, written out subset by subset."""
    g = np.random.default_rng(72)
    X = g.standard_normal((5, 4, 6, 3))
    Ap = [np.linalg.qr(g.standard_normal((s, r)))[0] for s, r in zip(X.shape, (2, 3, 2, 2))]
    ops, Mp = TO.pp_operators(X, Ap)
    D = [0.1 * g.standard_normal(a.shape) for a in Ap]
    A = [a + d for a, d in zip(Ap, D)]
    for n in range(4):
        others = [k for k in range(4) if k != n]
        rest = np.zeros_like(Mp[n])
        for size in (2, 3):
            for S in itertools.combinations(others, size):
                T = X
                for k in others:
                    T = TO.ttm(T, D[k] if k in S else Ap[k], k)
                rest = rest + T
        np.testing.assert_allclose(TO.ttmc(X, A, n) - TO.pp_ttmc(ops, Mp, D, n), rest,
                                   rtol=1e-10, atol=1e-12)
        zero = [np.zeros_like(a) for a in Ap]
        np.testing.assert_allclose(TO.pp_ttmc(ops, Mp, zero, n), TO.ttmc(X, Ap, n), atol=1e-12)


def test_tucker_hosvd_recovers_exact_multilinear_rank_order4():
    p = synth.tucker_problem([9, 8, 7, 6], [3, 2, 2, 3], seed=6, noise=0.0)
    A = TO.hosvd(p.X, p.R)
    G = TO.core(p.X, A)
    normX = float(np.linalg.norm(p.X))
    assert TO.fitness(normX, G) > 1 - 1e-7
    np.testing.assert_allclose(TO.reconstruct(G, A), p.X, rtol=0, atol=1e-10 * normX)


def test_pp_tucker_als_tracks_hooi_order4():
    p = synth.tucker_problem([10, 9, 8, 7], [3, 2, 2, 2], seed=7, noise=0.05)
    A0 = TO.hosvd(p.X, p.R)
    _, kinds, fit = TO.pp_tucker_als(p.X, A0, 12, eps=0.3)
    A = [a.copy() for a in A0]
    normX = float(np.linalg.norm(p.X))
    als = []
    for _ in range(12):
        _, G = TO.als_sweep(p.X, A)
        als.append(TO.fitness(normX, G))
    assert "pp_approx" in kinds
    assert max(abs(a - b) for a, b in zip(fit, als)) < 1e-6
