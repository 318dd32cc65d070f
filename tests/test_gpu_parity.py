"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances:
* FP64 mode: 1e-10 relative for factors, MTTKRP, operators; fitness within
  1e-10 absolute (the spec bar is 1e-10 relative for factors and
  fitness in FP64).
* FP32 mode: relative error of a length-K float32 dot product with float32
  inputs is below ~K * 2^-24 in the worst case and ~sqrt(K) * 2^-24 typically;
  the tests allow 2e-5 (small K) relative to max|ref|.
* MIXED_BF16 against the float64 oracle: X and the B operand are rounded to
  bf16 (relative 2^-9 each), so a product carries up to ~2^-8 and a sum of
  mixed-sign terms up to ~1e-2 relative to max|ref|; the tests allow 2e-2.
  (tests/test_gpu_umma.py checks the tensor-core kernel itself at 2e-5 on
  bf16-rounded inputs.)
"""
import numpy as np
import pytest
import torch

from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5, "mixed": 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    cpals.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def X64(p):
    return np.asarray(p.X, dtype=np.float64)


SHAPES = [([70, 45, 33], 10), ([33, 70, 45], 17), ([13, 17, 11, 9], 7), ([7, 6, 5, 8, 9], 5),
          ([9, 8, 7, 6, 5, 4], 3), ([130, 65, 40], 100), ([24, 24, 24], 1)]


def _ctx(p, prec):
    g = cpals.CPALS(p.dims, p.R, prec)
    g.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    g.init_factors(p.A0)
    return g


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("dims,R", SHAPES)
def test_mttkrp(dims, R, prec):
    storage = "f64" if prec == "fp64" else "f32"
    p = synth.make_problem("normal", dims, R, seed=3, storage=storage)
    with _ctx(p, prec) as g:
        for n in range(len(dims)):
            ref = O.mttkrp(X64(p), p.A0, n)
            assert rel(g.mttkrp(n), ref) < TOL[prec], (n, prec)


# float32 contractions with R > 32: 128-row tiles of 8 ceil(R/8) columns with
# 16-byte X loads when the contiguous dimension (K for the K-major launch, M
# for the other) is a multiple of 4, else the generic kernel; ragged row
# tiles, K not a multiple of the 16-deep slab, split K, TN = 5 to 16
WIDE = [([132, 36, 20], 33), ([20, 36, 132], 64), ([52, 44, 28], 128), ([36, 44, 130], 100),
        ([33, 35, 36], 40), ([9, 7, 2000], 100)]


@pytest.mark.parametrize("dims,R", WIDE)
def test_mttkrp_fp32_wide_rank(dims, R):
    p = synth.make_problem("normal", dims, R, seed=8, storage="f32")
    with _ctx(p, "fp32") as g:
        for n in range(len(dims)):
            ref = O.mttkrp(X64(p), p.A0, n)
            assert rel(g.mttkrp(n), ref) < TOL["fp32"], n


# float64 contractions with R = 4 (mod 8) above 64 (exact R-column tiles), and
# K-major launches whose 64-row tiles fill whole waves and part of another
# (40,000 and 32,300 rows): the last wave's rows run as a second launch with
# K split in two; the same 40,000-row shape on the float32 kernel (one launch)
TAIL = [([200, 200, 40], 100, "fp64"), ([190, 170, 48], 92, "fp64"), ([64, 48, 40], 68, "fp64"),
        ([200, 200, 40], 100, "fp32")]


@pytest.mark.parametrize("dims,R,prec", TAIL)
def test_mttkrp_exact_tiles_and_tail_split(dims, R, prec):
    p = synth.make_problem("normal", dims, R, seed=9, storage="f64" if prec == "fp64" else "f32")
    with _ctx(p, prec) as g:
        for n in range(len(dims)):
            ref = O.mttkrp(X64(p), p.A0, n)
            assert rel(g.mttkrp(n), ref) < TOL[prec], n


# the largest order (8), order 7, and modes of size 1 (degenerate unfoldings)
EDGE = [([3, 2, 4, 2, 3, 2, 2], 3), ([2, 3, 2, 2, 3, 2, 2, 3], 2), ([1, 9, 7], 4), ([8, 1, 6, 5], 3)]


@pytest.mark.parametrize("dims,R", [([40, 33, 27], 9), ([11, 13, 9, 10], 6), ([6, 7, 5, 6, 4], 4)] + EDGE)
def test_als_sweeps_fp64(dims, R):
    p = synth.make_problem("normal", dims, R, seed=5, storage="f64")
    A = [a.copy() for a in p.A0]
    S = [O.gram(a) for a in A]
    with _ctx(p, "fp64") as g:
        for sweep in range(4):
            f = g.als_sweep()
            dA_ref, _ = O.als_sweep(p.X, A, S)
            assert abs(f - O.fitness(p.X, A)) < 1e-10
            for a, b in zip(g.get_factors(), A):
                assert rel(a, b) < 1e-10, sweep
            ratios = g.get_dA_ratios()
            want = [np.linalg.norm(d) / np.linalg.norm(a) for d, a in zip(dA_ref, A)]
            # a mode of size 1 settles after one sweep: its ratio is then
            # rounding noise (~1e-16), compared absolutely
            np.testing.assert_allclose(ratios, want, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,R", [([40, 33, 27], 9), ([11, 13, 9, 10], 6), ([6, 7, 5, 6, 4], 4),
                                    ([5, 6, 4, 5, 3, 4], 3)])
def test_pp_operators(dims, R, prec):
    _check_operators(dims, R, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_pp_operators_short_modes_large(prec):
    """Order 5 with short modes: the operator tree's level-3 node (0, 3) has
    7.1 M entries and contracts a mode of 12, which takes the
    thread-per-output TTV (float64 scalar; float 16-byte with R % 4 = 0);
    in mixed precision the single-mode contractions of X (K = 12 and 48)
    run on the SIMT float32 kernels."""
    _check_operators([48, 12, 12, 48, 48], 64, prec)


def _check_operators(dims, R, prec):
    storage = "f64" if prec == "fp64" else "f32"
    p = synth.make_problem("normal", dims, R, seed=7, storage=storage)
    with _ctx(p, prec) as g:
        g.als_sweep()
        A = g.get_factors()
        g.pp_build_operators()
        ops, Mp = O.pp_operators(X64(p), A)
        N = len(dims)
        for i in range(N):
            for n in range(i + 1, N):
                assert rel(g.get_operator(i, n), ops[(i, n)]) < TOL[prec], (i, n)
            assert rel(g.get_operator(i, i), Mp[i]) < TOL[prec], i
        for n in range(N):
            np.testing.assert_array_equal(g.get_state("Ap", n), A[n])
            assert not np.any(g.get_state("dA", n))


def _dA_close(got, want, A):
    """dA agrees to 1e-9 relative, or to rounding (1e-13 of the factor) when
    the reference itself is rounding noise (a settled mode)."""
    return rel(got, want) < 1e-9 or np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(A))


@pytest.mark.parametrize("dims,R", [([40, 33, 27], 9), ([11, 13, 9, 10], 6), ([6, 7, 5, 6, 4], 4)])
def test_pp_sweeps_fp64(dims, R):
    """Algorithm 3's PP sweeps (with and without V) against the oracle, and the
    approximated right-hand sides of Eq. 3 for the state the GPU holds."""
    p = synth.make_problem("normal", dims, R, seed=9, storage="f64")
    with _ctx(p, "fp64") as g:
        for _ in range(2):
            g.als_sweep()
        A = g.get_factors()
        S = [O.gram(a) for a in A]
        g.pp_build_operators()
        Ap = [a.copy() for a in A]
        ops, Mp = O.pp_operators(p.X, Ap)
        dA = [np.zeros_like(a) for a in A]
        for sweep, useV in enumerate([True, False, True]):
            g.pp_sweep(use_V=useV)
            O.pp_sweep(ops, Mp, A, Ap, dA, S, useV)
            for n, (a, b) in enumerate(zip(g.get_factors(), A)):
                assert rel(a, b) < 1e-10, (sweep, n)
                assert _dA_close(g.get_state("dA", n), dA[n], A[n]), (sweep, n)
        A_g = g.get_factors()
        dA_g = [g.get_state("dA", n) for n in range(len(dims))]
        for n in range(len(dims)):
            for useV in (False, True):
                ref = O.pp_mttkrp(ops, Mp, A_g, dA_g, n, useV)
                assert rel(g.pp_mttkrp(n, useV), ref) < 1e-10, (n, useV)


@pytest.mark.parametrize("dims,R", EDGE)
def test_pp_sweep_edge_shapes_fp64(dims, R):
    """Orders 7 and 8 and modes of size 1: one PP sweep against the oracle,
    then the approximated right-hand sides (Eq. 3, with and without V) on the
    state the GPU holds.  Only one sweep: on these tiny tensors the PP
    iteration itself amplifies a 1e-15 perturbation of the factors to 1e-8
    within two sweeps (measured in the oracle), so later sweeps compare
    rounding paths, not the method."""
    p = synth.make_problem("normal", dims, R, seed=9, storage="f64")
    with _ctx(p, "fp64") as g:
        for _ in range(2):
            g.als_sweep()
        A = g.get_factors()
        S = [O.gram(a) for a in A]
        g.pp_build_operators()
        Ap = [a.copy() for a in A]
        ops, Mp = O.pp_operators(p.X, Ap)
        dA = [np.zeros_like(a) for a in A]
        g.pp_sweep(use_V=True)
        O.pp_sweep(ops, Mp, A, Ap, dA, S, True)
        for n, (a, b) in enumerate(zip(g.get_factors(), A)):
            assert rel(a, b) < 1e-10, n
            assert _dA_close(g.get_state("dA", n), dA[n], A[n]), n
        A_g = g.get_factors()
        dA_g = [g.get_state("dA", n) for n in range(len(dims))]
        for n in range(len(dims)):
            for useV in (False, True):
                ref = O.pp_mttkrp(ops, Mp, A_g, dA_g, n, useV)
                assert rel(g.pp_mttkrp(n, useV), ref) < 1e-10, (n, useV)


def test_fitness_exact_fp64():
    p = synth.make_problem("normal", [30, 20, 25], 5, seed=11, storage="f64")
    with _ctx(p, "fp64") as g:
        g.als_sweep()
        g.pp_build_operators()
        g.pp_sweep()
        f = g.fitness()
        A = g.get_factors()
        assert abs(f - O.fitness_explicit(p.X, A)) < 1e-10


def test_order3_60_rank10_run_fp64():
    """The 60^3 rank-10 FP64 workload end to end (Algorithm 3, eps = 0.2,
    50 sweeps): same sweep kinds as the oracle, fitness within 1e-10 for
    every sweep, final factors within 1e-8 relative."""
    p = synth.order3_60_rank10(seed=0)
    A_ref, tr = O.pp_cp_als(p.X, p.A0, p.sweeps, p.eps, use_V=True)
    with _ctx(p, "fp64") as g:
        out = g.run(p.sweeps, p.eps, use_V=True)
        assert out["kinds"] == tr.kinds
        assert g.pinv_modes() == 0                 # every Gamma positive definite
        # the GPU reports the exact fitness after ALS sweeps and the estimate
        # from M~^(N) after PP sweeps, as the oracle's trace of what the
        # algorithm sees does
        for k, (f, fr) in enumerate(zip(out["fitness"], tr.seen)):
            assert abs(f - fr) < 1e-10, (k, out["kinds"][k])
        assert abs(g.fitness() - tr.fitness[-1]) < 1e-10
        for a, b in zip(g.get_factors(), A_ref):
            assert rel(a, b) < 1e-8


def _zero_column_problem(R=5, col=2, seed=14, storage="f64"):
    p = synth.make_problem("normal", [12, 10, 9], R, seed=seed, storage=storage)
    A0 = [a.copy() for a in p.A0]
    A0[1][:, col] = 0.0
    return p, A0


def test_normal_solve_pinv_fp64():
    """Gamma^(0) with a zero row and column (zero column in A^(1)): the
    float64 path solves with Gamma^dagger (Algorithm 1) like the oracle's
    eigen pseudo-inverse fallback, for a consistent and an arbitrary
    right-hand side."""
    p, A0 = _zero_column_problem()
    g_ = np.random.default_rng(40)
    with cpals.CPALS(p.dims, p.R, "fp64") as g:
        g.set_tensor(p.X)
        g.init_factors(A0)
        S = [O.gram(a) for a in A0]
        G = O.gamma(S, 0)
        for rhs in (g_.standard_normal((p.dims[0], p.R)) @ G, g_.standard_normal((p.dims[0], p.R))):
            info = O.SolveInfo()
            ref = O.solve_normal(rhs, G, info)
            assert info.singular
            assert rel(g.normal_solve(0, rhs), ref) < 1e-11
            assert g.pinv_modes() & 1


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_normal_solve_pinv_double_float(prec):
    """The double-float normal equations of FP32/mixed contexts take the same
    Gamma^dagger fallback (Algorithm 1): a float64 Jacobi eigendecomposition
    of Gamma and the factor diag(w^+)^(1/2) V^T in double-float, applied as
    W^T W.  Against the oracle's eigen pseudo-inverse of the float-rounded
    right-hand side (the solve takes it in float), consistent and
    arbitrary."""
    p, A0 = _zero_column_problem(storage="f32")
    g_ = np.random.default_rng(41)
    with cpals.CPALS(p.dims, p.R, prec) as g:
        g.set_tensor(p.X)
        g.init_factors(A0)
        S = [O.gram(a) for a in A0]
        G = O.gamma(S, 0)
        for rhs in (g_.standard_normal((p.dims[0], p.R)) @ G, g_.standard_normal((p.dims[0], p.R))):
            rhs = rhs.astype(np.float32).astype(np.float64)
            info = O.SolveInfo()
            ref = O.solve_normal(rhs, G, info)
            assert info.singular
            assert rel(g.normal_solve(0, rhs), ref) < 1e-10
            assert g.pinv_modes() & 1


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("eps", [0.0, 0.2])
def test_run_with_singular_gamma_double_float_equals_lower_rank(prec, eps):
    """The double-float counterpart of the float64 run below: a zero column in
    every initial factor keeps every Gamma^(n) singular, the solves go
    through Gamma^dagger every mode, and the run equals the same context's
    rank R - 1 run without that column, with the column exactly zero
    throughout.  The contractions give the same columns; the solve's factor
    differs (double-float rounding, which can move a float compute copy by
    one unit) and the fitness sums R float terms in another order, so the
    two agree to float rounding: 1e-6 on the fitness, 1e-5 on the factors.
    The rank R - 1 run itself tracks the oracle within the contraction
    tolerance."""
    R, col = 5, 2
    p = synth.make_problem("normal", [12, 10, 9], R, seed=14, storage="f32")
    A0 = [a.copy() for a in p.A0]
    for a in A0:
        a[:, col] = 0.0
    keep = [r for r in range(R) if r != col]
    n = 12
    res = {}
    for rank, facs in ((R, A0), (R - 1, [a[:, keep] for a in A0])):
        with cpals.CPALS(p.dims, rank, prec) as g:
            g.set_tensor(p.X)
            g.init_factors(facs)
            out = g.run(n, eps, True, 0.0)
            assert g.pinv_modes() == (7 if rank == R else 0)
            res[rank] = (out, g.get_factors(), g.fitness())
    (o5, A5, f5), (o4, A4, f4) = res[R], res[R - 1]
    assert o5["kinds"] == o4["kinds"]
    np.testing.assert_allclose(o5["fitness"], o4["fitness"], rtol=0, atol=1e-6)
    assert abs(f5 - f4) < 1e-6
    for a, b in zip(A5, A4):
        assert np.all(a[:, col] == 0.0)
        assert rel(a[:, keep], b) < 1e-5
    if eps > 0:
        assert "pp_approx" in o5["kinds"]
    A_or, tr = O.pp_cp_als(X64(p), [a[:, keep] for a in A0], n, 0.0, use_V=True)
    if eps == 0.0:
        np.testing.assert_allclose(o4["fitness"], tr.seen, rtol=0, atol=50 * TOL[prec])


@pytest.mark.parametrize("eps", [0.0, 0.2])
def test_run_with_singular_gamma_fp64_equals_lower_rank(eps):
    """A zero column in every initial factor keeps every Gamma^(n) singular
    (a zero row and column) for the whole run; the float64 path then solves
    through Gamma^dagger every mode.  In exact arithmetic the run is the
    rank R - 1 decomposition without that column (its Gamma is the reduced
    Gamma, its MTTKRP columns the reduced ones), so ALS (eps 0) and PP-ALS
    (eps 0.2, second-order terms) must follow the oracle's rank R - 1 run
    sweep for sweep, with the column exactly zero throughout."""
    R, col = 5, 2
    p = synth.make_problem("normal", [12, 10, 9], R, seed=14, storage="f64")
    A0 = [a.copy() for a in p.A0]
    for a in A0:
        a[:, col] = 0.0
    keep = [r for r in range(R) if r != col]
    n = 12
    A_or, tr = O.pp_cp_als(p.X, [a[:, keep] for a in A0], n, eps, use_V=True)
    with cpals.CPALS(p.dims, R, "fp64") as g:
        g.set_tensor(p.X)
        g.init_factors(A0)
        out = g.run(n, eps, True, 0.0)
        assert g.pinv_modes() == 7
        A = g.get_factors()
        f = g.fitness()
    assert out["kinds"] == tr.kinds
    np.testing.assert_allclose(out["fitness"], tr.seen, rtol=0, atol=1e-10)
    assert abs(f - tr.fitness[-1]) < 1e-10
    for a, b in zip(A, A_or):
        assert np.all(a[:, col] == 0.0)
        assert rel(a[:, keep], b) < 1e-8
    if eps > 0:
        assert "pp_approx" in out["kinds"]


def test_call_order_errors():
    with cpals.CPALS([5, 6, 7], 2, "fp64") as g:
        with pytest.raises(cpals.CPALSError) as e:
            g.als_sweep()
        assert e.value.status == 4
        g.set_tensor(np.ones((5, 6, 7)))
        g.init_factors([np.ones((s, 2)) + np.arange(2) for s in (5, 6, 7)])
        with pytest.raises(cpals.CPALSError) as e:
            g.pp_sweep()
        assert e.value.status == 4


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_full_size_order3_400_sampled(prec):
    """400^3 rank 100 (FP32 storage), the launch configuration the benchmark
    times: sampled MTTKRP rows of every mode against the oracle row by row,
    then one ALS sweep's fitness against the oracle's formula."""
    p = synth.order3_400_rank100(seed=0)
    X = p.X
    rng = np.random.default_rng(0)
    with _ctx(p, prec) as g:
        for n in range(3):
            M = g.mttkrp(n)
            for y in rng.choice(p.dims[n], 4, replace=False):
                sub = np.take(X, [y], axis=n).astype(np.float64)
                A = [a if k != n else a[y:y + 1] for k, a in enumerate(p.A0)]
                ref = O.mttkrp(sub, A, n)[0]
                assert rel(M[y], ref) < (1e-4 if prec == "fp32" else 1e-2), (n, y)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("dims,R", [([40, 33, 27], 9), ([130, 120, 110], 100), ([11, 13, 9, 10], 6)])
def test_normal_solve(dims, R, prec):
    """Grams, Gamma^(n), its Cholesky factor and the row solves (Sec. 2.3)
    against the oracle's float64 solve for the Grams of the GPU's factors.
    float64 mode: IEEE float64; FP32/mixed: double-float (48-bit) kernels,
    which take the right-hand side in float (the contractions' precision),
    so the oracle solves the float-rounded right-hand side.  Both within
    1e-11 relative at these condition numbers."""
    storage = "f64" if prec == "fp64" else "f32"
    p = synth.make_problem("normal", dims, R, seed=31, storage=storage, init="normal")
    g_ = np.random.default_rng(32)
    with _ctx(p, prec) as g:
        g.als_sweep()
        A = g.get_factors()
        S = [O.gram(a) for a in A]
        for n in range(len(dims)):
            G = O.gamma(S, n)
            rhs = g_.standard_normal((dims[n], R)) @ G
            if prec != "fp64":
                rhs = rhs.astype(np.float32).astype(np.float64)
            ref = O.solve_normal(rhs, G)
            assert np.linalg.cond(G) < 1e6
            assert rel(g.normal_solve(n, rhs), ref) < 1e-11, (n, prec)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_normal_arith_fp64_and_double_float_agree(prec):
    """FP32/mixed contexts run the normal-equation work (Sec. 2.3) in
    double-float by default and in IEEE float64 on request.  The first mode
    update sees identical inputs in both (the same float right-hand side and
    Grams of the same factors), so the two agree within the double-float
    rounding amplified by the conditioning (1e-10); later updates see
    float compute copies that may differ in the last bit, so after ALS and
    PP sweeps they agree within the contraction tolerance.  The float64
    variant matches the float64 oracle sweep within that tolerance too.  An
    FP64 context refuses double-float."""
    p = synth.make_problem("normal", [40, 33, 27], 9, seed=5, storage="f32")
    out = {}
    for arith in ["double_float", "fp64"]:
        with _ctx(p, prec) as g:
            g.set_normal_arith(arith)
            with pytest.raises(cpals.CPALSError):
                g.als_sweep()                      # factors were dropped
            g.init_factors(p.A0)
            g.als_sweep()
            first = g.get_factors()
            for _ in range(2):
                g.als_sweep()
            g.pp_build_operators()
            g.pp_sweep(True)
            out[arith] = (first, g.get_factors())
    assert rel(out["fp64"][0][0], out["double_float"][0][0]) < 1e-10
    for a, b in zip(out["fp64"][1], out["double_float"][1]):
        assert rel(a, b) < TOL[prec]
    A = [a.copy() for a in p.A0]
    S = [O.gram(a) for a in A]
    O.als_sweep(X64(p), A, S)
    for a, b in zip(out["fp64"][0], A):
        assert rel(a, b) < 5 * TOL[prec]
    with cpals.CPALS(p.dims, p.R, "fp64") as g:
        with pytest.raises(cpals.CPALSError):
            g.set_normal_arith("double_float")


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("name", ["order4_120_rank64", "order6_24_rank50"])
def test_full_size_order4_order6_sampled(name, prec):
    """The 120^4 rank-64 and 24^6 rank-50 workloads (FP32 storage) at full
    size: sampled MTTKRP rows of every mode (Sec. 2.5 tree) and sampled
    entries of PP operators (Sec. 3.2.3 tree), each against the oracle's
    row-at-a-time contraction of the same slice."""
    p = getattr(synth, name)(seed=0)
    N = len(p.dims)
    tol = 1e-4 if prec == "fp32" else 1e-2
    rng = np.random.default_rng(2)
    with _ctx(p, prec) as g:
        for n in range(N):
            M = g.mttkrp(n)
            for y in rng.choice(p.dims[n], 2, replace=False):
                ref = O.partial_row(p.X, p.A0, {n: int(y)})
                assert rel(M[y], ref) < tol, (n, int(y))
        g.pp_build_operators()
        for i, n in [(0, 1), (0, N - 1), (N - 2, N - 1)]:
            op = g.get_operator(i, n)
            for _ in range(2):
                xi, xn = int(rng.integers(p.dims[i])), int(rng.integers(p.dims[n]))
                ref = O.partial_row(p.X, p.A0, {i: xi, n: xn})
                assert rel(op[xi, xn], ref) < tol, (i, n, xi, xn)
