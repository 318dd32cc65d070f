"""GPU parity of the ALS variants of Sec. 5.1 (update step size; symmetric
decomposition [[A, B, B]] with the B step 0.8) against the FP64 oracle, for
ALS sweeps, PP sweeps and whole Algorithm 3 runs, in every precision.
Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5, "mixed": 2e-2}
SYM_LAM = [1.0, 0.8, 1.0]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    cpals.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _ctx(p, prec, lam=None, tie=False):
    g = cpals.CPALS(p.dims, p.R, prec)
    g.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    if tie:
        g.set_symmetric(1, 2)
    if lam is not None:
        g.set_step_size(lam)
    g.init_factors(p.A0)
    return g


def X64(p):
    return np.asarray(p.X, dtype=np.float64)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("dims,R", [([40, 33, 27], 9), ([11, 13, 9, 10], 6)])
def test_step_size_als_and_pp_sweeps(dims, R, prec):
    """Three ALS sweeps then a PP initialisation and two approximated sweeps
    with step sizes 0.7 (and per-mode values), factor by factor against the
    oracle fed with the same state (precision-level tolerance)."""
    p = synth.make_problem("normal", dims, R, seed=5, storage="f64" if prec == "fp64" else "f32")
    lam = [0.7] * len(dims) if len(dims) == 3 else [0.6, 0.9, 1.0, 0.75]
    X = X64(p)
    with _ctx(p, prec, lam) as g:
        for sweep in range(3):
            A = g.get_factors()             # each sweep from the GPU's state
            S = [O.gram(a) for a in A]
            g.als_sweep()
            O.als_sweep(X, A, S, lam=lam)
            for n, (a, b) in enumerate(zip(g.get_factors(), A)):
                assert rel(a, b) < TOL[prec], (sweep, n, rel(a, b))
        g.pp_build_operators()
        Ap = g.get_factors()
        ops, Mp = O.pp_operators(X, Ap)
        for sweep in range(2):
            A = g.get_factors()
            dA = [g.get_state("dA", n) for n in range(len(dims))]
            S = [O.gram(a) for a in A]
            g.pp_sweep(use_V=True)
            O.pp_sweep(ops, Mp, A, Ap, dA, S, True, lam=lam)
            for n, (a, b) in enumerate(zip(g.get_factors(), A)):
                assert rel(a, b) < TOL[prec], ("pp", sweep, n, rel(a, b))


def test_step_size_run_fp64():
    """Algorithm 3 with step size 0.7 end to end: the same sweep kinds as the
    oracle and the exact fitness of every ALS sweep within 1e-10."""
    p = synth.make_problem("normal", [36, 30, 28], 6, seed=8, noise=1e-2, storage="f64")
    A_ref, tr = O.pp_cp_als(p.X, p.A0, 40, 0.2, use_V=True, lam=0.7)
    assert "pp_approx" in tr.kinds
    with _ctx(p, "fp64", 0.7) as g:
        out = g.run(40, 0.2, use_V=True)
        assert out["kinds"] == tr.kinds
        for k, (f, fr) in enumerate(zip(out["fitness"], tr.fitness)):
            if out["kinds"][k] == "als":
                assert abs(f - fr) < 1e-10, k
        for a, b in zip(g.get_factors(), A_ref):
            assert rel(a, b) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_symmetric_sweeps(prec):
    """[[A, B, B]] with the B step 0.8: ALS sweeps then PP sweeps against the
    oracle; modes 1 and 2 hold bit-identical factors throughout."""
    p = synth.symmetric_order3(44, 30, 7, seed=3, storage="f64" if prec == "fp64" else "f32")
    X = X64(p)
    tie = {2: 1}
    with _ctx(p, prec, SYM_LAM, tie=True) as g:
        A0 = g.get_factors()
        np.testing.assert_array_equal(A0[1], A0[2])
        np.testing.assert_array_equal(A0[2], p.A0[1])
        for sweep in range(3):
            A = g.get_factors()
            S = [O.gram(a) for a in A]
            g.als_sweep()
            O.als_sweep(X, A, S, lam=SYM_LAM, tie=tie)
            Ag = g.get_factors()
            np.testing.assert_array_equal(Ag[1], Ag[2])
            for n, (a, b) in enumerate(zip(Ag, A)):
                assert rel(a, b) < TOL[prec], (sweep, n, rel(a, b))
        g.pp_build_operators()
        Ap = g.get_factors()
        ops, Mp = O.pp_operators(X, Ap)
        for sweep in range(3):
            A = g.get_factors()
            dA = [g.get_state("dA", n) for n in range(3)]
            S = [O.gram(a) for a in A]
            g.pp_sweep(use_V=True)
            O.pp_sweep(ops, Mp, A, Ap, dA, S, True, lam=SYM_LAM, tie=tie)
            Ag = g.get_factors()
            np.testing.assert_array_equal(Ag[1], Ag[2])
            np.testing.assert_array_equal(g.get_state("dA", 1), g.get_state("dA", 2))
            for n, (a, b) in enumerate(zip(Ag, A)):
                assert rel(a, b) < TOL[prec], ("pp", sweep, n, rel(a, b))


def test_symmetric_run_fp64_and_exact_fitness():
    """Symmetric PP-ALS end to end against the oracle (sweep kinds, exact
    fitness of ALS sweeps, final factors); the exact fitness also matches the
    explicit reconstruction."""
    p = synth.symmetric_order3(40, 26, 6, seed=12, storage="f64")
    A_ref, tr = O.pp_cp_als(p.X, p.A0, 40, 0.2, use_V=True, lam=SYM_LAM, tie={2: 1})
    assert "pp_approx" in tr.kinds
    with _ctx(p, "fp64", SYM_LAM, tie=True) as g:
        out = g.run(40, 0.2, use_V=True)
        assert out["kinds"] == tr.kinds
        for k, (f, fr) in enumerate(zip(out["fitness"], tr.fitness)):
            if out["kinds"][k] == "als":
                assert abs(f - fr) < 1e-10, k
        A = g.get_factors()
        for a, b in zip(A, A_ref):
            assert rel(a, b) < 1e-8
        assert abs(g.fitness() - O.fitness_explicit(p.X, A)) < 1e-10


def test_variant_argument_errors():
    p = synth.make_problem("normal", [12, 10, 10], 3, seed=1, storage="f64")
    with _ctx(p, "fp64") as g:
        for bad in ([0.0, 1.0, 1.0], [1.0, 2.5, 1.0], [1.0, np.nan, 1.0]):
            with pytest.raises(cpals.CPALSError):
                g.set_step_size(bad)
        with pytest.raises(cpals.CPALSError):
            g.set_symmetric(0, 1)             # sizes 12 and 10
        with pytest.raises(cpals.CPALSError):
            g.set_symmetric(2, 1)             # m2 < m1
        g.set_symmetric(1, 2)
        with pytest.raises(cpals.CPALSError):
            g.als_sweep()                     # the tie dropped the factors
        g.init_factors(p.A0)
        g.als_sweep()
        A = g.get_factors()
        np.testing.assert_array_equal(A[1], A[2])
        g.set_symmetric(-1, -1)
        g.init_factors(p.A0)
        g.als_sweep()
        A = g.get_factors()
        assert not np.array_equal(A[1], A[2])
