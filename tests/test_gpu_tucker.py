"""GPU parity of Tucker-ALS (HOOI) and PP-Tucker-ALS (Algorithm 4), order 3,
float64, against the oracle fed with the same state; tolerance 1e-10 (the
subspace iteration converges to rounding on these spectrally separated
problems)."""
import numpy as np
import pytest
import torch

from oracle import tucker_oracle as TO
from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    cpals.lib()


def _setup(dims, ranks, seed, noise=0.05, init="hosvd"):
    p = synth.tucker_problem(dims, ranks, seed=seed, noise=noise)
    A0 = TO.hosvd(p.X, ranks) if init == "hosvd" else p.A0
    t = cpals.Tucker(dims, ranks)
    if init != "hosvd":
        t.set_iterations(100)                            # converged from a random start
    t.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    t.init_factors(A0)
    return p, A0, t


@pytest.mark.parametrize("dims,ranks,init", [([40, 36, 32], [4, 3, 5], "hosvd"),
                                             ([30, 50, 24], [6, 2, 3], "hosvd"),
                                             ([33, 29, 40], [5, 4, 3], "random")])
def test_tucker_als_sweeps(dims, ranks, init):
    p, A0, t = _setup(dims, ranks, seed=7, noise=0.05 if init == "hosvd" else 0.3, init=init)
    with t:
        normX = float(np.linalg.norm(p.X))
        for sweep in range(3):
            A = t.get_factors()
            f = t.als_sweep()
            _, G = TO.als_sweep(p.X, A)
            for n, (a, b) in enumerate(zip(t.get_factors(), A)):
                assert np.max(np.abs(a - b)) < 1e-10, (sweep, n, np.max(np.abs(a - b)))
            np.testing.assert_allclose(t.get_core(), G, rtol=0, atol=1e-9 * np.max(np.abs(G)))
            assert abs(f - TO.fitness(normX, G)) < 1e-10
        assert abs(t.fitness() - TO.fitness(normX, TO.core(p.X, t.get_factors()))) < 1e-10


def test_tucker_pp_sweeps():
    p, A0, t = _setup([36, 32, 28], [4, 4, 3], seed=8)
    with t:
        for _ in range(2):
            t.als_sweep()
        t.pp_build_operators()
        Ap = t.get_factors()
        ops, Mp = TO.pp_operators(p.X, Ap)
        A = [a.copy() for a in Ap]
        dA = [np.zeros_like(a) for a in Ap]
        normX = float(np.linalg.norm(p.X))
        for sweep in range(3):
            f = t.pp_sweep()
            G = TO.pp_sweep(ops, Mp, A, Ap, dA)
            for n, (a, b) in enumerate(zip(t.get_factors(), A)):
                assert np.max(np.abs(a - b)) < 1e-10, (sweep, n, np.max(np.abs(a - b)))
            assert abs(f - TO.fitness(normX, G)) < 1e-10


def test_tucker_run_matches_oracle():
    # random orthonormal start, 0.3 relative noise: ALS sweeps until every
    # ||dA|| < 0.3 ||A||, then PP-init and PP-approx sweeps (Algorithm 4)
    p = synth.tucker_problem([32, 30, 28], [3, 3, 2], seed=9, noise=0.3)
    A_ref, kinds, fit = TO.pp_tucker_als(p.X, p.A0, 16, eps=0.3)
    assert kinds[0] == "als" and "pp_init" in kinds and "pp_approx" in kinds
    with cpals.Tucker([32, 30, 28], [3, 3, 2]) as t:
        t.set_iterations(100)                            # eigen ratio up to 0.65 in sweep 1
        t.set_tensor(np.ascontiguousarray(p.X))
        t.init_factors(p.A0)
        out = t.run(16, 0.3)
        assert out["kinds"] == kinds
        for k, (f, fr) in enumerate(zip(out["fitness"], fit)):
            if kinds[k] == "als":
                assert abs(f - fr) < 1e-10, k
        for a, b in zip(t.get_factors(), A_ref):
            assert np.max(np.abs(a - b)) < 1e-9
        assert abs(t.fitness() - fit[-1]) < 1e-10


def test_tucker_errors():
    with pytest.raises(cpals.CPALSError):
        cpals.Tucker([10, 10, 10], [11, 2, 2])          # rank above the size
    with pytest.raises(cpals.CPALSError):
        cpals.Tucker([10, 10, 10], [2, 2, 49])          # rank above the cap
    p, A0, t = _setup([12, 10, 9], [2, 2, 2], seed=1)
    with t:
        with pytest.raises(cpals.CPALSError):
            t.pp_sweep()                                 # operators not built
        t.als_sweep()
        t.pp_build_operators()
        t.pp_sweep()


def test_tucker_full_size_sweeps():
    # the bench's tensor (400^3, ranks 20 = 0.05 s, 0.3 relative noise) from
    # the oracle's HOSVD, default subspace-iteration count: two ALS sweeps,
    # then an operator build and a PP sweep, against the oracle
    dims, ranks = [400] * 3, [20] * 3
    p = synth.tucker_problem(dims, ranks, seed=0, noise=0.3)
    A0 = TO.hosvd(p.X, ranks)
    normX = float(np.linalg.norm(p.X))
    A = [a.copy() for a in A0]
    with cpals.Tucker(dims, ranks) as t:
        t.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
        t.init_factors(A0)
        for _ in range(2):
            f = t.als_sweep()
            _, G = TO.als_sweep(p.X, A)
            assert abs(f - TO.fitness(normX, G)) < 1e-10
        for a, b in zip(t.get_factors(), A):
            assert np.max(np.abs(a - b)) < 1e-9
        t.pp_build_operators()
        ops, Mp = TO.pp_operators(p.X, A)
        Ap = [a.copy() for a in A]
        dA = [np.zeros_like(a) for a in A]
        f = t.pp_sweep()
        G = TO.pp_sweep(ops, Mp, A, Ap, dA)
        assert abs(f - TO.fitness(normX, G)) < 1e-10
        for a, b in zip(t.get_factors(), A):
            assert np.max(np.abs(a - b)) < 1e-9


@pytest.mark.parametrize("dims,ranks", [([40, 32, 48], [4, 3, 5]), ([64, 56, 40], [6, 5, 4])])
def test_tucker_mixed_precision(dims, ranks):
    # first-level TTMs on the tensor cores (X in bf16, factor hi + lo): ALS
    # sweeps, the operators and a PP sweep against the float64 oracle at the
    # bf16 tolerance of the CP path (2e-2 on factors), fitness to 5e-3
    p = synth.tucker_problem(dims, ranks, seed=11, noise=0.05)
    A0 = TO.hosvd(p.X, ranks)
    normX = float(np.linalg.norm(p.X))
    with cpals.Tucker(dims, ranks, "mixed") as t:
        t.set_tensor(np.ascontiguousarray(p.X))
        t.init_factors(A0)
        A = [a.copy() for a in A0]
        for _ in range(2):
            f = t.als_sweep()
            _, G = TO.als_sweep(p.X, A)
            assert abs(f - TO.fitness(normX, G)) < 5e-3
        for a, b in zip(t.get_factors(), A):
            assert np.max(np.abs(a - b)) < 2e-2 * np.max(np.abs(b))
        t.pp_build_operators()
        A = t.get_factors()
        ops, Mp = TO.pp_operators(p.X, A)
        Ap = [a.copy() for a in A]
        dA = [np.zeros_like(a) for a in A]
        f = t.pp_sweep()
        G = TO.pp_sweep(ops, Mp, A, Ap, dA)
        assert abs(f - TO.fitness(normX, G)) < 5e-3
        for a, b in zip(t.get_factors(), A):
            assert np.max(np.abs(a - b)) < 2e-2 * np.max(np.abs(b))
        assert abs(t.fitness() - TO.fitness(normX, TO.core(p.X, t.get_factors()))) < 5e-3


def test_tucker_mixed_unsupported_shape():
    with pytest.raises(cpals.CPALSError) as e:
        cpals.Tucker([12, 10, 9], [2, 2, 2], "mixed")    # s_3 = 9 is not a multiple of 8
    assert e.value.status == 8


def test_tucker_full_rank_is_exact():
    # R_n = s_n: the factors are orthogonal matrices, the core holds all of X
    # (||G|| = ||X||) and [[G; A]] reproduces X; which basis is returned is
    # not unique (noise-level eigenvalues may be close), so compare invariants
    dims = [8, 9, 10]
    p = synth.tucker_problem(dims, [3, 3, 3], seed=4, noise=0.05)
    A0 = TO.hosvd(p.X, dims)
    with cpals.Tucker(dims, dims) as t:
        t.set_tensor(np.ascontiguousarray(p.X))
        t.init_factors(A0)
        f = t.als_sweep()
        A = t.get_factors()
        G = t.get_core()
    assert f > 1.0 - 1e-6
    for a in A:
        assert np.max(np.abs(a.T @ a - np.eye(a.shape[1]))) < 1e-12
    Xr = TO.reconstruct(G, A)
    assert np.max(np.abs(Xr - p.X)) < 1e-10 * np.max(np.abs(p.X))


@pytest.mark.parametrize("dims,ranks", [([16, 24, 8], [1, 1, 1]), ([56, 48, 64], [48, 40, 48])])
def test_tucker_rank_extremes(dims, ranks):
    # rank 1 (one Jacobi slot and a dummy) and the largest supported rank
    p, A0, t = _setup(dims, ranks, seed=5)
    with t:
        normX = float(np.linalg.norm(p.X))
        A = [a.copy() for a in A0]
        for _ in range(2):
            f = t.als_sweep()
            _, G = TO.als_sweep(p.X, A)
            assert abs(f - TO.fitness(normX, G)) < 1e-10
        for a, b in zip(t.get_factors(), A):
            assert np.max(np.abs(a - b)) < 1e-9
        np.testing.assert_allclose(t.get_core(), G, rtol=0, atol=1e-9 * np.max(np.abs(G)))


ORDER_N = [([20, 18, 16, 14], [3, 3, 2, 2]), ([10, 9, 8, 7, 6], [2, 3, 2, 2, 2])]


@pytest.mark.parametrize("dims,ranks", ORDER_N, ids=["order4", "order5"])
def test_tucker_order_n_als_and_pp_sweeps(dims, ranks):
    """Orders 4 and 5 (the generic contraction chains): HOOI sweeps, then an
    operator build and PP sweeps (Sec. 3.2.2), each against the oracle fed
    with the same state: factors within 1e-10, the core within 1e-9 of its
    largest entry, fitness within 1e-10."""
    p, A0, t = _setup(dims, ranks, seed=11)
    with t:
        normX = float(np.linalg.norm(p.X))
        for sweep in range(2):
            A = t.get_factors()
            f = t.als_sweep()
            _, G = TO.als_sweep(p.X, A)
            for n, (a, b) in enumerate(zip(t.get_factors(), A)):
                assert np.max(np.abs(a - b)) < 1e-10, (sweep, n)
            np.testing.assert_allclose(t.get_core(), G, rtol=0, atol=1e-9 * np.max(np.abs(G)))
            assert abs(f - TO.fitness(normX, G)) < 1e-10
        t.pp_build_operators()
        Ap = t.get_factors()
        ops, Mp = TO.pp_operators(p.X, Ap)
        A = [a.copy() for a in Ap]
        dA = [np.zeros_like(a) for a in Ap]
        for sweep in range(3):
            f = t.pp_sweep()
            G = TO.pp_sweep(ops, Mp, A, Ap, dA)
            for n, (a, b) in enumerate(zip(t.get_factors(), A)):
                assert np.max(np.abs(a - b)) < 1e-10, (sweep, n)
            np.testing.assert_allclose(t.get_core(), G, rtol=0, atol=1e-9 * np.max(np.abs(G)))
            assert abs(f - TO.fitness(normX, G)) < 1e-10
        assert abs(t.fitness() - TO.fitness(normX, TO.core(p.X, t.get_factors()))) < 1e-10


def test_tucker_order4_run_matches_oracle():
    """Algorithm 4 at order 4 from a random orthonormal start: the same sweep
    kinds as the oracle's, the exact fitness after every ALS sweep within
    1e-10 and the final factors within 1e-9."""
    dims, ranks = [24, 20, 18, 16], [3, 2, 2, 2]
    p = synth.tucker_problem(dims, ranks, seed=12, noise=0.3)
    A_ref, kinds, fit = TO.pp_tucker_als(p.X, p.A0, 14, eps=0.3)
    assert kinds[0] == "als" and "pp_approx" in kinds
    with cpals.Tucker(dims, ranks) as t:
        t.set_iterations(100)
        t.set_tensor(np.ascontiguousarray(p.X))
        t.init_factors(p.A0)
        out = t.run(14, 0.3)
        assert out["kinds"] == kinds
        for k, (f, fr) in enumerate(zip(out["fitness"], fit)):
            if kinds[k] == "als":
                assert abs(f - fr) < 1e-10, k
        for a, b in zip(t.get_factors(), A_ref):
            assert np.max(np.abs(a - b)) < 1e-9
        assert abs(t.fitness() - fit[-1]) < 1e-10


def test_tucker_order4_mixed_unsupported():
    with cpals.Tucker([16, 16, 16, 16], [2, 2, 2, 2]) as t:
        with pytest.raises(cpals.CPALSError) as e:
            t._ck(cpals.cpals_tucker_set_precision(t.t, cpals.PRECISIONS["mixed"]))
        assert e.value.status == 8
