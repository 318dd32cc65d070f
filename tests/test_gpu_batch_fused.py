"""Many small order-3 decompositions in one set of launches (cpals_batch_*)
against the FP64 oracle.

In float64 every instance must follow the oracle's Algorithm 3 (pp_cp_als)
sweep for sweep: the same sweep kinds, the fitness the algorithm sees after
every sweep (exact after ALS sweeps, the M~ estimate after PP sweeps) within
1e-10, the final factors within 1e-8 relative and the final exact fitness
within 1e-10 -- with and without the stopping test inside PP runs.  The
instances differ in every size and rank, so each stage launch covers
instances in different sweep kinds at once.  In float32 (the contractions,
operators and corrections; double-float normal equations) the final fitness
stays within 1e-4 of the float64 batch.  One sweep of the batch launches the same
number of kernels whatever the number of instances.
"""
import numpy as np
import pytest
import torch

from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu
SWEEPS, EPS = 30, 0.1


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def probs():
    return synth.batch_order3(count=6, seed=3, smin=8, smax=20, rmin=2, rmax=6)


def _batch(probs, prec):
    b = cpals.Batch([q.dims for q in probs], [q.R for q in probs], prec)
    for i, q in enumerate(probs):
        b.set_tensor(i, np.ascontiguousarray(q.X))
        b.init_factors(i, q.A0)
    return b


@pytest.mark.parametrize("tol", [0.0, 1e-3])
def test_batch_fp64_follows_oracle(probs, tol):
    with _batch(probs, "fp64") as b:
        out = b.run(SWEEPS, EPS, True, tol)
        facs = [b.get_factors(i) for i in range(len(probs))]
    kinds_seen = set()
    for i, q in enumerate(probs):
        X = q.X.astype(np.float64)
        A_or, tr = O.pp_cp_als(X, q.A0, SWEEPS, EPS, use_V=True, pp_stop_tol=tol)
        assert out["status"][i] == 0
        assert out["sweeps"][i] == SWEEPS
        assert out["kinds"][i] == tr.kinds, i
        np.testing.assert_allclose(out["trace"][i], tr.seen, rtol=0, atol=1e-10)
        assert abs(out["fitness"][i] - tr.fitness[-1]) < 1e-10, i
        for a, ref in zip(facs[i], A_or):
            assert np.max(np.abs(a - ref)) / np.max(np.abs(ref)) < 1e-8, i
        kinds_seen.update(tr.kinds)
    assert kinds_seen == {"als", "pp_init", "pp_approx"}


def test_batch_fp32_close_to_fp64(probs):
    with _batch(probs, "fp64") as b64:
        f64 = b64.run(SWEEPS, EPS)["fitness"]
    with _batch(probs, "fp32") as b32:
        out = b32.run(SWEEPS, EPS)
    assert np.all(out["status"] == 0)
    assert np.max(np.abs(out["fitness"] - f64)) < 1e-4, (out["fitness"], f64)


def test_batch_one_launch_per_stage(probs):
    with _batch(probs[:2], "fp32") as b2, _batch(probs, "fp32") as b6:
        b2.run(3, EPS)
        b6.run(3, EPS)
        s2, s6 = b2.stats(), b6.stats()
    assert s2["launches_per_sweep"] == s6["launches_per_sweep"] > 0
    assert s6["launches_last_run"] == s2["launches_last_run"]


def test_batch_autotuner_cache_and_results(probs):
    """The first run times the three tile shapes of the four contraction
    stages; a second batch of the same shapes takes the cached choice
    without timing.  The tile shape does not change any sum's order, so
    both batches give bit-identical results."""
    sub = probs[:3]
    with _batch(sub, "fp32") as a:
        ra = a.run(8, EPS)
        ta = a.tiles()
    with _batch(sub, "fp32") as b:
        rb = b.run(8, EPS)
        tb = b.tiles()
    assert len(ta["tiles"]) == 4 and all(t in (0, 1, 2) for t in ta["tiles"]) and tb["tiles"] == ta["tiles"]
    assert all(m > 0 for m in ta["ms"])
    assert tb["from_cache"]
    assert np.array_equal(ra["fitness"], rb["fitness"])
    for x, y in zip(ra["trace"], rb["trace"]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_singular_gamma_pinv(prec):
    """An instance whose initial factors share a zero column keeps every
    Gamma^(n) singular (a zero row and column); the batch's normal equations
    then solve through Gamma^dagger (Algorithm 1: a Jacobi eigendecomposition
    and the dense factor diag(w^+)^(1/2) V^T), so that instance is the
    oracle's rank R - 1 run without the column (float64: sweep for sweep
    within 1e-10; float32: final fitness within 1e-4) with the column exactly
    zero, while the regular instance in the same launches is unaffected."""
    R, col = 5, 2
    qs = synth.batch_order3(count=2, seed=11, smin=10, smax=16, rmin=R, rmax=R)
    keep = [r for r in range(R) if r != col]
    A0s = [[a.copy() for a in q.A0] for q in qs]
    for a in A0s[1]:
        a[:, col] = 0.0
    b = cpals.Batch([q.dims for q in qs], [R, R], prec)
    with b:
        for i, q in enumerate(qs):
            b.set_tensor(i, np.ascontiguousarray(q.X))
            b.init_factors(i, A0s[i])
        out = b.run(SWEEPS, EPS, True, 0.0)
        facs = [b.get_factors(i) for i in range(2)]
    assert list(out["status"]) == [0, 0]
    refs = [O.pp_cp_als(qs[0].X.astype(np.float64), A0s[0], SWEEPS, EPS, use_V=True),
            O.pp_cp_als(qs[1].X.astype(np.float64), [a[:, keep] for a in A0s[1]], SWEEPS, EPS,
                        use_V=True)]
    for a in facs[1]:
        assert np.all(a[:, col] == 0.0)
    for i, (A_or, tr) in enumerate(refs):
        got = facs[i] if i == 0 else [a[:, keep] for a in facs[i]]
        if prec == "fp64":
            assert out["kinds"][i] == tr.kinds, i
            np.testing.assert_allclose(out["trace"][i], tr.seen, rtol=0, atol=1e-10)
            assert abs(out["fitness"][i] - tr.fitness[-1]) < 1e-10, i
            for a, ref in zip(got, A_or):
                assert np.max(np.abs(a - ref)) / np.max(np.abs(ref)) < 1e-8, i
        else:
            assert abs(out["fitness"][i] - tr.fitness[-1]) < 1e-4, i
    assert "pp_approx" in refs[1][1].kinds
