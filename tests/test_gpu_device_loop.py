"""Algorithm 3 with its decisions on the device (cpals_run's graph with a
while loop around a switch over the sweep kinds) against the host loop, and
the stopping test inside PP runs (cpals_set_pp_stop_tol) against the oracle.

The two loops launch the same captured kernels in the same order and take
the same decisions on the same device scalars, so their traces and factors
must agree bit for bit.  The stopping test follows the oracle's
pp_cp_als(pp_stop_tol=...) sweep for sweep: the same kinds, the fitness it
sees (exact after ALS sweeps, the first-order estimate after PP sweeps)
within 1e-10, the final factors within 1e-10 relative.
"""
import numpy as np
import pytest
import torch

from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _problem(storage="f64"):
    return synth.make_problem("collinear", [40, 36, 32], 6, seed=13, noise=1e-2, collinearity=0.8,
                              storage=storage)


def _run(g, p, loop, sweeps, eps, target, tol=0.0):
    g.set_device_loop(loop)
    g.set_pp_stop_tol(tol)
    assert g.device_loop_active() == loop
    g.init_factors(p.A0)
    out = g.run(sweeps, eps, True, target)
    return out, g.get_factors()


SCENARIOS = [
    ("als", 30, 0.0, 0.0, 0.0),
    ("pp", 60, 0.2, 0.0, 0.0),
    ("pp_first", 6, 2.0, 0.0, 0.0),          # eps > 1: the operators are built before any ALS sweep
    ("pp_target", 80, 0.2, None, 0.0),       # stops at a target (PP estimates confirmed exactly)
    ("pp_tol", 60, 0.2, 0.0, 1e-5),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("scen", SCENARIOS, ids=[s[0] for s in SCENARIOS])
def test_device_loop_equals_host_loop(prec, scen):
    name, sweeps, eps, target, tol = scen
    p = _problem("f64" if prec == "fp64" else "f32")
    X = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
    with cpals.CPALS(p.dims, p.R, prec) as g:
        g.set_tensor(X)
        if target is None:
            # a target the run reaches after some PP sweeps: ALS's fitness after 25 sweeps
            g.set_device_loop(False)
            g.init_factors(p.A0)
            target = float(g.run(25, 0.0, True, 0.0)["fitness"][-1])
        host, Ah = _run(g, p, False, sweeps, eps, target, tol)
        dev, Ad = _run(g, p, True, sweeps, eps, target, tol)
    assert dev["kinds"] == host["kinds"]
    assert np.array_equal(dev["fitness"], host["fitness"])
    assert dev["reached"] == host["reached"]
    for a, b in zip(Ad, Ah):
        assert np.array_equal(a, b)
    assert np.all(np.diff(dev["times"]) >= 0)
    if name.startswith("pp"):
        assert "pp_init" in dev["kinds"]
    if name == "pp_target":
        assert dev["reached"] and len(dev["kinds"]) < sweeps
    if name == "pp_first":
        assert dev["kinds"][0] == "pp_init"


@pytest.mark.parametrize("loop", [True, False])
def test_pp_stop_tolerance_follows_oracle(loop):
    p = synth.make_problem("collinear", [14, 13, 12], 4, seed=11, noise=1e-2, collinearity=0.8,
                           storage="f64")
    eps, tol, n = 0.0993, 1e-3, 45
    A_or, tr = O.pp_cp_als(p.X, p.A0, n, eps, use_V=True, pp_stop_tol=tol)
    with cpals.CPALS(p.dims, p.R, "fp64") as g:
        g.set_tensor(p.X)
        out, A = _run(g, p, loop, n, eps, 0.0, tol)
    assert out["kinds"] == tr.kinds
    np.testing.assert_allclose(out["fitness"], tr.seen, rtol=0, atol=1e-10)
    for a, b in zip(A, A_or):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-10
    # the test ended at least one PP run that the eps test alone would continue
    _, tr0 = O.pp_cp_als(p.X, p.A0, n, eps, use_V=True)
    assert tr0.kinds != tr.kinds
