"""Failure paths on the GPU, made without a GPU fault.

* A bounded wait that runs out: the tensor-core contraction's waits take
  their bound from the context (cpals_set_wait_limit).  With a bound of one
  cycle the first wait on a stage that the TMA has not filled yet gives up;
  the kernel records the error, lets the loads and MMAs it issued land, frees
  its tensor memory and returns, and the sweep reports CPALS_E_TIMEOUT.  With
  the default bound restored and the status cleared (cpals_init_factors) the
  same context runs the sweep again and gives the result of a fresh context,
  bit for bit.
* A NaN planted in the host tensor: the sweep reports CPALS_E_NUMERIC (not a
  singular Gamma, which the NaN would also cause), and the context recovers
  once a clean tensor is set.
"""
import numpy as np
import pytest
import torch

from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu

E_NUMERIC, E_TIMEOUT = 6, 7


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_wait_limit_timeout_then_recovery():
    p = synth.make_problem("normal", [64, 72, 80], 16, seed=21, storage="f32")
    X = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
    with cpals.CPALS(p.dims, p.R, "mixed") as ref:
        ref.set_tensor(X)
        ref.init_factors(p.A0)
        f_ref = ref.als_sweep()
        A_ref = ref.get_factors()
    with cpals.CPALS(p.dims, p.R, "mixed") as g:
        g.set_tensor(X)
        g.init_factors(p.A0)
        g.set_wait_limit(1)
        with pytest.raises(cpals.CPALSError) as ei:
            g.als_sweep()
        assert ei.value.status == E_TIMEOUT, ei.value
        # the status stays until init_factors clears it
        with pytest.raises(cpals.CPALSError) as ei:
            g.fitness()
        assert ei.value.status == E_TIMEOUT
        g.set_wait_limit(0)
        g.init_factors(p.A0)
        f = g.als_sweep()
        A = g.get_factors()
    assert f == f_ref
    for a, b in zip(A, A_ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_in_tensor_reports_numeric(prec):
    p = synth.make_problem("normal", [24, 32, 40], 6, seed=22, storage="f64")
    Xbad = p.X.copy()
    Xbad[3, 5, 7] = np.nan
    with cpals.CPALS(p.dims, p.R, prec) as g:
        g.set_tensor(Xbad)
        g.init_factors(p.A0)
        with pytest.raises(cpals.CPALSError) as ei:
            g.als_sweep()
        assert ei.value.status == E_NUMERIC, ei.value
        g.set_tensor(p.X)
        g.init_factors(p.A0)
        f = g.als_sweep()
        assert np.isfinite(f) and 0.0 < f <= 1.0


def test_wait_limit_timeout_in_device_loop():
    """The same bounded wait running out inside cpals_run's device loop: the
    loop stops at that sweep, the run reports CPALS_E_TIMEOUT, and the
    context runs normally once the bound is restored and the status cleared."""
    p = synth.make_problem("normal", [64, 72, 80], 16, seed=23, storage="f32")
    X = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
    with cpals.CPALS(p.dims, p.R, "mixed") as g:
        g.set_tensor(X)
        g.init_factors(p.A0)
        assert g.device_loop_active()
        g.set_wait_limit(1)
        with pytest.raises(cpals.CPALSError) as ei:
            g.run(10, 0.2, True, 0.0)
        assert ei.value.status == E_TIMEOUT, ei.value
        g.set_wait_limit(0)
        g.init_factors(p.A0)
        out = g.run(10, 0.2, True, 0.0)
        assert len(out["kinds"]) == 10 and np.all(np.isfinite(out["fitness"]))
