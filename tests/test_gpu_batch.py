"""Many independent decompositions at once (cpals_run_batch): every instance
gets exactly the result a lone cpals_run gives it (factors compared bit for
bit), FP64 instances match the oracle, and uneven instances (the 256-tensor
workload's shape mix, scaled down) all finish."""
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
    cpals.lib()


def _ctx(p, prec):
    g = cpals.CPALS(p.dims, p.R, prec)
    g.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    g.init_factors(p.A0)
    return g


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_batch_equals_lone_runs(prec):
    probs = synth.batch_order3(count=10, seed=5, smin=20, smax=56, rmin=3, rmax=16)
    lone = []
    for p in probs:
        with _ctx(p, prec) as g:
            out = g.run(40, 0.1, True, 0.0)
            lone.append((out["fitness"][-1], len(out["kinds"]), g.get_factors()))
    ctxs = [_ctx(p, prec) for p in probs]
    try:
        fit, sw, st = cpals.run_batch(ctxs, workers=4, max_sweeps=40, eps=0.1)
        assert np.all(st == 0)
        for k, g in enumerate(ctxs):
            assert fit[k] == lone[k][0] and sw[k] == lone[k][1], k
            for a, b in zip(g.get_factors(), lone[k][2]):
                np.testing.assert_array_equal(a, b)
    finally:
        for g in ctxs:
            g.close()


def test_batch_fp64_matches_oracle():
    probs = [synth.make_problem("normal", d, R, seed=40 + k, noise=1e-2, storage="f64", eps=0.2)
             for k, (d, R) in enumerate([([24, 20, 18], 4), ([18, 26, 22], 5), ([30, 16, 20], 3)])]
    ctxs = [_ctx(p, "fp64") for p in probs]
    try:
        fit, sw, st = cpals.run_batch(ctxs, workers=3, max_sweeps=25, eps=0.2)
        assert np.all(st == 0) and np.all(sw == 25)
        for p, g in zip(probs, ctxs):
            A_ref, tr = O.pp_cp_als(p.X, p.A0, 25, 0.2, use_V=True)
            for a, b in zip(g.get_factors(), A_ref):
                assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-8
            assert abs(g.fitness() - tr.fitness[-1]) < 1e-10
    finally:
        for g in ctxs:
            g.close()


def test_batch_targets_and_errors():
    probs = synth.batch_order3(count=6, seed=7, smin=16, smax=40, rmin=2, rmax=8)
    ctxs = [_ctx(p, "mixed") for p in probs]
    try:
        with pytest.raises(cpals.CPALSError):
            cpals.run_batch(ctxs, workers=0, max_sweeps=10, eps=0.1)
        fit, sw, st = cpals.run_batch([], workers=2, max_sweeps=10, eps=0.1)
        assert len(fit) == 0
        # a reachable target stops each instance early, an unreachable one runs the budget
        targets = np.array([0.5, 2.0, 0.5, 2.0, 0.5, 2.0])
        fit, sw, st = cpals.run_batch(ctxs, workers=3, max_sweeps=30, eps=0.1, targets=targets)
        assert np.all(st == 0)
        assert np.all(sw[1::2] == 30) and np.all(sw[0::2] < 30)
    finally:
        for g in ctxs:
            g.close()
