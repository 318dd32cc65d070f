"""The full 400^3 rank-100 benchmark workload (seed 0, FP32 storage) in
float64 on the GPU against the oracle's own trajectory.

``tests/golden/order3_400_rank100_schedule.json`` holds what the FP64 oracle
(and nothing else) computed on this tensor: the exact fitness after each of
200 plain ALS sweeps (Algorithm 1), and the sweep kinds and exact fitness of
200 sweeps of PP-ALS (Algorithm 3, eps 0.1, second-order terms on).  The
GPU's float64 path must follow both:

* ALS: every sweep's exact fitness within 1e-6 absolute, the final one
  (f*, the benchmark's target) within 1e-10 relative;
* PP-ALS: the library's own controller (cpals_run) takes the oracle's sweep
  kinds up to the sweep where the oracle reaches the target, and, with the
  same kinds, the exact fitness after every sweep (cpals_fitness after PP
  sweeps) is within 1e-6 absolute of the oracle's.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "order3_400_rank100_schedule.json")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def ctx(gold):
    p = synth.order3_400_rank100(seed=gold["seed"])
    assert p.dims == gold["dims"] and p.R == gold["R"]
    g = cpals.CPALS(p.dims, p.R, "fp64")
    g.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    yield g, p
    g.close()


def test_order3_400_fp64_als_trajectory(ctx, gold):
    g, p = ctx
    g.init_factors(p.A0)
    out = g.run(gold["sweeps"], 0.0, True, 0.0)
    assert out["kinds"] == ["als"] * gold["sweeps"]
    fit = np.asarray(out["fitness"])
    ref = np.asarray(gold["als_fitness"])
    err = np.abs(fit - ref)
    assert err.max() < 1e-6, (int(err.argmax()), float(err.max()))
    assert abs(fit[-1] - gold["f_star_als"]) < 1e-10 * gold["f_star_als"], (fit[-1], gold["f_star_als"])


def test_order3_400_fp64_pp_als_schedule(ctx, gold):
    g, p = ctx
    n = gold["pp_hit_index"] + 1
    kinds = gold["pp_kinds"][:n]
    g.init_factors(p.A0)
    out = g.run(n, gold["eps"], True, 0.0)
    assert out["kinds"] == kinds
    # exact fitness after every sweep along the same schedule
    g.init_factors(p.A0)
    fit = []
    for k in kinds:
        if k == "als":
            fit.append(g.als_sweep())
            continue
        if k == "pp_init":
            g.pp_build_operators()
        g.pp_sweep(use_V=True)
        fit.append(g.fitness())
    fit = np.asarray(fit)
    ref = np.asarray(gold["pp_fitness"][:n])
    err = np.abs(fit - ref)
    assert err.max() < 1e-6, (int(err.argmax()), float(err.max()))
    assert fit[-1] >= gold["target"] - 1e-9


def test_order3_400_fp64_pp_als_schedule_with_stop_test(ctx, gold):
    """The benchmark's setting: Algorithm 3's stopping test inside PP runs
    (tolerance 1e-6, cpals_set_pp_stop_tol) in the library's device loop
    against the oracle's run with the same test: the same sweep kinds up to
    the target and the fitness the algorithm sees (exact after ALS sweeps,
    the M~ estimate after PP sweeps) within 1e-6."""
    g, p = ctx
    n = gold["pp_tol_hit_index"] + 1
    g.set_pp_stop_tol(gold["pp_stop_tol"])
    try:
        g.init_factors(p.A0)
        out = g.run(n, gold["eps"], True, 0.0)
    finally:
        g.set_pp_stop_tol(0.0)
    assert out["kinds"] == gold["pp_tol_kinds"][:n]
    err = np.abs(np.asarray(out["fitness"]) - np.asarray(gold["pp_tol_seen"][:n]))
    assert err.max() < 1e-6, (int(err.argmax()), float(err.max()))
