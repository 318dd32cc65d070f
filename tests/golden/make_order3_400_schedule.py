"""Write order3_400_rank100_schedule.json with the FP64 oracle only.

Runs, on the 400^3 rank-100 workload (seed 0, FP32 storage upcast to
float64), plain CP-ALS (Algorithm 1) and PP-CP-ALS (Algorithm 3, eps 0.1,
with V) for 200 sweeps each and records the exact fitness after every sweep
and the sweep kinds.  The target fitness is ALS's final fitness minus 1e-6;
the file also records the first sweep at which each run reaches it.  A
second PP-CP-ALS run takes Algorithm 3's stopping test inside PP runs with
tolerance 1e-6 (pp_stop_tol, the setting of the benchmark) and also records
the fitness the algorithm itself sees after each sweep.

Usage: python tests/golden/make_order3_400_schedule.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cpals_oracle as O  # noqa: E402
from paper_1811_10573_gb300 import synth  # noqa: E402


def main():
    p = synth.order3_400_rank100(seed=0)
    X = p.X.astype(np.float64)
    t0 = time.time()
    _, als = O.cp_als(X, p.A0, p.sweeps)
    t1 = time.time()
    _, tr = O.pp_cp_als(X, p.A0, p.sweeps, p.eps, use_V=True)
    t2 = time.time()
    _, trt = O.pp_cp_als(X, p.A0, p.sweeps, p.eps, use_V=True, pp_stop_tol=1e-6)
    t3 = time.time()
    f_star = als[-1]
    target = f_star - 1e-6
    hit_pp = next((i for i, f in enumerate(tr.fitness) if f >= target), None)
    hit_als = next((i for i, f in enumerate(als) if f >= target), None)
    upto = tr.kinds[: (hit_pp + 1) if hit_pp is not None else len(tr.kinds)]
    hit_tol = next((i for i, f in enumerate(trt.fitness) if f >= target), None)
    upto_tol = trt.kinds[: (hit_tol + 1) if hit_tol is not None else len(trt.kinds)]
    out = {
        "workload": p.name, "seed": 0, "dims": p.dims, "R": p.R, "eps": p.eps,
        "sweeps": p.sweeps, "collinearity": p.meta.get("collinearity"),
        "f_star_als": f_star, "target": target,
        "als_fitness": als, "pp_kinds": tr.kinds, "pp_fitness": tr.fitness,
        "pp_hit_index": hit_pp, "als_hit_index": hit_als,
        "counts_to_target": {k: upto.count(k) for k in ("als", "pp_init", "pp_approx")},
        "pp_stop_tol": 1e-6, "pp_tol_kinds": trt.kinds, "pp_tol_fitness": trt.fitness,
        "pp_tol_seen": trt.seen, "pp_tol_hit_index": hit_tol,
        "counts_to_target_tol": {k: upto_tol.count(k) for k in ("als", "pp_init", "pp_approx")},
        "oracle_seconds": {"als_run": t1 - t0, "pp_run": t2 - t1, "pp_tol_run": t3 - t2},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "order3_400_rank100_schedule.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["counts_to_target"], hit_pp, hit_als, f_star)


if __name__ == "__main__":
    main()
