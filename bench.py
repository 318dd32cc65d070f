#!/usr/bin/env python
"""Benchmark: time-to-fitness of PP-CP-ALS (Algorithm 3) vs CP-ALS on one GB300.

Headline (the paper's arithmetic, float64): one step = one float64 PP-ALS
decomposition (eps = 0.1, second-order terms on) of the 400x400x400 rank-100
workload (FP32 storage, collinearity C ~ U[0.5,0.9) drawn per seed, 1e-2
relative noise, U[0,1] init) through the whole hot path: first-level
contractions, multi-TTV, PP operator construction, PP corrections, float64
Gram/Cholesky/solve and fitness, and the eps controller.  A step stops at the
first sweep whose exact fitness reaches f* - 1e-6, f* being the fitness
float64 GPU ALS reaches after 200 sweeps on the same tensor (that ALS run is
also the ALS time to the same target).  Steps cycle over seeds 0..S-1, each
seed a fresh tensor; value = mean seconds per step (lower is better), timed
with CUDA events, inputs resident in HBM, L2 flushed between steps.

Sub-entries: the same comparison in FP32 and in mixed precision (tensor-core
first level, with and without the learned controller), each against its own
ALS and with its error against the float64 oracle; the 60^3, 120^4 and 24^6
workloads; the ALS variants, many small tensors, and PP-Tucker.  The short
summary at the end of the JSON line repeats the medians over seeds.

--impl reference times the FP64 CPU oracle (the baseline arm) on the host
cores for the same workload and metric.
Under torchrun (--gpus N > 1) every rank decomposes its own instances
(replicas, no data-path collective); value is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-fitness (s) PP-ALS vs ALS on 1 GB300; MTTKRP TFLOP/s and HBM GB/s"
SCHEDULE = os.path.join(ROOT, "tests", "golden", "order3_400_rank100_schedule.json")
PROFILE_DIR = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_1811_10573_gb300", "csrc")
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2070 MHz
# (the 1.25 TFLOP/s FP64 figure of the part at its maximum SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithm 3's stopping test inside PP runs (fitness-difference form): a PP
# run goes on only while each sweep gains at least the target's own margin
PP_STOP_TOL = 1e-6
HOST_LOOP = False      # --host-loop: decisions on the host (for profilers)


def prep(g):
    """Settings every decomposition context of the benchmark gets."""
    g.set_pp_stop_tol(PP_STOP_TOL)
    if HOST_LOOP:
        g.set_device_loop(False)
    return g


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--seeds", type=int, default=10, help="headline steps cycle over this many seeds")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="order3_400_rank100")
    ap.add_argument("--precision", default="fp64", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-reduced", action="store_true", help="skip the FP32 and mixed sub-entries")
    ap.add_argument("--no-configs", action="store_true", help="skip the 60^3, 120^4 and 24^6 entries")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tucker", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline and FP32/mixed only")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the 256-tensor batch entry (its own JSON line)")
    ap.add_argument("--no-contexts", action="store_true",
                    help="batch entry: the fused batch only, without the per-tensor contexts")
    ap.add_argument("--host-loop", action="store_true",
                    help="Algorithm 3's decisions on the host in every run (for profilers)")
    return ap.parse_args()


WORKLOADS = ("order3_400_rank100", "order4_120_rank64", "order6_24_rank50", "order3_60_rank10")


def workload(name, seed):
    from paper_1811_10573_gb300 import synth
    assert name in WORKLOADS, name
    return getattr(synth, name)(seed=seed)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


def committed_traffic(kernel, workload_name, precision, source):
    """DRAM bytes per launch from a committed ncu summary, valid only for the
    workload and precision it was captured on and while the kernel source is
    unchanged (else None)."""
    path = os.path.join(PROFILE_DIR, f"{kernel}_{workload_name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        prof = json.load(f)
    with open(os.path.join(CSRC, source), "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()
    if prof.get("source_sha256") != h or prof.get("precision") != precision:
        return None
    return prof.get("traffic_bytes_per_launch")


def median(v):
    v = [x for x in v if x is not None]
    return round(statistics.median(v), 6) if v else None


# ----------------------------------------------------------------- oracle timing
ORACLE_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import synth
p = getattr(synth, %(name)r)(seed=%(seed)d)
X = p.X.astype(np.float64)
A = [a.copy() for a in p.A0]
S = [O.gram(a) for a in A]
t = time.perf_counter(); O.als_sweep(X, A, S); t_als = time.perf_counter() - t
t = time.perf_counter(); ops, Mp = O.pp_operators(X, A); t_build = time.perf_counter() - t
Ap = [a.copy() for a in A]; dA = [np.zeros_like(a) for a in A]
t = time.perf_counter(); O.pp_sweep(ops, Mp, A, Ap, dA, S, True); t_pp = time.perf_counter() - t
t = time.perf_counter(); O.fitness(X, A); t_fit = time.perf_counter() - t
print(json.dumps({"als": t_als, "build": t_build, "pp": t_pp, "fit": t_fit}))
"""


def oracle_sample(name, seed=0, threads=None):
    """One of each oracle step on the full workload (a bounded sample), in a
    child process; threads = 1 pins the BLAS and OpenMP pools to one thread."""
    env = dict(os.environ)
    if threads:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
    code = ORACLE_SAMPLE % {"root": ROOT, "name": name, "seed": seed}
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def project(ts, counts):
    """Oracle seconds for a sweep schedule: ALS sweeps, PP initialisation
    sweeps (build + one PP pass), PP approximated sweeps, one exact check."""
    return (counts.get("als", 0) * ts["als"] + counts.get("pp_init", 0) * (ts["build"] + ts["pp"])
            + counts.get("pp_approx", 0) * ts["pp"] + ts["fit"])


def oracle_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_counts(name):
    if name == "order3_400_rank100" and os.path.exists(SCHEDULE):
        with open(SCHEDULE) as f:
            return json.load(f)["counts_to_target"], "the oracle's own schedule to the target"
    return None, None


# ----------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- timing helpers
class Runner:
    """Times whole decompositions of one context with CUDA events on the
    caller's stream (the library joins it at the start and end of a call)."""

    def __init__(self, dist, flush):
        self.dist = dist
        self.flush = flush

    def run(self, ctx, A0, max_sweeps, eps, target, controlled=False):
        import torch
        ctx.init_factors(A0)
        self.flush.zero_()                      # 256 MB write: L2 holds nothing of the inputs
        torch.cuda.synchronize()
        self.dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if controlled:
            out = ctx.run_controlled(max_sweeps, eps, True, target)
        else:
            out = ctx.run(max_sweeps, eps, True, target)
        e1.record()
        torch.cuda.synchronize()
        return self.dist.max(e0.elapsed_time(e1) / 1e3), out


def counts_of(kinds):
    return {k: kinds.count(k) for k in ("als", "pp_init", "pp_approx")}


def als_to_target(dt, out, target):
    """Time of the first sweep of a full ALS run whose exact fitness reaches
    the target: the run's event-timed total scaled by the host-clock fraction
    at that sweep (the trace's time stamps are taken after each sweep's
    synchronisation)."""
    fit = list(out["fitness"])
    hit = next((i for i, f in enumerate(fit) if f >= target), None)
    if hit is None:
        return None, None
    t = out["times"]
    return dt * float(t[hit]) / float(t[-1]), hit + 1


def reference_errors(p, precisions, contexts):
    """Errors of each precision against the float64 oracle on the same state
    (seed 0): the exact MTTKRP of every mode at the initial factors, and the
    factors and exact fitness after one ALS sweep from them."""
    import numpy as np
    from oracle import cpals_oracle as O
    X = p.X.astype(np.float64)
    N = X.ndim
    M_or = [O.mttkrp(X, p.A0, n) for n in range(N)]
    A = [a.copy() for a in p.A0]
    S = [O.gram(a) for a in A]
    O.als_sweep(X, A, S)
    f_or = O.fitness(X, A)
    out = {}
    for prec in precisions:
        g = contexts[prec]
        g.init_factors(p.A0)
        merr = max(float(np.max(np.abs(g.mttkrp(n) - M_or[n])) / np.max(np.abs(M_or[n])))
                   for n in range(N))
        f = g.als_sweep()
        Ag = g.get_factors()
        aerr = max(float(np.max(np.abs(a - b)) / np.max(np.abs(b))) for a, b in zip(Ag, A))
        out[prec] = {"mttkrp_rel_err": float(f"{merr:.3e}"), "factor_rel_err_one_sweep": float(f"{aerr:.3e}"),
                     "fitness_abs_err_one_sweep": float(f"{abs(f - f_or):.3e}")}
    return out


def graph_replay_floor_us(n=200):
    """Host floor of one sweep with a per-sweep host decision: replay of a
    one-kernel CUDA graph plus a stream synchronisation."""
    import torch
    x = torch.zeros(32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x.add_(1.0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        x.add_(1.0)
    for _ in range(10):
        g.replay()
        torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(n):
        g.replay()
        torch.cuda.synchronize()
    return (time.perf_counter() - t) / n * 1e6


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_1811_10573_gb300 import build, cpals, harness

    dist = harness.init()
    torch.cuda.set_device(dist.local_rank)
    build.build()
    cpals.lib()
    t_start = time.time()
    if args.quick:
        args.no_configs = args.no_variants = args.no_batch = args.no_tucker = True
    name = args.workload
    nseed = max(1, args.seeds)
    seeds = [100 * dist.rank + s for s in range(nseed)]     # replicas: each rank its own tensors
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    runner = Runner(dist, flush)
    hp = args.precision
    probs, Xd, target, f_star, als64 = {}, {}, {}, {}, {}
    p0 = workload(name, seeds[0])
    dims, R, sweeps, eps = p0.dims, p0.R, p0.sweeps, p0.eps
    max_sweeps = 2 * sweeps
    ctx = {"fp64": cpals.CPALS(dims, R, "fp64")}
    prep(ctx["fp64"])

    def load(s):
        if s not in probs:
            p = p0 if s == seeds[0] else workload(name, s)
            probs[s] = p
            Xd[s] = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
        return probs[s]

    # f* and the float64 ALS time to f* - 1e-6 per seed: one full ALS run each
    g64 = ctx["fp64"]
    for i, s in enumerate(seeds):
        p = load(s)
        g64.set_tensor(Xd[s])
        if i == 0:
            runner.run(g64, p.A0, 2, 0.0, 0.0)              # graph capture
        dt, out = runner.run(g64, p.A0, p.sweeps, 0.0, 0.0)
        f_star[s] = float(out["fitness"][-1])
        target[s] = f_star[s] - 1e-6
        t_hit, n_hit = als_to_target(dt, out, target[s])
        als64[s] = {"value": t_hit, "sweeps": n_hit, "full_run_s": round(dt, 6),
                    "per_sweep_ms": round(dt / p.sweeps * 1e3, 3)}
        log(f"seed {s}: float64 ALS {p.sweeps} sweeps {dt:.3f} s, f* {f_star[s]:.12f}, "
            f"target reached after {n_hit} sweeps ({t_hit:.3f} s)")

    # ---- headline: PP-ALS in the headline precision (float64 by default)
    if hp not in ctx:
        ctx[hp] = cpals.CPALS(dims, R, hp)
        prep(ctx[hp])
    gh = ctx[hp]
    gh.set_profiling(True)
    gh.set_tensor(Xd[seeds[0]])
    for _ in range(args.warmup):
        runner.run(gh, probs[seeds[0]].A0, max_sweeps, eps, target[seeds[0]])
    gh.reset_stats()
    clocks = Clocks(dist.local_rank)
    clocks.start()
    steps = []
    for k in range(args.steps):
        s = seeds[k % nseed]
        gh.set_tensor(Xd[s])
        dt, out = runner.run(gh, probs[s].A0, max_sweeps, eps, target[s])
        steps.append({"seed": s, "s": round(dt, 6), "reached": bool(out["reached"]),
                      "sweeps": len(out["kinds"]), "counts": counts_of(out["kinds"]),
                      "final_fitness": float(out["fitness"][-1])})
        log(f"step {k} seed {s}: PP-ALS ({hp}) {dt:.3f} s, {len(out['kinds'])} sweeps "
            f"{counts_of(out['kinds'])}, reached {out['reached']}")
    clk = clocks.stop()
    fl, pc = gh.get_stats(0), gh.get_stats(2)
    launches = gh.get_stats(1)["launches"]
    gh.set_profiling(False)
    # the same runs with Algorithm 3's decisions on the device (the default
    # of cpals_run; the timed steps above keep the host loop because their
    # CUDA events, which time the contraction for the roofline, cannot sit
    # inside the device loop's conditional graph)
    loop_check = {}
    for s in ([] if HOST_LOOP else seeds[: min(3, nseed)]):
        gh.set_tensor(Xd[s])
        runner.run(gh, probs[s].A0, max_sweeps, eps, target[s])    # device-loop graph capture
        dd, od = runner.run(gh, probs[s].A0, max_sweeps, eps, target[s])
        hs = [x for x in steps if x["seed"] == s]
        loop_check[str(s)] = {"device_loop_s": round(dd, 6), "host_loop_s": hs[0]["s"] if hs else None,
                              "same_kinds": (counts_of(od["kinds"]) == hs[0]["counts"]) if hs else None,
                              "reached": bool(od["reached"])}
    value = statistics.mean(x["s"] for x in steps)
    pp_by_seed = {}
    for x in steps:
        pp_by_seed.setdefault(x["seed"], []).append(x["s"])
    pp_seed = {s: statistics.mean(v) for s, v in pp_by_seed.items()}

    # ---- FP32 and mixed precision: PP-ALS and ALS to each seed's float64 target
    reduced = {}
    if not args.no_reduced:
        for prec in ("fp32", "mixed"):
            reduced[prec] = precision_block(prec, ctx, dims, R, seeds, probs, Xd, target, f_star,
                                            runner, max_sweeps, eps, learned=(prec == "mixed"))
        log(f"reduced precision done at {time.time() - t_start:.0f} s")

    # the headline precision's own ALS (float64: the run that fixed f*)
    if hp == "fp64":
        als_seed = {s: als64[s]["value"] for s in seeds}
    else:
        als_seed = {int(k): v["als_s"] for k, v in reduced.get(hp, {}).get("per_seed", {}).items()}
    speed = [als_seed[s] / pp_seed[s] for s in pp_seed if als_seed.get(s)]

    # errors of every precision against the float64 oracle on the same state
    errors = None
    if not args.no_reduced and dist.rank == 0:
        ctx["fp64"].set_tensor(Xd[seeds[0]])
        for prec in ("fp32", "mixed"):
            ctx[prec].set_tensor(Xd[seeds[0]])
        errors = reference_errors(p0, ["fp64", "fp32", "mixed"], ctx)
        log(f"errors vs oracle: {errors}")

    # ---- the other workloads (one seed each)
    configs = {}
    if not args.no_configs:
        for cname in ("order3_60_rank10", "order4_120_rank64", "order6_24_rank50"):
            if cname != name:
                configs[cname] = run_config(cname, dist, runner)
                log(f"{cname}: {configs[cname].get('summary')}")

    variants = batch = tucker = None
    if not args.no_variants and name == "order3_400_rank100":
        variants = run_variants(args, dist, p0, Xd[seeds[0]], flush, max_sweeps, "mixed")
    if not args.no_batch and name == "order3_400_rank100":
        batch = run_batch_bench(args, dist, flush, "mixed")
    if not args.no_tucker and name == "order3_400_rank100":
        tucker = run_tucker_bench(args, dist, flush)

    # ---- end to end through the C ABI from pinned host buffers
    e2e_t, h2d, d2h = [], 0, 0
    for s in seeds[: max(1, min(args.steps, 3))]:
        p = probs[s]
        Xh = torch.from_numpy(np.ascontiguousarray(p.X)).pin_memory()
        A0h = [np.ascontiguousarray(a) for a in p.A0]
        flush.zero_()
        torch.cuda.synchronize()
        dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gh.set_tensor(Xh)
        gh.init_factors(A0h)
        out = gh.run(max_sweeps, eps, True, target[s])
        A_host = gh.get_factors()
        e1.record()
        torch.cuda.synchronize()
        e2e_t.append(dist.max(e0.elapsed_time(e1) / 1e3))
        fbytes = sum(a.nbytes for a in A_host)
        h2d = int(Xh.numel() * Xh.element_size() + fbytes)
        d2h = int(fbytes + len(out["kinds"]) * (32 * 8 + 4 * 4))

    # ---- roofline of the dominant kernel: the first-level contraction
    pk = peaks()
    sec = fl["total_ms"] / 1e3 if fl["total_ms"] > 0 else float("nan")
    nl = max(1, fl["launches"])
    common = {"launches": fl["launches"], "avg_launch_us": round(fl["total_ms"] * 1e3 / nl, 2),
              "algorithmic_bytes_per_launch": round(fl["bytes"] / nl),
              "algorithmic_flops_per_launch": round(fl["flops"] / nl)}
    if hp == "fp64":
        ach = fl["flops"] / sec / 1e12
        roofline = {"bound": "alu", "achieved": round(ach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                    "traffic": committed_traffic("gemm_simt_fp64", name, "fp64", "contract.cu"),
                    "kernel": "first-level contraction (float64 FMA, gemm_simt)",
                    "hbm_gbs": round(fl["bytes"] / sec / 1e9, 1), **common,
                    "peak_src": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (the part's "
                                "1.25 TFLOP/s FP64 rate); not a measured peak"}
    elif hp == "fp32":
        ach = fl["flops"] / sec / 1e12
        roofline = {"bound": "alu", "achieved": round(ach, 3), "peak": round(FP32_PEAK_TFLOPS, 3),
                    "unit": "TFLOP/s", "frac": round(ach / FP32_PEAK_TFLOPS, 4), "traffic": None,
                    "kernel": "first-level contraction (float32 FMA, gemm_f32 / gemm_simt)",
                    "hbm_gbs": round(fl["bytes"] / sec / 1e9, 1), **common,
                    "peak_src": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz; "
                                "not a measured peak"}
    else:
        ach = fl["bytes"] / sec / 1e9
        roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": round(ach / pk["hbm_gbs"], 4),
                    "traffic": committed_traffic("umma_gemm", name, hp, "umma.cu"),
                    "kernel": "first-level contraction (tcgen05 bf16)",
                    "tflops": round(fl["flops"] / sec / 1e12, 2), **common,
                    "peak_src": pk["src"] + " (copy bandwidth)"}
    pc_ach = pc["bytes"] / (pc["total_ms"] / 1e3) / 1e9 if pc["total_ms"] > 0 else 0.0
    roofline_pp = {"bound": "hbm", "achieved": round(pc_ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                   "frac": round(pc_ach / pk["hbm_gbs"], 4), "kernel": f"PP correction (Eq. 3), {hp}",
                   "launches": pc["launches"],
                   "avg_launch_us": round(pc["total_ms"] * 1e3 / max(1, pc["launches"]), 2),
                   "algorithmic_bytes_per_launch": round(pc["bytes"] / max(1, pc["launches"])),
                   "peak_src": pk["src"] + " (copy bandwidth)"}

    reached = all(x["reached"] for x in steps)
    last = steps[-1]
    result = {
        "metric": METRIC, "value": round(value, 6), "unit": "s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value * 1e3, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "bf16-tc/fp32/f32x2", "fp32": "fp32/f32x2", "fp64": "f64"}[hp],
        "data": "synthetic",
        "config": {"workload": p0.name, "dims": dims, "R": R, "eps": eps, "max_sweeps": max_sweeps,
                   "pp_stop_tol": PP_STOP_TOL,
                   "seeds": seeds, "precision": hp, "use_V": True,
                   "target": "f* - 1e-6, f* = float64 GPU ALS fitness after 200 sweeps, per seed",
                   "normal_eq": "fp64" if hp == "fp64" else "double-float (f32 pair)",
                   "l2": "flushed between steps (256 MB write); X is 256 MB fp32 (512 MB as float64)",
                   "parallelism": "replicas" if dist.world > 1 else "single GPU"},
        "reached": reached, "steps_detail": steps, "device_loop_check": loop_check,
        "f_star_per_seed": {str(s): f_star[s] for s in seeds},
        "als_fp64_per_seed": {str(s): als64[s] for s in seeds},
        "reduced_precision": reduced or None,
        "errors_vs_oracle": errors,
        "configs": configs or None,
        "variants": variants, "batch": batch, "tucker": tucker,
        "roofline": roofline,
        "roofline_pp_correct": roofline_pp,
        "e2e": {"value": round(statistics.mean(e2e_t), 6), "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "seeds": seeds[: len(e2e_t)]},
        "gpu_launches": int(launches), "gpu_launches_per_step": round(launches / max(1, args.steps), 1),
        "clocks": clk,
    }
    if dist.rank == 0 and not args.no_cpu_baseline:
        counts, how = oracle_counts(name)
        if counts is None:
            counts, how = counts_of(["als"] * sweeps), f"the workload's sweep budget ({sweeps} ALS sweeps)"
        ts = oracle_sample(name, seeds[0])
        ts1 = oracle_sample(name, seeds[0], threads=1)
        result["cpu_baseline"] = {
            "value": round(project(ts, counts), 3), "unit": "s", "cores": oracle_cores(),
            "kind": "oracle",
            "single_thread_value": round(project(ts1, counts), 3),
            "sample": ("float64 numpy oracle on the full seed-0 workload: one ALS sweep "
                       f"({ts['als']:.3f} s; one thread {ts1['als']:.3f} s), one PP operator build "
                       f"({ts['build']:.3f} s; {ts1['build']:.3f} s), one PP sweep ({ts['pp']:.3f} s; "
                       f"{ts1['pp']:.3f} s), one exact fitness ({ts['fit']:.3f} s; {ts1['fit']:.3f} s), "
                       f"projected onto {how} {counts}")}
    # the comparison last, so that a tail of the output keeps it
    pm = {}
    for prec, blk in reduced.items():
        pm[prec] = blk.get("summary")
    result["summary"] = {
        "precision": hp, "seeds": len(seeds),
        "pp_s_median": median(list(pp_seed.values())),
        "als_s_median": median([als_seed.get(s) for s in pp_seed]),
        "pp_vs_als_speedup_median": median(speed),
        "pp_vs_als_speedup_min": round(min(speed), 3) if speed else None,
        "per_precision": pm or None,
        "configs": {k: v.get("summary") for k, v in configs.items()} or None,
        "batch": (batch or {}).get("summary"),
        "roofline_frac": roofline["frac"],
        "bench_wall_s": round(time.time() - t_start, 1),
    }
    result["als_time_to_fitness_s"] = median([als_seed.get(s) for s in pp_seed])
    result["pp_vs_als_speedup"] = median(speed)
    if dist.rank == 0:
        print(json.dumps(result))
    for g in ctx.values():
        g.close()
    dist.close()


def precision_block(prec, ctx, dims, R, seeds, probs, Xd, target, f_star, runner, max_sweeps, eps,
                    learned=False):
    """PP-ALS (eps rule) and plain ALS in one precision on every seed, to
    that seed's float64 target; with learned, also PP-ALS with the learned
    sweep-type controller.  The tensor-core roofline is taken over the
    PP-ALS runs of the mixed context."""
    import numpy as np

    from paper_1811_10573_gb300 import controller as ctrl
    from paper_1811_10573_gb300 import cpals

    if prec not in ctx:
        ctx[prec] = cpals.CPALS(dims, R, prec)
        prep(ctx[prec])
    g = ctx[prec]
    params = ctrl.load() if learned else None
    per = {}
    for i, s in enumerate(seeds):
        p = probs[s]
        g.set_tensor(Xd[s])
        if i == 0:
            runner.run(g, p.A0, max_sweeps, eps, target[s])        # graph capture
            runner.run(g, p.A0, max_sweeps, 0.0, target[s])
        dpp, opp = runner.run(g, p.A0, max_sweeps, eps, target[s])
        dals, oals = runner.run(g, p.A0, max_sweeps, 0.0, target[s])
        e = {"pp_s": round(dpp, 6), "pp_reached": bool(opp["reached"]), "pp_sweeps": len(opp["kinds"]),
             "pp_counts": counts_of(opp["kinds"]),
             "pp_final_minus_f_star": float(f"{opp['fitness'][-1] - f_star[s]:.3e}"),
             "als_s": round(dals, 6) if oals["reached"] else None, "als_reached": bool(oals["reached"]),
             "als_sweeps": len(oals["kinds"]),
             "als_final_minus_f_star": float(f"{oals['fitness'][-1] - f_star[s]:.3e}")}
        e["speedup"] = round(dals / dpp, 3) if (oals["reached"] and opp["reached"]) else None
        per[str(s)] = e
    # the tensor-core roofline: CUDA events around every first-level
    # contraction of one more PP-ALS run of the first seed (host loop)
    g.set_profiling(prec in ("mixed", "fp32"))
    g.set_tensor(Xd[seeds[0]])
    runner.run(g, probs[seeds[0]].A0, max_sweeps, eps, target[seeds[0]])
    g.reset_stats()
    runner.run(g, probs[seeds[0]].A0, max_sweeps, eps, target[seeds[0]])
    st = g.get_stats(0)
    g.set_profiling(False)
    if params is not None:
        g.set_controller(params, 0.6)
        for i, s in enumerate(seeds):
            p = probs[s]
            g.set_tensor(Xd[s])
            if i == 0:
                runner.run(g, p.A0, max_sweeps, eps, target[s], controlled=True)
            dl, ol = runner.run(g, p.A0, max_sweeps, eps, target[s], controlled=True)
            per[str(s)].update({"learned_s": round(dl, 6), "learned_reached": bool(ol["reached"]),
                                "learned_counts": counts_of(ol["kinds"]),
                                "learned_network_decisions": round(float(np.mean(ol["learned"])), 3)
                                if len(ol["learned"]) else 0.0})
        g.set_controller(None)
    pp = [v["pp_s"] for v in per.values() if v["pp_reached"]]
    als = [v["als_s"] for v in per.values()]
    sp = [v["speedup"] for v in per.values()]
    summ = {"pp_s_median": median(pp), "als_s_median": median(als), "speedup_median": median(sp),
            "pp_reached": sum(v["pp_reached"] for v in per.values()),
            "als_reached": sum(v["als_reached"] for v in per.values()), "seeds": len(seeds)}
    if params is not None:
        lr = [v["learned_s"] for v in per.values() if v["learned_reached"]]
        summ["learned_s_median"] = median(lr)
        summ["learned_reached"] = sum(v["learned_reached"] for v in per.values())
    out = {"per_seed": per, "summary": summ}
    if prec == "mixed" and st["total_ms"] > 0:
        pk = peaks()
        ach = st["bytes"] / (st["total_ms"] / 1e3) / 1e9
        out["roofline_tc"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                              "kernel": "first-level contraction (tcgen05 bf16), one PP-ALS run of the first seed",
                              "launches": st["launches"],
                              "avg_launch_us": round(st["total_ms"] * 1e3 / max(1, st["launches"]), 2),
                              "algorithmic_bytes_per_launch": round(st["bytes"] / max(1, st["launches"])),
                              "traffic": committed_traffic("umma_gemm", "order3_400_rank100", "mixed",
                                                           "umma.cu"),
                              "tflops": round(st["flops"] / (st["total_ms"] / 1e3) / 1e12, 2),
                              "peak_src": pk["src"] + " (copy bandwidth)"}
        summ["roofline_tc_frac"] = out["roofline_tc"]["frac"]
    if prec == "fp32" and st["total_ms"] > 0:
        ach = st["flops"] / (st["total_ms"] / 1e3) / 1e12
        out["roofline_fp32"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(FP32_PEAK_TFLOPS, 3),
                                "unit": "TFLOP/s", "frac": round(ach / FP32_PEAK_TFLOPS, 4),
                                "kernel": "first-level contraction (float32 FMA), one PP-ALS run of the first seed",
                                "launches": st["launches"],
                                "avg_launch_us": round(st["total_ms"] * 1e3 / max(1, st["launches"]), 2),
                                "peak_src": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz"}
        summ["roofline_fp32_frac"] = out["roofline_fp32"]["frac"]
    return out


def run_config(cname, dist, runner):
    """One seed of another workload: float64 ALS for f*, then PP-ALS and ALS
    to f* - 1e-6 in float64 and in mixed precision; per-sweep times; on the
    60^3 tensor also the host floor of a per-sweep decision."""
    import numpy as np
    import torch

    from paper_1811_10573_gb300 import cpals

    p = workload(cname, 100 * dist.rank)
    X = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
    res = {"workload": p.name, "dims": p.dims, "R": p.R, "eps": p.eps, "sweeps": p.sweeps}
    summ = {}
    target = None
    for prec in ("fp64", "mixed"):
        with cpals.CPALS(p.dims, p.R, prec) as g:
            g.set_tensor(X)
            prep(g)
            runner.run(g, p.A0, 2, 0.0, 0.0)                      # graph capture
            if prec == "fp64":
                dt, out = runner.run(g, p.A0, p.sweeps, 0.0, 0.0)
                f_star = float(out["fitness"][-1])
                target = f_star - 1e-6
                t_als, n_als = als_to_target(dt, out, target)
                als = {"als_s": round(t_als, 6), "als_sweeps": n_als,
                       "als_per_sweep_us": round(dt / p.sweeps * 1e6, 1)}
                res["f_star"] = f_star
            else:
                dt, out = runner.run(g, p.A0, 2 * p.sweeps, 0.0, target)
                als = {"als_s": round(dt, 6) if out["reached"] else None, "als_sweeps": len(out["kinds"]),
                       "als_per_sweep_us": round(dt / max(1, len(out["kinds"])) * 1e6, 1),
                       "als_reached": bool(out["reached"])}
            runner.run(g, p.A0, 2 * p.sweeps, p.eps, target)       # PP graph capture
            dpp, opp = runner.run(g, p.A0, 2 * p.sweeps, p.eps, target)
            e = {"pp_s": round(dpp, 6), "pp_reached": bool(opp["reached"]), "pp_sweeps": len(opp["kinds"]),
                 "pp_counts": counts_of(opp["kinds"]),
                 "pp_per_sweep_us": round(dpp / max(1, len(opp["kinds"])) * 1e6, 1), **als}
            e["speedup"] = round(e["als_s"] / dpp, 3) if (e["als_s"] and opp["reached"]) else None
            if cname == "order3_60_rank10":
                # the same PP-ALS run with a host round trip per sweep
                g.set_device_loop(False)
                runner.run(g, p.A0, 2 * p.sweeps, p.eps, target)
                dh, oh = runner.run(g, p.A0, 2 * p.sweeps, p.eps, target)
                g.set_device_loop(True)
                e["host_loop_pp_s"] = round(dh, 6)
                e["host_loop_pp_per_sweep_us"] = round(dh / max(1, len(oh["kinds"])) * 1e6, 1)
            res[prec] = e
            summ[prec] = {"pp_s": e["pp_s"], "als_s": e["als_s"], "speedup": e["speedup"]}
    if cname == "order3_60_rank10":
        res["graph_replay_floor_us"] = round(graph_replay_floor_us(), 1)
        summ["fp64_pp_per_sweep_us"] = res["fp64"]["pp_per_sweep_us"]
        summ["fp64_host_loop_pp_per_sweep_us"] = res["fp64"].get("host_loop_pp_per_sweep_us")
        summ["graph_replay_floor_us"] = res["graph_replay_floor_us"]
    res["summary"] = summ
    return res


def run_batch_bench(args, dist, flush, prec, workers=16):
    """256 order-3 tensors (s_n ~ U{32..160}, R ~ U{8..64}, 100 sweeps of
    Algorithm 3 each): the fused batch (cpals_batch_*: one launch per sweep
    stage over all instances, one graph per batch sweep, tiles from the
    autotuner) in float32 and float64, against one context per tensor run
    by host worker threads (cpals_run_batch) in float32 and in the given
    precision."""
    import numpy as np
    import torch

    from paper_1811_10573_gb300 import cpals, synth

    probs = synth.batch_order3(count=256, seed=dist.rank)
    n = len(probs)
    q0 = probs[0]
    out = {"workload": "batch_order3: 256 order-3 tensors, s_n ~ U{32..160}, R ~ U{8..64}, "
                       f"1e-2 relative noise, eps {q0.eps}, {q0.sweeps} sweeps each (Algorithm 3 per tensor), "
                       f"stopping test {PP_STOP_TOL}"}

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        dist.barrier()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return dist.max(time.perf_counter() - t), r

    for bprec in ("fp32", "fp64"):
        with cpals.Batch([q.dims for q in probs], [q.R for q in probs], bprec) as b:
            for i, q in enumerate(probs):
                b.set_tensor(i, np.ascontiguousarray(q.X))
                b.init_factors(i, q.A0)
            b.run(2, q0.eps, True, PP_STOP_TOL)                  # tile autotuning
            dt, r = timed(lambda: b.run(q0.sweeps, q0.eps, True, PP_STOP_TOL))
            ks = [k for kk in r["kinds"] for k in kk]
            st = b.stats()
            out["fused_" + bprec] = {
                "value": round(dt, 4), "unit": "s", "decompositions_per_s": round(n / dt, 1),
                "launches_per_sweep": st["launches_per_sweep"],
                "launches_per_stage": 1, "kernel_launches_per_run": st["launches_last_run"],
                "sweep_counts": {k: ks.count(k) for k in ("als", "pp_init", "pp_approx")},
                "mean_final_fitness": round(float(np.mean(r["fitness"])), 6),
                "failed": int(np.sum(r["status"] != 0)), "autotuner": b.tiles()}
    for cprec in (() if args.no_contexts else ("fp32", prec)):
        if "contexts_" + cprec in out:
            continue
        ctxs = []
        try:
            for q in probs:
                g = cpals.CPALS(q.dims, q.R, cprec)
                prep(g)
                g.set_tensor(torch.from_numpy(np.ascontiguousarray(q.X)).cuda())
                ctxs.append(g)

            def go(w):
                for g, q in zip(ctxs, probs):
                    g.init_factors(q.A0)
                return cpals.run_batch(ctxs, workers=w, max_sweeps=q0.sweeps, eps=q0.eps)

            timed(lambda: go(workers))                       # warm-up: every context captures its graphs
            dt, (fit, sw, stt) = timed(lambda: go(workers))
            fe = np.array([g.fitness() for g in ctxs])
            out["contexts_" + cprec] = {"value": round(dt, 4), "unit": "s", "workers": workers,
                                        "decompositions_per_s": round(n / dt, 1),
                                        "mean_final_fitness": round(float(np.mean(fe)), 6),
                                        "failed": int(np.sum(stt != 0))}
        finally:
            for g in ctxs:
                g.close()
    f32 = out["fused_fp32"]
    out["summary"] = {"fused_fp32_per_s": f32["decompositions_per_s"]}
    if "contexts_fp32" in out:
        c32 = out["contexts_fp32"]["decompositions_per_s"]
        out["summary"].update({"contexts_fp32_per_s": c32,
                               "fused_vs_contexts_fp32": round(f32["decompositions_per_s"] / c32, 3)})
    return out


def run_tucker_bench(args, dist, flush, s=400, R=20, sweeps=20, eps=0.3):
    """Tucker rank R = 0.05 s on an order-3 s^3 tensor (the paper's Tucker
    sweep-time setting), float64 and with tensor-core first-level TTMs: mean
    time of each sweep kind, and a budget of sweeps with PP (eps 0.3, the
    paper's Tucker tolerance) and without."""
    import numpy as np
    import torch

    from paper_1811_10573_gb300 import cpals, synth

    p = synth.tucker_problem([s] * 3, [R] * 3, seed=dist.rank, noise=0.3)

    def ev_time(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    def one(precision, p):
        Xd = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
        with cpals.Tucker([int(d) for d in p.X.shape], p.R, precision) as t:
            t.set_tensor(Xd)
            t.init_factors(p.A0)
            for _ in range(3):
                t.als_sweep()
            als = [ev_time(t.als_sweep)[0] for _ in range(5)]
            build = [ev_time(t.pp_build_operators)[0] for _ in range(3)]
            pps = [ev_time(t.pp_sweep)[0] for _ in range(5)]
            runs = {}
            for name, e in (("pp", eps), ("als", 0.0)):
                t.init_factors(p.A0)
                t.run(2, e)                              # warm-up
                t.init_factors(p.A0)
                torch.cuda.synchronize()
                dist.barrier()
                dt, out = ev_time(lambda: t.run(sweeps, e))
                runs[name] = {"value": round(dist.max(dt), 6), "unit": "s", "sweeps": len(out["kinds"]),
                              "sweep_counts": {k: out["kinds"].count(k) for k in ("als", "pp_init", "pp_approx")},
                              "final_fitness": t.fitness()}
        ms = lambda v: round(statistics.mean(v) * 1e3, 3)
        return {"sweep_ms": {"als": ms(als), "pp_build": ms(build), "pp_approx": ms(pps)},
                "pp_approx_vs_als_sweep": round(statistics.mean(als) / statistics.mean(pps), 2),
                "pp": runs["pp"], "als": runs["als"],
                "pp_vs_als_speedup": round(runs["als"]["value"] / runs["pp"]["value"], 3)}

    out = {"workload": f"tucker_order3_{s}_rank{R}: X = [[G; A1, A2, A3]] + 0.3 relative noise, "
                       f"random orthonormal start, {sweeps} sweeps",
           "fp64": one("fp64", p)}
    out["mixed"] = one("mixed", p)
    out["mixed"]["note"] = "first-level TTMs on the tensor cores (X bf16, factor hi + lo), the rest float64"
    # order 4 (the generic contraction chains): 100^4, ranks 5 = 0.05 s, float64
    p4 = synth.tucker_problem([100] * 4, [5] * 4, seed=dist.rank, noise=0.3)
    out["order4"] = {"workload": f"tucker_order4_100_rank5: X = [[G; A1..A4]] + 0.3 relative noise, "
                                 f"random orthonormal start, {sweeps} sweeps", "fp64": one("fp64", p4)}
    return out


def run_variants(args, dist, p, Xd, flush, max_sweeps, prec):
    import numpy as np
    import torch

    from paper_1811_10573_gb300 import cpals, synth

    def timed(g, A0, eps, target):
        g.init_factors(A0)
        flush.zero_()
        torch.cuda.synchronize()
        dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = g.run(max_sweeps, eps, True, target)
        e1.record()
        torch.cuda.synchronize()
        return dist.max(e0.elapsed_time(e1) / 1e3), out

    def one_variant(q, X, setup, note):
        with cpals.CPALS(q.dims, q.R, "fp64") as g64:
            prep(g64)
            g64.set_tensor(X)
            setup(g64)
            g64.init_factors(q.A0)
            f_star = float(g64.run(q.sweeps, 0.0, True, 0.0)["fitness"][-1])
        target = f_star - 1e-6
        res = {"note": note, "target_fitness": target}
        with cpals.CPALS(q.dims, q.R, prec) as g:
            g.set_tensor(X)
            prep(g)
            setup(g)
            for kind, eps in (("pp", q.eps), ("als", 0.0)):
                ts, ok = [], True
                for i in range(3):
                    dt, out = timed(g, q.A0, eps, target)
                    if i == 0:
                        continue                    # warm-up (graph capture)
                    ts.append(dt)
                    ok = ok and out["reached"]
                kinds = out["kinds"]
                res[kind] = {"value": round(float(np.mean(ts)), 6), "unit": "s", "reached": ok,
                             "sweeps": len(kinds), "final_fitness": float(out["fitness"][-1]),
                             "sweep_counts": {k: kinds.count(k) for k in ("als", "pp_init", "pp_approx")}}
        res["pp_vs_als_speedup"] = round(res["als"]["value"] / res["pp"]["value"], 3)
        return res

    out = {}
    out["step_size_0.7"] = one_variant(
        p, Xd, lambda g: g.set_step_size(0.7),
        f"{p.name}, every mode A_new = 0.3 A + 0.7 M Gamma^-1")
    q = synth.symmetric_order3(400, 400, 100, seed=dist.rank, collinearity=0.7, eps=p.eps,
                               sweeps=p.sweeps)
    Xs = torch.from_numpy(np.ascontiguousarray(q.X)).cuda()

    def sym(g):
        g.set_symmetric(1, 2)
        g.set_step_size([1.0, 0.8, 1.0])
    out["symmetric_ABB"] = one_variant(
        q, Xs, sym, f"{q.name} (X = [[A, B, B]] + 1e-2 relative symmetric noise, collinearity "
        "0.7), A plain update, B step 0.8")
    del Xs
    return out


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores, on the headline's workload and
    metric: each step times one of each oracle step (ALS sweep, operator
    build, PP sweep, exact fitness) on the full seed-0 tensor and projects
    them onto the oracle's own schedule to the target."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workload(args.workload, seed=0)
    counts, how = oracle_counts(args.workload)
    if counts is None:
        counts, how = counts_of(["als"] * p.sweeps), f"the workload's sweep budget ({p.sweeps} ALS sweeps)"
    vals = []
    ts = None
    for i in range(args.warmup + args.steps):
        ts = oracle_sample(args.workload, 0)
        if i >= args.warmup:
            vals.append(project(ts, counts))
    value = statistics.mean(vals)
    sample = ("float64 numpy oracle on the full seed-0 workload, each step one ALS sweep, one PP "
              f"operator build, one PP sweep and one exact fitness, projected onto {how} {counts}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(value * 1e3, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": p.name, "dims": p.dims, "R": p.R, "eps": p.eps},
        "cpu_baseline": {"value": round(value, 4), "unit": "s", "cores": oracle_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "last_sample_seconds": ts,
    }))


def run_batch_only(args):
    """The 256-tensor batch entry alone: fused batch in float32 and float64
    against per-tensor contexts; the line's value is the fused float32
    batch's decompositions per second."""
    import torch

    from paper_1811_10573_gb300 import build, cpals, harness

    dist = harness.init()
    torch.cuda.set_device(dist.local_rank)
    build.build()
    cpals.lib()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = run_batch_bench(args, dist, flush, args.precision)
    if dist.rank == 0:
        v = out["fused_fp32"]["decompositions_per_s"] * dist.world
        print(json.dumps({"metric": "decompositions_per_s", "value": v, "unit": "1/s",
                          "n_gpus": dist.world, "higher_is_better": True, "scaling": "weak",
                          "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "batch_order3_256"}, "batch": out}))


if __name__ == "__main__":
    a = parse()
    HOST_LOOP = a.host_loop
    if a.impl == "reference":
        run_reference(a)
    elif a.batch_only:
        run_batch_only(a)
    else:
        run_ours(a)
