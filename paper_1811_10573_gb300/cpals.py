"""Thin ctypes binding of libcpals (include/cpals.h).

Argument marshalling only: every step of CP-ALS / PP-CP-ALS runs in the CUDA
library.  The module-level functions carry the C ABI's names; ``CPALS`` wraps
them for convenience.  Importing this module never falls back to anything:
if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpals.so")

FP64, FP32, MIXED_BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED_BF16, "mixed_bf16": MIXED_BF16}
SWEEP_KINDS = {0: "als", 1: "pp_init", 2: "pp_approx"}
STATUS = {0: "OK", 1: "E_INVALID", 2: "E_OOM", 3: "E_CUDA", 4: "E_STATE", 5: "E_SINGULAR",
          6: "E_NUMERIC", 7: "E_TIMEOUT", 8: "E_UNSUPPORTED"}

_lib = None
_ctx_p = C.c_void_p
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)

_SIGS = {
    "cpals_create": (C.c_int, [_i64p, C.c_int, C.c_int, C.c_int, C.POINTER(_ctx_p)]),
    "cpals_destroy": (None, [_ctx_p]),
    "cpals_set_stream": (C.c_int, [_ctx_p, C.c_void_p]),
    "cpals_set_tensor": (C.c_int, [_ctx_p, C.c_void_p, C.c_int, C.c_int]),
    "cpals_init_factors": (C.c_int, [_ctx_p, C.POINTER(_dp)]),
    "cpals_als_sweep": (C.c_int, [_ctx_p, _dp]),
    "cpals_pp_build_operators": (C.c_int, [_ctx_p]),
    "cpals_pp_sweep": (C.c_int, [_ctx_p, C.c_int, _dp]),
    "cpals_fitness": (C.c_int, [_ctx_p, _dp]),
    "cpals_get_factors": (C.c_int, [_ctx_p, C.POINTER(_dp)]),
    "cpals_get_dA_ratios": (C.c_int, [_ctx_p, _dp]),
    "cpals_pinv_modes": (C.c_int, [_ctx_p, _ip]),
    "cpals_run_batch": (C.c_int, [C.POINTER(_ctx_p), C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                  _dp, _dp, _ip, _ip]),
    "cpals_run": (C.c_int, [_ctx_p, C.c_int, C.c_double, C.c_int, C.c_double, _dp, _ip, _dp,
                            _ip, _ip]),
    "cpals_last_error": (C.c_char_p, [_ctx_p]),
    "cpals_mttkrp": (C.c_int, [_ctx_p, C.c_int, _dp]),
    "cpals_get_operator": (C.c_int, [_ctx_p, C.c_int, C.c_int, _dp]),
    "cpals_pp_mttkrp": (C.c_int, [_ctx_p, C.c_int, C.c_int, _dp]),
    "cpals_get_state": (C.c_int, [_ctx_p, C.c_int, C.c_int, _dp]),
    "cpals_normal_solve": (C.c_int, [_ctx_p, C.c_int, _dp, _dp]),
    "cpals_set_profiling": (C.c_int, [_ctx_p, C.c_int]),
    "cpals_reset_stats": (C.c_int, [_ctx_p]),
    "cpals_get_stats": (C.c_int, [_ctx_p, C.c_int, _i64p, _dp, _dp, _dp]),
    "cpals_set_graphs": (C.c_int, [_ctx_p, C.c_int]),
    "cpals_set_wait_limit": (C.c_int, [_ctx_p, C.c_uint64]),
    "cpals_set_device_loop": (C.c_int, [_ctx_p, C.c_int]),
    "cpals_set_pp_stop_tol": (C.c_int, [_ctx_p, C.c_double]),
    "cpals_batch_create": (C.c_int, [C.c_int, _i64p, _ip, C.c_int, C.POINTER(_ctx_p)]),
    "cpals_batch_destroy": (None, [_ctx_p]),
    "cpals_batch_set_tensor": (C.c_int, [_ctx_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "cpals_batch_init_factors": (C.c_int, [_ctx_p, C.c_int, C.POINTER(_dp)]),
    "cpals_batch_run": (C.c_int, [_ctx_p, C.c_int, C.c_double, C.c_int, C.c_double, _dp, _ip, _ip, _ip,
                                  _dp]),
    "cpals_batch_get_factors": (C.c_int, [_ctx_p, C.c_int, C.POINTER(_dp)]),
    "cpals_batch_stats": (C.c_int, [_ctx_p, _i64p, _i64p]),
    "cpals_batch_last_error": (C.c_char_p, [_ctx_p]),
    "cpals_batch_tiles": (C.c_int, [_ctx_p, _ip, _fp, _ip]),
    "cpals_device_loop_active": (C.c_int, [_ctx_p]),
    "cpals_set_normal_arith": (C.c_int, [_ctx_p, C.c_int]),
    "cpals_set_step_size": (C.c_int, [_ctx_p, _dp]),
    "cpals_set_symmetric": (C.c_int, [_ctx_p, C.c_int, C.c_int]),
    "cpals_set_controller": (C.c_int, [_ctx_p, _fp, C.c_int, C.c_double]),
    "cpals_tucker_create": (C.c_int, [_i64p, C.c_int, _ip, C.POINTER(_ctx_p)]),
    "cpals_tucker_destroy": (None, [_ctx_p]),
    "cpals_tucker_set_iterations": (C.c_int, [_ctx_p, C.c_int]),
    "cpals_tucker_set_precision": (C.c_int, [_ctx_p, C.c_int]),
    "cpals_tucker_set_tensor": (C.c_int, [_ctx_p, C.c_void_p, C.c_int, C.c_int]),
    "cpals_tucker_init_factors": (C.c_int, [_ctx_p, C.POINTER(_dp)]),
    "cpals_tucker_als_sweep": (C.c_int, [_ctx_p, _dp]),
    "cpals_tucker_pp_build_operators": (C.c_int, [_ctx_p]),
    "cpals_tucker_pp_sweep": (C.c_int, [_ctx_p, _dp]),
    "cpals_tucker_run": (C.c_int, [_ctx_p, C.c_int, C.c_double, _dp, _ip, _ip]),
    "cpals_tucker_fitness": (C.c_int, [_ctx_p, _dp]),
    "cpals_tucker_get_factors": (C.c_int, [_ctx_p, C.POINTER(_dp)]),
    "cpals_tucker_get_core": (C.c_int, [_ctx_p, _dp]),
    "cpals_tucker_last_error": (C.c_char_p, [_ctx_p]),
    "cpals_tucker_cost_model": (C.c_int, [_i64p, _ip, C.c_int, _dp]),
    "cpals_run_controlled": (C.c_int, [_ctx_p, C.c_int, C.c_double, C.c_int, C.c_double, _dp,
                                       _ip, _dp, _ip, _ip, _ip]),
    "cpals_set_controller_labels": (C.c_int, [_ctx_p, C.c_double, C.c_int]),
    "cpals_controller_last": (C.c_int, [_ctx_p, _fp, _fp]),
    "cpals_controller_log": (C.c_int, [_ctx_p, C.c_int, C.c_double, C.c_int, _fp, _ip, _dp, _dp,
                                       _ip]),
    "cpals_mlp_train": (C.c_int, [_fp, _ip, _fp, C.c_int, _fp, C.c_int, C.c_int, C.c_double,
                                  C.c_double, _dp]),
    "cpals_mlp_forward": (C.c_int, [_fp, C.c_int, _fp, C.c_int, _fp]),
    "cpals_cost_model": (C.c_int, [_i64p, C.c_int, C.c_int, C.c_int, _dp]),
    "cpals_contract_bf16_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                             C.c_int64, C.c_int64, C.c_int, C.c_int64, C.c_int,
                                             C.c_int, C.c_void_p]),
}
NOALLOC_SCRATCH_FLOATS = 4 << 20


def lib():
    """Load libcpals.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1811_10573_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CPALSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a):
    return a.ctypes.data_as(_dp)


# ---------------------------------------------------------------- C names
def cpals_create(dims, N, R, precision):
    d = (C.c_int64 * N)(*[int(x) for x in dims])
    out = _ctx_p()
    st = lib().cpals_create(d, N, R, precision, C.byref(out))
    return st, out


def cpals_destroy(ctx):
    lib().cpals_destroy(ctx)


def cpals_last_error(ctx):
    s = lib().cpals_last_error(ctx)
    return s.decode() if s else ""


def cpals_set_stream(ctx, stream):
    return lib().cpals_set_stream(ctx, C.c_void_p(int(stream)))


def cpals_set_tensor(ctx, ptr, dtype, on_device):
    return lib().cpals_set_tensor(ctx, C.c_void_p(int(ptr)), dtype, on_device)


def cpals_init_factors(ctx, factors):
    arr = (_dp * len(factors))(*[_dptr(f) for f in factors])
    return lib().cpals_init_factors(ctx, arr)


def cpals_als_sweep(ctx, fit):
    return lib().cpals_als_sweep(ctx, fit)


def cpals_pp_build_operators(ctx):
    return lib().cpals_pp_build_operators(ctx)


def cpals_pp_sweep(ctx, use_V, fit):
    return lib().cpals_pp_sweep(ctx, use_V, fit)


def cpals_fitness(ctx, out):
    return lib().cpals_fitness(ctx, out)


def cpals_get_factors(ctx, outs):
    arr = (_dp * len(outs))(*[_dptr(o) for o in outs])
    return lib().cpals_get_factors(ctx, arr)


def cpals_get_dA_ratios(ctx, out):
    return lib().cpals_get_dA_ratios(ctx, _dptr(out))


def cpals_pinv_modes(ctx, mask):
    return lib().cpals_pinv_modes(ctx, C.byref(mask))


def cpals_run(ctx, max_sweeps, eps, use_V, target, ftrace, ktrace, ttrace, n_done, reached):
    return lib().cpals_run(ctx, max_sweeps, eps, use_V, target, ftrace, ktrace, ttrace, n_done,
                           reached)


def cpals_run_batch(ctxs, n, workers, max_sweeps, eps, use_V, targets, fit, sweeps, status):
    return lib().cpals_run_batch(ctxs, n, workers, max_sweeps, eps, use_V, targets, fit, sweeps,
                                 status)


def run_batch(contexts, workers, max_sweeps, eps, use_V=True, targets=None):
    """Run Algorithm 3 on many contexts at once (cpals_run_batch).  Returns
    per-instance final fitness, sweeps run and status (numpy arrays)."""
    n = len(contexts)
    arr = (_ctx_p * max(n, 1))(*[c.ctx for c in contexts])
    fit = np.zeros(max(n, 1))
    sw = np.zeros(max(n, 1), dtype=np.int32)
    st = np.zeros(max(n, 1), dtype=np.int32)
    tg = None
    if targets is not None:
        tg = np.ascontiguousarray(targets, dtype=np.float64)
    rc = cpals_run_batch(arr, n, int(workers), int(max_sweeps), float(eps), 1 if use_V else 0,
                         _dptr(tg) if tg is not None else None, _dptr(fit),
                         sw.ctypes.data_as(_ip), st.ctypes.data_as(_ip))
    if rc != 0:
        raise CPALSError(rc, "cpals_run_batch: bad arguments")
    return fit[:n], sw[:n], st[:n]


CTRL_FEATURES = 20
CTRL_PARAMS = 32 * CTRL_FEATURES + 32 + 3 * 32 + 3
CTRL_ACTIONS = ["pp", "als", "rebuild"]


def _fptr(a):
    return a.ctypes.data_as(_fp)


def cpals_set_controller(ctx, params, nparams, confidence):
    return lib().cpals_set_controller(ctx, params, nparams, confidence)


def cpals_run_controlled(ctx, max_sweeps, eps, use_V, target, ftrace, ktrace, ttrace, strace,
                         n_done, reached):
    return lib().cpals_run_controlled(ctx, max_sweeps, eps, use_V, target, ftrace, ktrace, ttrace,
                                      strace, n_done, reached)


def cpals_controller_last(ctx, features, probs):
    return lib().cpals_controller_last(ctx, features, probs)


def cpals_set_controller_labels(ctx, target, max_rollout):
    return lib().cpals_set_controller_labels(ctx, target, max_rollout)


def cpals_controller_log(ctx, steps, eps, use_V, features, labels, gains, costs, n_out):
    return lib().cpals_controller_log(ctx, steps, eps, use_V, features, labels, gains, costs, n_out)


def cpals_mlp_train(X, y, w, n, params, nparams, epochs, lr, decay, loss_out):
    return lib().cpals_mlp_train(X, y, w, n, params, nparams, epochs, lr, decay, loss_out)


def cpals_mlp_forward(params, nparams, X, n, probs):
    return lib().cpals_mlp_forward(params, nparams, X, n, probs)


def mlp_train(X, y, w, params, epochs=2000, lr=1e-2, decay=1e-4):
    """Train the controller network (cpals_mlp_train); returns (params, loss)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    p = np.ascontiguousarray(params, dtype=np.float32).copy()
    loss = C.c_double()
    st = cpals_mlp_train(_fptr(X), y.ctypes.data_as(_ip), _fptr(w), len(y), _fptr(p), p.size,
                         epochs, lr, decay, C.byref(loss))
    if st != 0:
        raise CPALSError(st, "cpals_mlp_train")
    return p, loss.value


def mlp_forward(params, X):
    """Controller probabilities for feature rows X (cpals_mlp_forward)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    out = np.empty((X.shape[0], 3), dtype=np.float32)
    st = cpals_mlp_forward(_fptr(p), p.size, _fptr(X), X.shape[0], _fptr(out))
    if st != 0:
        raise CPALSError(st, "cpals_mlp_forward")
    return out


def cpals_mttkrp(ctx, n, out):
    return lib().cpals_mttkrp(ctx, n, _dptr(out))


def cpals_get_operator(ctx, i, n, out):
    return lib().cpals_get_operator(ctx, i, n, _dptr(out))


def cpals_pp_mttkrp(ctx, n, use_V, out):
    return lib().cpals_pp_mttkrp(ctx, n, use_V, _dptr(out))


def cpals_normal_solve(ctx, n, rhs, out):
    return lib().cpals_normal_solve(ctx, n, _dptr(rhs), _dptr(out))


def cpals_get_state(ctx, which, n, out):
    return lib().cpals_get_state(ctx, which, n, _dptr(out))


def cpals_set_profiling(ctx, enable):
    return lib().cpals_set_profiling(ctx, enable)


def cpals_reset_stats(ctx):
    return lib().cpals_reset_stats(ctx)


def cpals_get_stats(ctx, kind):
    n = C.c_int64()
    ms, b, f = C.c_double(), C.c_double(), C.c_double()
    st = lib().cpals_get_stats(ctx, kind, C.byref(n), C.byref(ms), C.byref(b), C.byref(f))
    return st, n.value, ms.value, b.value, f.value


def cpals_set_graphs(ctx, enable):
    return lib().cpals_set_graphs(ctx, enable)


NORMAL_ARITH = {"fp64": 0, "double_float": 1}


def cpals_set_pp_stop_tol(ctx, tol):
    return lib().cpals_set_pp_stop_tol(ctx, float(tol))


def cpals_set_device_loop(ctx, enable):
    return lib().cpals_set_device_loop(ctx, enable)


def cpals_device_loop_active(ctx):
    return lib().cpals_device_loop_active(ctx)


def cpals_set_wait_limit(ctx, cycles):
    return lib().cpals_set_wait_limit(ctx, int(cycles))


def cpals_set_normal_arith(ctx, arith):
    return lib().cpals_set_normal_arith(ctx, arith)


def cpals_set_step_size(ctx, lam):
    return lib().cpals_set_step_size(ctx, lam)


def cpals_set_symmetric(ctx, m1, m2):
    return lib().cpals_set_symmetric(ctx, m1, m2)


def cpals_cost_model(dims, N, R, kind):
    d = (C.c_int64 * N)(*[int(x) for x in dims])
    out = C.c_double()
    st = lib().cpals_cost_model(d, N, R, kind, C.byref(out))
    if st != 0:
        raise CPALSError(st, "cost model: bad sizes")
    return out.value


def cpals_contract_bf16_noalloc(Xb, Bt, out, batch, K, M, R, Kstride, kmajor, splits, stream=0):
    """Device pointers (ints) in, status out; see include/cpals.h."""
    return lib().cpals_contract_bf16_noalloc(C.c_void_p(int(Xb)), C.c_void_p(int(Bt)),
                                             C.c_void_p(int(out)), batch, K, M, R, Kstride,
                                             1 if kmajor else 0, splits, C.c_void_p(int(stream)))


# ---------------------------------------------------------------- convenience wrapper
class CPALS:
    """One decomposition context (owns its device memory)."""

    def __init__(self, dims, R, precision="fp64", stream=None):
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims)
        self.R = int(R)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        st, ctx = cpals_create(self.dims, self.N, self.R, prec)
        if st != 0:
            raise CPALSError(st, "cpals_create failed")
        self.ctx = ctx
        if stream is not None:
            self._ck(cpals_set_stream(ctx, stream))

    def _ck(self, st):
        if st != 0:
            raise CPALSError(st, cpals_last_error(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            cpals_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        self._ck(cpals_set_stream(self.ctx, stream))

    def set_tensor(self, X):
        """X: numpy array (host) or torch tensor (host or CUDA), float64/float32."""
        if hasattr(X, "data_ptr"):          # torch tensor
            import torch
            assert X.is_contiguous()
            dt = {torch.float64: 0, torch.float32: 1}[X.dtype]
            self._ck(cpals_set_tensor(self.ctx, X.data_ptr(), dt, 1 if X.is_cuda else 0))
            return
        X = np.ascontiguousarray(X)
        dt = {np.dtype(np.float64): 0, np.dtype(np.float32): 1}[X.dtype]
        self._ck(cpals_set_tensor(self.ctx, X.ctypes.data, dt, 0))

    def init_factors(self, factors):
        fs = [_f64(f) for f in factors]
        for f, s in zip(fs, self.dims):
            assert f.shape == (s, self.R)
        self._ck(cpals_init_factors(self.ctx, fs))

    def als_sweep(self):
        f = C.c_double()
        self._ck(cpals_als_sweep(self.ctx, C.byref(f)))
        return f.value

    def pp_build_operators(self):
        self._ck(cpals_pp_build_operators(self.ctx))

    def pp_sweep(self, use_V=True):
        f = C.c_double()
        self._ck(cpals_pp_sweep(self.ctx, 1 if use_V else 0, C.byref(f)))
        return f.value

    def fitness(self):
        f = C.c_double()
        self._ck(cpals_fitness(self.ctx, C.byref(f)))
        return f.value

    def get_factors(self):
        outs = [np.empty((s, self.R)) for s in self.dims]
        self._ck(cpals_get_factors(self.ctx, outs))
        return outs

    def get_dA_ratios(self):
        out = np.empty(self.N)
        self._ck(cpals_get_dA_ratios(self.ctx, out))
        return out

    def pinv_modes(self):
        """Bit n: the last update of mode n went through Gamma^dagger."""
        m = C.c_int()
        self._ck(cpals_pinv_modes(self.ctx, m))
        return m.value

    def run(self, max_sweeps, eps, use_V=True, target=0.0):
        ft = np.zeros(max_sweeps)
        kt = np.zeros(max_sweeps, dtype=np.int32)
        tt = np.zeros(max_sweeps)
        nd, rc = C.c_int(), C.c_int()
        self._ck(cpals_run(self.ctx, max_sweeps, eps, 1 if use_V else 0, target, _dptr(ft),
                           kt.ctypes.data_as(_ip), _dptr(tt), C.byref(nd), C.byref(rc)))
        n = nd.value
        return {"fitness": ft[:n], "kinds": [SWEEP_KINDS[int(k)] for k in kt[:n]],
                "times": tt[:n], "reached": bool(rc.value)}

    def set_controller(self, params, confidence=0.6):
        """Install the learned sweep-type controller (None removes it)."""
        if params is None:
            self._ck(cpals_set_controller(self.ctx, None, 0, confidence))
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._ck(cpals_set_controller(self.ctx, _fptr(p), p.size, confidence))

    def run_controlled(self, max_sweeps, eps, use_V=True, target=0.0):
        ft = np.zeros(max_sweeps)
        kt = np.zeros(max_sweeps, dtype=np.int32)
        tt = np.zeros(max_sweeps)
        st = np.zeros(max_sweeps, dtype=np.int32)
        nd, rc = C.c_int(), C.c_int()
        self._ck(cpals_run_controlled(self.ctx, max_sweeps, eps, 1 if use_V else 0, target,
                                      _dptr(ft), kt.ctypes.data_as(_ip), _dptr(tt),
                                      st.ctypes.data_as(_ip), C.byref(nd), C.byref(rc)))
        n = nd.value
        return {"fitness": ft[:n], "kinds": [SWEEP_KINDS[int(k)] for k in kt[:n]],
                "times": tt[:n], "learned": st[:n].astype(bool), "reached": bool(rc.value)}

    def controller_last(self):
        """Input and output of the controller's last decision (cpals_controller_last)."""
        x = np.zeros(CTRL_FEATURES, dtype=np.float32)
        pr = np.zeros(3, dtype=np.float32)
        self._ck(cpals_controller_last(self.ctx, _fptr(x), _fptr(pr)))
        return x, pr

    def set_controller_labels(self, target, max_rollout=0):
        """Label the controller log by the time to `target` (0: four-sweep
        gain per second); cpals_set_controller_labels."""
        self._ck(cpals_set_controller_labels(self.ctx, float(target), int(max_rollout)))

    def controller_log(self, steps, eps, use_V=True):
        """Self-generated training log (cpals_controller_log)."""
        f = np.zeros((steps, CTRL_FEATURES), dtype=np.float32)
        lab = np.zeros(steps, dtype=np.int32)
        g = np.zeros((steps, 3))
        c = np.zeros((steps, 3))
        n = C.c_int()
        st = cpals_controller_log(self.ctx, steps, eps, 1 if use_V else 0, _fptr(f),
                                  lab.ctypes.data_as(_ip), _dptr(g), _dptr(c), C.byref(n))
        if st not in (0, 5):          # a singular Gamma ends the log early; the rest stands
            self._ck(st)
        k = n.value
        return {"features": f[:k], "labels": lab[:k], "gains": g[:k], "costs": c[:k],
                "status": STATUS.get(st, st)}

    def mttkrp(self, n):
        out = np.empty((self.dims[n], self.R))
        self._ck(cpals_mttkrp(self.ctx, n, out))
        return out

    def get_operator(self, i, n):
        shape = (self.dims[n], self.R) if i == n else (self.dims[i], self.dims[n], self.R)
        out = np.empty(shape)
        self._ck(cpals_get_operator(self.ctx, i, n, out))
        return out

    def pp_mttkrp(self, n, use_V=True):
        out = np.empty((self.dims[n], self.R))
        self._ck(cpals_pp_mttkrp(self.ctx, n, 1 if use_V else 0, out))
        return out

    def normal_solve(self, n, rhs):
        rhs = _f64(rhs)
        out = np.empty((self.dims[n], self.R))
        self._ck(cpals_normal_solve(self.ctx, n, rhs, out))
        return out

    def get_state(self, which, n):
        out = np.empty((self.dims[n], self.R))
        self._ck(cpals_get_state(self.ctx, {"Ap": 0, "dA": 1}[which], n, out))
        return out

    def set_profiling(self, enable):
        self._ck(cpals_set_profiling(self.ctx, 1 if enable else 0))

    def reset_stats(self):
        self._ck(cpals_reset_stats(self.ctx))

    def get_stats(self, kind=0):
        st, n, ms, b, f = cpals_get_stats(self.ctx, kind)
        self._ck(st)
        return {"launches": n, "total_ms": ms, "bytes": b, "flops": f}

    def set_graphs(self, enable):
        self._ck(cpals_set_graphs(self.ctx, 1 if enable else 0))

    def set_pp_stop_tol(self, tol):
        """Fitness gain a PP sweep must make for its PP run to go on (0 = no test)."""
        self._ck(cpals_set_pp_stop_tol(self.ctx, tol))

    def set_device_loop(self, enable):
        """Algorithm 3's decisions on the device (True, default) or the host."""
        self._ck(cpals_set_device_loop(self.ctx, 1 if enable else 0))

    def device_loop_active(self):
        return bool(cpals_device_loop_active(self.ctx))

    def set_wait_limit(self, cycles):
        """Bound of the tensor-core kernel's waits in SM cycles (0 = default)."""
        self._ck(cpals_set_wait_limit(self.ctx, cycles))

    def set_normal_arith(self, arith):
        """'fp64' or 'double_float' (see cpals_set_normal_arith); the factors
        must be set again afterwards."""
        a = NORMAL_ARITH[arith] if isinstance(arith, str) else int(arith)
        self._ck(cpals_set_normal_arith(self.ctx, a))

    def set_step_size(self, lam):
        """Update step size per mode (a scalar applies to all; None = 1),
        see cpals_set_step_size."""
        if lam is None:
            self._ck(cpals_set_step_size(self.ctx, None))
            return
        v = np.full(len(self.dims), float(lam)) if np.ndim(lam) == 0 else np.asarray(lam, float)
        self._lam = np.ascontiguousarray(v)
        self._ck(cpals_set_step_size(self.ctx, _dptr(self._lam)))

    def set_symmetric(self, m1, m2):
        """Tie mode m2's factor to mode m1's (see cpals_set_symmetric);
        (-1, -1) removes the ties.  The factors must be set again."""
        self._ck(cpals_set_symmetric(self.ctx, int(m1), int(m2)))


def cost_model(dims, R, kind):
    """Host-only flop model (see cpals_cost_model)."""
    return cpals_cost_model(dims, len(dims), R, kind)


# ---------------------------------------------------------------- Tucker (order 3, float64)
def cpals_tucker_create(dims, ranks):
    n = len(dims)
    d = (C.c_int64 * n)(*[int(x) for x in dims])
    r = (C.c_int * len(ranks))(*[int(x) for x in ranks])
    out = _ctx_p()
    st = lib().cpals_tucker_create(d, n, r, C.byref(out))
    return st, out


def cpals_tucker_destroy(t):
    lib().cpals_tucker_destroy(t)


def cpals_tucker_set_iterations(t, iters):
    return lib().cpals_tucker_set_iterations(t, iters)


def cpals_tucker_cost_model(dims, ranks, kind):
    d = (C.c_int64 * 3)(*[int(x) for x in dims])
    r = (C.c_int * 3)(*[int(x) for x in ranks])
    f = C.c_double()
    st = lib().cpals_tucker_cost_model(d, r, int(kind), C.byref(f))
    return st, f.value


def cpals_tucker_set_precision(t, precision):
    return lib().cpals_tucker_set_precision(t, precision)


def cpals_tucker_set_tensor(t, ptr, dtype, on_device):
    return lib().cpals_tucker_set_tensor(t, C.c_void_p(int(ptr)), dtype, on_device)


def cpals_tucker_init_factors(t, factors):
    arr = (_dp * len(factors))(*[_dptr(f) for f in factors])
    return lib().cpals_tucker_init_factors(t, arr)


def cpals_tucker_als_sweep(t, fit):
    return lib().cpals_tucker_als_sweep(t, fit)


def cpals_tucker_pp_build_operators(t):
    return lib().cpals_tucker_pp_build_operators(t)


def cpals_tucker_pp_sweep(t, fit):
    return lib().cpals_tucker_pp_sweep(t, fit)


def cpals_tucker_run(t, max_sweeps, eps, ftrace, ktrace, n_done):
    return lib().cpals_tucker_run(t, max_sweeps, eps, ftrace, ktrace, n_done)


def cpals_tucker_fitness(t, out):
    return lib().cpals_tucker_fitness(t, out)


def cpals_tucker_get_factors(t, out):
    return lib().cpals_tucker_get_factors(t, out)


def cpals_tucker_get_core(t, out):
    return lib().cpals_tucker_get_core(t, out)


def cpals_tucker_last_error(t):
    s = lib().cpals_tucker_last_error(t)
    return s.decode() if s else ""


class Tucker:
    """Tucker-ALS / PP-Tucker-ALS context in float64 for orders 3 to 8 (owns
    its device memory); precision "mixed" (order 3) puts the first-level
    TTMs on the tensor cores."""

    def __init__(self, dims, ranks, precision="fp64"):
        self.dims = [int(d) for d in dims]
        self.ranks = [int(r) for r in ranks]
        st, t = cpals_tucker_create(self.dims, self.ranks)
        if st != 0:
            raise CPALSError(st, "cpals_tucker_create failed")
        self.t = t
        if precision != "fp64":
            try:
                self._ck(cpals_tucker_set_precision(self.t, PRECISIONS[precision]))
            except Exception:
                self.close()
                raise

    def _ck(self, st):
        if st != 0:
            raise CPALSError(st, cpals_tucker_last_error(self.t))

    def close(self):
        if self.t:
            cpals_tucker_destroy(self.t)
            self.t = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_iterations(self, iters):
        self._ck(cpals_tucker_set_iterations(self.t, int(iters)))

    def set_tensor(self, X):
        if hasattr(X, "data_ptr"):
            import torch
            assert X.is_contiguous()
            dt = {torch.float64: 0, torch.float32: 1}[X.dtype]
            self._ck(cpals_tucker_set_tensor(self.t, X.data_ptr(), dt, 1 if X.is_cuda else 0))
            return
        X = np.ascontiguousarray(X)
        dt = {np.dtype(np.float64): 0, np.dtype(np.float32): 1}[X.dtype]
        self._ck(cpals_tucker_set_tensor(self.t, X.ctypes.data, dt, 0))

    def init_factors(self, factors):
        fs = [_f64(f) for f in factors]
        for f, s, r in zip(fs, self.dims, self.ranks):
            assert f.shape == (s, r)
        self._ck(cpals_tucker_init_factors(self.t, fs))

    def als_sweep(self):
        f = C.c_double()
        self._ck(cpals_tucker_als_sweep(self.t, C.byref(f)))
        return f.value

    def pp_build_operators(self):
        self._ck(cpals_tucker_pp_build_operators(self.t))

    def pp_sweep(self):
        f = C.c_double()
        self._ck(cpals_tucker_pp_sweep(self.t, C.byref(f)))
        return f.value

    def run(self, max_sweeps, eps):
        ft = np.zeros(max(max_sweeps, 1))
        kt = np.zeros(max(max_sweeps, 1), dtype=np.int32)
        nd = C.c_int()
        self._ck(cpals_tucker_run(self.t, int(max_sweeps), float(eps), _dptr(ft),
                                  kt.ctypes.data_as(_ip), C.byref(nd)))
        n = nd.value
        return {"fitness": ft[:n], "kinds": [SWEEP_KINDS[int(k)] for k in kt[:n]]}

    def fitness(self):
        f = C.c_double()
        self._ck(cpals_tucker_fitness(self.t, C.byref(f)))
        return f.value

    def get_factors(self):
        out = [np.empty((s, r)) for s, r in zip(self.dims, self.ranks)]
        arr = (_dp * len(out))(*[_dptr(o) for o in out])
        self._ck(cpals_tucker_get_factors(self.t, arr))
        return out

    def get_core(self):
        out = np.empty(tuple(self.ranks))
        self._ck(cpals_tucker_get_core(self.t, _dptr(out)))
        return out


# ---------------------------------------------------------------- batches of small problems
def cpals_batch_create(n, dims, ranks, precision, out):
    return lib().cpals_batch_create(n, dims, ranks, precision, out)


def cpals_batch_destroy(b):
    return lib().cpals_batch_destroy(b)


def cpals_batch_set_tensor(b, i, ptr, dtype, on_device):
    return lib().cpals_batch_set_tensor(b, i, ptr, dtype, on_device)


def cpals_batch_init_factors(b, i, factors):
    return lib().cpals_batch_init_factors(b, i, factors)


def cpals_batch_run(b, max_sweeps, eps, use_V, pp_stop_tol, fit, sweeps, status, kinds, trace):
    return lib().cpals_batch_run(b, max_sweeps, eps, use_V, pp_stop_tol, fit, sweeps, status, kinds, trace)


def cpals_batch_get_factors(b, i, outs):
    return lib().cpals_batch_get_factors(b, i, outs)


def cpals_batch_stats(b, launches_per_sweep, launches_last_run):
    return lib().cpals_batch_stats(b, launches_per_sweep, launches_last_run)


def cpals_batch_last_error(b):
    return lib().cpals_batch_last_error(b)


def cpals_batch_tiles(b, tiles, ms, from_cache):
    return lib().cpals_batch_tiles(b, tiles, ms, from_cache)


class Batch:
    """n order-3 problems run by Algorithm 3 together (cpals_batch_*): every
    sweep stage is one launch over all of them."""

    def __init__(self, dims, ranks, precision="fp32"):
        self.dims = [[int(d) for d in ds] for ds in dims]
        self.ranks = [int(r) for r in ranks]
        self.n = len(self.dims)
        assert len(self.ranks) == self.n and all(len(d) == 3 for d in self.dims)
        flat = np.ascontiguousarray(np.asarray(self.dims, dtype=np.int64).reshape(-1))
        rk = np.ascontiguousarray(np.asarray(self.ranks, dtype=np.int32))
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = _ctx_p()
        st = lib().cpals_batch_create(self.n, flat.ctypes.data_as(_i64p), rk.ctypes.data_as(_ip), prec,
                                      C.byref(h))
        if st != 0:
            raise CPALSError(st, "cpals_batch_create failed")
        self.h = h

    def _ck(self, st):
        if st != 0:
            msg = lib().cpals_batch_last_error(self.h)
            raise CPALSError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            lib().cpals_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_tensor(self, i, X):
        if hasattr(X, "data_ptr"):
            import torch
            assert X.is_contiguous()
            dt = {torch.float64: 0, torch.float32: 1}[X.dtype]
            self._ck(lib().cpals_batch_set_tensor(self.h, i, X.data_ptr(), dt, 1 if X.is_cuda else 0))
            return
        X = np.ascontiguousarray(X)
        dt = {np.dtype(np.float64): 0, np.dtype(np.float32): 1}[X.dtype]
        self._ck(lib().cpals_batch_set_tensor(self.h, i, X.ctypes.data, dt, 0))

    def init_factors(self, i, factors):
        fs = [_f64(f) for f in factors]
        for f, s in zip(fs, self.dims[i]):
            assert f.shape == (s, self.ranks[i])
        arr = (_dp * 3)(*[f.ctypes.data_as(_dp) for f in fs])
        self._ck(lib().cpals_batch_init_factors(self.h, i, arr))

    def run(self, max_sweeps, eps, use_V=True, pp_stop_tol=0.0):
        fit = np.zeros(self.n)
        sw = np.zeros(self.n, dtype=np.int32)
        st = np.zeros(self.n, dtype=np.int32)
        kt = np.zeros((self.n, max_sweeps), dtype=np.int32)
        ft = np.zeros((self.n, max_sweeps))
        self._ck(lib().cpals_batch_run(self.h, max_sweeps, eps, 1 if use_V else 0, pp_stop_tol, _dptr(fit),
                                       sw.ctypes.data_as(_ip), st.ctypes.data_as(_ip),
                                       kt.ctypes.data_as(_ip), _dptr(ft)))
        kinds = [[SWEEP_KINDS[int(k)] for k in kt[i, :sw[i]]] for i in range(self.n)]
        return {"fitness": fit, "sweeps": sw, "status": st, "kinds": kinds,
                "trace": [ft[i, :sw[i]] for i in range(self.n)]}

    def get_factors(self, i):
        outs = [np.empty((s, self.ranks[i])) for s in self.dims[i]]
        arr = (_dp * 3)(*[o.ctypes.data_as(_dp) for o in outs])
        self._ck(lib().cpals_batch_get_factors(self.h, i, arr))
        return outs

    def stats(self):
        a, b = C.c_int64(), C.c_int64()
        self._ck(lib().cpals_batch_stats(self.h, C.byref(a), C.byref(b)))
        return {"launches_per_sweep": a.value, "launches_last_run": b.value}

    def tiles(self):
        """The autotuner's tile choice for the four contraction stages."""
        t = np.zeros(4, dtype=np.int32)
        ms = np.zeros(12, dtype=np.float32)
        fc = C.c_int()
        self._ck(lib().cpals_batch_tiles(self.h, t.ctypes.data_as(_ip), ms.ctypes.data_as(_fp), C.byref(fc)))
        return {"tiles": t.tolist(), "ms": ms.tolist(), "from_cache": bool(fc.value)}
