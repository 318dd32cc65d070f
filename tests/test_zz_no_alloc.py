"""The allocation-free tensor-core contraction (cpals_contract_bf16_noalloc).

It exists for callers that cannot allocate device memory when they need the
contraction (a framework that owns all device memory through its own pool, a
latency-critical loop that cannot pay for cudaMalloc's synchronisation, a
process whose memory budget is committed): its split-K partial sums live in a
fixed file-scope device array instead of a context workspace.

The test builds the bf16 inputs on the device, calls the entry point through
the C ABI twice in a row on different problems, and checks each output
against the existing entry point that runs the same contraction
(cpals_mttkrp of the last mode of an order-3 MIXED_BF16 context, which is the
split-K contraction X_(01)^T (A^(0) (.) A^(1)) with nothing after it), within
the 2e-5 bound the tensor-core tests use.  It also checks that a call whose
partial sums would not fit the array is rejected.  This file is collected
last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _splits(K, M, R, batch=1):
    """The split count the context path picks for this shape."""
    mtiles = -(-M // 128) * batch
    if mtiles >= 2 * 152:
        return 1
    return max(1, min(-(-2 * 152 // mtiles), -(-K // 256)))


def _inputs(p):
    s0, s1, s2 = p.dims
    R = p.R
    X = torch.from_numpy(np.ascontiguousarray(p.X)).cuda()
    Xb = X.to(torch.bfloat16).contiguous()
    A0 = torch.from_numpy(p.A0[0]).float().cuda()
    A1 = torch.from_numpy(p.A0[1]).float().cuda()
    K = s0 * s1
    v = (A0[:, None, :] * A1[None, :, :]).reshape(K, R)        # float32 products
    hi = v.to(torch.bfloat16)
    lo = (v - hi.float()).to(torch.bfloat16)
    Rpad = -(-R // 16) * 16
    Kstride = -(-K // 8) * 8
    Bt = torch.zeros((2, Rpad, Kstride), dtype=torch.bfloat16, device="cuda")
    Bt[0, :R, :K] = hi.t()
    Bt[1, :R, :K] = lo.t()
    return X, Xb, Bt, K, s2, Kstride


@pytest.mark.parametrize("first,second", [(([64, 48, 40], 100, 1), ([96, 80, 64], 50, 2))])
def test_noalloc_matches_context_contraction_twice(first, second):
    outs = []
    for dims, R, seed in (first, second):
        p = synth.make_problem("normal", dims, R, seed=seed, storage="f32")
        X, Xb, Bt, K, M, Kstride = _inputs(p)
        out = torch.empty((M, R), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        st = cpals.cpals_contract_bf16_noalloc(Xb.data_ptr(), Bt.data_ptr(), out.data_ptr(), 1,
                                               K, M, R, Kstride, False, _splits(K, M, R))
        assert st == 0, cpals.STATUS.get(st, st)
        with cpals.CPALS(p.dims, R, "mixed") as g:
            g.set_tensor(X)
            g.init_factors(p.A0)
            ref = g.mttkrp(2)
        got = out.double().cpu().numpy()
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert err < 2e-5, err
        outs.append(got)
    assert outs[0].shape != outs[1].shape


def test_noalloc_rejects_scratch_overflow():
    p = synth.make_problem("normal", [64, 48, 40], 100, seed=3, storage="f32")
    X, Xb, Bt, K, M, Kstride = _inputs(p)
    out = torch.empty((M, 100), dtype=torch.float32, device="cuda")
    too_many = cpals.NOALLOC_SCRATCH_FLOATS // (M * 100) + 1
    st = cpals.cpals_contract_bf16_noalloc(Xb.data_ptr(), Bt.data_ptr(), out.data_ptr(), 1, K, M,
                                           100, Kstride, False, too_many)
    assert st == 1          # CPALS_E_INVALID
