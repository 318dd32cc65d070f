"""The allocation-free tensor-core contraction (cpals_contract_bf16_noalloc).

It exists for callers that cannot allocate device memory when they need the
contraction (a framework that owns all device memory through its own pool, a
latency-critical loop that cannot pay for cudaMalloc's synchronisation, a
process whose memory budget is committed): its split-K partial sums live in a
fixed file-scope device array instead of a context workspace.

The tests build the bf16 inputs on the device and call the entry point
through the C ABI, two calls in a row on different problems.  Each output is
checked against a host emulation that takes the library's rounding decisions
(X rounded to bf16, the B operand as hi + lo bf16 planes of its float32
values) and contracts them in float64: what remains is the tensor cores' fp32
accumulation, 2e-5 relative to max |ref| (the bound of the tensor-core
tests).  The shapes cover every path the header documents: the MN-major
layout with split-K partials in the scratch array, the K-major layout (2-D
tensor map), a batched middle-mode contraction (3-D map) and a single K chunk
that writes the output directly.  A call whose partial sums would not fit the
array is rejected, and one whose requested split count the kernel would round
down to a count that fits is accepted.  This file is collected last on
purpose.
"""
import numpy as np
import pytest
import torch

from paper_1811_10573_gb300 import cpals, synth

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _bf16(a):
    """float32 -> bf16 (round to nearest even) -> float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def _planes(B32):
    """Device planes [2][Rpad][Kstride] of the K x R float32 operand B, and
    the host value hi + lo they carry."""
    K, R = B32.shape
    Bd = torch.from_numpy(np.ascontiguousarray(B32)).cuda()
    hi = Bd.to(torch.bfloat16)
    lo = (Bd - hi.float()).to(torch.bfloat16)
    Rpad = -(-R // 16) * 16
    Kstride = -(-K // 8) * 8
    Bt = torch.zeros((2, Rpad, Kstride), dtype=torch.bfloat16, device="cuda")
    Bt[0, :R, :K] = hi.t()
    Bt[1, :R, :K] = lo.t()
    hi64 = _bf16(B32)
    lo64 = _bf16((B32 - hi64.astype(np.float32)).astype(np.float32))
    return Bt, Kstride, hi64 + lo64


def _case(kind, dims, R, seed):
    """Inputs and the emulated reference of one contraction of an order-3
    tensor X (s0 x s1 x s2, float32 storage):
      mn:     out[x2][r]     = sum_{x0 x1} X[x0][x1][x2] (A0 (.) A1)[(x0 x1)][r]
      kmajor: out[(x0 x1)][r] = sum_{x2} X[x0][x1][x2] A2[x2][r]
      batch:  out[x0][x2][r] = sum_{x1} X[x0][x1][x2] A1[x1][r]"""
    p = synth.make_problem("normal", dims, R, seed=seed, storage="f32")
    s0, s1, s2 = p.dims
    X = np.ascontiguousarray(p.X)
    Xb = torch.from_numpy(X).cuda().to(torch.bfloat16).contiguous()
    Xr = _bf16(X)
    A = [a.astype(np.float32) for a in p.A0]
    if kind == "mn":
        B32 = (A[0][:, None, :] * A[1][None, :, :]).reshape(s0 * s1, R).astype(np.float32)
        Bt, Kstride, Bv = _planes(B32)
        ref = Xr.reshape(s0 * s1, s2).T @ Bv
        return dict(Xb=Xb, Bt=Bt, batch=1, K=s0 * s1, M=s2, R=R, Kstride=Kstride, kmajor=0,
                    ref=ref, shape=(s2, R))
    if kind == "kmajor":
        Bt, Kstride, Bv = _planes(A[2])
        ref = Xr.reshape(s0 * s1, s2) @ Bv
        return dict(Xb=Xb, Bt=Bt, batch=1, K=s2, M=s0 * s1, R=R, Kstride=Kstride, kmajor=1,
                    ref=ref, shape=(s0 * s1, R))
    Bt, Kstride, Bv = _planes(A[1])
    ref = np.matmul(Xr.transpose(0, 2, 1), Bv)
    return dict(Xb=Xb, Bt=Bt, batch=s0, K=s1, M=s2, R=R, Kstride=Kstride, kmajor=0, ref=ref,
                shape=(s0, s2, R))


def _call(c, splits):
    out = torch.full(c["shape"], float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    st = cpals.cpals_contract_bf16_noalloc(c["Xb"].data_ptr(), c["Bt"].data_ptr(), out.data_ptr(),
                                           c["batch"], c["K"], c["M"], c["R"], c["Kstride"],
                                           c["kmajor"], splits)
    return st, out


def _err(out, ref):
    got = out.double().cpu().numpy()
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


# (kind, dims, R, seed, splits): split-K partials in the scratch array
# (MN-major, 2-D box over a long K), K-major (2-D tensor map, one chunk),
# batched middle mode (3-D map, split-K), a single MN-major chunk (direct write)
CASES = [
    ("mn", [64, 48, 40], 100, 1, 12),
    ("mn", [96, 80, 64], 50, 2, 30),
    ("kmajor", [40, 48, 64], 64, 3, 1),
    ("kmajor", [32, 40, 128], 100, 4, 2),
    ("batch", [12, 256, 40], 48, 5, 3),
    ("mn", [8, 16, 48], 32, 6, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-R{c[2]}-s{c[4]}" for c in CASES])
def test_noalloc_matches_emulation_twice(case):
    kind, dims, R, seed, splits = case
    c = _case(kind, dims, R, seed)
    # two calls in a row: the second starts with the first one's leftovers in
    # the shared scratch array and error word
    for _ in range(2):
        st, out = _call(c, splits)
        assert st == 0, cpals.STATUS.get(st, st)
        assert torch.isfinite(out).all()
        assert _err(out, c["ref"]) < TOL


def test_noalloc_alternating_problems():
    a = _case("mn", [64, 48, 40], 100, 1)
    b = _case("batch", [12, 256, 40], 48, 5)
    for c, sp in ((a, 12), (b, 3), (a, 12)):
        st, out = _call(c, sp)
        assert st == 0, cpals.STATUS.get(st, st)
        assert _err(out, c["ref"]) < TOL


def test_noalloc_scratch_bound():
    """The bound applies to the K chunks the kernel runs: a batched
    contraction with batch M R = 2 Mi floats fits twice in the 4 Mi-float
    array.  K = 256 in 4 requested splits runs 4 chunks of 64 (8 Mi floats:
    rejected); in 3 requested splits it runs ceil(256/3) = 86 rounded up to 128,
    i.e. 2 chunks (4 Mi floats: accepted and correct)."""
    c = _case("batch", [32, 256, 512], 128, 7)
    assert c["batch"] * c["M"] * c["R"] == 2 * 1024 * 1024
    assert 2 * 1024 * 1024 * 2 == cpals.NOALLOC_SCRATCH_FLOATS
    st, _ = _call(c, 4)
    assert st == 1          # CPALS_E_INVALID: the partial sums do not fit
    st, out = _call(c, 3)
    assert st == 0, cpals.STATUS.get(st, st)
    assert _err(out, c["ref"]) < TOL
