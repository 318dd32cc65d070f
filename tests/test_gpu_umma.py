"""Sharp parity of the tcgen05 (bf16 tensor-core) first-level contraction.

In MIXED_BF16 mode the library rounds X to bf16 (round to nearest even) and
carries the B operand (one factor, or the float32 Khatri-Rao product of
several) as two bf16 planes hi = bf16(b), lo = bf16(b - hi); the tensor cores
accumulate X (hi + lo) in fp32.  These tests take the same rounding decisions
on the host (float32 products, then the two RNE roundings), contract the
rounded values in float64, and compare: what remains is fp32 accumulation
error only (~K 2^-24 worst case), so the bound is 2e-5 relative to max|ref|.
A dropped k-step, a wrong swizzle or a transposed operand shows up as errors
of order 1e-2..1.
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


def bf16(a):
    """float32 -> bf16 (round to nearest even) -> float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def bsplit(a):
    """float32 B operand -> hi + lo as the library stores it (float64)."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    hi = bf16(a32)
    lo = bf16((a32 - hi.astype(np.float32)).astype(np.float32))
    return hi + lo


def krp32(mats):
    """Khatri-Rao product of float32 factors in the library's order: the
    leading factors multiplied left to right, then the last one, in float32."""
    R = mats[0].shape[1]
    rows = int(np.prod([m.shape[0] for m in mats]))
    idx = np.indices([m.shape[0] for m in mats]).reshape(len(mats), rows)
    v = mats[0].astype(np.float32)[idx[0]]
    for j in range(1, len(mats)):
        v = (v * mats[j].astype(np.float32)[idx[j]]).astype(np.float32)
    return v


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _ctx(p):
    g = cpals.CPALS(p.dims, p.R, "mixed")
    g.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    g.init_factors(p.A0)
    return g


SHAPES3 = [([64, 48, 40], 100), ([200, 136, 96], 50), ([96, 24, 136], 64), ([40, 24, 8], 7),
           ([130, 72, 256], 128), ([33, 17, 16], 33)]


@pytest.mark.parametrize("dims,R", SHAPES3)
def test_mttkrp_order3(dims, R):
    p = synth.make_problem("normal", dims, R, seed=21, storage="f32")
    Xb = bf16(p.X)
    A32 = [a.astype(np.float32) for a in p.A0]
    s0, s1, s2 = dims
    with _ctx(p) as g:
        # left half {0,1}: X_(01) times A^(2) (tensor cores), then one TTV in fp32
        ML = (Xb.reshape(s0 * s1, s2) @ bsplit(A32[2])).reshape(s0, s1, R)
        ref0 = np.einsum("ijr,jr->ir", ML, A32[1].astype(np.float64))
        ref1 = np.einsum("ijr,ir->jr", ML, A32[0].astype(np.float64))
        # right half {2}: X_(01)^T times the split of A^(0) (.) A^(1)
        ref2 = Xb.reshape(s0 * s1, s2).T @ bsplit(krp32([A32[0], A32[1]]))
        for n, ref in enumerate([ref0, ref1, ref2]):
            assert rel(g.mttkrp(n), ref) < TOL, n


@pytest.mark.parametrize("dims,R", [([16, 24, 16, 8], 16), ([24, 8, 12, 16], 40)])
def test_mttkrp_order4(dims, R):
    p = synth.make_problem("normal", dims, R, seed=22, storage="f32")
    Xb = bf16(p.X).reshape(dims[0] * dims[1], dims[2] * dims[3])
    A32 = [a.astype(np.float32) for a in p.A0]
    A64 = [a.astype(np.float64) for a in A32]
    with _ctx(p) as g:
        ML = (Xb @ bsplit(krp32([A32[2], A32[3]]))).reshape(dims[0], dims[1], R)
        MR = (Xb.T @ bsplit(krp32([A32[0], A32[1]]))).reshape(dims[2], dims[3], R)
        refs = [np.einsum("ijr,jr->ir", ML, A64[1]), np.einsum("ijr,ir->jr", ML, A64[0]),
                np.einsum("klr,lr->kr", MR, A64[3]), np.einsum("klr,kr->lr", MR, A64[2])]
        for n, ref in enumerate(refs):
            assert rel(g.mttkrp(n), ref) < TOL, n


@pytest.mark.parametrize("dims,R", SHAPES3[:4])
def test_pp_operators_order3(dims, R):
    """Level 2 of the operator tree = three single-mode contractions of X
    (K-major for the last mode, batched MN-major for the others): on the
    tensor cores (bf16 X, hi + lo B) when the contracted mode has at least 64
    entries, else on the SIMT float32 kernels (float32 X and factor)."""
    p = synth.make_problem("normal", dims, R, seed=23, storage="f32")
    with _ctx(p) as g:
        g.pp_build_operators()
        A32 = [a.astype(np.float32) for a in p.A0]
        X = {w: (bf16(p.X) if dims[w] >= 64 else np.asarray(p.X, dtype=np.float32).astype(np.float64))
             for w in range(3)}
        B = {w: (bsplit(A32[w]) if dims[w] >= 64 else A32[w].astype(np.float64)) for w in range(3)}
        refs = {(0, 1): np.einsum("ijk,kr->ijr", X[2], B[2]),
                (0, 2): np.einsum("ijk,jr->ikr", X[1], B[1]),
                (1, 2): np.einsum("ijk,ir->jkr", X[0], B[0])}
        for (i, n), ref in refs.items():
            assert rel(g.get_operator(i, n), ref) < TOL, (i, n)


def test_als_sweeps_track_fp32():
    """Mixed ALS sweeps stay within the bf16 rounding of the float32 path."""
    p = synth.make_problem("normal", [96, 80, 64], 32, seed=24, storage="f32")
    with cpals.CPALS(p.dims, p.R, "fp32") as g32, _ctx(p) as gm:
        g32.set_tensor(p.X)
        g32.init_factors(p.A0)
        for _ in range(3):
            f32 = g32.als_sweep()
            fm = gm.als_sweep()
        assert abs(f32 - fm) < 5e-3
        assert fm > 0.2
