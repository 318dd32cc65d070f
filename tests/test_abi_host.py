"""Host-only checks of the C-ABI library: it builds for sm_103a without a GPU,
loads, exports every symbol include/cpals.h declares, rejects bad arguments
before touching a device, and its flop model is the paper's (Table 1, Sec. 3.2.3).
"""
import os
import re

import pytest

from oracle import cpals_oracle as O
from paper_1811_10573_gb300 import build as B
from paper_1811_10573_gb300 import cpals

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cpals.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "cpals.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cpals_[a-z_A-Z0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # and the binding marshals each of them under the same name
    for n in names:
        assert n in cpals._SIGS, n
        assert callable(getattr(cpals, n)), n


def test_invalid_arguments_rejected_on_host(lib):
    for dims, R, prec in [([4, 5], 2, 0), ([4, 5, 0], 2, 0), ([4, 5, 6], 0, 0),
                          ([4, 5, 6], 200, 0), ([4, 5, 6], 3, 7), ([2] * 9, 2, 0)]:
        st, ctx = cpals.cpals_create(dims, len(dims), R, prec)
        assert st == 1 and not ctx, (dims, R, prec)


def test_tucker_invalid_arguments_rejected_on_host(lib):
    # order below 3 or above 8, an empty mode, a rank above its mode size or
    # above 48, a mode above 4096: rejected before any device call
    for dims, ranks in [([4, 5], [2, 2]), ([2] * 9, [1] * 9), ([4, 5, 6, 0], [2, 2, 2, 1]), ([4, 0, 6], [2, 1, 2]),
                        ([4, 5, 6], [5, 2, 2]), ([60, 60, 60], [49, 2, 2]), ([4, 5, 6], [2, 0, 2]),
                        ([5000, 5, 6], [2, 2, 2])]:
        st, t = cpals.cpals_tucker_create(dims, ranks)
        assert st == 1 and not t, (dims, ranks)


@pytest.mark.parametrize("s,R", [(400, 20), (2000, 10), (120, 12)])
def test_tucker_costs_table1(lib, s, R):
    """The order-3 Tucker context's contraction counts against Table 1's
    Tucker row (DT-ALS 4 s^N R, PP operators 6 s^N R, approximated step at
    most 2 N^2 s^2 R^{N-1}) and the paper's operator-construction sum."""
    def cost(kind, dims=(s, s, s), ranks=(R, R, R)):
        st, f = cpals.cpals_tucker_cost_model(dims, ranks, kind)
        assert st == 0, kind
        return f
    als, build, pp, paper = cost(0), cost(1), cost(2), cost(3)
    assert paper == 6 * s**3 * R                               # 2 C(3,2) s^3 R
    assert 4 * s**3 * R < als <= 4 * s**3 * R * (1 + 3 * R / s)
    assert paper < build <= paper * (1 + 2 * R / s)           # + the Y_p^(n)
    # N(N-1) first-order corrections of 2 s^2 R^2 each, plus the core estimate
    assert 12 * s**2 * R**2 < pp <= 2 * 9 * s**2 * R**2 + 2 * s * R**3
    # uneven sizes and ranks: every term scales with its own modes
    f0 = cost(0, (30, 40, 50), (2, 3, 4))
    assert f0 == 2 * 60000 * 4 + 2 * 1200 * 12 + 2 * 1200 * 8 + 2 * 60000 * 2 + 2 * 2000 * 6 + 2 * 50 * 24
    for kind, dims, ranks in [(3, (30, 40, 50), (2, 2, 2)), (4, (8, 8, 8), (2, 2, 2)),
                              (0, (8, 0, 8), (2, 2, 2)), (0, (8, 8, 8), (2, 0, 2))]:
        st, _ = cpals.cpals_tucker_cost_model(dims, ranks, kind)
        assert st == 1, (kind, dims, ranks)


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_operator_tree_cost_is_papers(lib, N):
    """The operator dimension tree the library runs has exactly the paper's
    cost 2R sum_{l=2}^{N-1} C(l+1,2) s^{N-l+2} (Sec. 3.2.3)."""
    for s, R in [(7, 3), (24, 50), (40, 16)]:
        mine = cpals.cost_model([s] * N, R, 1)
        paper = cpals.cost_model([s] * N, R, 3)
        assert mine == paper == O.pp_operator_build_cost(s, N, R)


@pytest.mark.parametrize("N", [3, 4, 6])
def test_als_and_pp_costs_table1(lib, N):
    """ALS sweep 4 s^N R to leading order; PP approximated step within
    2N^2(s^2R + sR^2) (Table 1)."""
    R = 8
    s = 400 if N == 3 else (120 if N == 4 else 24)
    als = cpals.cost_model([s] * N, R, 0)
    assert 1.0 <= als / (4 * s ** N * R) < 1.0 + 2.0 / s
    pp = cpals.cost_model([s] * N, R, 2)
    assert pp <= O.table1_cp(s, N, R)["pp_approx"]
    assert pp >= 2 * N * (N - 1) * s * s * R


def test_cost_model_rejects_bad_sizes(lib):
    with pytest.raises(cpals.CPALSError):
        cpals.cost_model([4, 0, 3], 2, 0)
