"""The paper's analytic cost bounds (Thm. 1, Thm. 2 and its planar form, the
left-to-right and explicit-time-evolution costs after Thm. 2) as evaluated by
tnc_circuit_bounds_eval, pinned to values worked out by hand for a small
circuit, to the constants the paper prints, and to the plans the separator
planner produces.  Host only."""
import math

import numpy as np
import pytest

import circuits as C

tnc = pytest.importorskip("paper_2208_01498_gb300.tnc")


def _square_4cz():
    """2 x 2 grid, CZ on the four edges of the square: f = 2 on every qubit,
    sum f = 8, F = 2, l = r = 1, two time steps ((0,1),(2,3) then (0,2),(1,3))."""
    gl = C.GateList(4, np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]))
    for a, b in ((0, 1), (2, 3), (0, 2), (1, 3)):
        gl.add((a, b), C.CZ)
    return gl


def test_constants_printed_in_the_paper():
    b = tnc.Network(_square_4cz()).bounds()
    assert b["a_d"] == pytest.approx(2.0 / (2.0 - math.sqrt(3.0)))      # a_2 = c_2 / (2 - 2 sqrt(3/4))
    assert b["a_d"] == pytest.approx(7.464, abs=1e-3)
    assert b["a2_pst"] == pytest.approx(1.971 / (2.0 - 2.0 * math.sqrt(2.0 / 3.0)))
    assert b["a2_pst"] < b["a_d"]                                         # a_2' < a_2 (text after the PST)


def test_hand_worked_square():
    b = tnc.Network(_square_4cz()).bounds()
    assert (b["n_qubits"], b["dim"], b["depth"]) == (4, 2, 2)
    assert (b["sum_f"], b["max_f"], b["l"], b["r"]) == (8, 2, 1, 1)
    assert b["n_tensors"] == 16 and b["k"] == 2 * 2 * 2 ** 2
    a2 = 2.0 / (2.0 - math.sqrt(3.0))
    # Thm. 2: log2(16) / log2(4/3) + 1 + 8 a_2 (1 + 1) 2^(1/2) 8^(1/2) = 4 / log2(4/3) + 1 + 64 a_2
    assert b["thm2_log2"] == pytest.approx(4.0 / math.log2(4.0 / 3.0) + 1.0 + 64.0 * a2)
    assert b["thm1_log2"] == pytest.approx(b["thm2_log2"])               # Thm. 1 at the proof's n, M, k
    # planar form: W = 4 * 2 * (2 + 1) = 24
    a2p = 1.971 / (2.0 - 2.0 * math.sqrt(2.0 / 3.0))
    assert b["thm2_pst_log2"] == pytest.approx(math.log2(24.0) / math.log2(1.5) + 1.0 + 4.0 * a2p * math.sqrt(24.0))
    assert b["sidewise_log2"] == pytest.approx(18.0)                      # 1 + 4 F L + log2 L, L = 2
    assert b["explicit_log2"] == pytest.approx(9.0)                       # log2(T N) + 2 + N = 3 + 6


def test_sidewise_matches_the_lattice_form():
    """1 + 4 F L^(d-1) + log2 L for an L x L lattice equals the N form."""
    gl = C.random_2d(6, 6, 8, 1)
    b = tnc.Network(gl).bounds()
    assert b["sidewise_log2"] == pytest.approx(1 + 4 * b["max_f"] * 6 + math.log2(6))
    assert b["depth"] == 2 * 8 + 1                                        # Haar + CZ per cycle, final Haar layer


def test_not_applicable_cases():
    line = C.GateList(3, np.array([[0.0], [1.0], [2.0]]))
    line.add((0, 1), C.CZ)
    b = tnc.Network(line).bounds()
    assert math.isnan(b["thm2_log2"]) and math.isnan(b["thm2_pst_log2"])   # d = 1
    free = C.GateList(2, np.array([[0.0, 0.0], [1.0, 0.0]]))
    free.add((0,), C.H)
    assert math.isnan(tnc.Network(free).bounds()["thm2_log2"])           # no two-qubit gate
    iqp = tnc.Network(C.iqp(3, 3, 0)).bounds()
    assert iqp["l"] == pytest.approx(2.0) and math.isnan(iqp["thm2_pst_log2"])   # not nearest-neighbour


@pytest.mark.parametrize("seed", [0, 1])
def test_separator_plans_stay_under_the_bounds(seed):
    """The doubled network of a 4 x 4 depth-8 circuit: the planner's cost is
    below the planar form of Thm. 2, which is below Thm. 2 itself."""
    gl = C.random_2d(4, 4, 8, seed)
    b = tnc.Network(gl).bounds()
    cost = tnc.Plan(tnc.Network(C.doubled(gl, []))).report["tree_cost_log2"]
    assert cost < b["thm2_pst_log2"] < b["thm2_log2"]
