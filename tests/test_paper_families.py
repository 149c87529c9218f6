"""The paper's own example families (Examples section: short-range IQP,
Sycamore-type periods with inaccessible qubits, (2+1)D circuits with
Poisson cavities) on the host: the generators' structure and gate
statistics, agreement of independent oracle methods on them, and the
planner's tree and compiled program (emulated with NumPy) against the
oracle.  No GPU."""
import math

import numpy as np
import pytest

import circuits as C
import oracle as O

from host_emulator import contract_tree, emulate_program

tnc = pytest.importorskip("paper_2208_01498_gb300.tnc")


def test_iqp_paper_structure_and_rates():
    L, T = 6, 36
    gl = C.iqp_paper(L, 3, steps=T)
    n = L * L
    g = gl.gates
    assert all(q == (i,) and np.allclose(m, C.H) for i, (q, m) in enumerate(g[:n]))
    assert all(q == (i,) and np.allclose(m, C.H) for i, (q, m) in enumerate(g[-n:]))
    mid = g[n:-n]
    assert all(np.allclose(m, np.diag(np.diag(m))) for _, m in mid)
    one = [m for q, m in mid if len(q) == 1]
    two = [(q, m) for q, m in mid if len(q) == 2]
    # phase gates diag(1, e^{i pi m/4}), m = 1..7: probability 7/8 per qubit and step
    assert abs(len(one) / (n * T) - 7 / 8) < 0.03
    assert all(abs(m[0, 0] - 1) < 1e-15 and abs(m[1, 1] ** 8 - 1) < 1e-12 and abs(m[1, 1] - 1) > 1e-9 for m in one)
    # controlled phases diag(1, 1, 1, i^m), m = 1..3, on nearest neighbours only
    for (a, b), m in two:
        (ra, ca), (rb, cb) = divmod(a, L), divmod(b, L)
        assert abs(ra - rb) + abs(ca - cb) == 1
        assert np.allclose(np.diag(m)[:3], 1) and abs(m[3, 3] ** 4 - 1) < 1e-12 and abs(m[3, 3] - 1) > 1e-9
    # at most 3/4 gamma ln N / N per pair and step (pairs blocked in a step draw nothing)
    n_pairs = 2 * L * (L - 1)
    rate = len(two) / (n_pairs * T)
    assert 0.5 * 0.75 * 3 * math.log(n) / n < rate <= 0.75 * 3 * math.log(n) / n * 1.1


def test_iqp_paper_closed_form_equals_state_vector():
    gl = C.iqp_paper(4, 5)
    bits = C.random_bitstrings(16, 6, 2)
    ref = O.statevector_amplitudes(gl, bits, [3, 12])
    assert np.allclose(O.iqp_wht_amplitudes(gl, bits, [3, 12]), ref, atol=1e-13)
    assert np.allclose(O.iqp_transfer_amplitudes(gl, bits, [3, 12]), ref, atol=1e-13)


def test_sycamore_periods_structure():
    L, q = 5, 2
    full = C.sycamore_periods(L, q, 0.0, 1)
    per_period = sum(len(C._staggered_pattern(L, p)) for p in "ABCDCDAB")
    assert full.n_2q == q * per_period and full.n_1q == q * 8 * L * L
    assert all(len(qs) == 1 or np.allclose(m, C.fsim(math.pi / 2, math.pi / 6)) for qs, m in full.gates)
    assert C.sycamore_periods(L, q, 1.0, 1).gates == []
    part = C.sycamore_periods(L, q, 0.5, 1)
    assert 0 < part.n_2q < full.n_2q
    # single-qubit gates never repeat on a qubit
    last = {}
    for qs, m in part.gates:
        if len(qs) == 1:
            assert qs[0] not in last or not np.allclose(last[qs[0]], m)
            last[qs[0]] = m


def test_cavity_3d_structure():
    L, T = 6, 5
    dense = C.cavity_3d(L, 2, steps=T, lam=0.0)
    assert dense.meta["cavities"] == 0
    assert dense.n_1q == (T + 1) * L * L
    holed = C.cavity_3d(L, 2, steps=T, lam=30.0, S=2, sigma=10.0)
    assert holed.meta["cavities"] > 0
    assert holed.n_1q < dense.n_1q
    assert C.cavity_3d(20, 0).meta["steps"] == 2        # T = alpha L with alpha = 0.1


@pytest.mark.parametrize("family", ["iqp_paper", "sycamore_periods", "cavity_3d"])
def test_tree_and_program_of_paper_families(family):
    gl = {"iqp_paper": lambda: C.iqp_paper(3, 1),
          "sycamore_periods": lambda: C.sycamore_periods(3, 2, 0.2, 4),
          "cavity_3d": lambda: C.cavity_3d(3, 5, steps=4, lam=2.0, S=2)}[family]()
    n = gl.n_qubits
    bits = C.random_bitstrings(n, 3, 8)
    ref = O.statevector_amplitudes(gl, bits, [1])
    p = tnc.Plan(tnc.Network(gl), open_qubits=[1], max_batch=3)
    e = p.export()
    assert np.allclose(contract_tree(e, bits), ref, atol=1e-13)
    assert O.rel_error(emulate_program(e, bits), ref, n).max() < 1e-5


@pytest.mark.parametrize("seed", [0, 4])
def test_fuse_diagonal_keeps_the_circuit(seed):
    """Merging the commuting diagonal gates per pair leaves every amplitude
    unchanged (state vector and the IQP closed form on both circuits) and
    leaves at most one gate per coupled pair."""
    gl = C.iqp_paper(4, seed)
    f = C.fuse_diagonal(gl)
    pairs = [tuple(sorted(q)) for q, _ in f.gates if len(q) == 2]
    assert len(pairs) == len(set(pairs)) and f.n_2q < gl.n_2q
    bits = C.random_bitstrings(16, 5, seed)
    ref = O.statevector_amplitudes(gl, bits, [6])
    assert np.allclose(O.statevector_amplitudes(f, bits, [6]), ref, atol=1e-13)
    assert np.allclose(O.iqp_wht_amplitudes(f, bits, [6]), ref, atol=1e-13)
    # a pair listed in both orders is merged with the right bit order
    g2 = C.GateList(3, np.zeros((3, 2)))
    for q in range(3):
        g2.add((q,), C.H)
    g2.add((0, 1), np.diag([1, 1j, 1, 1]))
    g2.add((1, 0), np.diag([1, 1, -1j, 1]))
    g2.add((2,), np.diag([1, np.exp(0.3j)]))
    for q in range(3):
        g2.add((q,), C.H)
    b3 = C.random_bitstrings(3, 4, 1)
    assert np.allclose(O.statevector_amplitudes(C.fuse_diagonal(g2), b3), O.statevector_amplitudes(g2, b3),
                       atol=1e-14)
    with pytest.raises(ValueError):
        C.fuse_diagonal(C.random_2d(2, 2, 2, 0))


def test_op_count_trees_beyond_the_executor():
    """The op-count curves cost the separator tree of c = <0|U^dagger P U|0>
    with projectors on every qubit for the paper's IQP family up to L = 8,
    whose largest intermediates exceed the executor's 48 binary indices: a
    tree-only plan gives the tree, with the fused circuit far cheaper than the
    gate-by-gate one and both below left-to-right contraction."""
    gl = C.iqp_paper(8, 0)
    ops = C.projector_ops(range(gl.n_qubits), [0] * gl.n_qubits)
    full = tnc.Plan(tnc.Network(C.doubled(gl, ops)), seed=1, tree_only=True).report
    fused = tnc.Plan(tnc.Network(C.doubled(C.fuse_diagonal(gl), ops)), seed=1, tree_only=True).report
    assert full["max_rank"] > 48
    b = tnc.Network(gl).bounds()
    assert fused["tree_cost_log2"] + 40 < full["tree_cost_log2"] < b["sidewise_log2"]
