"""The doubled network c = <0| U^dagger P U |0> (Classical Simulation section)
on the host: the oracle's expectation values and marginal probabilities
pinned against textbook values, GHZ closed forms, an independent method
(side-wise amplitudes; CH-form for Clifford circuits) and invariants; then the
planner's tree and the compiled node program of doubled networks (emulated
with NumPy) against the oracle.  No GPU.
"""
import importlib

import numpy as np
import pytest

import circuits as C
import oracle as O
SV = importlib.import_module("oracle.statevector")  # the module (the package re-exports a function of that name)
from oracle.stabilizer import stabilizer_amplitudes

from host_emulator import contract_tree, emulate_program

tnc_mod = pytest.importorskip("paper_2208_01498_gb300.tnc")


def _one_qubit(*mats):
    gl = C.GateList(1, np.zeros((1, 2)))
    for m in mats:
        gl.add((0,), m)
    return gl


# ------------------------------------------------------------ oracle pins
def test_textbook_single_qubit_expectations():
    assert O.statevector_expectation(_one_qubit(C.X), C.pauli_ops({0: "Z"})) == pytest.approx(-1)
    assert O.statevector_expectation(_one_qubit(C.H), C.pauli_ops({0: "X"})) == pytest.approx(1)
    assert O.statevector_expectation(_one_qubit(C.H), C.pauli_ops({0: "Z"})) == pytest.approx(0, abs=1e-15)
    # S H |0> = |+i>: <Y> = +1 (a transposed or sign-flipped Y gives -1)
    assert O.statevector_expectation(_one_qubit(C.H, C.S), C.pauli_ops({0: "Y"})) == pytest.approx(1)
    assert O.statevector_expectation(_one_qubit(C.H, C.S), C.pauli_ops({0: "X"})) == pytest.approx(0, abs=1e-15)


@pytest.mark.parametrize("rows,cols", [(2, 3), (3, 3)])
def test_ghz_expectations(rows, cols):
    gl = C.ghz(rows, cols)
    n = rows * cols
    for q in range(n):
        assert abs(O.statevector_expectation(gl, C.pauli_ops({q: "Z"}))) < 1e-12
        if q:
            assert O.statevector_expectation(gl, C.pauli_ops({0: "Z", q: "Z"})) == pytest.approx(1)
    assert O.statevector_expectation(gl, C.pauli_ops({q: "X" for q in range(n)})) == pytest.approx(1)
    # Y Y X ... X maps |0..0> to -|1..1> and |1..1> to -|0..0>
    yy = {q: "X" for q in range(n)}
    yy[0] = yy[1] = "Y"
    assert O.statevector_expectation(gl, C.pauli_ops(yy)) == pytest.approx(-1)
    assert O.statevector_marginal(gl, [0, n - 1], [1, 1]) == pytest.approx(0.5)
    assert O.statevector_marginal(gl, [0, n - 1], [0, 1]) == pytest.approx(0, abs=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_expectation_invariants_random(seed):
    gl = C.random_2d(3, 3, 6, seed)
    assert O.statevector_expectation(gl, []) == pytest.approx(1)   # P = I: normalisation
    rng = np.random.default_rng(seed)
    for _ in range(4):
        spec = {int(q): "XYZ"[int(rng.integers(3))] for q in rng.choice(9, size=3, replace=False)}
        c = O.statevector_expectation(gl, C.pauli_ops(spec))
        assert abs(c.imag) < 1e-12 and abs(c.real) <= 1 + 1e-12          # Hermitian, norm <= 1
    qs = [1, 4, 7]
    total = 0.0
    for v in range(8):
        vals = [(v >> i) & 1 for i in range(3)]
        pm = O.statevector_marginal(gl, qs, vals)
        # projector expectation (operator applied, inner product) = Born-rule sum
        assert O.statevector_expectation(gl, C.projector_ops(qs, vals)) == pytest.approx(pm, abs=1e-13)
        total += pm
    assert total == pytest.approx(1)


@pytest.mark.parametrize("seed", [3, 4])
def test_full_projector_is_squared_sidewise_amplitude(seed):
    gl = C.random_2d(3, 3, 5, seed)
    bits = C.random_bitstrings(9, 3, seed)
    amps = O.sidewise_amplitudes(gl, bits).ravel()   # an independent method
    for b, a in zip(bits, amps):
        c = O.statevector_expectation(gl, C.projector_ops(range(9), b))
        assert c == pytest.approx(abs(a) ** 2, abs=1e-13)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_clifford_expectations_match_ch_form(seed):
    gl = C.random_2d(3, 3, 6, seed, clifford=True)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        spec = {int(q): "XYZ"[int(rng.integers(3))] for q in rng.choice(9, size=2, replace=False)}
        c = O.statevector_expectation(gl, C.pauli_ops(spec))
        ch = stabilizer_amplitudes(C.doubled(gl, C.pauli_ops(spec)), np.zeros((1, 9), np.uint8)).ravel()[0]
        assert abs(c - ch) < 1e-12
        assert min(abs(c - v) for v in (-1, 0, 1)) < 1e-12


def test_planted_transpose_in_observable_is_caught(monkeypatch):
    real = SV._apply

    def transposed(psi, qubits, mat):
        m = np.asarray(mat)
        return real(psi, qubits, m.T if m.shape == (2, 2) else m)

    monkeypatch.setattr(SV, "_apply", transposed)
    c = O.statevector_expectation(_one_qubit(C.H, C.S), C.pauli_ops({0: "Y"}))
    assert c != pytest.approx(1)


# ------------------------------------------------- planner / program (host)
@pytest.mark.parametrize("case", ["pauli", "projector", "ghz"])
def test_tree_and_program_of_doubled_networks(case):
    tnc = tnc_mod
    if case == "ghz":
        gl = C.ghz(2, 3)
        ops = C.pauli_ops({0: "Y", 1: "Y", 2: "X", 3: "X", 4: "X", 5: "X"})
    else:
        gl = C.random_2d(3, 3, 4, 11)
        ops = C.pauli_ops({4: "Z", 0: "X"}) if case == "pauli" else C.projector_ops([0, 4, 8], [1, 0, 1])
    ref = O.statevector_expectation(gl, ops)
    dg = C.doubled(gl, ops)
    p = tnc.Plan(tnc.Network(dg))
    e = p.export()
    zeros = np.zeros((1, gl.n_qubits), np.uint8)
    assert abs(contract_tree(e, zeros).ravel()[0] - ref) < 1e-12
    em = emulate_program(e, zeros).ravel()[0]
    assert abs(em - ref) <= 1e-5 * max(abs(ref), 2.0 ** (-gl.n_qubits / 2))


def test_doubled_rejects_bad_observable():
    gl = C.random_2d(2, 2, 2, 0)
    with pytest.raises(ValueError):
        C.doubled(gl, [(4, np.eye(2))])
    with pytest.raises(ValueError):
        C.doubled(gl, [(0, np.eye(4))])


@pytest.mark.parametrize("seed", [8, 9])
def test_light_cone_keeps_the_value(seed):
    """Dropping the gates outside P's backward light cone (with their
    mirrors) leaves <0|U^dagger P U|0> unchanged: the oracle's definition on
    the full circuit against the state-vector amplitude of the reduced
    doubled circuit, and the CH-form of the full and reduced doubled Clifford
    circuits."""
    gl = C.random_2d(3, 4, 6, seed)
    zeros = np.zeros((1, 12), np.uint8)
    for spec in ({5: "Z"}, {0: "X", 1: "Y"}, {11: "Z", 6: "X"}):
        ops = C.pauli_ops(spec)
        ref = O.statevector_expectation(gl, ops)
        lc = C.doubled(gl, ops, light_cone=True)
        assert len(lc.gates) < len(C.doubled(gl, ops).gates)
        assert abs(O.statevector_amplitudes(lc, zeros).ravel()[0] - ref) < 1e-12
    ops = C.projector_ops([2, 3], [1, 0])
    assert abs(O.statevector_amplitudes(C.doubled(gl, ops, light_cone=True), zeros).ravel()[0]
               - O.statevector_marginal(gl, [2, 3], [1, 0])) < 1e-12
    tw = C.random_2d(3, 4, 6, seed, clifford=True)
    ops = C.pauli_ops({5: "Z", 6: "Z"})
    full = stabilizer_amplitudes(C.doubled(tw, ops), zeros).ravel()[0]
    red = stabilizer_amplitudes(C.doubled(tw, ops, light_cone=True), zeros).ravel()[0]
    assert abs(full - red) < 1e-12


def test_light_cone_of_ghz_correlator_is_exact_on_the_host():
    gl = C.ghz(2, 4)
    for spec, want in (({0: "Z", 7: "Z"}, 1.0), ({3: "Z"}, 0.0),
                       ({q: "X" for q in range(8)}, 1.0)):
        dg = C.doubled(gl, C.pauli_ops(spec), light_cone=True)
        p = tnc_mod.Plan(tnc_mod.Network(dg))
        got = contract_tree(p.export(), np.zeros((1, 8), np.uint8)).ravel()[0]
        assert abs(got - want) < 1e-12
