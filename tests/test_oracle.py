"""Pins of the FP64 oracle against facts fixed by the mathematics: closed
forms, invariants, textbook special cases and agreement between independent
methods (state vector / side-wise contraction / CH-form / IQP closed forms).

Each method is written independently, so a dropped term, a wrong sign, a
transposed operand or a wrong bit order in any one of them fails a cross-check
here.
"""
import math

import numpy as np
import pytest

import circuits as C
import oracle as O
from oracle.stabilizer import stabilizer_amplitudes, CHForm

SQ = 1 / math.sqrt(2)


def _all_bits(n):
    return ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


# ------------------------------------------------------------ textbook cases
def test_single_gate_textbook_values():
    gl = C.GateList(3, np.zeros((3, 2)))
    gl.add((1,), C.X)            # |010> in qubit order (q0, q1, q2)
    bits = _all_bits(3)
    a = O.statevector_amplitudes(gl, bits).ravel()
    want = np.zeros(8)
    want[0b010] = 1.0            # index sum_q x_q 2^q: qubit 1 -> 2
    assert np.allclose(a, want)
    assert np.allclose(O.sidewise_amplitudes(gl, bits).ravel(), want)
    assert np.allclose(stabilizer_amplitudes(gl, bits).ravel(), want)


def test_two_qubit_gate_first_qubit_is_msb():
    # CNOT written as an explicit matrix on (control, target), control = MSB
    cnot = np.eye(4)[[0, 1, 3, 2]].astype(np.complex128)
    gl = C.GateList(2, np.zeros((2, 2)))
    gl.add((1,), C.X)
    gl.add((1, 0), cnot)         # control qubit 1, target qubit 0
    bits = _all_bits(2)
    for f in (O.statevector_amplitudes, O.sidewise_amplitudes, stabilizer_amplitudes):
        a = f(gl, bits).ravel()
        assert np.allclose(a, [0, 0, 0, 1]), f.__name__


def test_hadamard_and_phase():
    gl = C.GateList(1, np.zeros((1, 2)))
    gl.add((0,), C.H)
    gl.add((0,), C.S)
    bits = _all_bits(1)
    for f in (O.statevector_amplitudes, O.sidewise_amplitudes, stabilizer_amplitudes):
        assert np.allclose(f(gl, bits).ravel(), [SQ, 1j * SQ]), f.__name__


@pytest.mark.parametrize("rows,cols", [(1, 2), (2, 3), (3, 3), (2, 5)])
def test_ghz(rows, cols):
    gl = C.ghz(rows, cols)
    n = gl.n_qubits
    bits = np.array([[0] * n, [1] * n, [1] + [0] * (n - 1), [0] * (n - 1) + [1]], np.uint8)
    want = [SQ, SQ, 0, 0]
    for f in (O.statevector_amplitudes, O.sidewise_amplitudes, stabilizer_amplitudes):
        assert np.allclose(f(gl, bits).ravel(), want, atol=1e-14), f.__name__


def test_ghz_full_size_stabilizer():
    gl = C.ghz(8, 8)
    bits = np.array([[0] * 64, [1] * 64, [0, 1] * 32], np.uint8)
    assert np.allclose(stabilizer_amplitudes(gl, bits).ravel(), [SQ, SQ, 0], atol=1e-14)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", [0, 1])
def test_normalisation_all_open(seed):
    gl = C.random_2d(2, 3, 6, seed)
    a = O.statevector_amplitudes(gl, np.zeros((1, 6), np.uint8), list(range(6)))
    assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-12
    b = O.sidewise_amplitudes(gl, np.zeros((1, 6), np.uint8), list(range(6)))
    assert abs(np.sum(np.abs(b) ** 2) - 1) < 1e-12
    assert np.allclose(a, b, atol=1e-14)


def test_mirror_is_identity():
    gl = C.mirror(C.random_2d(3, 3, 6, 4))
    bits = np.vstack([np.zeros((1, 9), np.uint8), C.random_bitstrings(9, 3, 5)])
    want = np.array([1, 0, 0, 0]) * (bits.sum(1) == 0)
    assert np.allclose(O.statevector_amplitudes(gl, bits).ravel(), want, atol=1e-13)
    assert np.allclose(O.sidewise_amplitudes(gl, bits).ravel(), want, atol=1e-13)


def test_mirror_full_size_clifford_twin():
    gl = C.mirror(C.random_2d(8, 8, 16, 0, clifford=True))
    bits = np.vstack([np.zeros((1, 64), np.uint8), C.random_bitstrings(64, 2, 9)])
    a = stabilizer_amplitudes(gl, bits).ravel()
    assert np.allclose(a, [1, 0, 0], atol=1e-13)


# ------------------------------------------- independent-method agreement
@pytest.mark.parametrize("seed", range(4))
def test_sidewise_equals_statevector_random(seed):
    gl = C.random_2d(3, 4, 8, seed)
    bits = C.random_bitstrings(12, 4, seed)
    oq = [2, 7]
    a = O.statevector_amplitudes(gl, bits, oq)
    for order in ("columns", "rows", "reverse", "index"):
        b = O.sidewise_amplitudes(gl, bits, oq, order=order)
        assert np.allclose(a, b, atol=1e-15, rtol=1e-12), order


def test_sidewise_sycamore_reduction():
    gl = C.sycamore(3, 6, 2)
    bits = C.random_bitstrings(9, 2, 2)
    a = O.statevector_amplitudes(gl, bits, [0, 4])
    b = O.sidewise_amplitudes(gl, bits, [0, 4], order="rows")
    assert np.allclose(a, b, atol=1e-15, rtol=1e-12)


def test_rand2d_4x4_d8_statevector_vs_sidewise():
    gl, info = C.workload("rand2d_4x4_d8", 0)
    a = O.statevector_amplitudes(gl, info["bits"])
    b = O.sidewise_amplitudes(gl, info["bits"])
    assert abs(a - b).max() < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_stabilizer_random_clifford_vs_statevector(seed):
    rng = np.random.default_rng(seed)
    grp = C.clifford_1q_group()
    for _ in range(40):
        n = int(rng.integers(1, 7))
        gl = C.GateList(n, np.zeros((n, 2)))
        for _ in range(int(rng.integers(1, 40))):
            if n > 1 and rng.uniform() < 0.4:
                a, b = rng.choice(n, 2, replace=False)
                m = [C.CZ, C.fsim(np.pi / 2, 0), np.diag([1, -1j, -1j, 1]),
                     np.eye(4)[[0, 1, 3, 2]]][int(rng.integers(4))]
                gl.add((a, b), m)
            else:
                gl.add((int(rng.integers(n)),), grp[int(rng.integers(192))])
        bits = np.zeros((1, n), np.uint8)
        a = O.statevector_amplitudes(gl, bits, list(range(n)))
        s = stabilizer_amplitudes(gl, bits, list(range(n)))
        assert np.allclose(a, s, atol=1e-13)


@pytest.mark.parametrize("name", ["rand2d_4x4_d8", "sycamore_7x7_c14", "iqp_5x8"])
def test_stabilizer_twins_reduced_vs_statevector(name):
    gl, info = C.workload(name, 1, clifford=True, reduced=True)
    bits = info["bits"][:6]
    a = O.statevector_amplitudes(gl, bits, info["open"])
    s = stabilizer_amplitudes(gl, bits, info["open"])
    assert np.allclose(a, s, atol=1e-13)


def test_clifford_amplitude_values_are_exact():
    # |a| in {0, 2^{-r/2}}, phase in (pi/4) Z
    gl, info = C.workload("sycamore_7x7_c14", 0, clifford=True, reduced=True)
    a = stabilizer_amplitudes(gl, info["bits"], info["open"]).ravel()
    nz = a[np.abs(a) > 1e-12]
    assert len(nz) > 0
    r = -2 * np.log2(np.abs(nz))
    assert np.allclose(r, np.round(r), atol=1e-9)
    ph = np.angle(nz) / (np.pi / 4)
    assert np.allclose(ph, np.round(ph), atol=1e-9)


def test_iqp_closed_forms_agree():
    gl, _ = C.workload("iqp_5x8", 2, reduced=True)
    bits = C.random_bitstrings(20, 32, 3)
    a = O.statevector_amplitudes(gl, bits)
    b = O.iqp_wht_amplitudes(gl, bits)
    c = O.iqp_transfer_amplitudes(gl, bits)
    assert np.allclose(a, b, atol=1e-15)
    assert np.allclose(a, c, atol=1e-15)


def test_iqp_commuting_gate_reorder():
    gl, _ = C.workload("iqp_5x8", 4, reduced=True)
    n = gl.n_qubits
    mid = gl.gates[n:-n]
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(mid))
    gl2 = C.GateList(n, gl.coords, gl.gates[:n] + [mid[i] for i in perm] + gl.gates[-n:])
    bits = C.random_bitstrings(n, 8, 1)
    assert np.allclose(O.iqp_transfer_amplitudes(gl, bits), O.statevector_amplitudes(gl2, bits), atol=1e-15)


def test_iqp_full_size_twin_transfer_vs_stabilizer():
    gl, info = C.workload("iqp_5x8", 0, clifford=True)
    bits = info["bits"][:64]
    a = O.iqp_transfer_amplitudes(gl, bits)
    s = stabilizer_amplitudes(gl, bits)
    assert np.allclose(a, s, atol=1e-15)


def test_iqp_transfer_normalisation_small():
    gl = C.iqp(2, 4, 5)
    a = O.iqp_transfer_amplitudes(gl, np.zeros((1, 8), np.uint8), list(range(8)))
    assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-12


def test_rel_error_measure():
    e = O.rel_error([1.0 + 1e-6], [1.0], 4)
    assert abs(e[0] - 1e-6) < 1e-12
    e = O.rel_error([1e-3], [0.0], 4)      # floor 2^-2
    assert abs(e[0] - 4e-3) < 1e-12


# ---------------------------------------------- planted mistakes are caught
def test_planted_sign_error_in_ch_form_is_caught(monkeypatch):
    gl = C.ghz(2, 2)
    bits = _all_bits(4)
    ref = O.statevector_amplitudes(gl, bits)

    orig = CHForm.S

    def bad_S(self, q):          # drop the phase update of S
        self.M[q] ^= self.G[q]
    monkeypatch.setattr(CHForm, "S", bad_S)
    gl2 = C.GateList(2, np.zeros((2, 2)))
    gl2.add((0,), C.H)
    gl2.add((0,), C.S)
    bad = stabilizer_amplitudes(gl2, _all_bits(2))
    monkeypatch.setattr(CHForm, "S", orig)
    good = stabilizer_amplitudes(gl2, _all_bits(2))
    sv = O.statevector_amplitudes(gl2, _all_bits(2))
    assert np.allclose(good, sv) and not np.allclose(bad, sv)
    assert np.allclose(stabilizer_amplitudes(gl, bits), ref, atol=1e-14)


def test_planted_transpose_in_gate_is_caught():
    gl = C.random_2d(2, 2, 4, 3)
    bad = C.GateList(gl.n_qubits, gl.coords, [(q, m.T) for q, m in gl.gates])
    bits = _all_bits(4)
    a = O.statevector_amplitudes(gl, bits)
    b = O.sidewise_amplitudes(bad, bits)
    assert not np.allclose(a, b, atol=1e-6)
