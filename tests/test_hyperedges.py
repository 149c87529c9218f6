"""The hyper-edge form of the network (TNC_NET_HYPEREDGES), on the host.

Diagonal gates read their wire without changing it, so all diagonal gates
between two non-diagonal gates of a qubit share one wire label.  The
amplitudes must not change: the exported tree is contracted exactly (FP64,
per bitstring) and the compiled program is emulated step by step (FP32
kernels' arithmetic), both against the FP64 oracles on the unmodified
circuits, including diagonal single-qubit gates at every position (before
the first two-qubit gate, between diagonal gates, after the last), open legs
and bitstring batches.  The plans get cheaper where diagonal gates dominate.
"""
import numpy as np
import pytest

import circuits as C
import oracle as O
from host_emulator import contract_tree, emulate_program

tnc = pytest.importorskip("paper_2208_01498_gb300.tnc")


def _diag_mix(seed):
    """A 3 x 3 circuit mixing Haar gates, CZ, and diagonal single-qubit gates
    (S, T, Z, random phases) before, between and after the CZs."""
    rng = np.random.default_rng(seed)
    gl = C.GateList(9, np.array([(c, r) for r in range(3) for c in range(3)], np.float64))
    phase = lambda: np.diag([1.0, np.exp(1j * rng.uniform(0, 2 * np.pi))])
    for q in range(9):
        gl.add((q,), phase())  # diagonal on |0>: folded into the first tensor of the wire
    for q in (0, 4, 8):
        gl.add((q,), C.H)
    for t in range(6):
        pairs = [(0, 1), (3, 4), (6, 7), (1, 2), (4, 5), (7, 8)] if t % 2 == 0 else \
            [(0, 3), (1, 4), (2, 5), (3, 6), (4, 7), (5, 8)]
        for a, b in pairs[:3] if t % 3 else pairs:
            gl.add((a, b), C.CZ)
            if rng.uniform() < 0.5:
                gl.add((a,), phase())
        for q in rng.choice(9, size=3, replace=False):
            gl.add((int(q),), C.haar_1q(rng) if rng.uniform() < 0.6 else phase())
    for q in range(0, 9, 2):
        gl.add((q,), phase())
    return gl


CASES = {
    "rand2d_4x4_d8": (lambda: C.random_2d(4, 4, 8, 3), "sv"),
    "iqp_4x4": (lambda: C.iqp(4, 4, 2), "sv"),
    "iqp_paper_4": (lambda: C.iqp_paper(4, 1), "sv"),
    "ghz_3x4": (lambda: C.ghz(3, 4), "sv"),
    "sycamore_3x3": (lambda: C.sycamore(3, 6, 1), "sv"),
    "diag_mix_a": (lambda: _diag_mix(0), "sv"),
    "diag_mix_b": (lambda: _diag_mix(5), "sv"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_hyperedge_network_gives_the_same_amplitudes(case):
    make, _ = CASES[case]
    gl = make()
    n = gl.n_qubits
    bits = C.random_bitstrings(n, 3, 7)
    oq = [1, n - 2]
    ref = O.statevector_amplitudes(gl, bits, oq)
    p = tnc.Plan(tnc.Network(gl, hyperedges=True), open_qubits=oq, max_batch=3)
    e = p.export()
    assert np.allclose(contract_tree(e, bits), ref, atol=1e-13)
    assert O.rel_error(emulate_program(e, bits), ref, n).max() < 1e-5


def test_diagonal_gates_share_wire_labels():
    gl = C.iqp(4, 4, 0)
    plain = tnc.Plan(tnc.Network(gl)).export()
    hyper = tnc.Plan(tnc.Network(gl, hyperedges=True)).export()
    holders = {}
    for L in hyper["leaves"]:
        for x in L["labels"]:
            holders[x] = holders.get(x, 0) + 1
    # each qubit's wire between the two H layers carries all of its Z / ZZ phases
    assert max(holders.values()) >= 5
    assert len(hyper["leaves"]) < len(plain["leaves"])
    assert all(len(L["labels"]) <= 2 for L in hyper["leaves"])


def test_non_diagonal_circuits_keep_their_split_gates():
    gl = C.sycamore(3, 4, 0)  # fSim and sqrt gates: nothing diagonal
    plain = tnc.Plan(tnc.Network(gl)).export()
    hyper = tnc.Plan(tnc.Network(gl, hyperedges=True)).export()
    assert [L["labels"] for L in plain["leaves"]] == [L["labels"] for L in hyper["leaves"]]


@pytest.mark.parametrize("name,make,batch,gain_log2", [
    ("iqp_5x8", lambda: C.iqp(5, 8, 0), 256, 6.0),
    ("iqp_paper_6", lambda: C.iqp_paper(6, 0), 1, 20.0),
])
def test_hyperedges_cheapen_diagonal_circuits(name, make, batch, gain_log2):
    gl = make()
    a = tnc.Plan(tnc.Network(gl), max_batch=batch).report
    b = tnc.Plan(tnc.Network(gl, hyperedges=True), max_batch=batch).report
    assert b["tree_cost_log2"] < a["tree_cost_log2"] - gain_log2, (a["tree_cost_log2"], b["tree_cost_log2"])


def test_unknown_network_flags_are_refused():
    import ctypes
    gl = C.random_2d(2, 2, 2, 0)
    net = tnc.Network(gl)
    d = net.desc()
    h = ctypes.c_void_p()
    assert tnc.lib.tnc_load_network_opts(ctypes.byref(d), 6, ctypes.byref(h)) == tnc.TNC_EINVAL
