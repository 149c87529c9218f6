"""Explicit time evolution of the state vector, FP64 (test infrastructure only).

This is the "explicit time evolution" scheme the paper compares its bounds
against (Thm. 2 discussion, cost T N 2^{2+N}): start from |0...0>, apply each
gate of the circuit in order, read off amplitudes.  The state is a complex128
array of shape (2,)*n; qubit q lives on axis n-1-q so that the flat index is
sum_q x_q 2^q.
"""
from __future__ import annotations

import numpy as np

from .common import expand_open


def statevector(n_qubits: int, gates) -> np.ndarray:
    """Return the flat state C|0...0> (index sum_q x_q 2^q) for ``gates`` =
    iterable of (qubits, matrix); a 2-qubit matrix acts on |x_a x_b> with the
    first listed qubit as the most significant bit."""
    n = n_qubits
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for qubits, mat in gates:
        k = len(qubits)
        axes = [n - 1 - q for q in qubits]
        g = np.asarray(mat, dtype=np.complex128).reshape((2,) * (2 * k))
        # contract the gate's input legs with the state's axes; the output
        # legs come first in the result and are moved back into place
        psi = np.tensordot(g, psi, axes=(list(range(k, 2 * k)), axes))
        psi = np.moveaxis(psi, list(range(k)), axes)
    return psi.reshape(-1)


def statevector_amplitudes(gl, bits, open_qubits=()) -> np.ndarray:
    """Amplitudes ``out[b, j]`` of the full bitstrings built from ``bits[b]``
    and the open-qubit index ``j`` (see :func:`oracle.common.expand_open`)."""
    psi = statevector(gl.n_qubits, gl.gates)
    full = expand_open(bits, open_qubits)
    weights = (1 << np.arange(gl.n_qubits, dtype=np.int64))
    idx = (full.astype(np.int64) * weights).sum(axis=-1)
    return psi[idx]
