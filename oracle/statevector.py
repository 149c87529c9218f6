"""Explicit time evolution of the state vector, FP64 (test infrastructure only).

This is the "explicit time evolution" scheme the paper compares its bounds
against (Thm. 2 discussion, cost T N 2^{2+N}): start from |0...0>, apply each
gate of the circuit in order, read off amplitudes.  The state is a complex128
array of shape (2,)*n; qubit q lives on axis n-1-q so that the flat index is
sum_q x_q 2^q.

It also gives the paper's own quantity c = <0| U^dagger P U |0> (Classical
Simulation section) by its definition: the inner product of psi = U|0> with
P psi, for P a product of single-qubit operators; and marginal probabilities
by the Born rule, summing |psi_x|^2 over the unobserved bits.
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
        psi = _apply(psi, qubits, mat)
    return psi.reshape(-1)


def _apply(psi: np.ndarray, qubits, mat) -> np.ndarray:
    """One gate on the (2,)*n state tensor."""
    n = psi.ndim
    k = len(qubits)
    axes = [n - 1 - q for q in qubits]
    g = np.asarray(mat, dtype=np.complex128).reshape((2,) * (2 * k))
    # contract the gate's input legs with the state's axes; the output legs
    # come first in the result and are moved back into place
    out = np.tensordot(g, psi, axes=(list(range(k, 2 * k)), axes))
    return np.moveaxis(out, list(range(k)), axes)


def statevector_expectation(gl, ops) -> complex:
    """c = <0| U^dagger P U |0> = <psi| P |psi> with psi = U|0> (U the circuit
    ``gl``) and P the product of the single-qubit factors ``ops`` =
    [(qubit, 2 x 2 matrix), ...] (Classical Simulation section)."""
    n = gl.n_qubits
    psi = statevector(n, gl.gates).reshape((2,) * n)
    phi = psi
    for q, m in ops:
        phi = _apply(phi, (q,), m)
    return complex(np.vdot(psi.reshape(-1), phi.reshape(-1)))


def statevector_marginal(gl, qubits, values) -> float:
    """Probability that measuring ``qubits`` of U|0> gives ``values``: the sum
    of |<x|U|0>|^2 over every x that agrees with ``values`` there."""
    psi = statevector(gl.n_qubits, gl.gates)
    x = np.arange(psi.size, dtype=np.int64)
    keep = np.ones(psi.size, dtype=bool)
    for q, v in zip(qubits, values):
        keep &= ((x >> int(q)) & 1) == int(v)
    return float(np.sum(np.abs(psi[keep]) ** 2))


def statevector_amplitudes(gl, bits, open_qubits=()) -> np.ndarray:
    """Amplitudes ``out[b, j]`` of the full bitstrings built from ``bits[b]``
    and the open-qubit index ``j`` (see :func:`oracle.common.expand_open`)."""
    psi = statevector(gl.n_qubits, gl.gates)
    full = expand_open(bits, open_qubits)
    weights = (1 << np.arange(gl.n_qubits, dtype=np.int64))
    idx = (full.astype(np.int64) * weights).sum(axis=-1)
    return psi[idx]
