"""Shared helpers of the oracle (test infrastructure only; see the package
docstring)."""
from __future__ import annotations

import numpy as np


def expand_open(bits: np.ndarray, open_qubits) -> np.ndarray:
    """All full bitstrings requested: ``out[b, j, q]`` = ``bits[b, q]`` for a
    fixed qubit, and bit ``i`` of ``j`` for ``q = open_qubits[i]``."""
    bits = np.atleast_2d(np.asarray(bits, dtype=np.uint8))
    open_qubits = [int(q) for q in open_qubits]
    m = len(open_qubits)
    out = np.repeat(bits[:, None, :], 1 << m, axis=1).copy()
    for i, q in enumerate(open_qubits):
        out[:, :, q] = (np.arange(1 << m) >> i) & 1
    return out


def rel_error(a, ref, n_qubits: int) -> np.ndarray:
    """Error measure of the benchmark: |a - a_ref| / max(|a_ref|, 2^{-n/2})."""
    a = np.asarray(a, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    floor = 2.0 ** (-n_qubits / 2.0)
    return np.abs(a - ref) / np.maximum(np.abs(ref), floor)
