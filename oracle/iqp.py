"""Closed forms for IQP circuits C = H^n D H^n, D diagonal (test infrastructure
only).

With H^n |0> = 2^{-n/2} sum_z |z> and <x| H^n |z> = 2^{-n/2} (-1)^{x.z}:

    a(x) = 2^{-n} sum_z (-1)^{x.z} D(z),

D(z) the product of the diagonal entries of every diagonal gate at the bits of
z on its qubits (for exp(i theta Z) and exp(i phi Z Z):
D(z) = prod_q e^{i theta_q s_q} prod_(q,r) e^{i phi_qr s_q s_r}, s = 1 - 2 z).
Used for the paper's IQP family (Examples, item 1) in the benchmark's variant.

* :func:`iqp_wht_amplitudes` -- one fast Walsh-Hadamard transform of D over
  all 2^n bitstrings (n <= ~26).
* :func:`iqp_transfer_amplitudes` -- the same sum taken column by column on a
  grid layout: gates couple qubits at most ``w`` columns apart, so the partial
  sum is a function of the last ``w`` columns only (exact for 5 x 8 at 40
  qubits with w = 2).
"""
from __future__ import annotations

import numpy as np

from .common import expand_open


def _split_iqp(gl):
    n = gl.n_qubits
    g = gl.gates
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2.0)
    head, tail, mid = g[:n], g[len(g) - n:], g[n:len(g) - n]
    for part in (head, tail):
        qs = sorted(q[0] for q, m in part if len(q) == 1 and np.allclose(m, H, atol=1e-14))
        if qs != list(range(n)):
            raise ValueError("not an IQP circuit: expected an H layer on every qubit")
    diag = []
    for q, m in mid:
        m = np.asarray(m)
        if not np.allclose(m, np.diag(np.diag(m)), atol=1e-14):
            raise ValueError("not an IQP circuit: non-diagonal middle gate")
        diag.append((q, np.diag(m).astype(np.complex128)))
    return diag


def _fwht(v: np.ndarray, n: int) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform: out[x] = sum_z (-1)^{x.z} v[z]."""
    v = v.reshape((2,) * n).copy()
    for ax in range(n):
        a = np.take(v, 0, axis=ax)
        b = np.take(v, 1, axis=ax)
        v = np.stack([a + b, a - b], axis=ax)
    return v.reshape(-1)


def iqp_wht_amplitudes(gl, bits, open_qubits=()) -> np.ndarray:
    n = gl.n_qubits
    diag = _split_iqp(gl)
    z = np.arange(1 << n, dtype=np.int64)
    D = np.ones(1 << n, dtype=np.complex128)
    for qubits, d in diag:
        if len(qubits) == 1:
            D *= d[(z >> qubits[0]) & 1]
        else:
            a, b = qubits
            D *= d[2 * ((z >> a) & 1) + ((z >> b) & 1)]
    A = _fwht(D, n) / float(1 << n)
    full = expand_open(bits, open_qubits)
    idx = (full.astype(np.int64) * (1 << np.arange(n, dtype=np.int64))).sum(-1)
    return A[idx]


def iqp_transfer_amplitudes(gl, bits, open_qubits=()) -> np.ndarray:
    n = gl.n_qubits
    diag = _split_iqp(gl)
    full = expand_open(bits, open_qubits)
    B0, J = full.shape[:2]
    X = full.reshape(B0 * J, n).astype(np.int64)
    Bn = X.shape[0]

    col = np.rint(np.asarray(gl.coords)[:, 0]).astype(int)
    cols = sorted(set(col.tolist()))
    members = {c: [q for q in range(n) if col[q] == c] for c in cols}
    R = max(len(v) for v in members.values())
    ci = {c: i for i, c in enumerate(cols)}
    w = 0
    for qubits, _ in diag:
        cs = [ci[col[q]] for q in qubits]
        w = max(w, max(cs) - min(cs))
    w = max(w, 1)
    slot_row = {}
    for c in cols:
        for r, q in enumerate(members[c]):
            slot_row[q] = r

    # state over the last w columns, slot 0 = oldest; bit (slot*R + row)
    state = np.zeros((Bn, 1 << (w * R)), dtype=np.complex128)
    state[:, 0] = 1.0
    E = 1 << ((w + 1) * R)
    e = np.arange(E, dtype=np.int64)
    for k, c in enumerate(cols):
        def zbit(q):
            # slot of qubit q within the extended window [k-w, k]
            slot = ci[col[q]] - (k - w)
            return (e >> (slot * R + slot_row[q])) & 1
        fac = np.ones(E, dtype=np.complex128)
        for qubits, d in diag:
            if max(ci[col[q]] for q in qubits) != k:
                continue
            if len(qubits) == 1:
                fac *= d[zbit(qubits[0])]
            else:
                fac *= d[2 * zbit(qubits[0]) + zbit(qubits[1])]
        # sign (-1)^{x_q z_q} for the qubits of this column, per bitstring
        sgn = np.ones((Bn, E), dtype=np.float64)
        for q in members[c]:
            zb = zbit(q)
            sgn *= 1.0 - 2.0 * (X[:, q:q + 1] * zb[None, :])
        old = state[:, e & ((1 << (w * R)) - 1)]
        ext = old * fac[None, :] * sgn
        # sum out slot 0 (column k-w) and shift the window
        ext = ext.reshape(Bn, 1 << (w * R), 1 << R)  # [.., slots 1..w, slot 0]
        state = ext.sum(axis=2)
    amp = state.sum(axis=1) / float(2 ** n)
    return amp.reshape(B0, J)
