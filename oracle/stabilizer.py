"""Exact amplitudes of Clifford circuits in the CH form (test infrastructure
only).

Reference: S. Bravyi, D. Browne, P. Calpin, E. Campbell, D. Gosset, M. Howard,
"Simulation of quantum circuits by low-rank stabilizer decompositions",
Quantum 3, 181 (2019), Sec. 4.1.  A stabilizer state is kept as

    |phi> = omega * U_C * U_H |s>,

U_C a "C-type" Clifford (generated by S, CZ, CX; U_C|0> = |0>) stored by its
tableau  U_C^-1 Z_p U_C = prod_j Z_j^{G_pj},
         U_C^-1 X_p U_C = i^{gamma_p} prod_j X_j^{F_pj} Z_j^{M_pj},
U_H = prod_j H_j^{v_j}, s a bitstring and omega a complex scalar.  Gates S,
CZ, CX, SWAP multiply U_C from the left (row updates); H is rewritten through
the two-term superposition rule, which multiplies U_C from the right (column
updates).  Every update rule below was derived from the conjugation relations
of the Pauli operators; amplitudes <x|phi> follow from <x| U_C = <0| U_C^-1
X(x) U_C.

Used to pin the executor on the "Clifford twins" of the benchmark circuits at
full size: same layout, same schedule, single-qubit gates drawn from the
Clifford group (exact |a| in {0, 2^{-r/2}}, phase in (pi/4) Z).

Gate matrices are recognised by breadth-first search over the finite groups
generated by {H, S} (one qubit, 192 elements with phases) and by
{H x I, I x H, S x I, I x S, CZ} (two qubits, 92160 elements): the search
returns an exact word in those generators for each matrix of the gate list.
"""
from __future__ import annotations

import math

import numpy as np

from .common import expand_open

_SQ2 = math.sqrt(2.0)
_OMEGA = complex(math.cos(math.pi / 4), math.sin(math.pi / 4))
_IPOW = [1, 1j, -1, -1j]


class CHForm:
    def __init__(self, n: int):
        self.n = n
        self.F = np.eye(n, dtype=np.uint8)
        self.G = np.eye(n, dtype=np.uint8)
        self.M = np.zeros((n, n), dtype=np.uint8)
        self.gamma = np.zeros(n, dtype=np.int64)
        self.v = np.zeros(n, dtype=np.uint8)
        self.s = np.zeros(n, dtype=np.uint8)
        self.omega = complex(1.0)

    # ---------------------------------------------------- left multiplication
    # U_C <- Gamma U_C : the images U_C^-1 (Gamma^-1 P Gamma) U_C, row updates
    def S(self, q):
        # S^-1 X S = i^3 X Z, S^-1 Z S = Z
        self.M[q] ^= self.G[q]
        self.gamma[q] = (self.gamma[q] - 1) % 4

    def CZ(self, q, r):
        # CZ^-1 X_q CZ = X_q Z_r, X_r -> Z_q X_r (G_q . F_r = 0 for q != r)
        self.M[q] ^= self.G[r]
        self.M[r] ^= self.G[q]

    def CX(self, q, r):
        # control q, target r: X_q -> X_q X_r, Z_r -> Z_q Z_r
        ph = int(np.dot(self.M[q].astype(np.int64), self.F[r].astype(np.int64)) % 2)
        self.gamma[q] = (self.gamma[q] + self.gamma[r] + 2 * ph) % 4
        self.G[r] ^= self.G[q]
        self.F[q] ^= self.F[r]
        self.M[q] ^= self.M[r]

    def SWAP(self, q, r):
        for A in (self.F, self.G, self.M):
            A[[q, r]] = A[[r, q]]
        self.gamma[[q, r]] = self.gamma[[r, q]]

    # --------------------------------------------------- right multiplication
    # U_C <- U_C Gamma : conjugate every row's Pauli by Gamma, column updates
    def _S_right(self, q):
        mask = self.F[:, q].copy()
        self.M[:, q] ^= mask
        self.gamma = (self.gamma - mask.astype(np.int64)) % 4

    def _CZ_right(self, q, r):
        self.gamma = (self.gamma + 2 * (self.F[:, q].astype(np.int64) & self.F[:, r])) % 4
        self.M[:, q] ^= self.F[:, r]
        self.M[:, r] ^= self.F[:, q]

    def _CX_right(self, q, r):
        # control q, target r: X_q -> X_q X_r (column q of F toggles column
        # r), Z_r -> Z_q Z_r (column r of G and M toggles column q)
        self.F[:, r] ^= self.F[:, q]
        self.G[:, q] ^= self.G[:, r]
        self.M[:, q] ^= self.M[:, r]

    # ------------------------------------------------------------- Hadamard
    def H(self, p):
        v, s = self.v, self.s
        a, b = self.F[p], self.M[p]
        # term 1: i^gamma_p X(F_p) Z(M_p) U_H |s>
        t = s ^ np.where(v == 1, b, a)
        e1 = int(np.sum(np.where(v == 1, a & t, b & s)) % 2)
        # term 2: Z(G_p) U_H |s>
        g = self.G[p]
        u = s ^ np.where(v == 1, g, 0).astype(np.uint8)
        e2 = int(np.sum(np.where(v == 1, 0, g & s)) % 2)
        c1 = _IPOW[int(self.gamma[p]) % 4] * (-1) ** e1
        c2 = (-1) ** e2
        if np.array_equal(t, u):
            self.omega *= (c1 + c2) / _SQ2
            self.s = t.astype(np.uint8)
            return
        delta = (int(self.gamma[p]) + 2 * (e1 + e2)) % 4
        f = self._superpose(u.astype(np.uint8), t.astype(np.uint8), delta)
        self.omega *= c2 * f / _SQ2

    def _superpose(self, y, z, delta):
        """Rewrite U_H (|y> + i^delta |z>) (y != z) as f * W U_H' |s'> with W
        C-type; apply W to U_C from the right, update v, s; return f."""
        D = (y ^ z).astype(bool)
        v = self.v
        D0 = np.flatnonzero(D & (v == 0))
        D1 = np.flatnonzero(D & (v == 1))
        if len(D0):
            q = int(D0[0])
            # V = prod CX_{q->j} (j in D \ q); U_H V = W U_H with
            # W = prod_{j in D0} CX_{q->j} prod_{j in D1} CZ_{q,j}
            for j in D0[1:]:
                self._CX_right(q, int(j))
            for j in D1:
                self._CZ_right(q, int(j))
            case_a = True
        else:
            q = int(D1[0])
            # both H: U_H CX_{q->j} = CX_{j->q} U_H
            for j in D1[1:]:
                self._CX_right(int(j), q)
            case_a = False
        w = (y if y[q] == 0 else z).copy()
        if y[q] == 0:
            k, c = delta, 1
        else:
            k, c = (-delta) % 4, _IPOW[delta]
        w[q] = 0
        self.s = w
        if case_a:
            # qubit q (no H): |0> + i^k |1> = sqrt2 S^k H |0>
            for _ in range(k):
                self._S_right(q)
            self.v[q] = 1
            return c * _SQ2
        # qubit q (under H): H (|0> + i^k |1>)
        if k == 0:
            self.v[q] = 0
            return c * _SQ2
        if k == 2:
            self.v[q] = 0
            self.s[q] = 1
            return c * _SQ2
        if k == 1:  # = sqrt2 omega S^3 H |0>
            for _ in range(3):
                self._S_right(q)
            return c * _SQ2 * _OMEGA
        self._S_right(q)  # k == 3: = sqrt2 omega^-1 S H |0>
        return c * _SQ2 * np.conj(_OMEGA)

    # ------------------------------------------------------------ amplitude
    def amplitude(self, x) -> complex:
        x = np.asarray(x, dtype=np.uint8)
        mu = 0
        t = np.zeros(self.n, dtype=np.uint8)
        u = np.zeros(self.n, dtype=np.uint8)
        for p in np.flatnonzero(x):
            mu += int(self.gamma[p]) + 2 * int(np.dot(u.astype(np.int64), self.F[p].astype(np.int64)) % 2)
            t ^= self.F[p]
            u ^= self.M[p]
        v, s = self.v, self.s
        if np.any((v == 0) & (t != s)):
            return 0j
        sign = int(np.dot(u.astype(np.int64), t.astype(np.int64)) + np.sum(v & t & s)) % 2
        r = int(np.sum(v))
        return self.omega * _IPOW[mu % 4] * (-1) ** sign * 2.0 ** (-r / 2.0)

    def apply_word(self, word, qubits):
        """Apply a word of generators (applied left to right in time)."""
        for g in word:
            if g == "H0":
                self.H(qubits[0])
            elif g == "S0":
                self.S(qubits[0])
            elif g == "H1":
                self.H(qubits[1])
            elif g == "S1":
                self.S(qubits[1])
            elif g == "CZ":
                self.CZ(qubits[0], qubits[1])
            else:
                raise ValueError(g)


# --------------------------------------------------------------- recognition
def _key(m: np.ndarray) -> bytes:
    v = np.round(np.asarray(m).reshape(-1) * 1e8)
    return np.concatenate([v.real, v.imag]).astype(np.int64).tobytes()


class _GroupSearch:
    """Breadth-first closure of a finite matrix group; ``word(m)`` returns the
    generator names whose product (first applied first) equals ``m``."""

    def __init__(self, gens: dict, dim: int):
        self.names = list(gens)
        self.mats = np.stack([gens[k] for k in self.names])
        ident = np.eye(dim, dtype=np.complex128)
        self.elems = [ident]
        self.parent = [(-1, -1)]
        self.index = {_key(ident): 0}
        self.frontier = [0]

    def _grow(self):
        if not self.frontier:
            return False
        F = np.stack([self.elems[i] for i in self.frontier])
        nxt = []
        for gi in range(len(self.names)):
            prod = np.einsum("ij,njk->nik", self.mats[gi], F)
            for fi, p in zip(self.frontier, prod):
                k = _key(p)
                if k not in self.index:
                    self.index[k] = len(self.elems)
                    self.elems.append(p)
                    self.parent.append((fi, gi))
                    nxt.append(self.index[k])
        self.frontier = nxt
        return True

    def word(self, m: np.ndarray):
        k = _key(m)
        while k not in self.index:
            if not self._grow():
                raise ValueError("matrix is not in the Clifford group:\n%r" % (m,))
        i = self.index[k]
        out = []
        while i > 0:
            pi, gi = self.parent[i]
            out.append(self.names[gi])
            i = pi
        return out[::-1]


_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / _SQ2
_S = np.diag([1, 1j]).astype(np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_G1 = None
_G2 = None


def _group1():
    global _G1
    if _G1 is None:
        _G1 = _GroupSearch({"H0": _H, "S0": _S}, 2)
    return _G1


def _group2():
    global _G2
    if _G2 is None:
        _G2 = _GroupSearch({"H0": np.kron(_H, _I2), "H1": np.kron(_I2, _H),
                            "S0": np.kron(_S, _I2), "S1": np.kron(_I2, _S),
                            "CZ": np.diag([1, 1, 1, -1]).astype(np.complex128)}, 4)
    return _G2


def clifford_word(mat: np.ndarray):
    mat = np.asarray(mat, dtype=np.complex128)
    return (_group1() if mat.shape[0] == 2 else _group2()).word(mat)


def simulate(gl) -> CHForm:
    """CH form of C|0...0> for a Clifford gate list."""
    ch = CHForm(gl.n_qubits)
    cache = {}
    for qubits, mat in gl.gates:
        k = _key(mat)
        if k not in cache:
            cache[k] = clifford_word(mat)
        ch.apply_word(cache[k], qubits)
    return ch


def stabilizer_amplitudes(gl, bits, open_qubits=()) -> np.ndarray:
    ch = simulate(gl)
    full = expand_open(bits, open_qubits)
    out = np.empty(full.shape[:2], dtype=np.complex128)
    for b in range(full.shape[0]):
        for j in range(full.shape[1]):
            out[b, j] = ch.amplitude(full[b, j])
    return out
