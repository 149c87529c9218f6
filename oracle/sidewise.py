"""Naive-order ("side-wise") FP64 contraction of a circuit's tensor network
(test infrastructure only).

The paper's left-to-right baseline (Thm. 2 discussion, bound
t_side <= 2^{1+4FL} L): sweep the qubit lattice one qubit at a time in a fixed
geometric order and absorb every tensor of that qubit's world line, in time
order, into one running boundary tensor.  The network is the one of the
Classical-Simulation section: |0> vectors, single-qubit gates as rank-2
tensors, each two-qubit gate split by an SVD of its operator-Schmidt
reshaping into two rank-3 tensors joined by a bond (Thm. 2 proof), and the
projections <x_q| (or an open leg).  A batch of bitstrings is carried as one
extra axis of the boundary (a hyper-index shared by all output projections).

The sweep order changes only the cost, never the value: the ``order``
argument exists so the order-independence of the result can be checked.
"""
from __future__ import annotations

import numpy as np

from .common import expand_open


def _schmidt_split(mat: np.ndarray, tol: float = 1e-13):
    """Split a 4x4 two-qubit gate G[(a'b'),(ab)] into A[a', a, k] and
    B[k, b', b] with sum_k A B = G (operator-Schmidt decomposition via SVD)."""
    g = np.asarray(mat, dtype=np.complex128).reshape(2, 2, 2, 2)  # a', b', a, b
    g = g.transpose(0, 2, 1, 3).reshape(4, 4)                    # (a' a), (b' b)
    u, s, vh = np.linalg.svd(g)
    r = max(1, int(np.sum(s > tol * s[0])))
    sq = np.sqrt(s[:r])
    A = (u[:, :r] * sq[None, :]).reshape(2, 2, r)
    B = (sq[:, None] * vh[:r, :]).reshape(r, 2, 2)
    return A, B


class _Boundary:
    """A dense tensor with one label per axis."""

    def __init__(self):
        self.t = np.ones((), dtype=np.complex128)
        self.labels: list = []

    def axis(self, lab):
        return self.labels.index(lab)

    def contract(self, small: np.ndarray, small_labels: list):
        """Contract ``small`` into the boundary over every shared label; new
        labels of ``small`` are appended in front."""
        shared = [l for l in small_labels if l in self.labels]
        ax_small = [small_labels.index(l) for l in shared]
        ax_big = [self.labels.index(l) for l in shared]
        out = np.tensordot(small, self.t, axes=(ax_small, ax_big))
        new_small = [l for l in small_labels if l not in shared]
        rest = [l for i, l in enumerate(self.labels) if i not in ax_big]
        self.t = out
        self.labels = new_small + rest

    def select(self, lab, values: np.ndarray):
        """Project axis ``lab`` onto per-bitstring values: the batch axis
        ``'beta'`` (created on first use) indexes the bitstrings."""
        ax = self.axis(lab)
        if "beta" not in self.labels:
            t = np.take(self.t, values, axis=ax)  # new axis of size B at ax
            labels = list(self.labels)
            labels[ax] = "beta"
            t = np.moveaxis(t, ax, 0)
            labels.insert(0, labels.pop(ax))
        else:
            bax = self.axis("beta")
            t = np.moveaxis(self.t, (bax, ax), (0, 1))
            labels = [l for l in self.labels if l not in ("beta", lab)]
            t = t[np.arange(len(values)), values]
            labels = ["beta"] + labels
        self.t, self.labels = t, labels


def _sweep_order(gl, order: str):
    n = gl.n_qubits
    xy = np.asarray(gl.coords, dtype=np.float64)
    if order == "columns":
        return sorted(range(n), key=lambda q: (xy[q][0], xy[q][1] if xy.shape[1] > 1 else 0, q))
    if order == "rows":
        return sorted(range(n), key=lambda q: (xy[q][1] if xy.shape[1] > 1 else 0, xy[q][0], q))
    if order == "reverse":
        return list(reversed(_sweep_order(gl, "columns")))
    if order == "index":
        return list(range(n))
    raise ValueError(order)


def sidewise_amplitudes(gl, bits, open_qubits=(), order: str = "columns") -> np.ndarray:
    """Amplitudes ``out[b, j]`` by side-wise contraction (see module doc)."""
    n = gl.n_qubits
    bits = np.atleast_2d(np.asarray(bits, dtype=np.uint8))
    open_qubits = [int(q) for q in open_qubits]
    is_open = set(open_qubits)

    # world lines: per qubit the time-ordered list of (labels, tensor);
    # wire segment labels ('w', q, seg), bond labels ('k', gate index, j)
    seg = [0] * n
    lines = [[(np.array([1.0, 0.0], dtype=np.complex128), [("w", q, 0)])] for q in range(n)]
    for gi, (qubits, mat) in enumerate(gl.gates):
        if len(qubits) == 1:
            q = qubits[0]
            lines[q].append((np.asarray(mat, np.complex128), [("w", q, seg[q] + 1), ("w", q, seg[q])]))
            seg[q] += 1
        else:
            a, b = qubits
            A, B = _schmidt_split(mat)
            kl = ("k", gi)
            lines[a].append((A, [("w", a, seg[a] + 1), ("w", a, seg[a]), kl]))
            lines[b].append((B, [kl, ("w", b, seg[b] + 1), ("w", b, seg[b])]))
            seg[a] += 1
            seg[b] += 1

    T = _Boundary()
    for q in _sweep_order(gl, order):
        for tensor, labels in lines[q]:
            T.contract(tensor, labels)
        last = ("w", q, seg[q])
        if q not in is_open:
            T.select(last, bits[:, q].astype(np.int64))
    # remaining labels: optional 'beta' and the open wires
    want = (["beta"] if "beta" in T.labels else []) + \
        [("w", q, seg[q]) for q in reversed(open_qubits)]
    assert sorted(map(str, want)) == sorted(map(str, T.labels)), (want, T.labels)
    t = np.transpose(T.t, [T.labels.index(l) for l in want])
    m = len(open_qubits)
    if "beta" not in T.labels:
        t = np.broadcast_to(t, (bits.shape[0],) + t.shape)
    # open wires are now ordered most significant first = open_qubits[m-1]
    return np.ascontiguousarray(t).reshape(bits.shape[0], 1 << m)
