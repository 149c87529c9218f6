"""Seeded synthetic quantum-circuit workloads (gate lists) for the contraction
executor and for the oracle.

This module holds only input generation: qubit layouts, gate schedules and
explicit gate matrices drawn from seeded ``numpy.random.Generator(PCG64)``
streams.  It contains no tensor-network or simulation arithmetic; both the CUDA
path and the oracle consume the :class:`GateList` it produces as plain data.

Conventions (fixed here, shared by everything downstream as data):

* qubit ``q = r * W + c`` for grid position (row ``r``, column ``c``);
  ``coords[q] = (c, r)`` (2D) — the geometric embedding used by the separator
  planner (the circuit's time axis is collapsed, Thm. 2 proof).
* a gate on qubits ``(a, b)`` is a ``4 x 4`` matrix acting on ``|x_a x_b>``,
  the first listed qubit being the most significant bit; rows index outputs.
* a bitstring is a ``uint8[n_qubits]`` array, entry ``q`` = value of qubit
  ``q``; the amplitude requested is ``<x| C |0...0>``.

Workload families (the paper's Examples section and its Sycamore/IQP/(2+1)D
circuit families, in the variants the benchmark configurations fix):

* :func:`random_2d` — L x L lattice, per cycle a Haar-random single-qubit layer
  then CZ on one of four brick patterns A, B, C, D (cycle ``t`` uses pattern
  ``t mod 4``), final Haar layer.  ``clifford=True`` draws uniformly random
  single-qubit Cliffords instead (the "Clifford twin": same layout, same
  schedule, hence the same network structure and contraction plan).
* :func:`sycamore` — 7 x 7 grid, staggered ABCD fSim schedule, single-qubit
  gates from {sqrt X, sqrt Y, sqrt W} never repeating on a qubit.
* :func:`iqp` — H layer, exp(i theta Z) on every qubit, exp(i phi Z Z) on all
  pairs within Manhattan distance 2, H layer.
* :func:`layered_3d` — (2+1)D random circuits: per layer a Haar layer then a
  randomly oriented, randomly offset brick pattern whose CZ gates are each
  kept with a per-layer density rho ~ U[0.5, 1].
* :func:`ghz`, :func:`mirror` — circuits with exactly known amplitudes.
* The paper's own example families (Examples section): :func:`iqp_paper`
  (short-range IQP: random phase gates with probability 7/8, controlled
  phases on nearest-neighbour pairs with probability 3/4 gamma ln N / N per
  time step), :func:`sycamore_periods` (Sycamore-type periods of eight
  coupling cycles with qubits inaccessible for a whole period) and
  :func:`cavity_3d` ((2+1)D dense random circuits with Poisson-distributed
  space-time cavities).
* :func:`doubled` — the circuit ``U, P, U^dagger`` whose amplitude at
  ``x = 0...0`` is the paper's quantity ``c = <0| U^dagger P U |0>`` (Classical
  Simulation section) for an observable ``P`` given as a product of
  single-qubit operators: a Pauli string (:func:`pauli_ops`) gives an
  expectation value, a product of projectors (:func:`projector_ops`) a
  marginal probability.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "GateList", "haar_1q", "clifford_1q_group", "random_2d", "sycamore",
    "iqp", "layered_3d", "ghz", "mirror", "doubled", "pauli_ops", "projector_ops",
    "iqp_paper", "sycamore_periods", "cavity_3d", "fuse_diagonal",
    "random_bitstrings", "serving_pool",
    "workload", "WORKLOADS", "H", "S", "CZ", "X", "Y", "sqrt_pauli", "fsim",
]

# ---------------------------------------------------------------- matrices
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)


def sqrt_pauli(P: np.ndarray) -> np.ndarray:
    """Principal square root of an involutory Pauli-like matrix P (P^2 = I):
    eigenvalue +1 -> 1, -1 -> i."""
    return 0.5 * (1 + 1j) * I2 + 0.5 * (1 - 1j) * P


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def haar_1q(rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(2): QR of a complex Ginibre matrix with the phases of R's
    diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


_CLIFF_CACHE: list[np.ndarray] | None = None


def clifford_1q_group() -> list[np.ndarray]:
    """All 192 elements of the group generated by H and S (the 24 single-qubit
    Cliffords times the 8 global phases e^{i pi k / 4}), built by breadth-first
    closure so every matrix is an exact product of H and S."""
    global _CLIFF_CACHE
    if _CLIFF_CACHE is None:
        def key(m):
            v = np.round(m.reshape(-1) * 1e6)
            return tuple(v.real.astype(np.int64).tolist()) + tuple(v.imag.astype(np.int64).tolist())
        elems = [I2.copy()]
        seen = {key(I2)}
        frontier = [I2.copy()]
        while frontier:
            nxt = []
            for m in frontier:
                for g in (H, S):
                    p = g @ m
                    k = key(p)
                    if k not in seen:
                        seen.add(k)
                        elems.append(p)
                        nxt.append(p)
            frontier = nxt
        assert len(elems) == 192, len(elems)
        _CLIFF_CACHE = elems
    return _CLIFF_CACHE


# ---------------------------------------------------------------- gate list
@dataclass
class GateList:
    """A circuit as an ordered list of explicit gates.

    ``gates[i] = (qubits, matrix)`` with ``matrix`` of shape ``(2^k, 2^k)``,
    ``k = len(qubits)`` in {1, 2}.
    """
    n_qubits: int
    coords: np.ndarray
    gates: list = field(default_factory=list)
    name: str = ""
    meta: dict = field(default_factory=dict)

    def add(self, qubits, mat):
        qubits = tuple(int(q) for q in qubits)
        mat = np.asarray(mat, dtype=np.complex128)
        assert mat.shape == (1 << len(qubits),) * 2
        self.gates.append((qubits, mat))

    @property
    def n_2q(self) -> int:
        return sum(1 for q, _ in self.gates if len(q) == 2)

    @property
    def n_1q(self) -> int:
        return sum(1 for q, _ in self.gates if len(q) == 1)

    def arrays(self):
        """Flat arrays for the C-ABI network descriptor: ``coords`` float64
        [n][dim], ``arity`` int32 [g], ``qubits`` int32 [sum arity],
        ``mats`` float64 interleaved (re, im), row-major per gate."""
        arity = np.array([len(q) for q, _ in self.gates], dtype=np.int32)
        qubits = np.array([x for q, _ in self.gates for x in q], dtype=np.int32)
        mats = np.concatenate([m.reshape(-1) for _, m in self.gates]) if self.gates else \
            np.zeros(0, np.complex128)
        mats = np.ascontiguousarray(mats.astype(np.complex128)).view(np.float64)
        coords = np.ascontiguousarray(self.coords, dtype=np.float64)
        return coords, arity, qubits, mats


def _grid_coords(rows: int, cols: int) -> np.ndarray:
    return np.array([(c, r) for r in range(rows) for c in range(cols)], dtype=np.float64)


def _brick_pattern(rows: int, cols: int, pat: str):
    """Pattern A: horizontal (r,c)-(r,c+1), c even; B: horizontal, c odd;
    C: vertical (r,c)-(r+1,c), r even; D: vertical, r odd."""
    W = cols
    out = []
    if pat in "AB":
        par = 0 if pat == "A" else 1
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                out.append((r * W + c, r * W + c + 1))
    else:
        par = 0 if pat == "C" else 1
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                out.append((r * W + c, (r + 1) * W + c))
    return out


def random_2d(rows: int, cols: int, depth: int, seed: int, clifford: bool = False) -> GateList:
    """2D random circuit: ``depth`` cycles of (single-qubit layer, CZ pattern
    ABCD[t mod 4]) followed by a final single-qubit layer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rows * cols
    gl = GateList(n, _grid_coords(rows, cols),
                  name=f"rand2d_{rows}x{cols}_d{depth}_s{seed}{'_cliff' if clifford else ''}",
                  meta=dict(family="random_2d", rows=rows, cols=cols, depth=depth, seed=seed,
                            clifford=clifford))
    group = clifford_1q_group() if clifford else None

    def one_q():
        if clifford:
            return group[int(rng.integers(len(group)))]
        return haar_1q(rng)

    for t in range(depth):
        for q in range(n):
            gl.add((q,), one_q())
        for (a, b) in _brick_pattern(rows, cols, "ABCD"[t % 4]):
            gl.add((a, b), CZ)
    for q in range(n):
        gl.add((q,), one_q())
    return gl


def _staggered_pattern(L: int, pat: str):
    """Staggered matchings of the L x L grid graph: A horizontal edges whose
    left end has (r+c) even, B (r+c) odd; C vertical edges whose top end has
    (r+c) even, D odd."""
    out = []
    par = 0 if pat in "AC" else 1
    for r in range(L):
        for c in range(L):
            if (r + c) % 2 != par:
                continue
            if pat in "AB" and c + 1 < L:
                out.append((r * L + c, r * L + c + 1))
            if pat in "CD" and r + 1 < L:
                out.append((r * L + c, (r + 1) * L + c))
    return out


def sycamore(L: int, cycles: int, seed: int, clifford: bool = False) -> GateList:
    """Sycamore-type circuit on the L x L grid (the diagonal lattice drawn
    rotated by 45 degrees): per cycle a single-qubit layer drawn from
    {sqrt X, sqrt Y, sqrt W} (the first uniformly, later uniformly from the
    two gates that differ from the qubit's previous one), then fSim(pi/2,
    pi/6) on pattern ABCD[t mod 4]; a final single-qubit layer.  The Clifford
    twin uses {sqrt X, sqrt Y} and fSim(pi/2, 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = L * L
    if clifford:
        pool = [sqrt_pauli(X), sqrt_pauli(Y)]
        g2 = fsim(math.pi / 2, 0.0)
    else:
        Wm = (X + Y) / math.sqrt(2.0)
        pool = [sqrt_pauli(X), sqrt_pauli(Y), sqrt_pauli(Wm)]
        g2 = fsim(math.pi / 2, math.pi / 6)
    gl = GateList(n, _grid_coords(L, L),
                  name=f"sycamore_{L}x{L}_c{cycles}_s{seed}{'_cliff' if clifford else ''}",
                  meta=dict(family="sycamore", L=L, cycles=cycles, seed=seed, clifford=clifford))
    prev = [-1] * n

    def layer():
        for q in range(n):
            if prev[q] < 0:
                k = int(rng.integers(len(pool)))
            else:
                choices = [i for i in range(len(pool)) if i != prev[q]]
                k = choices[int(rng.integers(len(choices)))]
            prev[q] = k
            gl.add((q,), pool[k])

    for t in range(cycles):
        layer()
        for (a, b) in _staggered_pattern(L, "ABCD"[t % 4]):
            gl.add((a, b), g2)
    layer()
    return gl


def iqp(rows: int, cols: int, seed: int, clifford: bool = False) -> GateList:
    """IQP circuit: H layer; exp(i theta_q Z) on every qubit; exp(i phi Z Z)
    on every unordered pair at Manhattan distance 1 or 2; H layer.  theta, phi
    ~ U[0, 2 pi); the Clifford twin draws them from (pi/4) * {0..7}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rows * cols
    gl = GateList(n, _grid_coords(rows, cols),
                  name=f"iqp_{rows}x{cols}_s{seed}{'_cliff' if clifford else ''}",
                  meta=dict(family="iqp", rows=rows, cols=cols, seed=seed, clifford=clifford))

    def angle():
        if clifford:
            return math.pi / 4 * int(rng.integers(8))
        return float(rng.uniform(0.0, 2 * math.pi))

    for q in range(n):
        gl.add((q,), H)
    for q in range(n):
        th = angle()
        gl.add((q,), np.diag([np.exp(1j * th), np.exp(-1j * th)]))
    for q in range(n):
        r1, c1 = divmod(q, cols)
        for p in range(q + 1, n):
            r2, c2 = divmod(p, cols)
            if 1 <= abs(r1 - r2) + abs(c1 - c2) <= 2:
                ph = angle()
                e, f = np.exp(1j * ph), np.exp(-1j * ph)
                gl.add((q, p), np.diag([e, f, f, e]))
    for q in range(n):
        gl.add((q,), H)
    return gl


def layered_3d(L: int, layers: int, seed: int, clifford: bool = False) -> GateList:
    """(2+1)D non-homogeneous random circuit on L x L qubits and ``layers``
    time layers: each layer applies a Haar single-qubit layer, draws an
    orientation (horizontal/vertical), a brick offset (0/1) and a density rho
    ~ U[0.5, 1], and keeps each candidate CZ of that brick pattern with
    probability rho; a final Haar layer follows."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = L * L
    gl = GateList(n, _grid_coords(L, L),
                  name=f"layered3d_{L}x{L}x{layers}_s{seed}{'_cliff' if clifford else ''}",
                  meta=dict(family="layered_3d", L=L, layers=layers, seed=seed, clifford=clifford))
    group = clifford_1q_group() if clifford else None

    def one_q():
        if clifford:
            return group[int(rng.integers(len(group)))]
        return haar_1q(rng)

    for _ in range(layers):
        for q in range(n):
            gl.add((q,), one_q())
        orient = int(rng.integers(2))
        off = int(rng.integers(2))
        rho = float(rng.uniform(0.5, 1.0))
        pat = ("AB" if orient == 0 else "CD")[off]
        for (a, b) in _brick_pattern(L, L, pat):
            if rng.uniform() < rho:
                gl.add((a, b), CZ)
    for q in range(n):
        gl.add((q,), one_q())
    return gl


def _nn_pairs(L: int):
    out = []
    for r in range(L):
        for c in range(L):
            if c + 1 < L:
                out.append((r * L + c, r * L + c + 1))
            if r + 1 < L:
                out.append((r * L + c, (r + 1) * L + c))
    return out


def iqp_paper(L: int, seed: int, gamma: float = 3.0, steps: int | None = None) -> GateList:
    """The paper's short-range IQP family (Examples, item 1) on L x L qubits:
    an H layer; then ``steps`` time steps (default T = L^2), each placing
    diag(1, e^{i pi m / 4}) with m uniform in {0..7} on every qubit (m = 0 is
    the identity and is left out, so a phase gate appears with probability
    7/8), then visiting the nearest-neighbour pairs in random order and, for
    a pair neither of whose qubits has a two-qubit gate in this step yet,
    drawing with probability gamma ln N / N a gate diag(1, 1, 1, i^m) with m
    uniform in {0..3} (m = 0 again left out: probability 3/4 gamma ln N / N);
    a final H layer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = L * L
    T = n if steps is None else steps
    p = min(1.0, gamma * math.log(n) / n) if n > 1 else 0.0
    gl = GateList(n, _grid_coords(L, L), name=f"iqp_paper_{L}x{L}_T{T}_s{seed}",
                  meta=dict(family="iqp_paper", L=L, steps=T, gamma=gamma, seed=seed))
    pairs = _nn_pairs(L)
    for q in range(n):
        gl.add((q,), H)
    for _ in range(T):
        for q in range(n):
            m = int(rng.integers(8))
            if m:
                gl.add((q,), np.diag([1.0, np.exp(1j * math.pi * m / 4)]))
        used = set()
        for i in rng.permutation(len(pairs)):
            a, b = pairs[int(i)]
            if a in used or b in used or rng.uniform() >= p:
                continue
            m = int(rng.integers(4))
            if m:
                gl.add((a, b), np.diag([1.0, 1.0, 1.0, 1j ** m]))
                used.update((a, b))
    for q in range(n):
        gl.add((q,), H)
    return gl


def fuse_diagonal(gl: GateList) -> GateList:
    """An IQP circuit (an H layer, diagonal gates, an H layer) with its
    diagonal gates merged: diagonal gates commute, so all of them on the same
    qubit pair are one gate (the product of their diagonals, a pair's
    single-qubit phases folded into it) and the remaining single-qubit phases
    one gate per qubit.  The circuit's operator is unchanged; its tensor
    network has at most one two-qubit tensor pair per coupled pair."""
    n = gl.n_qubits
    g = gl.gates
    head, mid, tail = g[:n], g[n:len(g) - n], g[len(g) - n:]
    for part in (head, tail):
        if sorted(q[0] for q, m in part if len(q) == 1 and np.allclose(m, H)) != list(range(n)):
            raise ValueError("fuse_diagonal: expected an H layer on every qubit at both ends")
    one = {}
    two = {}
    for q, m in mid:
        d = np.diag(m)
        if not np.allclose(m, np.diag(d)):
            raise ValueError("fuse_diagonal: a middle gate is not diagonal")
        if len(q) == 1:
            one[q[0]] = one.get(q[0], np.ones(2, complex)) * d
        else:
            a, b = q
            if a > b:  # diag over |x_a x_b>: swap the middle entries for the (b, a) order
                a, b, d = b, a, d[[0, 2, 1, 3]]
            two[(a, b)] = two.get((a, b), np.ones(4, complex)) * d
    for (a, b), d in two.items():  # fold single-qubit phases into one pair each
        for qq, pos in ((a, 0), (b, 1)):
            if qq in one:
                ph = one.pop(qq)
                d = d * (np.repeat(ph, 2) if pos == 0 else np.tile(ph, 2))
        two[(a, b)] = d
    out = GateList(n, gl.coords.copy(), name=gl.name + "_fused", meta=dict(gl.meta, fused=True))
    for q, m in head:
        out.add(q, m)
    for q in sorted(one):
        out.add((q,), np.diag(one[q]))
    for (a, b) in sorted(two):
        out.add((a, b), np.diag(two[(a, b)]))
    for q, m in tail:
        out.add(q, m)
    return out


def sycamore_periods(L: int, periods: int, p_inaccessible: float, seed: int) -> GateList:
    """The paper's Sycamore-type family with inaccessible qubits (Examples,
    item 2) on the L x L grid: ``periods`` periods of eight cycles with the
    coupling patterns A B C D C D A B (so each pair is coupled twice per
    period); at the start of a period every qubit is made inaccessible with
    probability ``p_inaccessible`` for the whole period.  A cycle applies a
    single-qubit gate from {sqrt X, sqrt Y, sqrt W} (never the qubit's
    previous one) to every accessible qubit, then fSim(pi/2, pi/6) to the
    pattern's pairs whose qubits are both accessible."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = L * L
    Wm = (X + Y) / math.sqrt(2.0)
    pool = [sqrt_pauli(X), sqrt_pauli(Y), sqrt_pauli(Wm)]
    g2 = fsim(math.pi / 2, math.pi / 6)
    gl = GateList(n, _grid_coords(L, L), name=f"sycamore_periods_{L}x{L}_q{periods}_p{p_inaccessible}_s{seed}",
                  meta=dict(family="sycamore_periods", L=L, periods=periods, p=p_inaccessible, seed=seed))
    prev = [-1] * n
    for _ in range(periods):
        active = rng.uniform(size=n) >= p_inaccessible
        for pat in "ABCDCDAB":
            for q in range(n):
                if not active[q]:
                    continue
                choices = [i for i in range(len(pool)) if i != prev[q]]
                k = choices[int(rng.integers(len(choices)))]
                prev[q] = k
                gl.add((q,), pool[k])
            for (a, b) in _staggered_pattern(L, pat):
                if active[a] and active[b]:
                    gl.add((a, b), g2)
    return gl


def cavity_3d(L: int, seed: int, alpha: float = 0.1, S: int = 5, sigma: float = 10.0,
              lam: float | None = None, steps: int | None = None) -> GateList:
    """The paper's (2+1)D random circuits with Poisson-distributed cavities
    (Examples, item 3) on L x L qubits: T = max(1, round(alpha L)) time steps
    (or ``steps``), each a Haar single-qubit layer and then CZ gates densely
    placed on a brick pattern of random orientation and offset, except inside
    cavities.  The number of cavity candidates is Poisson(lam), lam = 5e4
    (L/200)^3.5 by default; each candidate corner (x, y, t) is uniform in the
    space-time box and is kept with probability exp(-(x^2/L^2 + y^2/L^2 +
    t^2/T^2)/sigma^2); a kept cavity removes every gate in the S x S x S
    block from its corner.  A final Haar layer follows."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = L * L
    T = max(1, int(round(alpha * L))) if steps is None else steps
    lam = 5e4 * (L / 200.0) ** 3.5 if lam is None else lam
    holes = []
    for _ in range(int(rng.poisson(lam))):
        x, y, t = int(rng.integers(L)), int(rng.integers(L)), int(rng.integers(T))
        if rng.uniform() < math.exp(-(x * x / L / L + y * y / L / L + t * t / T / T) / sigma ** 2):
            holes.append((x, y, t))

    def in_cavity(q, t):
        r, c = divmod(q, L)
        return any(x <= c < x + S and y <= r < y + S and tt <= t < tt + S for x, y, tt in holes)

    gl = GateList(n, _grid_coords(L, L), name=f"cavity3d_{L}x{L}_T{T}_s{seed}",
                  meta=dict(family="cavity_3d", L=L, steps=T, seed=seed, cavities=len(holes)))
    for t in range(T):
        for q in range(n):
            if not in_cavity(q, t):
                gl.add((q,), haar_1q(rng))
        pat = ("AB" if int(rng.integers(2)) == 0 else "CD")[int(rng.integers(2))]
        for (a, b) in _brick_pattern(L, L, pat):
            if not (in_cavity(a, t) or in_cavity(b, t)):
                gl.add((a, b), CZ)
    for q in range(n):
        gl.add((q,), haar_1q(rng))
    return gl


def ghz(rows: int, cols: int) -> GateList:
    """GHZ preparation: H on the first qubit of a snake path through the grid,
    then CNOT along the path, each CNOT written as (I x H) CZ (I x H)."""
    n = rows * cols
    gl = GateList(n, _grid_coords(rows, cols), name=f"ghz_{rows}x{cols}",
                  meta=dict(family="ghz", rows=rows, cols=cols))
    path = []
    for r in range(rows):
        cs = range(cols) if r % 2 == 0 else range(cols - 1, -1, -1)
        path += [r * cols + c for c in cs]
    gl.add((path[0],), H)
    for a, b in zip(path[:-1], path[1:]):
        gl.add((b,), H)
        gl.add((a, b), CZ)
        gl.add((b,), H)
    return gl


def mirror(gl: GateList) -> GateList:
    """C followed by C^dagger: the identity circuit with the layout and a
    doubled schedule of ``gl``."""
    out = GateList(gl.n_qubits, gl.coords.copy(), name=gl.name + "_mirror",
                   meta=dict(gl.meta, mirror=True))
    for q, m in gl.gates:
        out.add(q, m)
    for q, m in reversed(gl.gates):
        out.add(q, m.conj().T)
    return out


def pauli_ops(spec: dict) -> list:
    """Single-qubit factors of a Pauli string: ``spec`` maps qubit -> one of
    "I", "X", "Y", "Z"; returns ``[(qubit, 2 x 2 matrix), ...]``."""
    mats = {"I": I2, "X": X, "Y": Y, "Z": np.diag([1, -1]).astype(np.complex128)}
    return [(int(q), mats[p].copy()) for q, p in sorted(spec.items())]


def projector_ops(qubits, values) -> list:
    """Factors of the projector ``|v><v|`` onto the values ``values`` of
    ``qubits`` (identity elsewhere): ``[(qubit, |v_q><v_q|), ...]``."""
    out = []
    for q, v in zip(qubits, values):
        m = np.zeros((2, 2), dtype=np.complex128)
        m[int(v), int(v)] = 1.0
        out.append((int(q), m))
    return out


def doubled(gl: GateList, ops, light_cone: bool = False) -> GateList:
    """The circuit ``U``, then the observable's single-qubit factors ``ops``
    (``[(qubit, 2 x 2 matrix), ...]``, not necessarily unitary), then
    ``U^dagger``.  Its amplitude at ``x = 0...0`` with no open qubits is
    ``<0| U^dagger P U |0>``; its tensor network is the doubled network of the
    Classical Simulation section (twice the gates of ``U`` on the same
    layout).

    ``light_cone=True`` keeps only the gates of ``U`` in the backward light
    cone of ``P``'s support: walking ``U`` from its last gate to its first, a
    gate whose qubits all lie outside the support gathered so far commutes
    with everything after it in ``U^dagger P U`` and meets its own inverse
    (``g^dagger g = I``), so it and its mirror are dropped; a gate that
    touches the support is kept and adds its qubits to it.  The value is
    unchanged; the network shrinks to the light cone."""
    for q, m in ops:
        if not 0 <= q < gl.n_qubits or np.shape(m) != (2, 2):
            raise ValueError(f"observable factor on qubit {q} must be a 2 x 2 matrix on an existing qubit")
    gates = list(gl.gates)
    if light_cone:
        support = {int(q) for q, _ in ops}
        kept = []
        for q, m in reversed(gates):
            if support.intersection(q):
                support.update(q)
                kept.append((q, m))
        gates = kept[::-1]
    out = GateList(gl.n_qubits, gl.coords.copy(), name=gl.name + ("_doubled_lc" if light_cone else "_doubled"),
                   meta=dict(gl.meta, doubled=True, light_cone=light_cone))
    for q, m in gates:
        out.add(q, m)
    for q, m in ops:
        out.add((q,), np.asarray(m, dtype=np.complex128))
    for q, m in reversed(gates):
        out.add(q, m.conj().T)
    return out


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.integers(0, 2, size=(count, n_qubits)).astype(np.uint8)


def random_open_qubits(n_qubits: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    return np.sort(rng.choice(n_qubits, size=count, replace=False)).astype(np.int32)


def serving_pool(seed: int = 0, n_2d: int = 10):
    """The mixed serving pool: 2D L x L random circuits (L in 4..10, depth
    U{8..20}) and (2+1)D circuits on 4x4x4 and 5x5x4 qubit grids."""
    rng = np.random.Generator(np.random.PCG64(seed + 31337))
    pool = []
    for i in range(n_2d):
        L = int(rng.integers(4, 11))
        d = int(rng.integers(8, 21))
        pool.append(random_2d(L, L, d, seed=1000 * seed + i))
    pool.append(layered_3d(4, 4, seed=1000 * seed + 100))
    pool.append(layered_3d(5, 4, seed=1000 * seed + 101))
    return pool


WORKLOADS = ("rand2d_4x4_d8", "rand2d_8x8_d16", "sycamore_7x7_c14", "iqp_5x8")


def workload(name: str, seed: int = 0, clifford: bool = False, reduced: bool = False):
    """The benchmark workloads by name: returns ``(gatelist, info)`` where
    ``info`` holds the bitstrings / open qubits a request asks for.

    * rand2d_4x4_d8: 4x4 depth-8 random 2D circuit, <0...0|C|0...0>.
    * rand2d_8x8_d16: 8x8 depth-16 random 2D circuit (``reduced``: 6x6 depth
      16), one seed-random bitstring.
    * sycamore_7x7_c14: 7x7 Sycamore-type, 14 cycles, 6 seed-random open
      qubits and 43 fixed seed-random bits (``reduced``: 4x4, 6 open).
    * iqp_5x8: 5x8 IQP, 256 seed-random bitstrings (``reduced``: 4x5).
    """
    if name == "rand2d_4x4_d8":
        gl = random_2d(4, 4, 8, seed, clifford)
        return gl, dict(bits=np.zeros((1, 16), np.uint8), open=np.zeros(0, np.int32))
    if name == "rand2d_8x8_d16":
        L = 6 if reduced else 8
        gl = random_2d(L, L, 16, seed, clifford)
        return gl, dict(bits=random_bitstrings(L * L, 1, seed), open=np.zeros(0, np.int32))
    if name == "sycamore_7x7_c14":
        L = 4 if reduced else 7
        gl = sycamore(L, 14, seed, clifford)
        return gl, dict(bits=random_bitstrings(L * L, 1, seed),
                        open=random_open_qubits(L * L, 6, seed))
    if name == "iqp_5x8":
        r, c = (4, 5) if reduced else (5, 8)
        gl = iqp(r, c, seed, clifford)
        return gl, dict(bits=random_bitstrings(r * c, 256, seed), open=np.zeros(0, np.int32))
    raise ValueError(name)
