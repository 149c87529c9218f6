"""Properties of the separator planner (host, no GPU).

Algorithm 1 (Sphere Separator Algorithm) must return separators that satisfy
the Sphere Separator Theorem, Eqs. (1) and (2): |Gamma_O| <= c_d k^{1/d}
n^{1-1/d} and |Gamma_E|, |Gamma_I| <= (d+1)/(d+2) n, where k is the largest
number of spheres overlapping at a point.  Its centerpoint (step 2) must split
the lifted points evenly under every hyperplane through it (up to the
approximation factor of iterated Radon points).  The checks recompute the
classification and k here from the geometry.
"""
import math

import numpy as np
import pytest

from paper_2208_01498_gb300 import tnc

C_D = {1: 1.0, 2: 2.0, 3: 2.135}


def _k_bruteforce(pos, rad):
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    return int((d2 <= rad[None, :] ** 2).sum(1).max())


def _check_sst(pos, rad, side, k):
    n, d = pos.shape
    nI, nE, nO = (side == 0).sum(), (side == 1).sum(), (side == 2).sum()
    assert nI + nE + nO == n
    assert nO <= C_D[d] * k ** (1 / d) * n ** (1 - 1 / d) + 1e-9          # Eq. (1)
    assert max(nI, nE) <= (d + 1) / (d + 2) * n + 1e-9                    # Eq. (2)


def _point_sets():
    rng = np.random.default_rng(7)
    yield "uniform2d", rng.uniform(0, 20, (600, 2)), 0.3
    yield "clustered2d", np.vstack([rng.normal(0, 0.5, (540, 2)), rng.uniform(-20, 20, (60, 2))]), 0.05
    g = np.array([(x, y) for x in range(16) for y in range(16)], float)
    yield "lattice2d", g, 0.55
    yield "uniform3d", rng.uniform(0, 8, (500, 3)), 0.3
    yield "line1d", rng.uniform(0, 100, (300, 1)), 0.2


@pytest.mark.parametrize("name,pos,r", list(_point_sets()), ids=lambda v: v if isinstance(v, str) else "")
def test_ssa_separator_satisfies_sst(name, pos, r):
    rad = np.full(len(pos), r)
    side, valid, k = tnc.ssa_separate(pos, rad, seed=3, trials=32)
    assert valid
    assert k == _k_bruteforce(pos, rad)
    _check_sst(pos, rad, side, k)


def test_ssa_classification_is_geometric():
    """Every sphere labelled intersected must straddle the separator: the
    inside and outside sets are never linked by a sphere of the other side
    (their spheres are disjoint)."""
    rng = np.random.default_rng(1)
    pos = rng.uniform(0, 10, (400, 2))
    rad = np.full(400, 0.25)
    side, valid, _ = tnc.ssa_separate(pos, rad, seed=5)
    assert valid
    I, E = pos[side == 0], pos[side == 1]
    d = np.sqrt(((I[:, None, :] - E[None, :, :]) ** 2).sum(-1))
    assert d.min() >= 2 * 0.25 - 1e-9  # no inside sphere touches an outside sphere


def test_ssa_many_seeds_always_valid():
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, 30, (800, 2))
    rad = np.full(800, 0.4)
    for seed in range(8):
        side, valid, k = tnc.ssa_separate(pos, rad, seed=seed, trials=16)
        assert valid, seed
        _check_sst(pos, rad, side, k)


@pytest.mark.parametrize("D", [2, 3, 4])
def test_centerpoint_splits_every_hyperplane(D):
    rng = np.random.default_rng(D)
    # lifted points on the sphere S^{D-1}, strongly skewed towards one pole
    x = rng.normal(size=(3000, D))
    x[:, -1] += 2.0
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    c = tnc.centerpoint(x, seed=2)
    assert np.linalg.norm(c) < 1
    worst = 1.0
    for _ in range(400):
        u = rng.normal(size=D)
        s = (x - c) @ u
        worst = min(worst, (s > 0).mean(), (s < 0).mean())
    # a true centerpoint guarantees 1/(D+1); iterated Radon points get close
    assert worst >= 0.5 / (D + 1), worst


def test_separator_tree_covers_all_tensors_once():
    import circuits as C
    gl = C.random_2d(5, 5, 8, 1)
    e = tnc.Plan(tnc.Network(gl), seed=4).export()
    leaves = [n["leaf"] for n in e["nodes"] if n["left"] < 0]
    assert sorted(leaves) == list(range(len(e["leaves"])))
    internal = [n for n in e["nodes"] if n["left"] >= 0]
    assert len(internal) == len(leaves) - 1
    # each internal node's cost is the number of distinct labels of both children (Eq. 3)
    for n in internal:
        a, b = e["nodes"][n["left"]], e["nodes"][n["right"]]
        assert n["cost_log2"] == len(set(a["out"]) | set(b["out"]))


def test_theorem2_bound_dominates_the_plan():
    """The paper states the separator order is at least as good as Thm. 2;
    check log2 of the plan's cost against log2 of Thm. 2's first bound."""
    import circuits as C
    gl = C.random_2d(4, 4, 8, 0)
    n = gl.n_qubits
    f = np.zeros(n)
    for q, _ in gl.gates:
        if len(q) == 2:
            f[list(q)] += 1
    S, F, d, l_over_r = f.sum(), f.max(), 2, 1.0
    a_d = C_D[2] / (2 - 2 * ((d + 1) / (d + 2)) ** (1 - 1 / d))
    assert abs(a_d - 7.46) < 0.01  # the constant a_2 ~ 7.46 of Thm. 1
    log2_bound = math.log2(2 * S) / math.log2((d + 2) / (d + 1)) + 1 + \
        8 * a_d * (1 + l_over_r) * F ** (1 / d) * S ** (1 - 1 / d)
    rep = tnc.Plan(tnc.Network(gl)).report
    assert rep["tree_cost_log2"] < log2_bound
