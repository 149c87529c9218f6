"""The doubled network c = <0| U^dagger P U |0> (Classical Simulation section)
on the GPU: the circuit U, the observable's single-qubit factors, then
U^dagger, contracted at x = 0...0 through the C ABI with the same executor as
amplitudes.  Expectation values of Pauli strings and marginal probabilities
(products of projectors) are compared with the FP64 oracle's definitions,
with the benchmark's error measure |c - c_ref| / max(|c_ref|, 2^{-n/2}):
at most 1e-5 (FP32, 3xTF32) or 1e-4 (split-BF16).  At 64 qubits the GHZ
correlators are exact closed forms and the Clifford twin's expectation values
come from the CH form, checked with an absolute tolerance of the same size
(c is normalised, |c| <= 1, and a zero there cancels O(1) terms).
"""
import itertools

import numpy as np
import pytest

import circuits as C
import oracle as O
from oracle.stabilizer import stabilizer_amplitudes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "3xtf32": 1e-5, "split_bf16": 1e-4}
FORMS = ["fp32", "3xtf32", "split_bf16"]


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _c(tnc, gl, ops, form, light_cone=False):
    dg = C.doubled(gl, ops, light_cone=light_cone)
    p = tnc.Plan(tnc.Network(dg), form=form)
    out = tnc.contract_amplitudes(p, np.zeros((1, gl.n_qubits), np.uint8))
    torch.cuda.synchronize()
    return complex(out.cpu().numpy().ravel()[0])


SPECS = [{5: "Z"}, {5: "Z", 6: "Z"}, {4: "X", 5: "X", 6: "X", 7: "X"}, {0: "Y", 10: "Z", 15: "X"}]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("light_cone", [False, True])
def test_pauli_expectations_4x4_depth8(tnc, form, light_cone):
    gl = C.random_2d(4, 4, 8, 0)
    for spec in SPECS:
        ops = C.pauli_ops(spec)
        ref = O.statevector_expectation(gl, ops)
        got = _c(tnc, gl, ops, form, light_cone)
        err = O.rel_error(np.array([got]), np.array([ref]), 16).max()
        assert err <= TOL[form], f"{spec} {form}: {got} vs {ref} ({err:.3g})"


@pytest.mark.parametrize("form", FORMS)
def test_marginal_probabilities(tnc, form):
    gl = C.random_2d(4, 4, 8, 2)
    qs = [3, 6, 9]
    total = 0.0
    for v in range(8):
        vals = [(v >> i) & 1 for i in range(3)]
        ref = O.statevector_marginal(gl, qs, vals)
        got = _c(tnc, gl, C.projector_ops(qs, vals), form, light_cone=True)
        err = O.rel_error(np.array([got]), np.array([ref]), 16).max()
        assert err <= TOL[form], f"{vals} {form}: {got} vs {ref}"
        total += got.real
    assert abs(total - 1.0) <= 8 * TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_full_projector_is_squared_amplitude(tnc, form):
    gl = C.random_2d(3, 3, 6, 4)
    bits = C.random_bitstrings(9, 3, 4)
    p = tnc.Plan(tnc.Network(gl), max_batch=3, form=form)
    amps = tnc.contract_amplitudes(p, bits).cpu().numpy().ravel()
    ref_amps = O.statevector_amplitudes(gl, bits).ravel()
    for b, a, ra in zip(bits, amps, ref_amps):
        got = _c(tnc, gl, C.projector_ops(range(9), b), form)
        err = O.rel_error(np.array([got]), np.array([abs(ra) ** 2]), 9).max()
        assert err <= TOL[form]
        assert abs(got - abs(a) ** 2) <= 2 * TOL[form] * max(abs(ra) ** 2, 2.0 ** -4.5)


@pytest.mark.parametrize("form", FORMS)
def test_ghz_correlators_64_qubits(tnc, form):
    gl = C.ghz(8, 8)
    yy = {q: "X" for q in range(64)}
    yy[0] = yy[1] = "Y"
    for spec, want in (({0: "Z", 63: "Z"}, 1.0), ({q: "X" for q in range(64)}, 1.0), (yy, -1.0),
                       ({17: "Z", 40: "Z"}, 1.0)):
        got = _c(tnc, gl, C.pauli_ops(spec), form, light_cone=True)
        assert abs(got - want) <= TOL[form], f"{form}: {got} vs {want}"


_PM = {"I": np.eye(2, dtype=complex), "X": C.X, "Y": C.Y, "Z": np.diag([1, -1]).astype(complex)}


def _stabilizer_string(gl, j):
    """The Pauli string P with U Z_j U^dagger = +-P for a Clifford circuit U
    (conjugated gate by gate with the gates' own matrices), so that
    <0|U^dagger P U|0> = +-1: an observable with a nonzero value to test."""
    spec = {j: "Z"}
    for qs, m in gl.gates:
        if not any(q in spec for q in qs):
            continue
        local = np.array([[1.0]], dtype=complex)
        for q in qs:
            local = np.kron(local, _PM[spec.get(q, "I")])
        r = m @ local @ m.conj().T
        for labs in itertools.product("IXYZ", repeat=len(qs)):
            cand = np.array([[1.0]], dtype=complex)
            for lab in labs:
                cand = np.kron(cand, _PM[lab])
            if abs(abs(np.trace(cand.conj().T @ r)) / cand.shape[0] - 1) < 1e-9:
                break
        for q, lab in zip(qs, labs):
            if lab == "I":
                spec.pop(q, None)
            else:
                spec[q] = lab
    return spec


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("depth,j", [(8, 9), (6, 36)])
def test_clifford_twin_8x8_light_cone(tnc, form, depth, j):
    """64 qubits: light-cone-reduced doubled networks on the GPU against the
    CH-form value of the full doubled circuit (exact, in {-1, 0, 1}): a
    stabilizer string of U|0> (value +-1) and two strings with value 0."""
    tw = C.random_2d(8, 8, depth, 3, clifford=True)
    zeros = np.zeros((1, 64), np.uint8)
    specs = [_stabilizer_string(tw, j), {27: "Z", 28: "Z"}, {35: "X"}]
    for k, spec in enumerate(specs):
        ops = C.pauli_ops(spec)
        want = stabilizer_amplitudes(C.doubled(tw, ops), zeros).ravel()[0]
        if k == 0:
            assert abs(abs(want) - 1) < 1e-9
        got = _c(tnc, tw, ops, form, light_cone=True)
        assert abs(got - want) <= TOL[form], f"{spec} {form}: {got} vs {want}"
