"""Parity of the CUDA path with the FP64 oracle on the paper's own example
families (Examples section): short-range IQP (against the column
transfer-matrix closed form, and at 16 qubits also the Walsh-Hadamard form
and the state vector), Sycamore-type periods with inaccessible
qubits, and (2+1)D circuits with Poisson cavities (state vector), in all
three forms, with the benchmark's error measure |a - a_ref| / max(|a_ref|,
2^{-n/2}): at most 1e-5 (FP32, 3xTF32) or 1e-4 (split-BF16)."""
import numpy as np
import pytest

import circuits as C
import oracle as O

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


def _run(tnc, gl, bits, oq, form):
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=bits.shape[0], form=form)
    out = tnc.contract_amplitudes(p, bits)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,steps,seed", [(4, None, 0), (6, 12, 1)])
def test_iqp_paper(tnc, form, L, steps, seed):
    gl = C.iqp_paper(L, seed, steps=steps)
    n = L * L
    bits = C.random_bitstrings(n, 8, seed)
    oq = [0, n - 1]
    ref = O.iqp_transfer_amplitudes(gl, bits, oq)
    if n <= 16:
        assert np.allclose(ref, O.iqp_wht_amplitudes(gl, bits, oq), atol=1e-13)
        assert np.allclose(ref, O.statevector_amplitudes(gl, bits, oq), atol=1e-13)
    err = O.rel_error(_run(tnc, gl, bits, oq, form), ref, n).max()
    assert err <= TOL[form], f"{gl.name} {form}: {err:.3g}"


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,periods,p,seed", [(4, 2, 0.3, 0), (4, 3, 0.6, 2)])
def test_sycamore_periods(tnc, form, L, periods, p, seed):
    gl = C.sycamore_periods(L, periods, p, seed)
    n = L * L
    bits = C.random_bitstrings(n, 4, seed)
    ref = O.statevector_amplitudes(gl, bits, [2])
    err = O.rel_error(_run(tnc, gl, bits, [2], form), ref, n).max()
    assert err <= TOL[form], f"{gl.name} {form}: {err:.3g}"


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,steps,lam,seed", [(4, 8, 3.0, 0), (4, 12, 6.0, 3)])
def test_cavity_3d(tnc, form, L, steps, lam, seed):
    gl = C.cavity_3d(L, seed, steps=steps, lam=lam, S=2)
    n = L * L
    bits = C.random_bitstrings(n, 4, seed)
    ref = O.statevector_amplitudes(gl, bits, [5])
    err = O.rel_error(_run(tnc, gl, bits, [5], form), ref, n).max()
    assert err <= TOL[form], f"{gl.name} {form}: {err:.3g}"


@pytest.mark.parametrize("form", FORMS)
def test_iqp_paper_8x8_full_depth_fused(tnc, form):
    """The paper's IQP parameters at L = 8 (64 qubits, T = L^2 = 64 steps,
    gamma = 3): the circuit with its commuting diagonal gates fused per pair
    on the GPU, against the transfer-matrix closed form of the circuit as
    generated."""
    gl = C.iqp_paper(8, 2)
    bits = C.random_bitstrings(64, 16, 2)
    oq = [0, 63]
    ref = O.iqp_transfer_amplitudes(gl, bits, oq)
    err = O.rel_error(_run(tnc, C.fuse_diagonal(gl), bits, oq, form), ref, 64).max()
    assert err <= TOL[form], f"{form}: {err:.3g}"
