"""Parity of the CUDA path with the FP64 oracle on the hyper-edge form of the
network (diagonal gates on shared wire labels, TNC_NET_HYPEREDGES), on the
unmodified circuits, in all three forms, with the benchmark's error measure
|a - a_ref| / max(|a_ref|, 2^{-n/2}): at most 1e-5 (FP32, 3xTF32) or 1e-4
(split-BF16).  The 4 x 4 depth-8 random circuit (state vector), the 5 x 8 IQP
benchmark workload at full size with 256 bitstrings (transfer-matrix closed
form; its Clifford twin against the CH form) and the paper's short-range IQP
family, at L = 8 with T = L^2 steps unfused (transfer-matrix closed form)."""
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


def _run(tnc, gl, bits, oq, form, **kw):
    p = tnc.Plan(tnc.Network(gl, hyperedges=True), open_qubits=oq, max_batch=bits.shape[0], form=form, **kw)
    out = tnc.contract_amplitudes(p, bits)
    torch.cuda.synchronize()
    return out.cpu().numpy(), p


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("seed", [0, 1])
def test_rand2d_4x4_d8_hyperedges(tnc, form, seed):
    gl, info = C.workload("rand2d_4x4_d8", seed)
    bits = C.random_bitstrings(16, 4, seed)
    ref = O.statevector_amplitudes(gl, bits, [3])
    got, _ = _run(tnc, gl, bits, [3], form)
    assert O.rel_error(got, ref, 16).max() <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_iqp_5x8_full_size_hyperedges(tnc, form):
    gl, info = C.workload("iqp_5x8", 0)
    ref = O.iqp_transfer_amplitudes(gl, info["bits"])
    got, p = _run(tnc, gl, info["bits"], [], form)
    assert p.report["tree_cost_log2"] < 30  # against about 2^34.6 without hyper-edges
    assert O.rel_error(got, ref, 40).max() <= TOL[form]


def test_iqp_5x8_clifford_twin_hyperedges(tnc):
    gl, info = C.workload("iqp_5x8", 1, clifford=True)
    bits = info["bits"][:32]
    ref = stabilizer_amplitudes(gl, bits)
    got, _ = _run(tnc, gl, bits, [], "split_bf16")
    assert O.rel_error(got, ref, 40).max() <= TOL["split_bf16"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("L,steps,seed", [(4, None, 0), (8, None, 2)])
def test_iqp_paper_hyperedges(tnc, form, L, steps, seed):
    gl = C.iqp_paper(L, seed, steps=steps)
    n = L * L
    bits = C.random_bitstrings(n, 8, seed)
    oq = [0, n - 1]
    ref = O.iqp_transfer_amplitudes(gl, bits, oq)
    got, _ = _run(tnc, gl, bits, oq, form, n_starts=1)
    err = O.rel_error(got, ref, n).max()
    assert err <= TOL[form], f"{gl.name} {form}: {err:.3g}"
