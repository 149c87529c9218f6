"""The entry point that allocates nothing (tnc_contract_amplitudes_static).

It serves callers that cannot allocate device memory when they need
amplitudes -- e.g. code inside a host framework whose allocator owns the
GPU's memory, or a latency-bound handler that may not call cudaMalloc/cudaFree
(both can synchronise the device) -- by using a workspace the
library holds statically.  Its results must equal those of the ordinary entry
point with a caller-provided workspace, call after call (the static array
keeps the previous call's contents, so the second call checks that nothing
stale leaks through), and the device's free memory must not change across
the calls (its set-up happens in tnc_plan_upload).  The tensor-core plans put
their hi/lo operand planes in the same static array.  Collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

import circuits as C
import oracle as O
from plan_cases import TC_CASE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _call(tnc, p, bits, out):
    stream = torch.cuda.current_stream().cuda_stream
    return tnc.lib.tnc_contract_amplitudes_static(p.handle, bits.ctypes.data_as(ctypes.c_void_p), bits.shape[0],
                                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


# (circuit, open qubits, batch, form, kernel choice of the tensor-core steps, tolerance vs the oracle)
CASES = {
    "fp32_4x4": (lambda: C.random_2d(4, 4, 8, 21), [1, 6], 4, "fp32", None, 1e-5),
    "split_bf16_4x5": (lambda: C.random_2d(*TC_CASE["shape"]), TC_CASE["open"], TC_CASE["batch"], "split_bf16", None,
                       1e-4),
    # every tensor-core step on the plane-fed tile: its hi/lo planes are scratch inside the static array
    "split_bf16_4x5_planes": (lambda: C.random_2d(*TC_CASE["shape"]), TC_CASE["open"], TC_CASE["batch"], "split_bf16",
                              1, 1e-4),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_workspace_matches_caller_workspace(tnc, case):
    make, oq, batch, form, tc_tile, tol = CASES[case]
    gl = make()
    n = gl.n_qubits
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=batch, form=form)
    assert p.ws_bytes <= 64 << 20
    if tc_tile is not None:
        ch = [[k, tc_tile if k == tnc.KG["tc"] else t] for k, t in p.get_kernels()]
        p.set_kernels(ch)
    if form != "fp32":
        assert any(k == tnc.KG["tc"] for k, _ in p.get_kernels()), "the plan has no tensor-core step"
    p.upload()
    seeds = (3, 4)
    bits = [C.random_bitstrings(n, batch, s) for s in seeds]
    refs = [tnc.contract_amplitudes(p, b).cpu().numpy() for b in bits]
    outs = [torch.full((batch, 1 << len(oq)), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            for _ in seeds]
    free0 = _free_bytes()
    for call in range(len(seeds)):
        assert _call(tnc, p, bits[call], outs[call]) == tnc.TNC_OK, tnc.lib.tnc_last_error()
        assert _free_bytes() == free0, f"call {call} changed the device's free memory"
    for call in range(len(seeds)):
        got = outs[call].cpu().numpy()
        assert O.rel_error(got, refs[call], n).max() <= 1e-5, f"call {call}"
        assert O.rel_error(got, O.statevector_amplitudes(gl, bits[call], oq), n).max() <= tol, f"call {call}"


def test_static_workspace_limits(tnc):
    # a plan that was never uploaded is refused (uploading would allocate)
    gl = C.random_2d(3, 3, 4, 2)
    p = tnc.Plan(tnc.Network(gl))
    out = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    assert _call(tnc, p, np.zeros((1, 9), np.uint8), out) == tnc.TNC_ESTATE
    # a plan larger than the static workspace is refused with TNC_ENOMEM
    big = tnc.Plan(tnc.Network(C.iqp(5, 8, 0)), max_batch=256)
    assert big.ws_bytes > 64 << 20
    out = torch.empty((256, 1), dtype=torch.complex128, device="cuda")
    assert _call(tnc, big, np.zeros((256, 40), np.uint8), out) == tnc.TNC_ENOMEM
    assert b"static workspace" in tnc.lib.tnc_last_error()
