"""The entry point that allocates nothing (tnc_contract_amplitudes_static).

It serves callers that cannot allocate device memory when they need
amplitudes -- e.g. code inside a host framework whose allocator owns the
GPU's memory, or a latency-bound handler that may not call cudaMalloc/cudaFree
(both can synchronise the device) -- by using a workspace the
library holds statically.  Its results must equal those of the ordinary entry
point with a caller-provided workspace, call after call (the static array
keeps the previous call's contents, so the second call checks that nothing
stale leaks through).  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import circuits as C
import oracle as O

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


def test_static_workspace_matches_caller_workspace(tnc):
    gl = C.random_2d(4, 4, 8, 21)
    oq = [1, 6]
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=4)
    assert p.ws_bytes <= 64 << 20
    p.upload()
    for call, seed in enumerate((3, 4)):
        bits = C.random_bitstrings(16, 4, seed)
        ref = tnc.contract_amplitudes(p, bits).cpu().numpy()
        out = torch.full((4, 4), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        assert _call(tnc, p, bits, out) == tnc.TNC_OK, tnc.lib.tnc_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert O.rel_error(got, ref, 16).max() <= 1e-5, f"call {call}"
        assert O.rel_error(got, O.statevector_amplitudes(gl, bits, oq), 16).max() <= 1e-5


def test_static_workspace_limits(tnc):
    # a plan that was never uploaded is refused (uploading would allocate)
    gl = C.random_2d(3, 3, 4, 2)
    p = tnc.Plan(tnc.Network(gl))
    out = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    assert _call(tnc, p, np.zeros((1, 9), np.uint8), out) == tnc.TNC_ESTATE
    # a plan larger than the static workspace is refused with TNC_ENOMEM
    big = tnc.Plan(tnc.Network(C.iqp(4, 6, 0)), max_batch=256)
    assert big.ws_bytes > 64 << 20
    out = torch.empty((256, 1), dtype=torch.complex128, device="cuda")
    assert _call(tnc, big, np.zeros((256, 24), np.uint8), out) == tnc.TNC_ENOMEM
    assert b"static workspace" in tnc.lib.tnc_last_error()
