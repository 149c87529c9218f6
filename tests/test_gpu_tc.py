"""Parity of the tensor-core forms (split-BF16 and 3xTF32 on tcgen05) with the
FP64 oracle and with the FP32 CUDA-core form (GPU)."""
import numpy as np
import pytest

import circuits as C
import oracle as O
from plan_cases import TC_CASE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "3xtf32": 1e-5, "split_bf16": 1e-4}


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _run(tnc, gl, bits, form, oq=(), **kw):
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=bits.shape[0], form=form, **kw)
    out = tnc.contract_amplitudes(p, bits)
    torch.cuda.synchronize()
    return out.cpu().numpy(), p


def _n_tc(p):
    return sum(1 for s in p.export()["steps"] if s["kind"] == 1 and s["kernel"] == 4)




@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
def test_single_tensor_core_node(tnc, form):
    gl = C.random_2d(*TC_CASE["shape"])
    bits = C.random_bitstrings(20, TC_CASE["batch"], 4)
    ref = O.statevector_amplitudes(gl, bits, TC_CASE["open"])
    got, p = _run(tnc, gl, bits, form, oq=TC_CASE["open"])
    assert _n_tc(p) >= 1
    assert O.rel_error(got, ref, 20).max() <= TOL[form]


@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
def test_iqp_5x8_full_size(tnc, form):
    """The benchmark workload (40 qubits, 256 bitstrings) against the
    transfer-matrix closed form, and against the FP32 form."""
    gl, info = C.workload("iqp_5x8", 0)
    ref = O.iqp_transfer_amplitudes(gl, info["bits"])
    got, p = _run(tnc, gl, info["bits"], form)
    assert _n_tc(p) >= 3
    assert O.rel_error(got, ref, 40).max() <= TOL[form]
    fp32, _ = _run(tnc, gl, info["bits"], "fp32")
    assert O.rel_error(got, fp32, 40).max() <= TOL[form] + TOL["fp32"]


@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
def test_dense_batched_nodes_random_2d(tnc, form):
    gl = C.random_2d(5, 5, 12, 9)
    bits = C.random_bitstrings(25, 64, 2)
    ref = O.statevector_amplitudes(gl, bits)
    got, p = _run(tnc, gl, bits, form)
    assert O.rel_error(got, ref, 25).max() <= TOL[form]


def test_tensor_core_error_flag_clear(tnc):
    """No bounded wait of the tcgen05 kernel timed out during the tests."""
    import ctypes
    gl = C.random_2d(*TC_CASE["shape"])
    _, p = _run(tnc, gl, C.random_bitstrings(20, TC_CASE["batch"], 4), "split_bf16", oq=TC_CASE["open"])
    assert _n_tc(p) >= 1
    flag = ctypes.c_int(-1)
    assert tnc.lib.tnc_device_error(ctypes.byref(flag)) == 0
    assert flag.value == 0


def test_bounded_wait_gives_up_and_device_stays_usable(tnc):
    """The kernels' bounded mbarrier wait, on a phase nothing completes, gives
    up after its limit with TNC_ETIMEOUT; the context stays usable and the
    kernels' error flag is untouched."""
    import ctypes
    timed_out = ctypes.c_int(-1)
    rc = tnc.lib.tnc_selftest_bounded_wait(20000, ctypes.byref(timed_out))  # 20 ms
    assert rc == tnc.TNC_ETIMEOUT and timed_out.value == 1
    gl = C.random_2d(3, 3, 6, 1)
    bits = C.random_bitstrings(9, 4, 2)
    got, _ = _run(tnc, gl, bits, "split_bf16")
    assert O.rel_error(got, O.statevector_amplitudes(gl, bits), 9).max() <= TOL["split_bf16"]
    flag = ctypes.c_int(-1)
    assert tnc.lib.tnc_device_error(ctypes.byref(flag)) == 0
    assert flag.value == 0


def test_iqp_5x8_full_size_autotuned_as_benchmarked(tnc):
    """The benchmark's own plan (5 x 8 IQP, 256 bitstrings, split-BF16, the
    same planner seed and trials), autotuned as the benchmark does, against
    the transfer-matrix closed form: the kernel variants the benchmark times
    (persistent on-chip-split, plane-fed, hybrid and ring-fed tiles) on their real
    shapes and scattered layouts."""
    gl = C.iqp(5, 8, 0)
    bits = C.random_bitstrings(40, 256, 11)
    p = tnc.Plan(tnc.Network(gl), max_batch=256, form="split_bf16", seed=1, ssa_trials=64)
    ws = tnc.alloc_workspace(p)
    p.autotune(ws, reps=2)
    tiles = {t for k, t in p.get_kernels() if k == 4}
    assert tiles & {9, 11, 12, 13, 14, 15, 16, 17, 18}, tiles  # persistent tiles chosen somewhere
    got = tnc.contract_amplitudes(p, bits, ws=ws).cpu().numpy()
    ref = O.iqp_transfer_amplitudes(gl, bits)
    assert O.rel_error(got, ref, 40).max() <= TOL["split_bf16"]
