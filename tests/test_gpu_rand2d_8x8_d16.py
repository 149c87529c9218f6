"""The 8 x 8 depth-16 random circuit at full size (64 qubits, 448 CZ): one
amplitude of a seed-random bitstring, contracted along the refined separator
tree sliced under a 180 GB memory cap, in the split-BF16 and 3xTF32 forms.

No FP64 oracle reaches a random 64-qubit amplitude, so the pins at this size
are (i) the Clifford twin (same layout and schedule, single-qubit gates drawn
from the Clifford group; its plan is of the same size, about 4.9e15 real
flops), whose amplitude the oracle's CH form gives exactly, and (ii) agreement
of the two tensor-core forms on the random circuit.  Error measure |a - a_ref| /
max(|a_ref|, 2^{-n/2}) with n = 64: at most 1e-5 for 3xTF32, 1e-4 for
split-BF16.  The plan costs about 5.4e15 real flops (about 2^50 paper ops);
each contraction takes seconds to tens of seconds.
"""
import numpy as np
import pytest

import circuits as C
import oracle as O
from oracle.stabilizer import stabilizer_amplitudes
from plan_cases import RAND8X8_D16_CAP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"3xtf32": 1e-5, "split_bf16": 1e-4}
CAP = RAND8X8_D16_CAP


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < CAP:
        pytest.skip(f"needs {CAP / 1e9:.0f} GB of free device memory")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _amp(tnc, gl, bits, form):
    p = tnc.Plan(tnc.Network(gl), max_batch=1, form=form, mem_cap_bytes=CAP, ssa_trials=64)
    assert p.ws_bytes <= CAP and p.report["real_flops"] < 1e16
    ws = tnc.alloc_workspace(p)
    got = tnc.contract_amplitudes(p, bits, ws=ws).cpu().numpy()
    torch.cuda.synchronize()
    rep = p.report
    del ws, p
    torch.cuda.empty_cache()
    return got, rep


def _nonzero_clifford_bits(gl, seed):
    # a bitstring whose exact amplitude is nonzero (|a| = 2^{-r/2}); the error
    # measure of an exact zero at 64 qubits would sit below FP32 resolution
    for s in range(seed, seed + 64):
        bits = C.random_bitstrings(64, 1, s)
        ref = stabilizer_amplitudes(gl, bits)
        if abs(ref[0, 0]) > 0:
            return bits, ref
    pytest.fail("no nonzero Clifford-twin amplitude among 64 bitstrings")


@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
def test_rand2d_8x8_d16_clifford_twin_full_size(tnc, form):
    gl, _ = C.workload("rand2d_8x8_d16", 0, clifford=True)
    bits, ref = _nonzero_clifford_bits(gl, 0)
    got, rep = _amp(tnc, gl, bits, form)
    assert rep["n_sliced"] >= 1
    err = O.rel_error(got, ref, 64).max()
    assert err <= TOL[form], f"{form}: rel error {err:.3g} (|a_ref| = {abs(ref[0, 0]):.3g})"


def test_rand2d_8x8_d16_forms_agree(tnc):
    gl, info = C.workload("rand2d_8x8_d16", 0)
    bits = info["bits"][:1]
    a_bf16, _ = _amp(tnc, gl, bits, "split_bf16")
    a_tf32, _ = _amp(tnc, gl, bits, "3xtf32")
    # a random 64-qubit amplitude is of order 2^-32 (Porter-Thomas)
    assert 2.0**-40 < abs(a_tf32[0, 0]) < 2.0**-24
    err = O.rel_error(a_bf16, a_tf32, 64).max()
    assert err <= TOL["split_bf16"] + TOL["3xtf32"], f"split-BF16 vs 3xTF32: {err:.3g}"
