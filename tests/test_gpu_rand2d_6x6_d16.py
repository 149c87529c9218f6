"""The 6 x 6 depth-16 random circuit (the reduction of the 8 x 8 depth-16
workload: Haar single-qubit gates, CZ on brick patterns A, B, C, D) contracted
along its separator tree on the GPU, against the stored amplitude that the
FP64 side-wise oracle computed (tests/golden/make_golden.py, which calls only
the oracle).  36 qubits put this beyond the state-vector oracle; the refined
separator tree costs about 1.4e12 real flops, with the largest nodes on the
tensor cores.

Error measure |a - a_ref| / max(|a_ref|, 2^{-n/2}) with n = 36: at most 1e-5
for the FP32 and 3xTF32 forms, 1e-4 for split-BF16.  Unsliced the refined
tree needs about 1 GB; with a 256 MiB memory cap the planner slices two to four
labels, so the serial slice loop and the FP64 accumulation run at full size
too.
"""
import json
import os

import numpy as np
import pytest

import circuits as C
import oracle as O
from plan_cases import RAND6X6_D16_CAP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rand2d_6x6_d16_sidewise.json")
TOL = {"fp32": 1e-5, "3xtf32": 1e-5, "split_bf16": 1e-4}


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(GOLDEN):
        pytest.skip("golden amplitude not generated")
    with open(GOLDEN) as f:
        g = json.load(f)
    gl, info = C.workload("rand2d_8x8_d16", 0, reduced=True)
    bits = np.asarray(g["bits"], np.uint8)[None, :]
    assert np.array_equal(bits, info["bits"][:1])  # the generator still yields the stored case
    ref = np.array([[complex(*g["amplitude"])]])
    from paper_2208_01498_gb300 import tnc
    return tnc, gl, bits, ref


@pytest.mark.parametrize("form", ["fp32", "split_bf16", "3xtf32"])
def test_rand2d_6x6_d16_against_sidewise_oracle(case, form):
    tnc, gl, bits, ref = case
    p = tnc.Plan(tnc.Network(gl), max_batch=1, form=form, mem_cap_bytes=RAND6X6_D16_CAP, ssa_trials=64)
    assert p.ws_bytes < 1.5 * RAND6X6_D16_CAP
    assert p.report["n_sliced"] >= 1
    got = tnc.contract_amplitudes(p, bits).cpu().numpy()
    torch.cuda.synchronize()
    err = O.rel_error(got, ref, 36).max()
    assert err <= TOL[form], f"{form}: rel error {err:.3g}"
    del p
    torch.cuda.empty_cache()
