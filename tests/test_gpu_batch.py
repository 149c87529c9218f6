"""Several requests on different circuits contracted together
(tnc_contract_batch): their nodes run wave by wave in grouped launches across
requests (grouped narrow nodes, grouped CUDA-core cGEMMs per tile shape), the
tensor-core and split-K nodes per request.  Each result must equal the same
request contracted alone (the nodes do the same arithmetic: bit for bit) and
the FP64 oracle within the form's tolerance, |a - a_ref| / max(|a_ref|,
2^{-n/2}) <= 1e-5 (FP32, 3xTF32) or 1e-4 (split-BF16)."""
import numpy as np
import pytest

import circuits as C
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "3xtf32": 1e-5, "split_bf16": 1e-4}


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


# (circuit, open qubits, batch): circuits of the serving mix, 16 to 20 qubits
POOL = [
    (lambda: C.random_2d(4, 4, 19, 1), [], 16),
    (lambda: C.random_2d(4, 5, 10, 2), [0, 3], 16),  # a tensor-core node in the split forms
    (lambda: C.layered_3d(4, 4, 100), [5], 3),
    (lambda: C.iqp(4, 4, 2), [1], 8),
    (lambda: C.sycamore(4, 8, 1), [2, 9], 2),
    (lambda: C.random_2d(4, 4, 8, 7), [], 1),
]


@pytest.mark.parametrize("form", ["fp32", "split_bf16", "3xtf32"])
def test_batch_equals_each_request_alone(tnc, form):
    reqs = []
    for i, (make, oq, batch) in enumerate(POOL):
        gl = make()
        p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=batch, form=form)
        reqs.append((gl, oq, p, C.random_bitstrings(gl.n_qubits, batch, 31 + i)))
    alone = [tnc.contract_amplitudes(p, bits).cpu().numpy() for _, _, p, bits in reqs]
    outs = tnc.contract_batch([r[2] for r in reqs], [r[3] for r in reqs])
    torch.cuda.synchronize()
    for (gl, oq, p, bits), a, o in zip(reqs, alone, outs):
        got = o.cpu().numpy()
        assert np.array_equal(got, a), f"{gl.name}: batch differs from alone by {np.abs(got - a).max():.3g}"
        ref = O.statevector_amplitudes(gl, bits, oq)
        assert O.rel_error(got, ref, gl.n_qubits).max() <= TOL[form], gl.name


def test_batch_twice_and_of_one(tnc):
    """The same plan twice in one batch, and a batch of one request."""
    gl = C.random_2d(4, 4, 10, 3)
    p = tnc.Plan(tnc.Network(gl), open_qubits=[2], max_batch=4)
    b1, b2 = C.random_bitstrings(16, 4, 1), C.random_bitstrings(16, 3, 2)
    o1, o2 = tnc.contract_batch([p, p], [b1, b2])
    (o3,) = tnc.contract_batch([p], [b2])
    assert np.array_equal(o1.cpu().numpy(), tnc.contract_amplitudes(p, b1).cpu().numpy())
    assert np.array_equal(o2.cpu().numpy(), o3.cpu().numpy())
    assert O.rel_error(o2.cpu().numpy(), O.statevector_amplitudes(gl, b2, [2]), 16).max() <= 1e-5


def test_batch_refuses_sliced_plans_and_small_workspaces(tnc):
    gl = C.random_2d(4, 5, 10, 2)
    sliced = tnc.Plan(tnc.Network(gl), max_batch=2, mem_cap_bytes=1 << 16, max_group_log2=0)
    assert sliced.report["n_slice_groups"] > 1
    plain = tnc.Plan(tnc.Network(gl), max_batch=2)
    bits = C.random_bitstrings(20, 2, 0)
    with pytest.raises(tnc.TncError) as ei:
        tnc.contract_batch([plain, sliced], [bits, bits])
    assert ei.value.status == tnc.TNC_EINVAL
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(tnc.TncError) as ei:
        tnc.contract_batch([plain, plain], [bits, bits], ws=small)
    assert ei.value.status == tnc.TNC_ENOMEM
