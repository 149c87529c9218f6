"""Parity of the CUDA path with the FP64 oracle (GPU).

Every test calls the C ABI through the binding and compares amplitudes
element by element with an oracle evaluated on the same seeded circuit, using
the benchmark's error measure |a - a_ref| / max(|a_ref|, 2^{-n/2}): at most
1e-5 for the FP32 and 3xTF32 forms, 1e-4 for split-BF16.
"""
import math

import numpy as np
import pytest

import circuits as C
import oracle as O
from oracle.stabilizer import stabilizer_amplitudes
from plan_cases import GROUPED_CASE, PARTIAL_CASE, SLICING_CAPS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "3xtf32": 1e-5, "split_bf16": 1e-4}


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _run(tnc, gl, bits, oq=(), form="fp32", **kw):
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=max(1, bits.shape[0]), form=form, **kw)
    out = tnc.contract_amplitudes(p, bits)
    torch.cuda.synchronize()
    return out.cpu().numpy(), p


def _check(got, ref, n, form="fp32"):
    err = O.rel_error(got, ref, n)
    assert err.max() <= TOL[form], f"max rel error {err.max():.3g} ({form})"
    return err.max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rand2d_4x4_d8_single_amplitude(tnc, seed):
    gl, info = C.workload("rand2d_4x4_d8", seed)
    ref = O.statevector_amplitudes(gl, info["bits"])
    got, _ = _run(tnc, gl, info["bits"])
    _check(got, ref, 16)


@pytest.mark.parametrize("family", ["rand2d", "sycamore", "iqp", "layered", "ghz"])
def test_families_batch_and_open_legs(tnc, family):
    gl = {"rand2d": lambda: C.random_2d(4, 4, 10, 3), "sycamore": lambda: C.sycamore(4, 8, 1),
          "iqp": lambda: C.iqp(4, 4, 3), "layered": lambda: C.layered_3d(4, 4, 5),
          "ghz": lambda: C.ghz(4, 4)}[family]()
    bits = C.random_bitstrings(16, 5, 7)
    oq = [2, 9, 13]
    ref = O.statevector_amplitudes(gl, bits, oq)
    got, _ = _run(tnc, gl, bits, oq)
    _check(got, ref, 16)


def test_batch_smaller_than_planned(tnc):
    gl = C.random_2d(3, 4, 8, 8)
    bits = C.random_bitstrings(12, 3, 2)
    p = tnc.Plan(tnc.Network(gl), open_qubits=[5], max_batch=16)
    out = tnc.contract_amplitudes(p, bits)
    ref = O.statevector_amplitudes(gl, bits, [5])
    _check(out.cpu().numpy(), ref, 12)


def test_all_legs_open_normalisation(tnc):
    gl = C.random_2d(3, 3, 6, 4)
    got, _ = _run(tnc, gl, np.zeros((1, 9), np.uint8), list(range(9)))
    assert abs(np.sum(np.abs(got) ** 2) - 1.0) < 1e-5
    ref = O.statevector_amplitudes(gl, np.zeros((1, 9), np.uint8), list(range(9)))
    _check(got, ref, 9)


def test_single_qubit_and_gate_free_networks(tnc):
    gl = C.GateList(3, np.zeros((3, 2)))
    gl.add((0,), C.H)
    gl.add((1,), C.haar_1q(np.random.default_rng(1)))
    bits = C.random_bitstrings(3, 4, 1)
    ref = O.statevector_amplitudes(gl, bits, [1])
    got, _ = _run(tnc, gl, bits, [1])
    _check(got, ref, 3)


def test_ghz_full_size(tnc):
    gl = C.ghz(8, 8)
    bits = np.array([[0] * 64, [1] * 64], np.uint8)
    got, _ = _run(tnc, gl, bits)
    assert np.allclose(got.ravel(), [1 / math.sqrt(2)] * 2, rtol=1e-5, atol=0)


def test_mirror_identity(tnc):
    gl = C.mirror(C.random_2d(4, 4, 6, 2))
    bits = np.vstack([np.zeros((1, 16), np.uint8), C.random_bitstrings(16, 3, 3)])
    got, _ = _run(tnc, gl, bits)
    assert abs(got[0, 0] - 1) < 1e-5
    assert np.abs(got[1:]).max() < 1e-5


def test_tree_order_independence(tnc):
    gl = C.random_2d(4, 5, 10, 6)
    bits = C.random_bitstrings(20, 4, 5)
    ref = O.statevector_amplitudes(gl, bits)
    vals = []
    for seed in (1, 2, 3):
        got, _ = _run(tnc, gl, bits, seed=seed)
        _check(got, ref, 20)
        vals.append(got)
    assert O.rel_error(vals[0], vals[1], 20).max() < 2e-5
    assert O.rel_error(vals[0], vals[2], 20).max() < 2e-5


@pytest.mark.parametrize("cap,group", SLICING_CAPS)
def test_slicing(tnc, cap, group):
    gl = C.random_2d(4, 5, 10, 2)
    bits = C.random_bitstrings(20, 2, 3)
    oq = [0, 7]
    ref = O.statevector_amplitudes(gl, bits, oq)
    got, p = _run(tnc, gl, bits, oq, mem_cap_bytes=cap, max_group_log2=group)
    assert p.report["n_sliced"] >= 1
    _check(got, ref, 20)


def test_grouped_and_serial_slices(tnc):
    gl = C.random_2d(*GROUPED_CASE["shape"])
    bits = C.random_bitstrings(20, GROUPED_CASE["batch"], 5)
    ref = O.statevector_amplitudes(gl, bits)
    got, p = _run(tnc, gl, bits, mem_cap_bytes=GROUPED_CASE["cap"], max_group_log2=GROUPED_CASE["max_group_log2"])
    ex = p.export()
    assert len(ex["sliced_par"]) >= 1 and len(ex["sliced_serial"]) >= 1
    _check(got, ref, 20)


def test_partial_slice_groups_add_up(tnc):
    gl = C.random_2d(4, 5, 10, 2)
    bits = C.random_bitstrings(20, 2, 3)
    p = tnc.Plan(tnc.Network(gl), open_qubits=PARTIAL_CASE["open"], max_batch=PARTIAL_CASE["batch"],
                 mem_cap_bytes=PARTIAL_CASE["cap"], max_group_log2=PARTIAL_CASE["max_group_log2"])
    ng = p.report["n_slice_groups"]
    assert ng >= 4
    db = torch.from_numpy(bits).cuda()
    full = tnc.contract_amplitudes_dbits(p, db)
    a = tnc.contract_partial(p, db, 0, ng // 3)
    b = tnc.contract_partial(p, db, ng // 3, ng)
    torch.cuda.synchronize()
    assert O.rel_error((a + b).cpu().numpy(), full.cpu().numpy(), 20).max() < 1e-9


def test_rand2d_4x4_d8_clifford_twin(tnc):
    gl, _ = C.workload("rand2d_4x4_d8", 3, clifford=True)
    bits = C.random_bitstrings(16, 8, 2)
    ref = stabilizer_amplitudes(gl, bits, [0, 5])
    got, _ = _run(tnc, gl, bits, [0, 5])
    _check(got, ref, 16)


def test_sycamore_4x4_c14(tnc):
    gl, info = C.workload("sycamore_7x7_c14", 0, reduced=True)
    ref = O.statevector_amplitudes(gl, info["bits"], info["open"])
    got, _ = _run(tnc, gl, info["bits"], info["open"])
    _check(got, ref, 16)


@pytest.fixture(scope="module")
def sycamore_5x5_c14():
    """The Sycamore-type rules on a 5 x 5 grid (14 cycles of fSim(pi/2, pi/6)
    on the staggered ABCD matchings, 6 seed-random open qubits, one
    seed-random bitstring for the other 19): 25 qubits, within the state
    vector (about two minutes on the host)."""
    gl = C.sycamore(5, 14, 0)
    bits = C.random_bitstrings(25, 1, 0)
    oq = [int(q) for q in C.random_open_qubits(25, 6, 0)]
    return gl, bits, oq, O.statevector_amplitudes(gl, bits, oq)


@pytest.mark.parametrize("form", ["fp32", "split_bf16", "3xtf32"])
def test_sycamore_5x5_c14(tnc, sycamore_5x5_c14, form):
    gl, bits, oq, ref = sycamore_5x5_c14
    got, p = _run(tnc, gl, bits, oq, form=form)
    assert got.shape == (1, 64)
    _check(got, ref, 25, form)


def test_iqp_4x5_wht(tnc):
    gl, info = C.workload("iqp_5x8", 0, reduced=True)
    ref = O.iqp_wht_amplitudes(gl, info["bits"])
    got, _ = _run(tnc, gl, info["bits"])
    _check(got, ref, 20)


@pytest.mark.parametrize("L", [4, 5])
def test_serving_pool_layered_instances(tnc, L):
    gl = C.layered_3d(L, 4, seed=100 + L)
    bits = C.random_bitstrings(L * L, 16, 1)
    ref = O.statevector_amplitudes(gl, bits)
    got, _ = _run(tnc, gl, bits)
    _check(got, ref, L * L)


def test_iqp_5x8_full_size_transfer_matrix(tnc):
    """40 qubits, 256 bitstrings: the benchmark workload, FP32 form."""
    gl, info = C.workload("iqp_5x8", 0)
    ref = O.iqp_transfer_amplitudes(gl, info["bits"])
    got, _ = _run(tnc, gl, info["bits"])
    _check(got, ref, 40)


def test_iqp_5x8_full_size_clifford_twin(tnc):
    gl, info = C.workload("iqp_5x8", 1, clifford=True)
    bits = info["bits"][:64]
    ref = stabilizer_amplitudes(gl, bits)
    got, _ = _run(tnc, gl, bits)
    _check(got, ref, 40)


def test_workspace_errors(tnc):
    gl = C.random_2d(3, 3, 4, 1)
    p = tnc.Plan(tnc.Network(gl))
    small = torch.empty(max(p.ws_bytes // 2, 256), dtype=torch.uint8, device="cuda")
    with pytest.raises(tnc.TncError) as ei:
        tnc.contract_amplitudes(p, np.zeros((1, 9), np.uint8), ws=small)
    assert ei.value.status == tnc.TNC_ENOMEM
    big = torch.empty(p.ws_bytes + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(tnc.TncError) as ei:
        tnc.contract_amplitudes(p, np.zeros((1, 9), np.uint8), ws=big[8:])
    assert ei.value.status == tnc.TNC_EINVAL
    with pytest.raises(tnc.TncError) as ei:
        tnc.contract_amplitudes(p, np.zeros((2, 9), np.uint8))
    assert ei.value.status == tnc.TNC_EINVAL


def test_profiling_counts_every_step(tnc):
    gl = C.random_2d(3, 4, 8, 2)
    p = tnc.Plan(tnc.Network(gl))
    p.set_profiling(True)
    for _ in range(3):
        tnc.contract_amplitudes(p, np.zeros((1, 12), np.uint8))
    prof = p.profile()
    assert (prof["runs"] == 3).all()
    assert (prof["ms"] > 0).all()
    assert abs(prof["flops"].sum() - p.report["real_flops"]) / p.report["real_flops"] < 1e-12


def test_autotuned_plan_stays_correct(tnc):
    gl = C.random_2d(4, 5, 10, 6)
    bits = C.random_bitstrings(20, 8, 5)
    ref = O.statevector_amplitudes(gl, bits)
    for form in ("fp32", "split_bf16"):
        p = tnc.Plan(tnc.Network(gl), max_batch=8, form=form)
        ws = tnc.alloc_workspace(p)
        p.autotune(ws, reps=2)
        got = tnc.contract_amplitudes(p, bits, ws=ws).cpu().numpy()
        _check(got, ref, 20, form)
