"""Host-side tests of the C ABI (no GPU): the library loads and exports every
declared entry point, argument checks return the documented status codes,
and the planner's tree and the compiled node program reproduce the FP64
oracle when executed on the host."""
import os
import re

import numpy as np
import pytest

import circuits as C
import oracle as O
from paper_2208_01498_gb300 import tnc
from host_emulator import contract_tree, emulate_program
from plan_cases import GROUPED_CASE, SLICING_CAPS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "tnc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnc_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(tnc.lib, n), n
    assert set(names) <= set(tnc.EXPORTED)


def test_status_strings():
    assert tnc.lib.tnc_status_string(0) == b"ok"
    assert tnc.lib.tnc_status_string(-2).startswith(b"out of memory")


def _arrays(gl):
    return gl.arrays()


def test_invalid_networks_are_rejected():
    gl = C.random_2d(2, 2, 2, 0)
    coords, arity, qubits, mats = _arrays(gl)
    bad_q = qubits.copy()
    bad_q[0] = 17
    with pytest.raises(tnc.TncError) as ei:
        tnc.Network(arrays=(coords, arity, bad_q, mats))
    assert ei.value.status == tnc.TNC_EINVAL
    bad_a = arity.copy()
    bad_a[0] = 3
    with pytest.raises(tnc.TncError):
        tnc.Network(arrays=(coords, bad_a, qubits, mats))
    twice = qubits.copy()
    i2 = int(np.flatnonzero(arity == 2)[0])
    off = int(arity[:i2].sum())
    twice[off + 1] = twice[off]
    with pytest.raises(tnc.TncError):
        tnc.Network(arrays=(coords, arity, twice, mats))
    nan = mats.copy()
    nan[3] = np.nan
    with pytest.raises(tnc.TncError):
        tnc.Network(arrays=(coords, arity, qubits, nan))


def test_invalid_plan_options_are_rejected():
    net = tnc.Network(C.random_2d(2, 2, 2, 0))
    for kw in (dict(open_qubits=[7]), dict(open_qubits=[1, 1]), dict(max_batch=0), dict(form=5)):
        with pytest.raises(tnc.TncError) as ei:
            tnc.Plan(net, **kw)
        assert ei.value.status == tnc.TNC_EINVAL


def test_unsatisfiable_memory_cap():
    net = tnc.Network(C.random_2d(3, 3, 6, 1))
    with pytest.raises(tnc.TncError) as ei:
        tnc.Plan(net, mem_cap_bytes=64)
    assert ei.value.status == tnc.TNC_ENOMEM


@pytest.mark.parametrize("oq,batch", [([], 1), ([1, 5], 1), ([], 4), ([3, 9, 12], 3)])
def test_tree_and_program_match_oracle_rand2d_4x4_d8(oq, batch):
    gl, _ = C.workload("rand2d_4x4_d8", 0)
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=batch)
    e = p.export()
    bits = C.random_bitstrings(16, batch, 3)
    ref = O.statevector_amplitudes(gl, bits, oq)
    assert np.allclose(contract_tree(e, bits), ref, atol=1e-14)
    em = emulate_program(e, bits)
    assert O.rel_error(em, ref, 16).max() < 1e-5


@pytest.mark.parametrize("family", ["sycamore", "iqp", "layered", "ghz", "single"])
def test_program_matches_oracle_families(family):
    if family == "sycamore":
        gl = C.sycamore(3, 6, 4)
    elif family == "iqp":
        gl = C.iqp(3, 3, 2)
    elif family == "layered":
        gl = C.layered_3d(3, 4, 7)
    elif family == "ghz":
        gl = C.ghz(2, 3)
    else:
        gl = C.GateList(3, np.zeros((3, 2)))
        gl.add((0,), C.H)
        gl.add((2,), C.haar_1q(np.random.default_rng(0)))
    n = gl.n_qubits
    bits = C.random_bitstrings(n, 3, 9)
    oq = [0] if n > 1 else []
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=3)
    e = p.export()
    ref = O.statevector_amplitudes(gl, bits, oq)
    assert np.allclose(contract_tree(e, bits), ref, atol=1e-14)
    assert O.rel_error(emulate_program(e, bits), ref, n).max() < 1e-5


@pytest.mark.parametrize("cap,group", SLICING_CAPS)
def test_slicing_sums_to_the_unsliced_result(cap, group):
    gl = C.random_2d(4, 5, 10, 2)
    bits = C.random_bitstrings(20, 2, 3)
    oq = [0, 7]
    ref = O.statevector_amplitudes(gl, bits, oq)
    p = tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=2, mem_cap_bytes=cap, max_group_log2=group)
    e = p.export()
    assert len(e["sliced_serial"]) + len(e["sliced_par"]) >= 1
    assert p.report["n_slice_groups"] == 2 ** len(e["sliced_serial"])
    assert O.rel_error(emulate_program(e, bits), ref, 20).max() < 1e-5
    # the slice groups add up: each group alone is a partial sum
    parts = sum(emulate_program(e, bits, groups=[g]) for g in range(min(4, e["program"]["n_groups"])))
    rest = emulate_program(e, bits, groups=range(min(4, e["program"]["n_groups"]), e["program"]["n_groups"]))
    assert O.rel_error(parts + rest, ref, 20).max() < 1e-5


def test_grouped_case_sums_to_the_unsliced_result():
    gl = C.random_2d(*GROUPED_CASE["shape"])
    bits = C.random_bitstrings(20, GROUPED_CASE["batch"], 5)
    ref = O.statevector_amplitudes(gl, bits)
    p = tnc.Plan(tnc.Network(gl), max_batch=GROUPED_CASE["batch"], mem_cap_bytes=GROUPED_CASE["cap"],
                 max_group_log2=GROUPED_CASE["max_group_log2"])
    e = p.export()
    assert len(e["sliced_par"]) >= 1
    assert O.rel_error(emulate_program(e, bits), ref, 20).max() < 1e-5


def test_grouped_slices_run_as_batch():
    gl = C.random_2d(3, 4, 8, 5)
    bits = C.random_bitstrings(12, 1, 1)
    ref = O.statevector_amplitudes(gl, bits)
    # one candidate tree, so that the cap cannot be met by another tree unsliced
    one = dict(n_starts=1, embedding="collapsed")
    full = tnc.Plan(tnc.Network(gl), **one).report
    p = tnc.Plan(tnc.Network(gl), mem_cap_bytes=int(full["peak_bytes"] * 0.3), max_group_log2=2, **one)
    e = p.export()
    assert len(e["sliced_serial"]) + len(e["sliced_par"]) >= 1
    assert O.rel_error(emulate_program(e, bits), ref, 12).max() < 1e-5


def test_plan_cost_equals_counted_work():
    """Sum over nodes of 2 M (Eq. 3) equals the work the program issues."""
    gl, _ = C.workload("rand2d_4x4_d8", 1)
    p = tnc.Plan(tnc.Network(gl), open_qubits=[4], max_batch=2)
    e = p.export()
    eq3 = sum(2 * 2.0 ** n["cost_log2"] for n in e["nodes"] if n["left"] >= 0)
    flat = [q for s in e["steps"] for q in (s["problems"] if s["kind"] == 2 else [s] if s["kind"] == 1 else [])]
    counted = sum(2.0 * s["batch"] * s["M"] * s["N"] * s["K"] for s in flat)
    assert abs(eq3 - counted) / counted < 1e-12
    assert abs(p.report["paper_ops"] - counted) / counted < 1e-12
    assert abs(p.report["real_flops"] - 4 * counted) / counted < 1e-12
    assert abs(np.log2(counted) - p.report["tree_cost_log2"]) < 1e-9


def test_tree_order_independence_on_host():
    gl = C.random_2d(3, 4, 8, 3)
    bits = C.random_bitstrings(12, 2, 4)
    vals = []
    for seed in (1, 2, 3):
        e = tnc.Plan(tnc.Network(gl), max_batch=2, seed=seed).export()
        vals.append(contract_tree(e, bits))
    assert np.allclose(vals[0], vals[1], atol=1e-14) and np.allclose(vals[0], vals[2], atol=1e-14)


def test_every_leaf_and_label_is_used_once():
    gl, _ = C.workload("sycamore_7x7_c14", 0, reduced=True)
    e = tnc.Plan(tnc.Network(gl), open_qubits=[1, 3]).export()
    leaves_in_tree = sorted(n["leaf"] for n in e["nodes"] if n["left"] < 0)
    assert leaves_in_tree == list(range(len(e["leaves"])))
    # every non-final label is held by exactly two leaves (a wire or a bond)
    finals = set(e["final_label"])
    count = {}
    for L in e["leaves"]:
        for x in L["labels"]:
            count[x] = count.get(x, 0) + 1
    assert all(c == 2 for x, c in count.items() if x not in finals)
    assert all(count[x] == 1 for x in finals)


def test_batch_workspace_covers_every_request():
    plans = [tnc.Plan(tnc.Network(C.random_2d(3, 4, 8, s)), max_batch=4) for s in range(3)]
    need = tnc.batch_ws_bytes(plans)
    assert need >= sum((p.ws_bytes + 255) // 256 * 256 for p in plans)
    assert need % 256 == 0
