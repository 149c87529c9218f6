"""Host-side checks of the plans the GPU tests and the benchmark rely on.

The planner (separator hierarchy over two embeddings and several seeds,
refined, then sliced under a memory cap) decides which kernels a contraction
runs.  These checks make sure the GPU tests' workloads still exercise what
they name (a tcgen05 step, sliced and grouped labels) and pin the planner's
invariants: the refinement never raises the Eq. 3 cost nor enlarges the
largest intermediate, slicing meets the cap, the 8 x 8 depth-16 workload
plans under 180 GB, and trees beyond the executor's 48 binary indices are
refused for execution (and costed with tree_only).
"""
import pytest

import circuits as C
from plan_cases import RAND8X8_D16_CAP, RAND6X6_D16_CAP, GROUPED_CASE, PARTIAL_CASE, SLICING_CAPS, TC_CASE

tnc = pytest.importorskip("paper_2208_01498_gb300.tnc")


def _n_tc(p):
    return sum(1 for k, _ in p.get_kernels() if k == tnc.KG["tc"])


@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
def test_tc_case_has_a_tensor_core_step(form):
    gl = C.random_2d(*TC_CASE["shape"])
    p = tnc.Plan(tnc.Network(gl), open_qubits=TC_CASE["open"], max_batch=TC_CASE["batch"], form=form)
    assert _n_tc(p) >= 1
    assert p.ws_bytes <= 64 << 20  # also the no-allocation test's tensor-core case


def test_slicing_cases_slice():
    gl = C.random_2d(4, 5, 10, 2)
    for cap, group in SLICING_CAPS:
        p = tnc.Plan(tnc.Network(gl), open_qubits=[0, 7], max_batch=2, mem_cap_bytes=cap, max_group_log2=group)
        assert p.report["n_sliced"] >= 1, cap
    p = tnc.Plan(tnc.Network(gl), open_qubits=PARTIAL_CASE["open"], max_batch=PARTIAL_CASE["batch"],
                 mem_cap_bytes=PARTIAL_CASE["cap"], max_group_log2=PARTIAL_CASE["max_group_log2"])
    assert p.report["n_slice_groups"] >= 4


def test_grouped_case_groups_a_label():
    gl = C.random_2d(*GROUPED_CASE["shape"])
    p = tnc.Plan(tnc.Network(gl), max_batch=GROUPED_CASE["batch"], mem_cap_bytes=GROUPED_CASE["cap"],
                 max_group_log2=GROUPED_CASE["max_group_log2"])
    ex = p.export()
    assert len(ex["sliced_par"]) >= 1 and len(ex["sliced_serial"]) >= 1


@pytest.mark.parametrize("form", ["fp32", "split_bf16", "3xtf32"])
def test_rand2d_6x6_d16_slices_under_its_cap(form):
    gl, _ = C.workload("rand2d_8x8_d16", 0, reduced=True)
    p = tnc.Plan(tnc.Network(gl), max_batch=1, form=form, mem_cap_bytes=RAND6X6_D16_CAP, ssa_trials=64)
    assert p.report["n_sliced"] >= 1
    assert p.ws_bytes < 1.5 * RAND6X6_D16_CAP
    if form != "fp32":
        assert _n_tc(p) >= 1


@pytest.mark.parametrize("clifford", [False, True])
def test_rand2d_8x8_d16_plans_under_180_gb(clifford):
    """The 8 x 8 depth-16 workload: sliced under 180 GB at a small multiple of
    its unsliced tree's work (about 5e15 real flops, against 8e18 for the
    greedy slicer over the plain separator tree)."""
    gl, _ = C.workload("rand2d_8x8_d16", 0, clifford=clifford)
    net = tnc.Network(gl)
    for form in ("split_bf16", "3xtf32"):
        p = tnc.Plan(net, max_batch=1, form=form, mem_cap_bytes=RAND8X8_D16_CAP, ssa_trials=64)
        r = p.report
        assert r["ws_bytes"] <= RAND8X8_D16_CAP
        assert 1e15 < r["real_flops"] < 1e16, r["real_flops"]
        assert r["n_sliced"] >= 1
        unsliced = 4 * 2.0 ** r["tree_cost_log2"]  # real flops of the tree without slicing
        assert r["real_flops"] < 4 * unsliced
        assert _n_tc(p) >= 10


@pytest.mark.parametrize("case", ["r4x4d19", "r5x5d13", "iqp5x8", "syc4x4"])
def test_refinement_never_raises_cost_or_rank(case):
    gl = {"r4x4d19": lambda: C.random_2d(4, 4, 19, 1), "r5x5d13": lambda: C.random_2d(5, 5, 13, 7),
          "iqp5x8": lambda: C.iqp(5, 8, 0), "syc4x4": lambda: C.sycamore(4, 14, 0)}[case]()
    net = tnc.Network(gl)
    for seed in (1, 2):
        # one candidate tree (one embedding, one seed): refined against itself
        kw = dict(max_batch=16, embedding="collapsed", n_starts=1, seed=seed)
        a = tnc.Plan(net, refine_window=0, **kw).report
        b = tnc.Plan(net, refine_window=8, **kw).report
        assert abs(b["sep_cost_log2"] - a["tree_cost_log2"]) < 1e-9  # same separator tree
        assert b["tree_cost_log2"] <= a["tree_cost_log2"] + 1e-9
        assert b["max_rank"] <= a["max_rank"]
        # several candidates (four layer distances): the cheapest refined tree is no costlier
        kw = dict(max_batch=16, embedding="spacetime", n_starts=1, seed=seed)
        a = tnc.Plan(net, refine_window=0, **kw).report
        b = tnc.Plan(net, refine_window=8, **kw).report
        assert b["tree_cost_log2"] <= a["tree_cost_log2"] + 1e-9


def test_space_time_embedding_helps_deep_circuits():
    """On a deep, narrow circuit the separators of the (d+1)-dimensional
    embedding can cut in time; the automatic choice keeps the cheaper tree."""
    net = tnc.Network(C.random_2d(4, 4, 19, 1))
    kw = dict(max_batch=16, refine_window=0, n_starts=4)
    col = tnc.Plan(net, embedding="collapsed", **kw).report
    st = tnc.Plan(net, embedding="spacetime", **kw).report
    auto = tnc.Plan(net, embedding="auto", **kw).report
    assert st["tree_cost_log2"] < col["tree_cost_log2"] - 2
    assert auto["tree_cost_log2"] == min(st["tree_cost_log2"], col["tree_cost_log2"])
    assert auto["embedding_used"] == 2 and auto["time_scale"] > 0


def test_rank_beyond_the_executor_is_refused():
    net = tnc.Network(C.random_2d(10, 10, 20, 3))
    with pytest.raises(tnc.TncError) as ei:
        tnc.Plan(net, max_batch=16, n_starts=1)
    assert ei.value.status == tnc.TNC_ENOMEM
    assert "binary indices" in str(ei.value)


def test_tree_only_costs_trees_beyond_the_executor():
    """tree_only: the same network gets its tree and Eq. 3 cost (no device
    program, so no rank limit), costed no higher than any compiled tree the
    planner could pick; the plan refuses upload and autotuning."""
    net = tnc.Network(C.random_2d(10, 10, 20, 3))
    p = tnc.Plan(net, max_batch=16, n_starts=1, tree_only=True)
    r = p.report
    assert r["max_rank"] > 48 and 0 < r["tree_cost_log2"] < 200
    assert abs(r["paper_ops"] - 2.0 ** r["tree_cost_log2"]) <= 1e-9 * r["paper_ops"]
    assert r["ws_bytes"] == 0 and r["n_launches"] == 0
    e = p.export()
    assert len(e["nodes"]) == 2 * r["n_leaves"] - 1 and e["program"]["ws_bytes"] == 0
    assert tnc.lib.tnc_plan_upload(p.handle, None) == tnc.TNC_ESTATE  # refused before any CUDA call
    # a compilable network: tree_only reports the same tree cost as the full plan
    small = tnc.Network(C.random_2d(4, 4, 8, 1))
    full = tnc.Plan(small, max_batch=16).report
    only = tnc.Plan(small, max_batch=16, tree_only=True).report
    assert abs(full["tree_cost_log2"] - only["tree_cost_log2"]) < 1e-9


def test_invalid_planner_options():
    net = tnc.Network(C.random_2d(3, 3, 4, 1))
    for kw in (dict(refine_window=2), dict(refine_window=13), dict(n_starts=65), dict(embedding=3)):
        with pytest.raises(tnc.TncError) as ei:
            tnc.Plan(net, **kw)
        assert ei.value.status == tnc.TNC_EINVAL
