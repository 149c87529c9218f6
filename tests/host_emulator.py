"""Host-side checks of the planner and plan compiler (no GPU).

``contract_tree`` contracts the exported leaves along the exported tree with
NumPy complex128 (labels summed as soon as no tensor outside the subtree holds
them), projecting the final wires onto the requested bits itself.
``emulate_program`` executes the compiled node program (gather, permute,
GEMM, FP64 accumulation) exactly as the descriptors say, on a NumPy
workspace.  Both are test code: they read only the plan's JSON export.
"""
from __future__ import annotations

import numpy as np


def _leaf_tensor(leaf):
    data = np.array(leaf["re"], np.float64) + 1j * np.array(leaf["im"], np.float64)
    r = len(leaf["labels"])
    return data.reshape((2,) * r) if r else data.reshape(())


def contract_tree(e: dict, bits: np.ndarray) -> np.ndarray:
    """Amplitudes out[b, j] by contracting the exported tree per bitstring."""
    bits = np.atleast_2d(bits)
    n_open = len(e["open_qubits"])
    open_final = [e["final_label"][q] for q in e["open_qubits"]]
    fixed = {e["final_label"][q]: q for q in range(e["n_qubits"]) if q not in e["open_qubits"]}
    leaves = e["leaves"]
    nodes = e["nodes"]
    holders = {}
    for li, L in enumerate(leaves):
        for x in L["labels"]:
            if x not in fixed:
                holders.setdefault(x, set()).add(li)
    leafsets = {}

    def leafset(v):
        if v in leafsets:
            return leafsets[v]
        nd = nodes[v]
        s = {nd["leaf"]} if nd["left"] < 0 else leafset(nd["left"]) | leafset(nd["right"])
        leafsets[v] = s
        return s

    out = np.zeros((bits.shape[0], 1 << n_open), np.complex128)
    for b in range(bits.shape[0]):
        def rec(v):
            nd = nodes[v]
            if nd["left"] < 0:
                L = leaves[nd["leaf"]]
                t = _leaf_tensor(L)
                labs = list(L["labels"])
                for x in list(labs):
                    if x in fixed:
                        ax = labs.index(x)
                        t = np.take(t, int(bits[b, fixed[x]]), axis=ax)
                        labs.pop(ax)
                return t, labs
            ta, la = rec(nd["left"])
            tb, lb = rec(nd["right"])
            inside = leafset(v)
            allabs = list(dict.fromkeys(la + lb))
            keep = [x for x in allabs if x in open_final or not holders.get(x, set()) <= inside]
            sym = {x: i for i, x in enumerate(allabs)}
            r = np.einsum(ta, [sym[x] for x in la], tb, [sym[x] for x in lb], [sym[x] for x in keep])
            return r, keep
        t, labs = rec(e["root"])
        # order: open qubits, bit i of j = open_qubits[i]
        want = [e["final_label"][q] for q in reversed(e["open_qubits"])]
        assert sorted(labs) == sorted(want), (labs, want)
        t = np.transpose(t, [labs.index(x) for x in want]) if labs else t
        out[b] = np.asarray(t).reshape(-1)
    return out


def emulate_program(e: dict, bits: np.ndarray, groups=None) -> np.ndarray:
    """Run the compiled program on the host; returns complex128 out[b, j]."""
    bits = np.atleast_2d(np.asarray(bits, np.uint8))
    batch = bits.shape[0]
    pr = e["program"]
    base = (np.array(pr["base_re"], np.float32) + 1j * np.array(pr["base_im"], np.float32)).astype(np.complex64)
    nq = e["n_qubits"]
    maxb = 1 << e["beta_bits"]
    ws = np.full(pr["ws_bytes"] // 8 + 1, np.nan + 1j * np.nan, np.complex64)
    bitsbuf = np.zeros((maxb, nq), np.uint8)
    bitsbuf[:batch] = bits
    acc = pr["accum"]
    n_open = acc["n_open"]
    out = np.zeros((batch, 1 << n_open), np.complex128)
    if groups is None:
        groups = range(pr["n_groups"])
    for g in groups:
        for gd in pr["gathers"]:
            r = len(gd["out_src"])
            o = np.arange(1 << r, dtype=np.int64)
            src = np.zeros_like(o)
            beta = np.zeros_like(o)
            for j, s in enumerate(gd["out_src"]):
                bit = (o >> j) & 1
                if s >= 0:
                    src |= bit << s
                else:
                    beta |= bit << (-1 - s)
            for pos, q in zip(gd["fixed_pos"], gd["fixed_qubit"]):
                src |= (bitsbuf[beta, q].astype(np.int64) & 1) << pos
            for pos, k in zip(gd["sliced_pos"], gd["sliced_bit"]):
                src |= ((g >> k) & 1) << pos
            ws[gd["dst"] + o] = base[gd["src"] + src]
        flat = []
        for st in e["steps"]:
            flat += st["problems"] if st["kind"] == 2 else [st]
        for st in flat:
            if st.get("kind", 1) == 0:
                r = st["rank"]
                j = np.arange(1 << r, dtype=np.int64)
                i = np.zeros_like(j)
                for k, sb in enumerate(st["src_bit"]):
                    i |= ((j >> k) & 1) << sb
                ws[st["dst"] + j] = ws[st["src"] + i]
            else:
                Bn, M, N, K = st["batch"], st["M"], st["N"], st["K"]
                Ab = base if st["a_buf"] else ws
                Bb = base if st["b_buf"] else ws
                A = Ab[st["a"]: st["a"] + Bn * M * K].astype(np.complex128)
                A = A.reshape(Bn, K, M).transpose(0, 2, 1) if st["tA"] else A.reshape(Bn, M, K)
                Bm = Bb[st["b"]: st["b"] + Bn * K * N].astype(np.complex128)
                Bm = Bm.reshape(Bn, N, K).transpose(0, 2, 1) if st["tB"] else Bm.reshape(Bn, K, N)
                assert np.isfinite(A).all() and np.isfinite(Bm).all(), "read of an unwritten workspace slot"
                Cv = (A @ Bm).astype(np.complex64).reshape(-1)
                if st.get("c_ident", 1):
                    ws[st["c"]: st["c"] + Bn * M * N] = Cv
                else:
                    # element (b, m, n) at the bit positions c_pos: n bits, m bits, batch bits
                    idx = np.arange(Bn * M * N, dtype=np.int64)
                    nN, nM = int(np.log2(N)), int(np.log2(M))
                    n_, m_, b_ = idx % N, (idx // N) % M, idx // (N * M)
                    off = np.zeros_like(idx)
                    pos = st["c_pos"]
                    for i in range(nN):
                        off |= ((n_ >> i) & 1) << pos[i]
                    for i in range(nM):
                        off |= ((m_ >> i) & 1) << pos[nN + i]
                    for i in range(len(pos) - nN - nM):
                        off |= ((b_ >> i) & 1) << pos[nN + nM + i]
                    ws[st["c"] + off] = Cv
        rank = len(acc["role"])
        root = ws[acc["src"]: acc["src"] + (1 << rank)].astype(np.complex128)
        for beta in range(batch):
            for j in range(1 << n_open):
                base_off = 0
                for k in range(rank):
                    if acc["role"][k] == 0:
                        base_off |= ((beta >> acc["idx"][k]) & 1) << k
                    elif acc["role"][k] == 1:
                        base_off |= ((j >> acc["idx"][k]) & 1) << k
                s = 0
                for p in range(1 << acc["n_par"]):
                    off = base_off
                    for k in range(rank):
                        if acc["role"][k] == 2:
                            off |= ((p >> acc["idx"][k]) & 1) << k
                    s += root[off]
                out[beta, j] += s
    return out
