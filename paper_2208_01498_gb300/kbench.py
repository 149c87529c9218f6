"""Micro-benchmarks of the node kernels at chosen sizes (CUDA events, one
GPU), for roofline checks and for profiler captures of a single kernel:

    python -m paper_2208_01498_gb300.kbench permute --rank 26
    python -m paper_2208_01498_gb300.kbench gemm --batch 256 --M 256 --N 256 --K 4096 --form split_bf16
    python -m paper_2208_01498_gb300.kbench gemm ... --kernel tc --tile 3
    python -m paper_2208_01498_gb300.kbench gemm --batch 256 --M 2048 --N 64 --K 32 --iqp-node

(--iqp-node: the operand layout and output bit order of the node of that
shape in the plan of the 5 x 8 IQP circuit for 256 bitstrings.)

Prints one JSON line: the kernel's average time and its algorithmic GB/s
(permute: 16 bytes per element) or useful TFLOP/s (8 flops per complex
multiply-add).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import tnc


def _time(fn, iters, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(iters):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / iters


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("kernel", choices=["permute", "gemm"])
    ap.add_argument("--rank", type=int, default=26)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--M", type=int, default=4096)
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--K", type=int, default=4096)
    ap.add_argument("--tA", type=int, default=0)
    ap.add_argument("--tB", type=int, default=1)
    ap.add_argument("--form", default="split_bf16")
    ap.add_argument("--kernel", default=None, help="variant name of tnc.KG (default: chosen by shape)")
    ap.add_argument("--tile", type=int, default=None, help="tensor-core tile variant (see tnc_cgemm_variant)")
    ap.add_argument("--c-pos", default=None,
                    help="output bit order as a comma-separated list (n bits, m bits, batch bits; see tnc.h)")
    ap.add_argument("--iqp-node", action="store_true",
                    help="take tA, tB and the output bit order from the node of this shape in the plan of the "
                         "5 x 8 IQP circuit (256 bitstrings, the form given)")
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args()
    rng = np.random.default_rng(a.seed)
    if a.kernel == "permute":
        x = torch.randn(1 << a.rank, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        perm = rng.permutation(a.rank).astype(np.int32)
        ms = _time(lambda: tnc.permute(x, perm, out=y), a.iters, a.warmup)
        gbs = 16.0 * (1 << a.rank) / (ms / 1e3) / 1e9
        print(json.dumps({"kernel": "permute", "rank": a.rank, "ms": ms, "GB/s": gbs}))
        return
    if a.iqp_node:
        import circuits
        plan = tnc.Plan(tnc.Network(circuits.iqp(5, 8, seed=0)), max_batch=256, form=a.form, seed=1, ssa_trials=64)
        hit = [s for s in plan.export()["steps"]
               if s.get("kind") == 1 and (s["batch"], s["M"], s["N"], s["K"]) == (a.batch, a.M, a.N, a.K)]
        if not hit:
            raise SystemExit(f"no node of shape {a.batch} x {a.M} x {a.N} x {a.K} in the plan")
        a.tA, a.tB = int(hit[0]["tA"]), int(hit[0]["tB"])
        a.c_pos = None if hit[0]["c_ident"] else ",".join(str(int(x)) for x in hit[0]["c_pos"])
    A = torch.randn(a.batch * a.M * a.K, dtype=torch.complex64, device="cuda")
    B = torch.randn(a.batch * a.K * a.N, dtype=torch.complex64, device="cuda")
    C = torch.empty((a.batch, a.M, a.N), dtype=torch.complex64, device="cuda")
    f = tnc.FORMS[a.form]
    cpos = None if a.c_pos is None else [int(x) for x in a.c_pos.split(",")]
    need = tnc.lib.tnc_cgemm_scratch_bytes(a.batch, a.M, a.N, a.K, f)
    scr = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    ms = _time(lambda: tnc.cgemm(A, B, a.batch, a.M, a.N, a.K, a.tA, a.tB, a.form, out=C, scratch=scr,
                                   kernel=a.kernel, tile=a.tile, c_pos=cpos),
               a.iters, a.warmup)
    flops = 8.0 * a.batch * a.M * a.N * a.K
    byts = 8.0 * a.batch * (a.M * a.K + a.K * a.N + a.M * a.N)
    print(json.dumps({"kernel": "cgemm", "variant": a.kernel, "tile": a.tile, "form": a.form, "batch": a.batch, "M": a.M, "N": a.N, "K": a.K,
                      "ms": ms, "useful_TFLOP/s": flops / (ms / 1e3) / 1e12, "GB/s": byts / (ms / 1e3) / 1e9}))


if __name__ == "__main__":
    main()
