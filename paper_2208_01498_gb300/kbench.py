"""Micro-benchmarks of the node kernels at chosen sizes (CUDA events, one
GPU), for roofline checks and for profiler captures of a single kernel:

    python -m paper_2208_01498_gb300.kbench permute --rank 26
    python -m paper_2208_01498_gb300.kbench gemm --batch 256 --M 256 --N 256 --K 4096 --form split_bf16
    python -m paper_2208_01498_gb300.kbench gemm ... --kernel tc --tile 3

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
