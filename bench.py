#!/usr/bin/env python
"""Throughput benchmark of the separator-tree contraction executor.

Workload (one step = one request): the 5 x 8 IQP circuit (40 qubits; H layer,
exp(i theta Z) on every qubit, exp(i phi ZZ) on the 177 pairs within
Manhattan distance 2, H layer; theta, phi ~ U[0, 2 pi)), amplitudes of 256
seed-random bitstrings per request, contracted along the separator tree in
the chosen form with the FP64 slice/beta accumulation.  Bitstrings of every
step are resident on the device before the timed region (``value``); ``e2e``
repeats the measurement through the public host-buffer call with the
host->device copy of the bitstrings and the device->host read of the
amplitudes inside the timed region.

Under torchrun each rank serves its own requests (independent problems:
weak scaling, no collective on the data path); the timed region is bracketed
by a barrier and a device synchronisation, and the maximum time over ranks is
used.  ``--impl reference`` times the FP64 oracle (the column transfer-matrix
closed form of the IQP amplitudes) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import circuits as C  # noqa: E402

REQ_BATCH = 256
def workload_name(rows, cols):
    return f"iqp_{rows}x{cols}_{rows * cols}q_256_bitstrings"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        with open(self.f.name) as g:
            rows = [r.strip().split(", ") for r in g if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _workload(seed: int, steps: int, rows: int = 5, cols: int = 8):
    gl = C.iqp(rows, cols, seed)
    bits = np.stack([C.random_bitstrings(gl.n_qubits, REQ_BATCH, seed * 100003 + i) for i in range(steps)])
    return gl, bits


def _cpu_oracle(gl, bits, max_seconds: float = 20.0):
    """Time the oracle (transfer-matrix closed form) on a bounded sample."""
    import oracle as O
    n_done = 0
    t0 = time.perf_counter()
    for req in bits:
        O.iqp_transfer_amplitudes(gl, req)
        n_done += req.shape[0]
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return n_done / dt, n_done, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    gl, bits = _workload(args.seed, args.warmup + args.steps, args.rows, args.cols)
    import oracle as O
    sample = 16  # bitstrings per step: a bounded slice of one request
    for w in range(args.warmup):
        O.iqp_transfer_amplitudes(gl, bits[w][:sample])
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.iqp_transfer_amplitudes(gl, bits[args.warmup + k][:sample])
    dt = time.perf_counter() - t0
    val = args.steps * sample / dt
    line = {
        "impl": "reference", "metric": "amplitudes/s", "value": val, "unit": "amplitudes/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.rows, args.cols), "bitstrings_per_step": sample,
                   "seed": args.seed},
        "cpu_baseline": {"value": val, "unit": "amplitudes/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample} of the 256 bitstrings of each request, IQP transfer-matrix "
                                   f"closed form (numpy, single thread; host has {os.cpu_count()} cores)"},
        "e2e": {"value": val, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_measure(tnc, torch, form: str, seed: int = 0, n_req: int = 240, cost_cap_log2: float = 36.0,
                    ws_cap_bytes: int = 8 << 30):
    """Poisson-arriving amplitude requests over the mixed pool (2D L x L
    random circuits and (2+1)D layered circuits), 1-256 bitstrings each
    (log-uniform), served by the continuous-batching loop; p50/p99 latency and
    amplitudes/s at two arrival rates relative to the measured single-stream
    capacity.  Instances planned above 2^cost_cap_log2 paper ops are excluded
    and listed, as are those whose workspace exceeds ws_cap_bytes."""
    rng = np.random.default_rng(seed + 17)
    buckets = [1, 16, 256]
    pool, excluded = [], []
    for gl in C.serving_pool(seed):
        net = tnc.Network(gl)
        big = tnc.Plan(net, max_batch=buckets[-1], form=form)
        if big.report["tree_cost_log2"] > cost_cap_log2 or big.ws_bytes > ws_cap_bytes:
            excluded.append({"circuit": gl.name, "paper_ops_log2": round(big.report["tree_cost_log2"], 1),
                             "ws_GB": round(big.ws_bytes / 1e9, 1)})
            continue
        pool.append((gl, {b: (big if b == buckets[-1] else tnc.Plan(net, max_batch=b, form=form))
                          for b in buckets}))
    if not pool:
        return {"excluded": excluded}
    reqs = []
    for i in range(n_req):
        gl, plans = pool[int(rng.integers(len(pool)))]
        nb = int(round(float(np.exp(rng.uniform(0.0, np.log(256.0))))))
        bucket = next(b for b in buckets if b >= nb)
        reqs.append((gl, plans[bucket], C.random_bitstrings(gl.n_qubits, nb, 5000 + i)))
    # single-stream service time of the mix (alone, warm)
    ws = {id(p): tnc.alloc_workspace(p) for _, plans in pool for p in plans.values()}
    for gl, p, bits in reqs[:len(pool) * 3]:
        tnc.contract_amplitudes(p, bits, ws=ws[id(p)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for gl, p, bits in reqs[:60]:
        tnc.contract_amplitudes(p, bits, ws=ws[id(p)])
        torch.cuda.synchronize()
    service = (time.perf_counter() - t0) / 60
    del ws
    arena_bytes = (2 * max(p.ws_bytes for _, pl in pool for p in pl.values()) + (64 << 20)) // 256 * 256
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    result = {"pool": len(pool), "excluded": excluded, "requests": n_req, "streams": 4,
              "single_stream_ms_per_request": 1e3 * service, "rates": []}
    for factor in (0.5, 0.9):
        rate = factor / service
        gaps = rng.exponential(1.0 / rate, size=n_req)
        srv = tnc.Server(arena, n_streams=4)
        outs, tickets = [], []
        start = time.perf_counter()
        due = start
        for (gl, p, bits), gap in zip(reqs, gaps):
            due += gap
            while time.perf_counter() < due:
                pass
            out = torch.empty((bits.shape[0], 1 << p.n_open), dtype=torch.complex128, device="cuda")
            outs.append(out)
            tickets.append(srv.submit(p, bits, out))
        lat = [srv.wait(t, 120000) for t in tickets]
        span = time.perf_counter() - start
        srv.close()
        amps = sum(b.shape[0] for _, _, b in reqs)
        result["rates"].append({"rate_factor": factor, "requests_per_s": rate,
                                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                "amplitudes_per_s": amps / span})
    return result


def expectation_measure(tnc, torch, form: str, seed: int = 0, reps: int = 20, warmup: int = 3):
    """The paper's quantity c = <0|U^dagger P U|0> (Classical Simulation
    section) for P = Z_27 Z_28 on the 8 x 8 depth-8 random circuit (64 qubits,
    Haar single-qubit gates): the light-cone-reduced doubled network
    contracted at x = 0 by the same executor, autotuned, timed with CUDA
    events per value after ``warmup`` untimed values; the same value in the
    FP32 form gives the relative difference."""
    gl = C.random_2d(8, 8, 8, seed)
    ops = C.pauli_ops({27: "Z", 28: "Z"})
    dg = C.doubled(gl, ops, light_cone=True)
    stream = torch.cuda.current_stream()
    d_bits = torch.zeros((1, gl.n_qubits), dtype=torch.uint8, device="cuda")
    res = {"workload": "rand2d_8x8_d8 <Z27 Z28>, doubled network, light cone", "form": form}
    vals = {}
    for f in dict.fromkeys((form, "fp32")):
        p = tnc.Plan(tnc.Network(dg), form=f, seed=1, ssa_trials=64)
        ws = tnc.alloc_workspace(p)
        out = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
        p.upload(stream)
        p.autotune(ws, stream)
        for _ in range(warmup):
            tnc.contract_amplitudes_dbits(p, d_bits, out=out, ws=ws, stream=stream)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tnc.contract_amplitudes_dbits(p, d_bits, out=out, ws=ws, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        vals[f] = complex(out.cpu().numpy().ravel()[0])
        if f == form:
            rep_ = p.report
            bd = tnc.Network(gl).bounds()
            res["bounds_log2"] = {k: (round(bd[k], 1) if math.isfinite(bd[k]) else None)
                                  for k in ("thm2_log2", "thm2_pst_log2", "sidewise_log2", "explicit_log2")}
            res.update({"paper_ops_log2": rep_["tree_cost_log2"], "real_tflop": rep_["real_flops"] / 1e12,
                        "ms_p50": float(np.percentile(times, 50)), "ms_p99": float(np.percentile(times, 99)),
                        "values_per_s": 1e3 / float(np.percentile(times, 50)),
                        "effective_tflops": rep_["real_flops"] / (float(np.percentile(times, 50)) / 1e3) / 1e12})
        del ws
    res["c"] = [vals[form].real, vals[form].imag]
    res["rel_diff_vs_fp32"] = abs(vals[form] - vals["fp32"]) / max(abs(vals["fp32"]), 2.0 ** -32)
    return res


def op_counts(reps: int = 10, seed: int = 0):
    """The shape of the paper's op-count curves (Examples section; the IQP
    figure and its Sycamore-type and Poisson-cavity counterparts) for the
    paper's own families: per lattice size L, the mean and standard error over
    ``reps`` seeded realizations of log2 of explicit time evolution (idle
    qubits removed, as in the figure), left-to-right contraction, Thm. 2 (its
    planar form where it applies) and the separator planner's tree for c =
    <0|U^dagger P U|0> with P projectors on every qubit.  For the IQP family
    the planner also runs on the circuit with its commuting diagonal gates
    fused per pair.  Host only: no GPU is used."""
    from paper_2208_01498_gb300 import tnc

    def stats(v):
        v = np.asarray(v, float)
        return [round(float(v.mean()), 2), round(float(v.std(ddof=1) / math.sqrt(len(v))) if len(v) > 1 else 0.0, 2)]

    def ssa(gl):
        ops = C.projector_ops(range(gl.n_qubits), [0] * gl.n_qubits)
        return tnc.Plan(tnc.Network(C.doubled(gl, ops)), seed=1).report["tree_cost_log2"]

    families = {
        "iqp_paper (T = L^2, gamma = 3)": ([3, 4, 5, 6, 7, 8], lambda L, s: C.iqp_paper(L, s)),
        "sycamore_periods (q = 5, p = 0.88)": ([4, 8, 12, 16], lambda L, s: C.sycamore_periods(L, 5, 0.88, s)),
        "cavity_3d (alpha = 0.1, S = 5, sigma = 10)": ([10, 20, 30], lambda L, s: C.cavity_3d(L, s)),
    }
    out = {}
    for name, (sizes, make) in families.items():
        rows = []
        for L in sizes:
            acc = {"explicit": [], "sidewise": [], "thm2": [], "ssa": [], "ssa_fused": []}
            for r in range(reps):
                gl = make(L, seed + r)
                b = tnc.Network(gl).bounds()
                touched = {q for qs, _ in gl.gates if len(qs) == 2 for q in qs}
                acc["explicit"].append(b["explicit_log2"] - (gl.n_qubits - len(touched)))
                acc["sidewise"].append(b["sidewise_log2"])
                t2 = b["thm2_pst_log2"] if math.isfinite(b["thm2_pst_log2"]) else b["thm2_log2"]
                if math.isfinite(t2):
                    acc["thm2"].append(t2)
                acc["ssa"].append(ssa(gl))
                if name.startswith("iqp"):
                    acc["ssa_fused"].append(ssa(C.fuse_diagonal(gl)))
            rows.append(dict({"L": L}, **{k: stats(v) for k, v in acc.items() if v}))
        out[name] = rows
    return {"op_counts_log2": out, "reps": reps, "columns": "[mean, standard error] of log2 scalar operations"}


def _traffic(step, kernel, form, tile=0):
    """DRAM bytes per launch of this step from the committed ncu summary
    (profiles/traffic.json), scaled by batch; None if that shape and kernel
    variant were not captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or not step.get("batch"):
        return None
    with open(p) as f:
        for e in json.load(f)["entries"]:
            if e["kernel"] == kernel and e["form"] == form and e.get("tile", 0) == tile and \
                    all(e[k] == step.get(k) for k in ("M", "N", "K")):
                return e["dram_bytes_captured"] * step["batch"] / e["captured_batch"]
    return None


def _tune(plan, ws, stream, cache_path, key):
    """Autotune the plan's kernel per step (outside any timed region), or
    reuse the choices saved under ``key`` in ``cache_path`` so that repeated
    runs (e.g. one under a profiler) execute the same kernels."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache and len(cache[key]) == len(plan.get_kernels()):
            plan.set_kernels(cache[key])
            return -1
    changed = plan.autotune(ws, stream)
    if cache_path:
        cache[key] = plan.get_kernels()
        with open(cache_path, "w") as f:
            json.dump(cache, f)
    return changed


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2208_01498_gb300 import tnc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    gl, bits = _workload(args.seed + rank, args.warmup + args.steps, args.rows, args.cols)
    net = tnc.Network(gl)
    plan = tnc.Plan(net, max_batch=REQ_BATCH, form=args.form, seed=1, ssa_trials=64)
    rep = plan.report
    ws = tnc.alloc_workspace(plan)
    out = torch.empty((REQ_BATCH, 1), dtype=torch.complex128, device=dev)
    d_bits = torch.from_numpy(bits).to(dev)
    stream = torch.cuda.current_stream()
    plan.upload(stream)
    tuned = _tune(plan, ws, stream, args.tune_cache, f"{workload_name(args.rows, args.cols)}:{args.form}:{rank}")
    rep = plan.report

    for w in range(args.warmup):
        tnc.contract_amplitudes_dbits(plan, d_bits[w], out=out, ws=ws, stream=stream)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs, the library's default launch
    # path (each slice group replayed as a CUDA graph)
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        tnc.contract_amplitudes_dbits(plan, d_bits[args.warmup + k], out=out, ws=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    # ---- the same requests again with CUDA events around every step on the
    # launch stream (eager launches): per-kernel durations for the roofline
    plan.set_profiling(True)
    torch.cuda.synchronize()
    for k in range(args.steps):
        tnc.contract_amplitudes_dbits(plan, d_bits[args.warmup + k], out=out, ws=ws, stream=stream)
    torch.cuda.synchronize()
    prof = plan.profile()
    plan.set_profiling(False)
    if world > 1:
        t = torch.tensor([t_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    amps = world * args.steps * REQ_BATCH
    value = amps / (t_ms / 1e3)

    last_out = out.clone()

    # ---- the FP32 CUDA-core form on the same requests (the metric's reference form)
    fp32_form = None
    if args.form != "fp32":
        p32 = tnc.Plan(net, max_batch=REQ_BATCH, form="fp32", seed=1, ssa_trials=64)
        ws32 = tnc.alloc_workspace(p32)
        _tune(p32, ws32, stream, args.tune_cache, f"{workload_name(args.rows, args.cols)}:fp32:{rank}")
        out32 = torch.empty_like(out)
        for w in range(args.warmup):
            tnc.contract_amplitudes_dbits(p32, d_bits[w], out=out32, ws=ws32, stream=stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(args.steps):
            tnc.contract_amplitudes_dbits(p32, d_bits[args.warmup + k], out=out32, ws=ws32, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize()
        t32 = f0.elapsed_time(f1)
        a, r = last_out.cpu().numpy(), out32.cpu().numpy()
        floor = 2.0 ** (-gl.n_qubits / 2)
        rel = float(np.max(np.abs(a - r) / np.maximum(np.abs(r), floor)))
        fp32_form = {"value": world * args.steps * REQ_BATCH / (t32 / 1e3), "unit": "amplitudes/s",
                     "ms_per_step": t32 / args.steps, "max_rel_err_vs_fp32": rel}
        del ws32

    # ---- end to end through the host-buffer API
    pinned = torch.from_numpy(bits).pin_memory()
    res = torch.empty((REQ_BATCH, 1), dtype=torch.complex128).pin_memory()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        tnc.contract_amplitudes(plan, pinned[args.warmup + k].numpy(), out=out, ws=ws, stream=stream)
        res.copy_(out, non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": amps / e2e_s, "unit": "amplitudes/s", "h2d_bytes_per_step": int(REQ_BATCH * gl.n_qubits),
           "d2h_bytes_per_step": int(REQ_BATCH * 16)}

    # ---- roofline of the dominant step (largest share of the live CUDA-event time)
    peaks, src = _peaks()
    names = {0: "cgemm_simt_128x64", 1: "cgemm_simt_64x32", 2: "cgemm_narrow", 3: "cgemm_dot",
             4: "cgemm_tc", 5: "cgemm_simt_32x128", 100: "permute", 101: "grouped_narrow"}
    kinds = {}
    for ms, runs, kind, fl, by in zip(prof["ms"], prof["runs"], prof["kind"], prof["flops"], prof["bytes"]):
        if runs == 0:
            continue
        d = kinds.setdefault(int(kind), {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
        d["ms"] += float(ms)
        d["flops"] += float(fl) * int(runs)
        d["bytes"] += float(by) * int(runs)
        d["launches"] += int(runs)
    total_ms = sum(d["ms"] for d in kinds.values())
    di = int(np.argmax(prof["ms"]))
    steps_all = plan.export()["steps"]
    step = steps_all[di]
    dkind, druns = int(prof["kind"][di]), int(prof["runs"][di])
    avg_s = float(prof["ms"][di]) / druns / 1e3
    fl, by = float(prof["flops"][di]), float(prof["bytes"][di])
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # three bf16 (tf32) products per useful product; tf32 peak = half the bf16 peak
    tc_peak = float(peaks["bf16_tflops"]) * (1.0 if args.form == "split_bf16" else 0.5)
    hbm = float(peaks["hbm_gbs"])
    if dkind in (100, 101, 2) or (dkind == 4 and by / hbm / 1e9 > 3.0 * fl / tc_peak / 1e12):
        # tensor-core nodes whose algorithmic bytes take longer than their MMAs at peak are HBM-bound
        roof = {"bound": "hbm", "achieved": by / avg_s / 1e9, "peak": hbm, "unit": "GB/s"}
    elif dkind == 4:
        roof = {"bound": "tensor", "achieved": 3.0 * fl / avg_s / 1e12, "peak": tc_peak, "unit": "TFLOP/s"}
    else:
        pk = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x max SM clock
        roof = {"bound": "alu", "achieved": fl / avg_s / 1e12, "peak": pk, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    choices = plan.get_kernels()
    dtile = int(choices[di][1]) if dkind == 4 else 0
    roof["traffic"] = _traffic(step, names.get(dkind), args.form, dtile)
    roof["kernel"] = names.get(dkind, str(dkind))
    roof["step"] = {k: step.get(k) for k in ("batch", "M", "N", "K")}
    if dkind == 4:
        roof["step"]["tile"] = dtile
    roof["launches_timed"] = druns
    roof["avg_launch_ms"] = avg_s * 1e3
    roof["algorithmic_bytes_per_launch"] = by
    roof["algorithmic_flops_per_launch"] = fl
    roof["share_of_device_time"] = float(prof["ms"][di]) / total_ms if total_ms else None
    roof["peak_source"] = src + (" burst" if dkind == 4 else "")
    if args.steps_detail and rank == 0:
        rows = []
        for i, (ms, runs, kind, fl_i, by_i) in enumerate(zip(prof["ms"], prof["runs"], prof["kind"], prof["flops"],
                                                              prof["bytes"])):
            if runs == 0:
                continue
            st_i = steps_all[i]
            t_launch = float(ms) / int(runs)
            mult = 3.0 if int(kind) == 4 else 1.0
            bound_ms = max(float(by_i) / hbm / 1e6, mult * float(fl_i) / tc_peak / 1e9)
            rows.append({"step": i, "kernel": names.get(int(kind), str(int(kind))),
                         "tile": int(choices[i][1]), "shape": {k: st_i.get(k) for k in ("batch", "M", "N", "K")},
                         "ms": t_launch, "bound_ms": bound_ms, "x_over_bound": t_launch / bound_ms if bound_ms else None})
        rows.sort(key=lambda r: -r["ms"])
        with open(args.steps_detail, "w") as f:
            json.dump(rows, f, indent=1)
    breakdown = {}
    for kd, v in sorted(kinds.items(), key=lambda kv: -kv[1]["ms"]):
        s = v["ms"] / 1e3
        breakdown[names.get(kd, str(kd))] = {"share": v["ms"] / total_ms, "launches": v["launches"],
                                              "GB/s": v["bytes"] / s / 1e9, "TFLOP/s": v["flops"] / s / 1e12}

    line = {
        "metric": "amplitudes/s", "value": value, "unit": "amplitudes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "c64", "3xtf32": "tf32x3 (fp32 acc)", "split_bf16": "bf16x3 (fp32 acc)"}[args.form],
        "data": "synthetic",
        "config": {"workload": workload_name(args.rows, args.cols), "form": args.form, "bitstrings_per_request": REQ_BATCH,
                   "seed": args.seed, "real_tflop_per_request": rep["real_flops"] / 1e12,
                   "paper_ops_log2": rep["tree_cost_log2"], "ws_bytes": rep["ws_bytes"],
                   "paper_bounds_log2": {k: (round(v, 1) if math.isfinite(v) else None)
                                         for k, v in net.bounds().items()
                                         if k in ("thm2_log2", "thm2_pst_log2", "sidewise_log2", "explicit_log2")},
                   "l2": f"working set {rep['ws_bytes'] / 1e9:.1f} GB per request > 129 MB L2",
                   "parallelism": f"dp{world} (independent requests)", "autotuned_steps": tuned,
                   "timing": "value: CUDA events around the K steps, device-resident bitstrings, CUDA-graph "
                             "replay per slice group; roofline and kernel_breakdown: a second pass over the same "
                             "K requests with CUDA events around every step (eager launches); e2e: host buffers "
                             "through tnc_contract_amplitudes, wall clock"},
        "effective_tflops": world * args.steps * rep["real_flops"] / (t_ms / 1e3) / 1e12,
        "roofline": roof,
        "kernel_breakdown": breakdown,
        "fp32_form": fp32_form,
        "e2e": e2e,
        "clocks": ck,
        "gpu_launches": int(args.steps * rep["n_launches"]),
    }
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_measure(tnc, torch, args.form, args.seed)
    if rank == 0 and not args.no_expectation:
        line["expectation"] = expectation_measure(tnc, torch, args.form, args.seed)
    if rank == 0 and not args.no_cpu_baseline:
        v, n_done, dt = _cpu_oracle(gl, bits[args.warmup:args.warmup + 1])
        line["cpu_baseline"] = {"value": v, "unit": "amplitudes/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n_done} bitstrings (one request) of the same workload by the IQP "
                                          f"transfer-matrix closed form, {dt:.1f} s, numpy single thread "
                                          f"(host has {os.cpu_count()} cores)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["fp32", "3xtf32", "split_bf16"], default="split_bf16")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-mix latency measurement")
    ap.add_argument("--op-counts", action="store_true",
                    help="print the op-count curves of the paper's example families (host only) and exit")
    ap.add_argument("--no-expectation", action="store_true",
                    help="skip the doubled-network expectation-value measurement")
    ap.add_argument("--tune-cache", default=None, help="JSON file to save / reuse the autotuner's kernel choices")
    ap.add_argument("--rows", type=int, default=5, help="IQP lattice rows (the benchmark uses 5 x 8)")
    ap.add_argument("--cols", type=int, default=8)
    ap.add_argument("--steps-detail", default=None,
                    help="write a JSON table of every program step (shape, kernel, ms per launch, roofline ms)")
    args = ap.parse_args()
    if args.op_counts:
        print(json.dumps(op_counts()), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
