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


def _oracle_chunk(job):
    """One worker's share of the all-cores oracle timing (spawned process)."""
    gl, bits = job
    import oracle as O
    O.iqp_transfer_amplitudes(gl, bits)
    return bits.shape[0]


def _cpu_oracle_all_cores(gl, bits, per_core: int = 32):
    """The same oracle on every host core: a spawned process pool (the oracle
    itself is elementwise NumPy, one thread), per_core bitstrings per
    worker; returns amplitudes/s, workers, bitstrings, seconds."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    flat = bits.reshape(-1, bits.shape[-1])
    need = per_core * ncores
    flat = np.concatenate([flat] * (need // flat.shape[0] + 1))[:need]
    jobs = [(gl, flat[i * per_core:(i + 1) * per_core]) for i in range(ncores)]
    with mp.get_context("spawn").Pool(ncores) as pool:
        pool.map(_oracle_chunk, jobs[:ncores])  # start-up and imports outside the timing
        t0 = time.perf_counter()
        n = sum(pool.map(_oracle_chunk, jobs))
        dt = time.perf_counter() - t0
    return n / dt, ncores, n, dt


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


SERVING_RATES = (0.25, 0.5, 0.75, 0.9, 1.0, 1.2)
SERVING_BUCKETS = (1, 16, 256)


def _serve(tnc, torch, arena, reqs, gaps, n_streams, batching=1):
    """Submit the requests at their Poisson arrival times; latencies and span."""
    srv = tnc.Server(arena, n_streams=n_streams)
    srv.set_batching(batching)
    tickets = []
    start = time.perf_counter()
    due = start
    for (_, p, bits), gap in zip(reqs, gaps):
        due += gap
        while time.perf_counter() < due:
            pass
        out = torch.empty((bits.shape[0], 1 << p.n_open), dtype=torch.complex128, device="cuda")
        tickets.append(srv.submit(p, bits, out))
    lat = [srv.wait(t, 600000) for t in tickets]
    span = time.perf_counter() - start
    srv.close()
    return np.asarray(lat), span


def serving_measure(tnc, torch, forms=("split_bf16", "fp32"), seed: int = 0, n_req: int = 1000,
                    cost_cap_flops: float = 2.0 ** 50, arena_bytes: int = 64 << 30, n_streams: int = 4,
                    rates=SERVING_RATES, batching: int = 16, n_req_by_form=None):
    """Poisson-arriving amplitude requests over the mixed pool (2D L x L random
    circuits, L 4..10, depth 8..20, and (2+1)D layered circuits), 1-256
    bitstrings each (log-uniform), served by the continuous-batching loop over
    a device arena.  Every pool instance is planned under half the arena
    (sliced where needed) and autotuned, per form and batch bucket; an
    instance whose plan exceeds cost_cap_flops real flops (or cannot be
    planned) is listed as excluded with its planned cost.  Per form: the
    single-stream service time of the mix (the capacity), then n_req requests
    at each rate factor of that capacity, p50/p99 latency and amplitudes/s,
    with waiting requests admitted together up to `batching` at a time (their
    nodes grouped across requests); for the first form also without
    batching (each request its own launches, overlapped on the streams) and a
    serial queue (one stream, no overlap) at rate factors 0.9 and 1.2.
    n_req_by_form: fewer requests per rate for a form (a prefix of the same
    sequence), e.g. the slower FP32 form."""
    n_req_by_form = dict(n_req_by_form or {})
    rng = np.random.default_rng(seed + 17)
    pool, excluded = [], []
    for gl in C.serving_pool(seed):
        net = tnc.Network(gl)
        plans, why = {}, None
        for f in forms:
            try:
                big = tnc.Plan(net, max_batch=SERVING_BUCKETS[-1], form=f, mem_cap_bytes=arena_bytes // 2)
            except tnc.TncError as e:
                why = f"{f}: {str(e)[:120]}"
                break
            if big.report["real_flops"] > cost_cap_flops:
                why = f"planned {big.report['real_flops']:.3g} real flops > 2^{math.log2(cost_cap_flops):.0f}"
                plans[f] = {SERVING_BUCKETS[-1]: big}
                break
            plans[f] = {b: (big if b == SERVING_BUCKETS[-1] else
                            tnc.Plan(net, max_batch=b, form=f, mem_cap_bytes=arena_bytes // 2))
                        for b in SERVING_BUCKETS}
        if why:
            r = next(iter(plans.values()))[SERVING_BUCKETS[-1]].report if plans else None
            excluded.append({"circuit": gl.name, "reason": why,
                             "real_flops": r["real_flops"] if r else None,
                             "paper_ops_log2": round(r["tree_cost_log2"], 1) if r else None,
                             "ws_GB": round(r["ws_bytes"] / 1e9, 2) if r else None})
            continue
        pool.append((gl, plans))
    result = {"pool": [{"circuit": gl.name, "qubits": gl.n_qubits,
                        "real_flops_256": pl[forms[0]][SERVING_BUCKETS[-1]].report["real_flops"],
                        "ws_GB_256": round(pl[forms[0]][SERVING_BUCKETS[-1]].ws_bytes / 1e9, 3)} for gl, pl in pool],
              "excluded": excluded, "cost_cap_real_flops": cost_cap_flops, "arena_GB": arena_bytes / 1e9,
              "requests_per_rate": n_req, "streams": n_streams, "forms": {}}
    if not pool:
        return result
    # one request sequence for every form and rate
    seq = []
    for i in range(n_req):
        k = int(rng.integers(len(pool)))
        nb = int(round(float(np.exp(rng.uniform(0.0, np.log(256.0))))))
        seq.append((k, nb, C.random_bitstrings(pool[k][0].n_qubits, nb, 5000 + i)))
    gaps_unit = rng.exponential(1.0, size=n_req)
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    for f in forms:
        # autotune every plan of this form in the arena (outside any timing)
        for _, plans in pool:
            for p in plans[f].values():
                p.autotune(arena[:p.ws_bytes // 256 * 256 + 256] if p.ws_bytes < arena_bytes else None, reps=2)
        n_f = min(n_req, int(n_req_by_form.get(f, n_req)))
        reqs = []
        for k, nb, bits in seq[:n_f]:
            bucket = next(b for b in SERVING_BUCKETS if b >= nb)
            reqs.append((k, pool[k][1][f][bucket], bits))
        # single-stream service time of the mix (one request at a time through
        # the serving loop, warm): the capacity
        srv = tnc.Server(arena, n_streams=1)

        def one_by_one(rs):
            for _, p, bits in rs:
                out = torch.empty((bits.shape[0], 1 << p.n_open), dtype=torch.complex128, device="cuda")
                srv.wait(srv.submit(p, bits, out), 600000)

        one_by_one(reqs[:3 * len(pool)])
        timed = reqs[:min(200, n_f)]
        t0 = time.perf_counter()
        one_by_one(timed)
        service = (time.perf_counter() - t0) / len(timed)
        srv.close()
        amps = sum(b.shape[0] for _, _, b in reqs)
        fr = {"single_stream_ms_per_request": 1e3 * service, "capacity_requests_per_s": 1.0 / service,
              "requests_per_rate": n_f, "batching": batching, "rates": [], "no_batching": [], "serial_queue": []}

        def point(factor, lat, span):
            return {"rate_factor": factor, "requests_per_s": factor / service,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "amplitudes_per_s": amps / span}

        for factor in rates:
            rate = factor / service
            gaps = gaps_unit[:n_f] / rate
            fr["rates"].append(point(factor, *_serve(tnc, torch, arena, reqs, gaps, n_streams, batching)))
            if f == forms[0]:
                fr["no_batching"].append(point(factor, *_serve(tnc, torch, arena, reqs, gaps, n_streams)))
                if factor in (0.9, 1.2):
                    fr["serial_queue"].append(point(factor, *_serve(tnc, torch, arena, reqs, gaps, 1)))
        if f == forms[0]:
            fr["small_mix"] = _small_mix(tnc, torch, arena, pool, f, seed, n_f, n_streams, batching)
        result["forms"][f] = fr
    del arena
    torch.cuda.empty_cache()
    return result


def _small_mix(tnc, torch, arena, pool, form, seed, n_req, n_streams, batching,
               max_flops=2.0 ** 34, rates=(0.9, 1.5, 3.0)):
    """The same serving loop on the pool's small instances only (planned at
    most max_flops real flops for 256 bitstrings, the size cross-request
    batching merges): n_req Poisson requests at each rate factor of their
    single-stream capacity, with and without batching."""
    small = [i for i, (_, pl) in enumerate(pool) if pl[form][SERVING_BUCKETS[-1]].report["real_flops"] <= max_flops]
    if not small:
        return None
    rng = np.random.default_rng(seed + 29)
    reqs = []
    for i in range(n_req):
        k = small[int(rng.integers(len(small)))]
        nb = int(round(float(np.exp(rng.uniform(0.0, np.log(256.0))))))
        bucket = next(b for b in SERVING_BUCKETS if b >= nb)
        reqs.append((k, pool[k][1][form][bucket], C.random_bitstrings(pool[k][0].n_qubits, nb, 9000 + i)))
    gaps_unit = rng.exponential(1.0, size=n_req)
    srv = tnc.Server(arena, n_streams=1)
    for _, p, bits in reqs[:3 * len(small)] + reqs[:min(200, n_req)]:
        out = torch.empty((bits.shape[0], 1 << p.n_open), dtype=torch.complex128, device="cuda")
        srv.wait(srv.submit(p, bits, out), 600000)
    t0 = time.perf_counter()
    for _, p, bits in reqs[:min(200, n_req)]:
        out = torch.empty((bits.shape[0], 1 << p.n_open), dtype=torch.complex128, device="cuda")
        srv.wait(srv.submit(p, bits, out), 600000)
    service = (time.perf_counter() - t0) / min(200, n_req)
    srv.close()
    amps = sum(b.shape[0] for _, _, b in reqs)
    res = {"circuits": [pool[i][0].name for i in small], "requests_per_rate": n_req,
           "single_stream_ms_per_request": 1e3 * service, "batching": batching, "rates": [], "no_batching": []}
    for factor in rates:
        gaps = gaps_unit / (factor / service)
        for key, b in (("rates", batching), ("no_batching", 1)):
            lat, span = _serve(tnc, torch, arena, reqs, gaps, n_streams, b)
            res[key].append({"rate_factor": factor, "requests_per_s": factor / service,
                             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "amplitudes_per_s": amps / span})
    return res


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
        return tnc.Plan(tnc.Network(C.doubled(gl, ops)), seed=1, tree_only=True).report["tree_cost_log2"]

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


def _form_peaks(torch):
    """TF32 and FP32 GEMM rates of this GPU measured in the run: cuBLAS through
    torch.matmul on 8192^3 fp32 operands with TF32 allowed (tensor cores) and
    not allowed (CUDA cores), CUDA events after warm-up."""
    n, reps = 8192, 10
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    res = {}
    try:
        for name, tf32 in (("tf32_tflops", True), ("fp32_tflops", False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            for _ in range(3):
                a @ b
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                a @ b
            e1.record()
            torch.cuda.synchronize()
            res[name] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b
    torch.cuda.empty_cache()
    return res


WORKLOADS = ("iqp_5x8", "rand2d_8x8_d16")


def _make_workload(args, rank):
    """(name, gate list, bitstrings [steps][batch][n], plan options) of the
    benchmark workload: the 5 x 8 IQP circuit with 256 bitstrings per request,
    or the 8 x 8 depth-16 random circuit with one seed-random bitstring per
    request, sliced under 180 GB."""
    nsteps = args.warmup + args.steps
    if args.workload == "rand2d_8x8_d16":
        gl, _ = C.workload("rand2d_8x8_d16", args.seed + rank)
        bits = np.stack([C.random_bitstrings(gl.n_qubits, 1, 7919 * (args.seed + rank) + i) for i in range(nsteps)])
        return "rand2d_8x8_d16_1amp", gl, bits, dict(max_batch=1, mem_cap_bytes=180 * 10**9)
    gl, bits = _workload(args.seed + rank, nsteps, args.rows, args.cols)
    return workload_name(args.rows, args.cols), gl, bits, dict(max_batch=REQ_BATCH)


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

    wname, gl, bits, popts = _make_workload(args, rank)
    batch = bits.shape[1]
    net = tnc.Network(gl)
    t_plan = time.perf_counter()
    plan = tnc.Plan(net, form=args.form, seed=1, ssa_trials=64, **popts)
    plan_s = time.perf_counter() - t_plan
    rep = plan.report
    ws = tnc.alloc_workspace(plan)
    out = torch.empty((batch, 1), dtype=torch.complex128, device=dev)
    d_bits = torch.from_numpy(bits).to(dev)
    stream = torch.cuda.current_stream()
    plan.upload(stream)
    tuned = _tune(plan, ws, stream, args.tune_cache, f"{wname}:{args.form}:{rank}") if args.autotune else 0
    rep = plan.report

    for w in range(args.warmup):
        if args.shard_slices and args.workload == "rand2d_8x8_d16" and world > 1:
            from paper_2208_01498_gb300 import shard as shard_w
            shard_w.contract_amplitudes_sharded(plan, d_bits[w], out=out, ws=ws, stream=stream)
        else:
            tnc.contract_amplitudes_dbits(plan, d_bits[w], out=out, ws=ws, stream=stream)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs, the library's default launch
    # path (each slice group replayed as a CUDA graph)
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # slice sharding: every rank contracts its range of the serial slice
    # groups of the same request, one FP64 all-reduce of the amplitudes
    sharded = args.shard_slices and args.workload == "rand2d_8x8_d16"
    if sharded:
        from paper_2208_01498_gb300 import shard as shard_mod

    def one_step(k):
        if sharded:
            out.copy_(shard_mod.contract_amplitudes_sharded(plan, d_bits[k], out=out, ws=ws, stream=stream))
        else:
            tnc.contract_amplitudes_dbits(plan, d_bits[k], out=out, ws=ws, stream=stream)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        one_step(args.warmup + k)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    # ---- the same requests again with CUDA events around every step on the
    # launch stream (eager launches): per-kernel durations for the roofline
    prof_steps = args.steps if args.workload == "iqp_5x8" else 1
    plan.set_profiling(True)
    torch.cuda.synchronize()
    for k in range(prof_steps):
        tnc.contract_amplitudes_dbits(plan, d_bits[args.warmup + k], out=out, ws=ws, stream=stream)
    torch.cuda.synchronize()
    prof = plan.profile()
    plan.set_profiling(False)
    if world > 1:
        t = torch.tensor([t_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    amps = (1 if sharded else world) * args.steps * batch
    value = amps / (t_ms / 1e3)

    last_out = out.clone()

    # ---- the FP32 CUDA-core form on the same requests (the metric's reference form)
    fp32_form = None
    if args.form != "fp32" and (args.workload == "iqp_5x8" or args.compare_forms):
        p32 = tnc.Plan(net, form="fp32", seed=1, ssa_trials=64, **popts)
        ws32 = tnc.alloc_workspace(p32) if args.workload == "iqp_5x8" else None
        if ws32 is None:  # the 8 x 8 workload: one workspace at a time
            del ws
            torch.cuda.empty_cache()
            ws32 = tnc.alloc_workspace(p32)
        if args.autotune:
            _tune(p32, ws32, stream, args.tune_cache, f"{wname}:fp32:{rank}")
        out32 = torch.empty_like(out)
        n32 = args.steps if args.workload == "iqp_5x8" else 1
        for w in range(args.warmup if args.workload == "iqp_5x8" else 0):
            tnc.contract_amplitudes_dbits(p32, d_bits[w], out=out32, ws=ws32, stream=stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(n32):
            tnc.contract_amplitudes_dbits(p32, d_bits[args.warmup + args.steps - n32 + k], out=out32, ws=ws32,
                                          stream=stream)
        f1.record(stream)
        torch.cuda.synchronize()
        t32 = f0.elapsed_time(f1)
        a, r = last_out.cpu().numpy(), out32.cpu().numpy()
        floor = 2.0 ** (-gl.n_qubits / 2)
        rel = float(np.max(np.abs(a - r) / np.maximum(np.abs(r), floor)))
        fp32_form = {"value": world * n32 * batch / (t32 / 1e3), "unit": "amplitudes/s",
                     "ms_per_step": t32 / n32, "steps": n32, "max_rel_err_vs_fp32": rel}
        del ws32, p32
        torch.cuda.empty_cache()
        if args.workload != "iqp_5x8":
            ws = tnc.alloc_workspace(plan)

    # ---- the same requests on the hyper-edge form of the network (diagonal
    # gates on shared wire labels): another plan for the same amplitudes
    hyper_form = None
    if args.workload == "iqp_5x8" and args.hyperedges:
        ph = tnc.Plan(tnc.Network(gl, hyperedges=True), form=args.form, seed=1, ssa_trials=64, **popts)
        wsh = tnc.alloc_workspace(ph)
        if args.autotune:
            _tune(ph, wsh, stream, args.tune_cache, f"{wname}:{args.form}:hyper:{rank}")
        outh = torch.empty_like(out)
        for w in range(args.warmup):
            tnc.contract_amplitudes_dbits(ph, d_bits[w], out=outh, ws=wsh, stream=stream)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for k in range(args.steps):
            tnc.contract_amplitudes_dbits(ph, d_bits[args.warmup + k], out=outh, ws=wsh, stream=stream)
        h1.record(stream)
        torch.cuda.synchronize()
        th = h0.elapsed_time(h1)
        a, r = last_out.cpu().numpy(), outh.cpu().numpy()
        floor = 2.0 ** (-gl.n_qubits / 2)
        hyper_form = {"value": world * args.steps * batch / (th / 1e3), "unit": "amplitudes/s",
                      "ms_per_step": th / args.steps, "tree_cost_log2": ph.report["tree_cost_log2"],
                      "real_tflop_per_request": ph.report["real_flops"] / 1e12, "ws_bytes": ph.report["ws_bytes"],
                      "gpu_launches_per_step": ph.report["n_launches"],
                      "max_rel_diff_vs_default_network": float(np.max(np.abs(a - r) / np.maximum(np.abs(r), floor)))}
        del wsh, ph
        torch.cuda.empty_cache()

    # ---- end to end through the host-buffer API
    pinned = torch.from_numpy(bits).pin_memory()
    res = torch.empty((batch, 1), dtype=torch.complex128).pin_memory()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n_e2e = args.steps
    t0 = time.perf_counter()
    for k in range(n_e2e):
        if sharded:
            # host bitstrings in, this rank's slice groups, the FP64 all-reduce, the amplitudes out
            db = pinned[args.warmup + k].to(dev, non_blocking=True)
            res.copy_(shard_mod.contract_amplitudes_sharded(plan, db, out=out, ws=ws, stream=stream),
                      non_blocking=True)
        else:
            tnc.contract_amplitudes(plan, pinned[args.warmup + k].numpy(), out=out, ws=ws, stream=stream)
            res.copy_(out, non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": (1 if sharded else world) * n_e2e * batch / e2e_s, "unit": "amplitudes/s",
           "h2d_bytes_per_step": int(batch * gl.n_qubits), "d2h_bytes_per_step": int(batch * 16)}
    del ws
    torch.cuda.empty_cache()

    # ---- roofline of the dominant step (largest share of the live CUDA-event time)
    peaks, src = _peaks()
    fpk = _form_peaks(torch)
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
    # the MMA peak of the form's operand type: bf16 measured; tf32 measured in
    # this run (cuBLAS through torch), else the nominal tf32 / bf16 ratio
    tf32_peak = fpk.get("tf32_tflops") or float(peaks["bf16_tflops"]) * 1.1 / 2.25
    # a kernel timed inside a seconds-long step runs under the power cap: the
    # sustained bf16 figure; the burst figure for the short steps
    sustained = t_ms > 1000.0 and "bf16_tflops_sustained" in peaks
    bf16_peak = float(peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"])
    tc_peak = bf16_peak if args.form == "split_bf16" else tf32_peak
    hbm = float(peaks["hbm_gbs"])
    fp32_peak = fpk.get("fp32_tflops") or 152 * 128 * 2 * sm_max * 1e6 / 1e12
    # useful peak of the form: three MMA products per useful product on the tensor cores
    form_peak = fp32_peak if args.form == "fp32" else tc_peak / 3.0
    if dkind in (100, 101, 2) or (dkind == 4 and by / hbm / 1e9 > 3.0 * fl / tc_peak / 1e12):
        # tensor-core nodes whose algorithmic bytes take longer than their MMAs at peak are HBM-bound
        roof = {"bound": "hbm", "achieved": by / avg_s / 1e9, "peak": hbm, "unit": "GB/s"}
    elif dkind == 4:
        roof = {"bound": "tensor", "achieved": 3.0 * fl / avg_s / 1e12, "peak": tc_peak, "unit": "TFLOP/s"}
    else:
        roof = {"bound": "alu", "achieved": fl / avg_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    choices = plan.get_kernels()
    dtile = int(choices[di][1]) if choices[di][1] >= 0 else 0
    roof["traffic"] = _traffic(step, names.get(dkind), args.form, dtile)
    roof["kernel"] = names.get(dkind, str(dkind))
    roof["step"] = {k: step.get(k) for k in ("batch", "M", "N", "K")}
    roof["step"]["tile"] = dtile
    roof["launches_timed"] = druns
    roof["avg_launch_ms"] = avg_s * 1e3
    roof["algorithmic_bytes_per_launch"] = by
    roof["algorithmic_flops_per_launch"] = fl
    roof["share_of_device_time"] = float(prof["ms"][di]) / total_ms if total_ms else None
    roof["peak_source"] = (src + (" sustained" if sustained else " burst")) if (dkind == 4 and args.form == "split_bf16") else \
        ("measured in this run (cuBLAS tf32)" if dkind == 4 else
         ("measured in this run (cuBLAS fp32)" if dkind in (0, 1, 3, 5) else src))
    # request-level roofline: sum over the steps of max(flops / form peak,
    # bytes / HBM) against the measured time per request
    bound_ms_req = 0.0
    rows = []
    for i, (ms, runs, kind, fl_i, by_i) in enumerate(zip(prof["ms"], prof["runs"], prof["kind"], prof["flops"],
                                                          prof["bytes"])):
        if runs == 0:
            continue
        b_i = max(float(by_i) / hbm / 1e6, float(fl_i) / form_peak / 1e9)  # ms per launch
        bound_ms_req += b_i * int(runs) / prof_steps
        st_i = steps_all[i]
        t_launch = float(ms) / int(runs)
        mult = 3.0 if int(kind) == 4 else 1.0
        kb_ms = max(float(by_i) / hbm / 1e6, mult * float(fl_i) / (tc_peak if int(kind) == 4 else fp32_peak) / 1e9)
        rows.append({"step": i, "kernel": names.get(int(kind), str(int(kind))), "tile": int(choices[i][1]),
                     "shape": {k: st_i.get(k) for k in ("batch", "M", "N", "K")}, "launches": int(runs),
                     "ms": t_launch, "flops": float(fl_i), "bytes": float(by_i), "form_bound_ms": b_i,
                     "kernel_bound_ms": kb_ms, "x_over_kernel_bound": t_launch / kb_ms if kb_ms else None})
    roof["request_bound_ms"] = bound_ms_req
    roof["request_frac"] = bound_ms_req / (t_ms / args.steps)
    roof["request_peak"] = {"form_peak_tflops": form_peak, "hbm_gbs": hbm,
                            "note": "sum over steps of max(flops / form peak, bytes / HBM), form peak = tensor "
                                    "peak / 3 products (fp32 form: cuBLAS fp32), over ms_per_step"}
    if args.steps_detail and rank == 0:
        rows.sort(key=lambda r: -r["ms"] * r["launches"])
        with open(args.steps_detail, "w") as f:
            json.dump({"workload": wname, "form": args.form, "ms_per_step": t_ms / args.steps,
                       "request_bound_ms": bound_ms_req, "request_frac": roof["request_frac"],
                       "form_peak_tflops": form_peak, "tc_peak_tflops": tc_peak, "fp32_peak_tflops": fp32_peak,
                       "hbm_gbs": hbm, "steps": rows}, f, indent=1)
    breakdown = {}
    for kd, v in sorted(kinds.items(), key=lambda kv: -kv[1]["ms"]):
        sec = v["ms"] / 1e3
        breakdown[names.get(kd, str(kd))] = {"share": v["ms"] / total_ms, "launches": v["launches"],
                                              "GB/s": v["bytes"] / sec / 1e9, "TFLOP/s": v["flops"] / sec / 1e12}

    line = {
        "metric": "amplitudes/s", "value": value, "unit": "amplitudes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": {"fp32": "c64", "3xtf32": "tf32x3 (fp32 acc)", "split_bf16": "bf16x3 (fp32 acc)"}[args.form],
        "data": "synthetic",
        "config": {"workload": wname, "form": args.form, "bitstrings_per_request": batch,
                   "seed": args.seed, "real_tflop_per_request": rep["real_flops"] / 1e12,
                   "paper_ops_log2": math.log2(rep["paper_ops"]), "tree_cost_log2": rep["tree_cost_log2"],
                   "separator_tree_cost_log2": rep["sep_cost_log2"], "n_sliced": rep["n_sliced"],
                   "slice_groups": rep["n_slice_groups"], "ws_bytes": rep["ws_bytes"],
                   "embedding": {1: "time collapsed", 2: "space-time"}.get(rep["embedding_used"]),
                   "plan_s": plan_s,
                   "paper_bounds_log2": {k: (round(v, 1) if math.isfinite(v) else None)
                                         for k, v in net.bounds().items()
                                         if k in ("thm2_log2", "thm2_pst_log2", "sidewise_log2", "explicit_log2")},
                   "l2": f"working set {rep['ws_bytes'] / 1e9:.2f} GB per request > 129 MB L2",
                   "parallelism": (f"slice groups of one request over {world} ranks, one FP64 all-reduce" if sharded
                                   else f"dp{world} (independent requests)"), "autotuned_steps": tuned,
                   "timing": "value: CUDA events around the K steps, device-resident bitstrings, CUDA-graph "
                             "replay per slice group; roofline and kernel_breakdown: a second pass with CUDA events "
                             "around every step (eager launches); e2e: host buffers through "
                             "tnc_contract_amplitudes, wall clock"},
        "effective_tflops": world * args.steps * rep["real_flops"] / (t_ms / 1e3) / 1e12,
        "measured_peaks": dict(fpk, hbm_gbs=hbm, bf16_tflops=float(peaks["bf16_tflops"]),
                               bf16_tflops_sustained=float(peaks.get("bf16_tflops_sustained", 0.0)) or None,
                               source=src),
        "roofline": roof,
        "kernel_breakdown": breakdown,
        "fp32_form": fp32_form,
        "hyperedge_form": hyper_form,
        "e2e": e2e,
        "clocks": ck,
        "gpu_launches": int(args.steps * rep["n_launches"]),
    }
    if args.workload == "iqp_5x8":
        if rank == 0 and not args.no_serving:
            forms = tuple(dict.fromkeys((args.form, "fp32")))
            line["serving"] = serving_measure(tnc, torch, forms=forms, seed=args.seed,
                                              n_req=max(args.serving_requests, args.serving_requests_fp32),
                                              n_req_by_form={args.form: args.serving_requests,
                                                             "fp32": args.serving_requests_fp32})
        if rank == 0 and not args.no_expectation:
            line["expectation"] = expectation_measure(tnc, torch, args.form, args.seed)
        if rank == 0 and not args.no_cpu_baseline:
            v, n_done, dt = _cpu_oracle(gl, bits[args.warmup:args.warmup + 1])
            va, ncores, na, dta = _cpu_oracle_all_cores(gl, bits[args.warmup:args.warmup + 1])
            line["cpu_baseline"] = {
                "value": v, "unit": "amplitudes/s", "cores": 1, "kind": "oracle",
                "sample": f"{n_done} bitstrings (one request) of the same workload by the IQP transfer-matrix "
                          f"closed form, {dt:.1f} s, numpy on one thread (elementwise, no BLAS calls; host has "
                          f"{os.cpu_count()} cores)",
                "all_cores": {"value": va, "unit": "amplitudes/s", "cores": ncores,
                              "sample": f"{na} bitstrings over {ncores} spawned processes (one thread each), "
                                        f"{dta:.1f} s"}}
    elif rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_oracle_rand2d_8x8_twin()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _cpu_oracle_rand2d_8x8_twin():
    """No CPU oracle reaches a random 64-qubit amplitude; the reported baseline
    is the oracle's CH form on the workload's Clifford twin (same 8 x 8 layout
    and depth-16 schedule, Clifford single-qubit gates), one thread, on a
    bounded sample of seed-random bitstrings."""
    from oracle.stabilizer import stabilizer_amplitudes
    gl, _ = C.workload("rand2d_8x8_d16", 0, clifford=True)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 10.0 and n < 256:
        stabilizer_amplitudes(gl, C.random_bitstrings(64, 1, 1000 + n))
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "amplitudes/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} amplitudes of the workload's Clifford twin by the CH form, {dt:.1f} s, one thread; "
                      f"no CPU oracle reaches a random 64-qubit amplitude"}


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
    ap.add_argument("--workload", choices=WORKLOADS, default="iqp_5x8",
                    help="iqp_5x8: 5 x 8 IQP, 256 bitstrings per request (default); rand2d_8x8_d16: 8 x 8 "
                         "depth-16 random circuit, one amplitude per request, sliced under 180 GB")
    ap.add_argument("--compare-forms", action="store_true",
                    help="rand2d_8x8_d16: also time one amplitude in the FP32 form")
    ap.add_argument("--serving-requests", type=int, default=1000, help="requests per arrival rate")
    ap.add_argument("--serving-requests-fp32", type=int, default=250,
                    help="requests per arrival rate in the FP32 form (5.5x slower; 1000 takes three minutes)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the compiler's default kernel per step")
    ap.add_argument("--no-hyperedges", dest="hyperedges", action="store_false",
                    help="skip timing the hyper-edge form of the network")
    ap.add_argument("--shard-slices", action="store_true",
                    help="rand2d_8x8_d16 under torchrun: split each request's slice groups over the ranks "
                         "(strong scaling, one FP64 all-reduce) instead of independent requests per rank")
    args = ap.parse_args()
    if args.op_counts:
        print(json.dumps(op_counts()), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
