"""Thin Python binding of the C ABI in ``include/tnc.h`` (ctypes).

Argument marshalling only: every step of the contraction runs inside
``libtnc.so`` (planning on the host, kernels on the GPU).  PyTorch provides
device memory and streams.  Importing this module fails loudly if the library
has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtnc.so")

TNC_OK = 0
TNC_EINVAL = -1
TNC_ENOMEM = -2
TNC_ECUDA = -3
TNC_ETIMEOUT = -4
TNC_EBUSY = -5
TNC_ESTATE = -6
TNC_ENOTFOUND = -7
TNC_NET_HYPEREDGES = 1

FORMS = {"fp32": 0, "3xtf32": 1, "split_bf16": 2}
EMBEDDINGS = {"auto": 0, "collapsed": 1, "spacetime": 2}


class TncError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class NetworkDesc(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("dim", C.c_int), ("coords", C.POINTER(C.c_double)),
                ("n_gates", C.c_int), ("arity", C.POINTER(C.c_int)), ("qubits", C.POINTER(C.c_int)),
                ("mats", C.POINTER(C.c_double))]


class CircuitBounds(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("dim", C.c_int), ("depth", C.c_int), ("sum_f", C.c_double),
                ("max_f", C.c_double), ("l", C.c_double), ("r", C.c_double), ("n_tensors", C.c_double),
                ("k", C.c_double), ("a_d", C.c_double), ("a2_pst", C.c_double), ("thm1_log2", C.c_double),
                ("thm2_log2", C.c_double), ("thm2_pst_log2", C.c_double), ("sidewise_log2", C.c_double),
                ("explicit_log2", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanOpts(C.Structure):
    _fields_ = [("n_open", C.c_int), ("open_qubits", C.POINTER(C.c_int)), ("max_batch", C.c_int),
                ("mem_cap_bytes", C.c_size_t), ("form", C.c_int), ("seed", C.c_uint64),
                ("ssa_trials", C.c_int), ("leaf_size", C.c_int), ("max_group_log2", C.c_int),
                ("use_graph", C.c_int), ("embedding", C.c_int), ("n_starts", C.c_int),
                ("refine_window", C.c_int), ("tree_only", C.c_int)]


class PlanReport(C.Structure):
    _fields_ = [("paper_ops", C.c_double), ("real_flops", C.c_double), ("bytes", C.c_double),
                ("peak_bytes", C.c_double), ("ws_bytes", C.c_size_t), ("n_slices", C.c_double),
                ("n_slice_groups", C.c_int), ("n_sliced", C.c_int), ("n_nodes", C.c_int),
                ("n_leaves", C.c_int), ("max_rank", C.c_int), ("n_launches", C.c_int),
                ("plan_ms", C.c_double), ("tree_cost_log2", C.c_double), ("embedding_used", C.c_int),
                ("seed_used", C.c_int), ("time_scale", C.c_double), ("sep_cost_log2", C.c_double),
                ("n_refined", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = [
    "tnc_status_string", "tnc_last_error", "tnc_load_network", "tnc_load_network_opts", "tnc_free_network",
    "tnc_plan_opts_default", "tnc_plan", "tnc_free_plan", "tnc_plan_get_report",
    "tnc_plan_export_json", "tnc_plan_upload", "tnc_contract_amplitudes",
    "tnc_contract_amplitudes_dbits", "tnc_contract_partial", "tnc_server_create",
    "tnc_server_submit", "tnc_server_poll", "tnc_server_wait", "tnc_server_cancel",
    "tnc_server_destroy", "tnc_plan_set_profiling", "tnc_plan_get_profile", "tnc_device_error",
    "tnc_contract_amplitudes_static", "tnc_permute", "tnc_cgemm_scratch_bytes", "tnc_cgemm",
    "tnc_ssa_separate", "tnc_centerpoint", "tnc_plan_autotune", "tnc_plan_get_kernels",
    "tnc_plan_set_kernels", "tnc_cgemm_variant", "tnc_selftest_bounded_wait", "tnc_circuit_bounds_eval",
    "tnc_contract_batch", "tnc_batch_ws_bytes", "tnc_server_set_batching",
]

# kernel variants of a contraction step (TNC_KG_* in tnc.h)
KG = {"simt_128x64": 0, "simt_64x32": 1, "narrow": 2, "dot": 3, "tc": 4, "simt_32x128": 5}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libtnc.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(_LIB_PATH)
    vp, i, sz, u64 = C.c_void_p, C.c_int, C.c_size_t, C.c_uint64
    sig = {
        "tnc_status_string": (C.c_char_p, [i]),
        "tnc_last_error": (C.c_char_p, []),
        "tnc_load_network": (i, [C.POINTER(NetworkDesc), C.POINTER(vp)]),
        "tnc_load_network_opts": (i, [C.POINTER(NetworkDesc), i, C.POINTER(vp)]),
        "tnc_free_network": (None, [vp]),
        "tnc_plan_opts_default": (None, [C.POINTER(PlanOpts)]),
        "tnc_plan": (i, [vp, C.POINTER(PlanOpts), C.POINTER(vp), C.POINTER(PlanReport)]),
        "tnc_free_plan": (None, [vp]),
        "tnc_plan_get_report": (i, [vp, C.POINTER(PlanReport)]),
        "tnc_plan_export_json": (i, [vp, C.c_char_p, sz, C.POINTER(sz)]),
        "tnc_plan_upload": (i, [vp, vp]),
        "tnc_contract_amplitudes": (i, [vp, vp, i, vp, vp, sz, vp]),
        "tnc_contract_amplitudes_dbits": (i, [vp, vp, i, vp, vp, sz, vp]),
        "tnc_contract_partial": (i, [vp, vp, i, i, i, vp, vp, sz, vp]),
        "tnc_contract_batch": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(i), C.POINTER(vp), vp, sz, vp]),
        "tnc_batch_ws_bytes": (sz, [i, C.POINTER(vp)]),
        "tnc_server_set_batching": (i, [vp, i, C.c_double, C.c_double]),
        "tnc_server_create": (i, [vp, sz, i, C.POINTER(vp)]),
        "tnc_server_submit": (i, [vp, vp, vp, i, vp, C.POINTER(u64)]),
        "tnc_server_poll": (i, [vp, u64, C.POINTER(i)]),
        "tnc_server_wait": (i, [vp, u64, i, C.POINTER(C.c_double)]),
        "tnc_server_cancel": (i, [vp, u64]),
        "tnc_server_destroy": (i, [vp]),
        "tnc_plan_set_profiling": (i, [vp, i]),
        "tnc_device_error": (i, [C.POINTER(i)]),
        "tnc_contract_amplitudes_static": (i, [vp, vp, i, vp, vp]),
        "tnc_permute": (i, [vp, vp, i, C.POINTER(i), vp]),
        "tnc_ssa_separate": (i, [C.POINTER(C.c_double), C.POINTER(C.c_double), i, i, u64, i, C.POINTER(i),
                                 C.POINTER(i), C.POINTER(i)]),
        "tnc_centerpoint": (i, [C.POINTER(C.c_double), i, i, u64, C.POINTER(C.c_double)]),
        "tnc_circuit_bounds_eval": (i, [C.POINTER(NetworkDesc), C.POINTER(CircuitBounds)]),
        "tnc_plan_autotune": (i, [vp, vp, sz, vp, i, C.POINTER(i)]),
        "tnc_plan_get_kernels": (i, [vp, C.POINTER(i), i, C.POINTER(i)]),
        "tnc_plan_set_kernels": (i, [vp, C.POINTER(i), i]),
        "tnc_cgemm_scratch_bytes": (sz, [C.c_int64] * 4 + [i]),
        "tnc_cgemm": (i, [vp, vp, vp] + [C.c_int64] * 4 + [i, i, i, vp, sz, vp]),
        "tnc_cgemm_variant": (i, [vp, vp, vp] + [C.c_int64] * 4 + [i, i, i, i, i, vp, vp, sz, vp]),
        "tnc_selftest_bounded_wait": (i, [C.c_uint, C.POINTER(C.c_int)]),
        "tnc_plan_get_profile": (i, [vp, C.POINTER(i), i, C.POINTER(C.c_double), C.POINTER(i),
                                     C.POINTER(i), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int, what: str):
    if status != TNC_OK:
        msg = lib.tnc_last_error().decode(errors="replace")
        raise TncError(status, f"{what}: {lib.tnc_status_string(status).decode()}: {msg}")


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Network:
    """``tnc_load_network`` on a gate list (``circuits.GateList``) or on the
    flat arrays (coords, arity, qubits, mats)."""

    def __init__(self, gatelist=None, *, arrays=None, hyperedges: bool = False):
        if gatelist is not None:
            coords, arity, qubits, mats = gatelist.arrays()
            n = gatelist.n_qubits
        else:
            coords, arity, qubits, mats = arrays
            n = coords.shape[0]
        coords = np.ascontiguousarray(coords, np.float64)
        self._n = int(n)
        self._keep = (coords, np.ascontiguousarray(arity, np.int32),
                      np.ascontiguousarray(qubits, np.int32), np.ascontiguousarray(mats, np.float64))
        desc = self.desc()
        h = C.c_void_p()
        _check(lib.tnc_load_network_opts(C.byref(desc), TNC_NET_HYPEREDGES if hyperedges else 0, C.byref(h)),
               "tnc_load_network_opts")
        self.handle = h
        self.n_qubits = int(n)

    def desc(self) -> NetworkDesc:
        """The descriptor of the arrays this object keeps alive."""
        c, a, q, m = self._keep
        return NetworkDesc(self._n, int(c.shape[1]) if c.ndim == 2 else 1, _ptr(c, C.c_double),
                           int(a.shape[0]), _ptr(a, C.c_int), _ptr(q, C.c_int), _ptr(m, C.c_double))

    def bounds(self) -> dict:
        """``tnc_circuit_bounds_eval``: the paper's cost bounds (Thm. 1, Thm. 2
        and its planar form, left-to-right, explicit time evolution) for this
        circuit's c = <0|U^dagger P U|0>, in log2 of scalar operations."""
        out = CircuitBounds()
        d = self.desc()
        _check(lib.tnc_circuit_bounds_eval(C.byref(d), C.byref(out)), "tnc_circuit_bounds_eval")
        return out.as_dict()

    def close(self):
        if self.handle:
            lib.tnc_free_network(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_network(gatelist) -> Network:
    return Network(gatelist)


class Plan:
    """``tnc_plan``: separator tree, slicing and compiled program (options as
    in ``tnc_plan_opts``; ``tree_only``: the tree and its Eq. 3 cost only, for
    cost studies of networks the executor cannot run)."""

    def __init__(self, net: Network, open_qubits=(), max_batch: int = 1, mem_cap_bytes: int = 0,
                 form: str = "fp32", seed: int = 1, ssa_trials: int = 32, leaf_size: int = 8,
                 max_group_log2: int = 6, use_graph: bool = True, embedding: str = "auto",
                 n_starts: int = 0, refine_window: int | None = None, tree_only: bool = False):
        o = PlanOpts()
        lib.tnc_plan_opts_default(C.byref(o))
        self._open = np.ascontiguousarray(sorted(int(q) for q in open_qubits), np.int32)
        o.n_open = len(self._open)
        o.open_qubits = _ptr(self._open, C.c_int) if len(self._open) else None
        o.max_batch = int(max_batch)
        o.mem_cap_bytes = int(mem_cap_bytes)
        o.form = FORMS[form] if isinstance(form, str) else int(form)
        o.seed = int(seed)
        o.ssa_trials = int(ssa_trials)
        o.leaf_size = int(leaf_size)
        o.max_group_log2 = int(max_group_log2)
        o.use_graph = int(bool(use_graph))
        o.embedding = EMBEDDINGS[embedding] if isinstance(embedding, str) else int(embedding)
        if n_starts:
            o.n_starts = int(n_starts)
        if refine_window is not None:
            o.refine_window = int(refine_window)
        o.tree_only = int(bool(tree_only))
        rep = PlanReport()
        h = C.c_void_p()
        _check(lib.tnc_plan(net.handle, C.byref(o), C.byref(h), C.byref(rep)), "tnc_plan")
        self.handle = h
        self.report = rep.as_dict()
        self.n_qubits = net.n_qubits
        self.n_open = len(self._open)
        self.open_qubits = self._open.copy()
        self.max_batch = int(max_batch)
        self.form = form

    @property
    def ws_bytes(self) -> int:
        return int(self.report["ws_bytes"])

    def export(self) -> dict:
        need = C.c_size_t()
        _check(lib.tnc_plan_export_json(self.handle, None, 0, C.byref(need)), "export")
        buf = C.create_string_buffer(need.value + 1)
        _check(lib.tnc_plan_export_json(self.handle, buf, need.value + 1, C.byref(need)), "export")
        return json.loads(buf.value.decode())

    def upload(self, stream=None):
        _check(lib.tnc_plan_upload(self.handle, _stream_ptr(stream)), "tnc_plan_upload")

    def autotune(self, ws=None, stream=None, reps: int = 3) -> int:
        """``tnc_plan_autotune``: pick the fastest kernel variant per step on
        this GPU; returns the number of steps that changed."""
        if ws is None:
            ws = alloc_workspace(self)
        n = C.c_int()
        _check(lib.tnc_plan_autotune(self.handle, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream),
                                     int(reps), C.byref(n)), "tnc_plan_autotune")
        rep = PlanReport()
        _check(lib.tnc_plan_get_report(self.handle, C.byref(rep)), "tnc_plan_get_report")
        self.report = rep.as_dict()
        return n.value

    def get_kernels(self):
        """Kernel choice per step ([kernel, tile] pairs; -1 for non-GEMM steps)."""
        n = C.c_int()
        _check(lib.tnc_plan_get_kernels(self.handle, None, 0, C.byref(n)), "tnc_plan_get_kernels")
        arr = np.zeros(2 * n.value, np.int32)
        _check(lib.tnc_plan_get_kernels(self.handle, _ptr(arr, C.c_int), arr.size, C.byref(n)), "tnc_plan_get_kernels")
        return arr.reshape(-1, 2).tolist()

    def set_kernels(self, choices):
        arr = np.ascontiguousarray(np.asarray(choices, np.int32).reshape(-1))
        _check(lib.tnc_plan_set_kernels(self.handle, _ptr(arr, C.c_int), arr.size // 2), "tnc_plan_set_kernels")
        rep = PlanReport()
        _check(lib.tnc_plan_get_report(self.handle, C.byref(rep)), "tnc_plan_get_report")
        self.report = rep.as_dict()

    def set_profiling(self, enable: bool):
        _check(lib.tnc_plan_set_profiling(self.handle, int(bool(enable))), "tnc_plan_set_profiling")

    def profile(self) -> dict:
        """Per-step event timings: arrays ms, runs, kind, flops, bytes."""
        n = C.c_int()
        _check(lib.tnc_plan_get_profile(self.handle, C.byref(n), 0, None, None, None, None, None), "profile")
        k = n.value
        ms = np.zeros(k, np.float64)
        runs = np.zeros(k, np.int32)
        kind = np.zeros(k, np.int32)
        fl = np.zeros(k, np.float64)
        by = np.zeros(k, np.float64)
        _check(lib.tnc_plan_get_profile(self.handle, C.byref(n), k, _ptr(ms, C.c_double), _ptr(runs, C.c_int),
                                        _ptr(kind, C.c_int), _ptr(fl, C.c_double), _ptr(by, C.c_double)),
               "profile")
        return dict(ms=ms, runs=runs, kind=kind, flops=fl, bytes=by)

    def close(self):
        if self.handle:
            lib.tnc_free_plan(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan(net: Network, **kw) -> Plan:
    return Plan(net, **kw)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def alloc_workspace(p: Plan, device="cuda"):
    import torch
    return torch.empty(max(p.ws_bytes, 256), dtype=torch.uint8, device=device)


def contract_amplitudes(p: Plan, bits, out=None, ws=None, stream=None):
    """Amplitudes for host bitstrings ``bits`` (uint8 [batch][n_qubits]).
    Returns (or fills) a complex128 CUDA tensor [batch][2^n_open]."""
    import torch
    bits = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint8)
    batch = bits.shape[0]
    if out is None:
        out = torch.empty((batch, 1 << p.n_open), dtype=torch.complex128, device="cuda")
    if ws is None:
        ws = alloc_workspace(p)
    _check(lib.tnc_contract_amplitudes(p.handle, bits.ctypes.data_as(C.c_void_p), batch,
                                       C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()),
                                       ws.numel(), _stream_ptr(stream)), "tnc_contract_amplitudes")
    return out


def contract_amplitudes_dbits(p: Plan, d_bits, out=None, ws=None, stream=None):
    """Same with a uint8 CUDA tensor of bitstrings."""
    import torch
    batch = d_bits.shape[0]
    if out is None:
        out = torch.empty((batch, 1 << p.n_open), dtype=torch.complex128, device="cuda")
    if ws is None:
        ws = alloc_workspace(p)
    _check(lib.tnc_contract_amplitudes_dbits(p.handle, C.c_void_p(d_bits.data_ptr()), batch,
                                             C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()),
                                             ws.numel(), _stream_ptr(stream)), "tnc_contract_amplitudes_dbits")
    return out


def contract_partial(p: Plan, d_bits, group_begin: int, group_end: int, out=None, ws=None, stream=None):
    import torch
    batch = d_bits.shape[0]
    if out is None:
        out = torch.empty((batch, 1 << p.n_open), dtype=torch.complex128, device="cuda")
    if ws is None:
        ws = alloc_workspace(p)
    _check(lib.tnc_contract_partial(p.handle, C.c_void_p(d_bits.data_ptr()), batch, int(group_begin),
                                    int(group_end), C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()),
                                    ws.numel(), _stream_ptr(stream)), "tnc_contract_partial")
    return out


def batch_ws_bytes(plans) -> int:
    """``tnc_batch_ws_bytes``: workspace of ``contract_batch`` for these plans."""
    arr = (C.c_void_p * len(plans))(*[p.handle.value for p in plans])
    return int(lib.tnc_batch_ws_bytes(len(plans), arr))


def contract_batch(plans, bits_list, outs=None, ws=None, stream=None):
    """``tnc_contract_batch``: several requests (plan, host bitstrings) in one
    go, their nodes grouped across requests wave by wave.  Returns (or fills)
    one complex128 CUDA tensor [batch][2^n_open] per request."""
    import torch
    n = len(plans)
    bl = [np.ascontiguousarray(np.atleast_2d(b), dtype=np.uint8) for b in bits_list]
    if outs is None:
        outs = [torch.empty((b.shape[0], 1 << p.n_open), dtype=torch.complex128, device="cuda")
                for p, b in zip(plans, bl)]
    if ws is None:
        ws = torch.empty(max(batch_ws_bytes(plans), 256), dtype=torch.uint8, device="cuda")
    ph = (C.c_void_p * n)(*[p.handle.value for p in plans])
    bp = (C.c_void_p * n)(*[b.ctypes.data for b in bl])
    nb = (C.c_int * n)(*[b.shape[0] for b in bl])
    op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(lib.tnc_contract_batch(n, ph, bp, nb, op, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)),
           "tnc_contract_batch")
    return outs


def contract_amplitudes_static(p: Plan, bits, out, stream=None):
    """``tnc_contract_amplitudes_static``: same result as
    :func:`contract_amplitudes` with the library's static 64 MiB workspace;
    the plan must be uploaded first and ``out`` preallocated (nothing is
    allocated by this call)."""
    bits = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint8)
    _check(lib.tnc_contract_amplitudes_static(p.handle, bits.ctypes.data_as(C.c_void_p), bits.shape[0],
                                              C.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "tnc_contract_amplitudes_static")
    return out


def permute(x, src_bit, out=None, stream=None):
    """``tnc_permute`` on a complex64 CUDA tensor of 2^rank elements."""
    import torch
    rank = len(src_bit)
    if out is None:
        out = torch.empty_like(x)
    sb = np.ascontiguousarray(src_bit, np.int32)
    _check(lib.tnc_permute(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), rank,
                           sb.ctypes.data_as(C.POINTER(C.c_int)), _stream_ptr(stream)), "tnc_permute")
    return out


def cgemm(A, B, batch, M, N, K, transA=0, transB=0, form="fp32", out=None, scratch=None, stream=None,
          kernel=None, tile=None, c_pos=None):
    """``tnc_cgemm`` (``tnc_cgemm_variant`` when ``kernel`` is given, a name
    of ``KG`` or its number): batched complex GEMM of one tree node on
    complex64 CUDA tensors.  ``c_pos``: output bit order (see tnc.h)."""
    import torch
    f = FORMS[form] if isinstance(form, str) else int(form)
    need = lib.tnc_cgemm_scratch_bytes(batch, M, N, K, f)
    if out is None:
        out = torch.empty((batch, M, N), dtype=torch.complex64, device=A.device)
    if scratch is None and need:
        scratch = torch.empty(need, dtype=torch.uint8, device=A.device)
    kg = -1 if kernel is None else (KG[kernel] if isinstance(kernel, str) else int(kernel))
    cp = None if c_pos is None else np.ascontiguousarray(c_pos, np.int32)
    _check(lib.tnc_cgemm_variant(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_void_p(out.data_ptr()),
                                 batch, M, N, K, int(transA), int(transB), f, kg, -1 if tile is None else int(tile),
                                 _ptr(cp, C.c_int) if cp is not None else None,
                                 C.c_void_p(scratch.data_ptr() if scratch is not None else 0),
                                 scratch.numel() if scratch is not None else 0, _stream_ptr(stream)), "tnc_cgemm")
    return out


def ssa_separate(pos, rad, seed: int = 1, trials: int = 32):
    """Algorithm 1 on spheres (centres ``pos`` [n][dim], radii ``rad``):
    returns (side array: 0 inside, 1 outside, 2 intersected; valid; k)."""
    pos = np.ascontiguousarray(pos, np.float64)
    rad = np.ascontiguousarray(rad, np.float64)
    n, dim = pos.shape
    side = np.zeros(n, np.int32)
    valid, k = C.c_int(), C.c_int()
    _check(lib.tnc_ssa_separate(_ptr(pos, C.c_double), _ptr(rad, C.c_double), n, dim, seed, trials,
                                _ptr(side, C.c_int), C.byref(valid), C.byref(k)), "tnc_ssa_separate")
    return side, bool(valid.value), k.value


def centerpoint(pts, seed: int = 1):
    pts = np.ascontiguousarray(pts, np.float64)
    c = np.zeros(pts.shape[1], np.float64)
    _check(lib.tnc_centerpoint(_ptr(pts, C.c_double), pts.shape[0], pts.shape[1], seed, _ptr(c, C.c_double)),
           "tnc_centerpoint")
    return c


class Server:
    """``tnc_server_*``: continuous batching of amplitude requests over a
    device arena (a uint8 CUDA tensor owned by the caller)."""

    def __init__(self, arena, n_streams: int = 4):
        self.arena = arena
        h = C.c_void_p()
        _check(lib.tnc_server_create(C.c_void_p(arena.data_ptr()), arena.numel(), n_streams, C.byref(h)),
               "tnc_server_create")
        self.handle = h
        self._keep = {}

    def set_batching(self, max_requests: int, max_request_flops: float = 2.0 ** 34,
                     max_request_bytes: float = 2.0 ** 28):
        """``tnc_server_set_batching``: admit up to this many waiting small
        requests together (planned real flops and bytes at most the limits;
        0: no limit), their nodes grouped across requests (1: each alone)."""
        _check(lib.tnc_server_set_batching(self.handle, int(max_requests), float(max_request_flops),
                                           float(max_request_bytes)), "tnc_server_set_batching")

    def submit(self, plan: Plan, bits, out) -> int:
        bits = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint8)
        t = C.c_uint64()
        _check(lib.tnc_server_submit(self.handle, plan.handle, bits.ctypes.data_as(C.c_void_p), bits.shape[0],
                                     C.c_void_p(out.data_ptr()), C.byref(t)), "tnc_server_submit")
        self._keep[t.value] = out
        return t.value

    def poll(self, ticket: int):
        done = C.c_int()
        st = lib.tnc_server_poll(self.handle, ticket, C.byref(done))
        return bool(done.value), st

    def wait(self, ticket: int, timeout_ms: int = 60000) -> float:
        lat = C.c_double()
        _check(lib.tnc_server_wait(self.handle, ticket, timeout_ms, C.byref(lat)), "tnc_server_wait")
        self._keep.pop(ticket, None)
        return lat.value

    def cancel(self, ticket: int) -> int:
        return lib.tnc_server_cancel(self.handle, ticket)

    def close(self):
        if self.handle:
            lib.tnc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
