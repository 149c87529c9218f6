"""Slice sharding across processes (one per GPU).

The slices of a plan are independent sub-networks with identical shapes
(index slicing, named as future work in the paper's Conclusion), so the
serial slice groups split into contiguous ranges, one per rank; each rank
computes its partial amplitudes with ``tnc_contract_partial`` and one FP64
sum over the ranks (the only exchange step) gives the amplitudes.
"""
from __future__ import annotations

import numpy as np


def group_range(n_groups: int, rank: int, world: int):
    """Contiguous, balanced range [begin, end) of slice groups of ``rank``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_groups, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist, dist.get_rank(), dist.get_world_size()
    return None, 0, 1


def allreduce_sum_fp64(values):
    """Sum complex128 partial amplitudes over all ranks (FP64).  Accepts a
    torch tensor (CUDA tensors go through the process group's device backend)
    or a NumPy array (summed through a CPU tensor)."""
    import torch
    dist, _, world = _dist()
    if dist is None or world == 1:
        return values
    if isinstance(values, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(values).view(np.float64).copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy().view(np.complex128).reshape(values.shape)
    t = torch.view_as_real(values).contiguous()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return torch.view_as_complex(t)


def contract_amplitudes_sharded(plan, d_bits, compute=None, out=None, ws=None, stream=None):
    """Amplitudes of ``plan`` for device bitstrings ``d_bits`` with the slice
    groups split over the ranks of the default process group.  ``compute``
    (begin, end) -> partial amplitudes replaces the GPU call (for host tests)."""
    _, rank, world = _dist()
    g0, g1 = group_range(int(plan.report["n_slice_groups"]), rank, world)
    if compute is not None:
        part = compute(g0, g1)
    else:
        from . import tnc
        part = tnc.contract_partial(plan, d_bits, g0, g1, out=out, ws=ws, stream=stream)
    return allreduce_sum_fp64(part)
