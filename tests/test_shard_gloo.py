"""Slice sharding over two CPU ranks (gloo, world size 2): each rank computes
its range of slice groups (the compiled program emulated on the host) and one
FP64 all-reduce gives the amplitudes of the FP64 oracle."""
import os
import socket

import numpy as np
import pytest

import circuits as C
import oracle as O
from paper_2208_01498_gb300 import shard, tnc
from host_emulator import emulate_program

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_group_range_partitions():
    for n in (1, 2, 7, 64, 513):
        for w in (1, 2, 3, 8):
            ranges = [shard.group_range(n, r, w) for r in range(w)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        gl = C.random_2d(4, 5, 10, 2)
        bits = C.random_bitstrings(20, 2, 3)
        p = tnc.Plan(tnc.Network(gl), open_qubits=[0, 7], max_batch=2, mem_cap_bytes=1 << 16, max_group_log2=0)
        e = p.export()
        res = shard.contract_amplitudes_sharded(p, None, compute=lambda g0, g1: emulate_program(e, bits, range(g0, g1)))
        q.put((rank, p.report["n_slice_groups"], res))
    finally:
        dist.destroy_process_group()


def test_two_rank_slice_sharding_matches_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=300) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    gl = C.random_2d(4, 5, 10, 2)
    bits = C.random_bitstrings(20, 2, 3)
    ref = O.statevector_amplitudes(gl, bits, [0, 7])
    assert results[0][1] >= 2
    for _, _, res in results:
        assert O.rel_error(res, ref, 20).max() < 1e-5
    assert np.allclose(results[0][2], results[1][2], rtol=0, atol=0)


def _dying_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(3)  # a rank that leaves before the exchange
    try:
        shard.allreduce_sum_fp64(np.ones(4, np.complex128))
        q.put("no error")
    except Exception as ex:  # the surviving rank sees an error, not a hang
        q.put(type(ex).__name__)


def test_lost_rank_surfaces_as_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    msg = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        if pr.is_alive():
            pr.kill()
    assert msg != "no error"
