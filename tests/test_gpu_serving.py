"""The serving loop (GPU): continuous batching of requests from different
circuits over a device arena.  Each result must equal the same request run
alone; admission refuses what can never fit; queued requests can be
cancelled; latencies are reported.  Also: CUDA-graph replay of a slice group
equals eager execution."""
import numpy as np
import pytest

import circuits as C
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _pool(tnc):
    circuits = [C.random_2d(4, 4, 8, 1), C.random_2d(5, 5, 8, 2), C.layered_3d(4, 4, 3), C.iqp(4, 5, 4),
                C.sycamore(4, 6, 5)]
    plans = []
    for i, gl in enumerate(circuits):
        oq = [1, 2] if i == 4 else []
        plans.append((gl, tnc.Plan(tnc.Network(gl), open_qubits=oq, max_batch=16, form="split_bf16")))
    return plans


@pytest.mark.parametrize("batching", [1, 8])
def test_alone_and_in_the_mix_agree(tnc, batching):
    """batching 8: waiting requests are admitted together and their nodes run
    in grouped launches across requests (tnc_contract_batch)."""
    plans = _pool(tnc)
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(40):
        gl, p = plans[i % len(plans)]
        b = int(rng.integers(1, 17))
        reqs.append((gl, p, C.random_bitstrings(gl.n_qubits, b, 100 + i)))
    alone = [tnc.contract_amplitudes(p, bits).cpu().numpy() for gl, p, bits in reqs]
    arena = torch.empty(max(p.ws_bytes for _, p in plans) * 3 + (1 << 20), dtype=torch.uint8, device="cuda")
    srv = tnc.Server(arena, n_streams=4)
    srv.set_batching(batching, 0, 0)  # every request of this pool may join a batch
    outs, tickets = [], []
    for gl, p, bits in reqs:
        out = torch.full((bits.shape[0], 1 << p.n_open), complex(np.nan, np.nan), dtype=torch.complex128,
                         device="cuda")
        outs.append(out)
        tickets.append(srv.submit(p, bits, out))
    lat = [srv.wait(t) for t in tickets]
    srv.close()
    for (gl, p, bits), a, o in zip(reqs, alone, outs):
        got = o.cpu().numpy()
        assert O.rel_error(got, a, gl.n_qubits).max() <= 1e-12
    ref = O.statevector_amplitudes(reqs[0][0], reqs[0][2], [])
    assert O.rel_error(outs[0].cpu().numpy(), ref, 16).max() <= 1e-4
    assert all(l > 0 for l in lat)
    p50, p99 = np.percentile(lat, [50, 99])
    assert p99 >= p50 > 0


def test_admission_refuses_what_cannot_fit(tnc):
    gl = C.random_2d(4, 4, 8, 1)
    p = tnc.Plan(tnc.Network(gl))
    arena = torch.empty(max(p.ws_bytes // 2, 256) // 256 * 256, dtype=torch.uint8, device="cuda")
    srv = tnc.Server(arena, n_streams=2)
    out = torch.empty((1, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(tnc.TncError) as ei:
        srv.submit(p, np.zeros((1, 16), np.uint8), out)
    assert ei.value.status == tnc.TNC_EBUSY
    srv.close()


def test_cancel_queued_request(tnc):
    gl = C.random_2d(5, 5, 10, 3)
    p = tnc.Plan(tnc.Network(gl), max_batch=4)
    arena = torch.empty((p.ws_bytes + 4096) // 256 * 256 + 256, dtype=torch.uint8, device="cuda")
    srv = tnc.Server(arena, n_streams=1)  # one request at a time: the rest queue
    outs = [torch.empty((4, 1), dtype=torch.complex128, device="cuda") for _ in range(12)]
    tickets = [srv.submit(p, C.random_bitstrings(25, 4, i), o) for i, o in enumerate(outs)]
    st = srv.cancel(tickets[-1])
    assert st in (tnc.TNC_OK, tnc.TNC_ESTATE)
    for t in tickets[:-1]:
        srv.wait(t)
    done, status = srv.poll(tickets[-1])
    if st == tnc.TNC_OK:
        assert done and status == tnc.TNC_ESTATE
    assert srv.poll(987654321)[1] == tnc.TNC_ENOTFOUND
    srv.close()


def test_graph_replay_equals_eager(tnc):
    gl = C.random_2d(4, 5, 10, 2)
    bits = C.random_bitstrings(20, 8, 1)
    for cap in (0, 1 << 17):
        pg = tnc.Plan(tnc.Network(gl), max_batch=8, form="split_bf16", mem_cap_bytes=cap, use_graph=True)
        pe = tnc.Plan(tnc.Network(gl), max_batch=8, form="split_bf16", mem_cap_bytes=cap, use_graph=False)
        ws = tnc.alloc_workspace(pg)
        g1 = tnc.contract_amplitudes(pg, bits, ws=ws).cpu().numpy()
        g2 = tnc.contract_amplitudes(pg, bits[::-1].copy(), ws=ws).cpu().numpy()  # replay, new inputs
        e1 = tnc.contract_amplitudes(pe, bits).cpu().numpy()
        e2 = tnc.contract_amplitudes(pe, bits[::-1].copy()).cpu().numpy()
        assert np.array_equal(g1, e1) and np.array_equal(g2, e2)
