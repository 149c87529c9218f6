"""Kernel-level parity (GPU): the permute and the complex GEMM of one tree
node, called through tnc_permute / tnc_cgemm, against NumPy complex128."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative Frobenius error bound per form (random normal operands)
TOL = {"fp32": 2e-6, "3xtf32": 4e-6, "split_bf16": 4e-5}
# per-element bound: max |C - C_ref| / max(|C_ref|, TAU * rms(C_ref)) <= ELEM_TOL.  Every element is
# judged on its own, so a few wrong ones (a ragged edge, a collision of the scattered output) cannot
# hide behind the norm.  With TAU = 1 the bound is max |err| / rms(C_ref) for the small elements; the
# rounding errors of an FP32 sum have a Gaussian-like tail, whose maximum over 10^6 elements is about
# 4x their rms, hence 5x the Frobenius bound.
TAU = 1.0
ELEM_TOL = {f: 5 * t for f, t in TOL.items()}


def _assert_close(got, ref, form, what):
    got = np.asarray(got).astype(np.complex128).reshape(ref.shape)
    diff = np.abs(got - ref)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2)) if ref.size else 0.0
    frob = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    assert frob <= TOL[form], f"{what} {form}: Frobenius {frob:.3g} > {TOL[form]}"
    if rms == 0.0:
        assert diff.max(initial=0.0) == 0.0, f"{what} {form}: nonzero result for a zero product"
        return
    elem = diff / np.maximum(np.abs(ref), TAU * rms)
    worst = int(np.argmax(elem))
    assert elem.flat[worst] <= ELEM_TOL[form], (
        f"{what} {form}: element {np.unravel_index(worst, ref.shape)} off by {elem.flat[worst]:.3g} "
        f"(> {ELEM_TOL[form]})")


@pytest.fixture(scope="module")
def tnc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_01498_gb300 import tnc as t
    return t


def _crand(shape, rng):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("rank", [0, 1, 3, 5, 8, 11, 16, 21])
@pytest.mark.parametrize("kind", ["random", "identity", "reverse"])
def test_permute_matches_numpy(tnc, rank, kind):
    rng = np.random.default_rng(rank)
    src_bit = {"random": rng.permutation(rank), "identity": np.arange(rank),
               "reverse": np.arange(rank)[::-1]}[kind].astype(np.int32)
    x = _crand(1 << rank, rng)
    got = tnc.permute(torch.from_numpy(x).cuda(), src_bit).cpu().numpy()
    # out bit k = in bit src_bit[k]; numpy axis a <-> bit rank-1-a
    perm = [rank - 1 - src_bit[rank - 1 - a] for a in range(rank)]
    ref = np.transpose(x.reshape((2,) * rank), perm).reshape(-1) if rank else x
    assert np.array_equal(got, ref)


def test_permute_rejects_non_permutation(tnc):
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(tnc.TncError) as ei:
        tnc.permute(x, [0, 0, 1])
    assert ei.value.status == tnc.TNC_EINVAL


SHAPES = [  # batch, M, N, K, transA, transB
    (1, 1, 1, 1, 0, 0), (3, 5, 7, 9, 0, 0), (2, 64, 48, 100, 1, 0), (2, 33, 65, 17, 0, 1),
    (1, 1000, 4, 2, 0, 1), (4, 513, 16, 16, 1, 1), (1, 2, 2, 100000, 0, 1), (2, 8, 8, 20000, 1, 0),
    (1, 4, 4, 3000, 0, 0), (8, 16, 256, 8, 0, 1), (3, 1, 1, 70000, 0, 1), (2, 1, 1, 4099, 1, 0),
    (5, 1, 1, 1 << 16, 0, 1),
    # split-K dot with 16-byte loads (K-major operands): FP32 per thread and warp, FP64 across
    (256, 4, 4, 16384, 0, 1), (3, 2, 4, 1000, 0, 1), (2, 4, 1, 1 << 20, 0, 1), (1, 3, 3, 70000, 0, 1),
]
TC_SHAPES = [(4, 128, 64, 64, 0, 1), (2, 256, 128, 512, 0, 1), (1, 512, 256, 4096, 0, 1),
             (2, 128, 32, 64, 0, 1), (1, 1024, 512, 8192, 0, 1),
             (3, 128, 32, 32, 1, 0), (2, 128, 128, 1024, 0, 0)]


def _ref(A, B, batch, M, N, K, tA, tB):
    a = A.reshape(batch, K, M).transpose(0, 2, 1) if tA else A.reshape(batch, M, K)
    b = B.reshape(batch, N, K).transpose(0, 2, 1) if tB else B.reshape(batch, K, N)
    return a.astype(np.complex128) @ b.astype(np.complex128)


def _check_gemm(tnc, shape, form):
    batch, M, N, K, tA, tB = shape
    rng = np.random.default_rng(batch * 7 + M + N + K)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, tA, tB, form)
    torch.cuda.synchronize()
    ref = _ref(A, B, batch, M, N, K, tA, tB)
    _assert_close(got.cpu().numpy(), ref, form, f"{shape}")


@pytest.mark.parametrize("shape", SHAPES)
def test_cgemm_cuda_cores(tnc, shape):
    _check_gemm(tnc, shape, "fp32")


@pytest.mark.parametrize("shape", TC_SHAPES)
@pytest.mark.parametrize("form", ["split_bf16", "3xtf32", "fp32"])
def test_cgemm_tensor_cores(tnc, shape, form):
    _check_gemm(tnc, shape, form)


def test_cgemm_scratch_too_small(tnc):
    A = torch.zeros(128 * 64, dtype=torch.complex64, device="cuda")
    B = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(tnc.TncError) as ei:
        tnc.cgemm(A, B, 1, 128, 64, 64, 0, 1, "split_bf16", scratch=small)
    assert ei.value.status == tnc.TNC_ENOMEM


TILE_SHAPES = [(2, 128, 128, 64, 0, 1), (1, 256, 256, 4096, 0, 1), (3, 512, 128, 128, 0, 1), (1, 256, 512, 1024, 1, 0),
               (4, 256, 32, 128, 0, 1), (2, 128, 64, 1024, 0, 1), (2, 256, 512, 256, 0, 1), (3, 128, 256, 32, 0, 1)]


@pytest.mark.parametrize("shape", TILE_SHAPES)
@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15])
@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
def test_cgemm_tensor_core_tile_widths(tnc, shape, tile, form):
    """Every tcgen05 tile width (128 x 64, 128 x 128, 128 x 256 real outputs
    per CTA; 128 x 128, 128 x 64 and 128 x 256 with the split on chip,
    without and with prefetch; 128 x 256 and 128 x 128 persistent from the
    planes) on the same shapes, through tnc_cgemm_variant."""
    batch, M, N, K, tA, tB = shape
    if (4 <= tile <= 8 or tile >= 14) and (form != "split_bf16" or tA or not tB):
        pytest.skip("the on-chip split takes split-BF16 with K-major operands only")
    if tile >= 9 and form != "split_bf16":  # 9..12
        pytest.skip("the persistent plane kernel takes split-BF16 only")
    if tile == 13 and (form != "split_bf16" or tA):
        pytest.skip("the hybrid tile splits a K-major A on chip (split-BF16)")
    if (tile == 2 and N < 64) or (tile in (3, 8, 9, 11, 13, 14, 15) and N < 128) or (tile in (4, 5, 10) and N < 64):
        pytest.skip("tile wider than N")
    if tile in (8, 9, 11, 13) and K > 256:
        pytest.skip("the 256-column persistent tiles take K <= 256")
    rng = np.random.default_rng(batch + M + N + K + tile)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, tA, tB, form,
                    kernel="tc", tile=tile)
    torch.cuda.synchronize()
    ref = _ref(A, B, batch, M, N, K, tA, tB)
    _assert_close(got.cpu().numpy(), ref, form, f"{shape} tile {tile}")


def test_cgemm_variant_rejects_impossible_choice(tnc):
    A = torch.zeros(128 * 64, dtype=torch.complex64, device="cuda")
    B = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(tnc.TncError) as ei:  # N = 64 complex is too narrow for 256 real columns
        tnc.cgemm(A, B, 1, 128, 64, 64, 0, 1, "split_bf16", kernel="tc", tile=3)
    assert ei.value.status == tnc.TNC_EINVAL
    with pytest.raises(tnc.TncError) as ei:  # no tensor cores in the FP32 form
        tnc.cgemm(A, B, 1, 128, 64, 64, 0, 1, "fp32", kernel="tc", tile=2)
    assert ei.value.status == tnc.TNC_EINVAL


def test_cgemm_on_chip_split_unaligned_operands(tnc):
    """Operands that are not 16-byte aligned go through the hi/lo planes
    instead of the on-chip split, with the same result."""
    batch, M, N, K = 2, 128, 64, 256
    rng = np.random.default_rng(5)
    A = _crand(batch * M * K + 1, rng)
    B = _crand(batch * K * N + 1, rng)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    got = tnc.cgemm(dA[1:], dB[1:], batch, M, N, K, 0, 1, "split_bf16", kernel="tc", tile=4)
    ref = _ref(A[1:], B[1:], batch, M, N, K, 0, 1)
    _assert_close(got.cpu().numpy(), ref, "split_bf16", "unaligned operands")


SCATTER_CASES = [  # batch, M, N, K, kernel, tile, form
    (4, 64, 32, 8, "simt_64x32", 0, "fp32"), (2, 128, 64, 4, "simt_128x64", 0, "fp32"),
    (8, 32, 128, 16, "simt_32x128", 0, "fp32"), (16, 256, 8, 4, "narrow", 0, "fp32"),
    (4, 1, 1, 4096, "dot", 0, "fp32"), (4, 256, 128, 128, "tc", 2, "split_bf16"),
    (4, 256, 128, 128, "tc", 4, "split_bf16"), (4, 256, 128, 256, "tc", 8, "split_bf16"),
    (4, 256, 128, 256, "tc", 9, "split_bf16"), (4, 256, 128, 64, "tc", 11, "split_bf16"),
    (2, 512, 256, 8, "tc", 11, "split_bf16"), (8, 128, 32, 64, "tc", 6, "split_bf16"),
    (8, 256, 32, 4, "tc", 12, "split_bf16"), (4, 128, 64, 128, "tc", 12, "split_bf16"),
    (4, 256, 128, 128, "tc", 13, "split_bf16"), (2, 512, 256, 16, "tc", 13, "split_bf16"),
    (2, 256, 128, 2048, "tc", 14, "split_bf16"), (2, 128, 256, 1024, "tc", 15, "split_bf16"),
    (2, 128, 64, 1024, "tc", 5, "split_bf16"), (2, 256, 64, 128, "tc", 10, "split_bf16"),
    (4, 128, 64, 64, "tc", 2, "3xtf32"), (4, 256, 32, 32, "tc", 16, "split_bf16"),
    (4, 256, 64, 128, "tc", 17, "split_bf16"), (2, 256, 128, 256, "tc", 18, "split_bf16"),
    (4, 256, 64, 8, "tc", 17, "split_bf16"),
]


@pytest.mark.parametrize("case", SCATTER_CASES, ids=lambda c: f"{c[4]}{c[5]}-{c[6]}")
def test_cgemm_scattered_output(tnc, case):
    """Every kernel variant writing C in a shuffled bit order (as a plan's
    consumer layout), element by element against NumPy."""
    batch, M, N, K, kernel, tile, form = case
    nN, nM, nB = N.bit_length() - 1, M.bit_length() - 1, batch.bit_length() - 1
    rng = np.random.default_rng(M + N + K + tile)
    c_pos = rng.permutation(nN + nM + nB)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, 0, 1, form,
                    kernel=kernel, tile=tile, c_pos=c_pos).reshape(-1).cpu().numpy()
    ref = _ref(A, B, batch, M, N, K, 0, 1)
    b, m, n = np.meshgrid(np.arange(batch), np.arange(M), np.arange(N), indexing="ij")
    addr = np.zeros(b.shape, np.int64)
    for i in range(nN):
        addr |= ((n >> i) & 1) << int(c_pos[i])
    for i in range(nM):
        addr |= ((m >> i) & 1) << int(c_pos[nN + i])
    for i in range(nB):
        addr |= ((b >> i) & 1) << int(c_pos[nN + nM + i])
    placed = got[addr]
    _assert_close(placed, ref, form, f"{case}")
    # the scatter is a bijection: no output slot is left unwritten or written twice
    assert np.array_equal(np.sort(addr.reshape(-1)), np.arange(addr.size))


@pytest.mark.parametrize("case", [(4, 256, 128, 128, 4), (8, 256, 32, 64, 6), (2, 256, 128, 256, 8),
                                  (2, 256, 64, 128, 10), (4, 256, 128, 128, 13), (2, 256, 128, 512, 14),
                                  (4, 256, 32, 32, 16), (4, 256, 64, 128, 17), (2, 256, 128, 256, 18)],
                         ids=lambda c: f"tile{c[4]}")
@pytest.mark.parametrize("low", [("m", 0, "m", 1), ("n", 1, None, None), ("n", 2, "m", 3), ("m", 2, "n", 2),
                                 ("m", 4, "n", 0)], ids=lambda x: "".join(str(t) for t in x if t is not None))
def test_cgemm_direct_store_layout(tnc, case, low):
    """Output orders whose lowest address bits are bits of an epilogue warp's
    32 x 8 block: row bits at bits 0 and 1 (direct 8-byte stores), a column
    bit at bit 0 (direct 16-byte column pairs), a row bit at 0 and a column
    bit at 1 (through the staging block).  Element by element against NumPy;
    the scatter is a bijection."""
    batch, M, N, K, tile = case
    nN, nM, nB = N.bit_length() - 1, M.bit_length() - 1, batch.bit_length() - 1
    rng = np.random.default_rng(11 * tile + K)
    c_pos = np.full(nN + nM + nB, -1, np.int64)
    fixed = []
    for at, (kind, bit) in enumerate([(low[0], low[1]), (low[2], low[3])]):
        if kind is None:
            continue
        idx = bit if kind == "n" else nN + bit
        c_pos[idx] = at
        fixed.append(at)
    others = [i for i in range(nN + nM + nB) if c_pos[i] < 0]
    c_pos[others] = rng.permutation([p for p in range(nN + nM + nB) if p not in fixed])
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, 0, 1, "split_bf16",
                    kernel="tc", tile=tile, c_pos=c_pos).reshape(-1).cpu().numpy()
    ref = _ref(A, B, batch, M, N, K, 0, 1)
    b, m, n = np.meshgrid(np.arange(batch), np.arange(M), np.arange(N), indexing="ij")
    addr = np.zeros(b.shape, np.int64)
    for i in range(nN):
        addr |= ((n >> i) & 1) << int(c_pos[i])
    for i in range(nM):
        addr |= ((m >> i) & 1) << int(c_pos[nN + i])
    for i in range(nB):
        addr |= ((b >> i) & 1) << int(c_pos[nN + nM + i])
    assert np.array_equal(np.sort(addr.reshape(-1)), np.arange(addr.size))
    _assert_close(got[addr], ref, "split_bf16", f"{case} direct stores")


@pytest.mark.parametrize("shape,tile", [((2, 256, 128, 8, 0, 1), 9), ((2, 256, 128, 8, 0, 1), 10),
                                        ((4, 128, 64, 4, 0, 1), 10), ((1, 512, 256, 16, 1, 0), 9),
                                        ((2, 256, 128, 8, 0, 1), 11), ((1, 256, 256, 4, 0, 1), 11),
                                        ((4, 256, 32, 4, 0, 1), 12), ((2, 128, 64, 16, 1, 0), 12)])
def test_cgemm_short_k_plane_tiles(tnc, shape, tile):
    """The persistent plane tiles on K < 32 (the k-block beyond the plane
    rows is zero-filled by TMA), on plain and scattered outputs."""
    batch, M, N, K, tA, tB = shape
    rng = np.random.default_rng(M + N + K + tile)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    ref = _ref(A, B, batch, M, N, K, tA, tB)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, tA, tB, "split_bf16",
                    kernel="tc", tile=tile)
    _assert_close(got.cpu().numpy(), ref, "split_bf16", f"{shape} tile {tile}")


@pytest.mark.parametrize("shape,tile", [((2, 256, 32, 2), 16), ((4, 128, 64, 8), 17), ((2, 256, 128, 4), 18),
                                        ((1, 512, 64, 16), 16), ((8, 4096, 32, 32), 16), ((2, 2048, 64, 64), 17),
                                        ((4, 1024, 128, 256), 18), ((2, 256, 64, 2048), 17),
                                        ((1, 128, 32, 1024), 16), ((16, 512, 128, 32), 18)])
def test_cgemm_f32_ring_tiles(tnc, shape, tile):
    """The on-chip split fed by TMA from FP32 tiles (tiles 16-18): short K
    (the k-block beyond K zero-filled by TMA), CTAs with several tiles, rings
    that wrap many times, long K with several accumulation chunks, element by
    element against NumPy."""
    batch, M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 5 * K + tile)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    ref = _ref(A, B, batch, M, N, K, 0, 1)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, 0, 1, "split_bf16",
                    kernel="tc", tile=tile)
    _assert_close(got.cpu().numpy(), ref, "split_bf16", f"{shape} tile {tile}")


@pytest.mark.parametrize("form", ["split_bf16", "3xtf32"])
@pytest.mark.parametrize("shape,scatter", [((1, 256, 64, 65536), False), ((2, 128, 32, 8192), True),
                                           ((1, 128, 128, 4096), True), ((4, 256, 32, 1024), False)])
def test_cgemm_tc_split_k(tnc, shape, scatter, form):
    """Tile 19: the plane tiles with K split over CTAs (FP32 partial tiles
    summed in FP64 into the consumer's layout), for nodes with few output
    tiles and long K; element by element against NumPy."""
    batch, M, N, K = shape
    rng = np.random.default_rng(M + N + K + batch)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    ref = _ref(A, B, batch, M, N, K, 0, 1)
    c_pos = None
    if scatter:
        nN, nM, nB = N.bit_length() - 1, M.bit_length() - 1, batch.bit_length() - 1
        c_pos = rng.permutation(nN + nM + nB)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, 0, 1, form,
                    kernel="tc", tile=19, c_pos=c_pos).reshape(-1).cpu().numpy()
    if scatter:
        b, m, n = np.meshgrid(np.arange(batch), np.arange(M), np.arange(N), indexing="ij")
        addr = np.zeros(b.shape, np.int64)
        for i in range(nN):
            addr |= ((n >> i) & 1) << int(c_pos[i])
        for i in range(nM):
            addr |= ((m >> i) & 1) << int(c_pos[nN + i])
        for i in range(nB):
            addr |= ((b >> i) & 1) << int(c_pos[nN + nM + i])
        got = got[addr]
    _assert_close(got.reshape(ref.shape), ref, form, f"{shape} split K")


@pytest.mark.parametrize("kernel", ["simt_128x64", "simt_64x32", "simt_32x128"])
@pytest.mark.parametrize("shape", [(1, 64, 64, 4096, 0, 1), (2, 100, 36, 1000, 1, 0), (1, 32, 128, 600, 0, 0),
                                   (256, 32, 16, 2048, 0, 1)])
def test_cgemm_cuda_cores_split_k_small_grid(tnc, kernel, shape):
    """Nodes with fewer output tiles than SMs and K >= 512, or one to four
    waves of tiles and K >= 2048 (batch 256, M 32, N 16), run the CUDA-core
    kernels with K split over blocks and an FP64 reduction: every tile shape,
    ragged sizes included, against NumPy; the power-of-two shape also with a
    scattered output."""
    batch, M, N, K, tA, tB = shape
    rng = np.random.default_rng(M + N + K)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    ref = _ref(A, B, batch, M, N, K, tA, tB)
    got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, tA, tB, "fp32",
                    kernel=kernel)
    _assert_close(got.cpu().numpy(), ref, "fp32", f"{shape} {kernel}")
    if shape[0] == 1 and M == 64:
        c_pos = np.random.default_rng(1).permutation(12)
        got = tnc.cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), batch, M, N, K, tA, tB, "fp32",
                        kernel=kernel, c_pos=c_pos).reshape(-1).cpu().numpy()
        m, n = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
        addr = np.zeros(m.shape, np.int64)
        for i in range(6):
            addr |= ((n >> i) & 1) << int(c_pos[i])
            addr |= ((m >> i) & 1) << int(c_pos[6 + i])
        placed = got[addr]
        _assert_close(placed, ref[0], "fp32", f"scattered {kernel}")


NARROW_CASES = [  # batch, M, N, K
    (256, 8192, 16, 16), (4, 2048, 8, 16), (2, 4096, 4, 4), (1, 1 << 16, 2, 2), (8, 512, 1, 16), (3, 256, 16, 1),
    (16, 4, 16, 8), (2, 1, 4, 4), (5, 64, 8, 2), (3, 768, 4, 8), (5, 1 << 16, 2, 16), (2, 4096, 16, 8),
    (256, 1024, 4, 4), (3, 1280, 16, 4), (1, 1 << 20, 8, 4),
]
NARROW_TILES = (0, 1, 2, 3)  # unrolled; one row per thread; tiled, output staged; A tiles staged by TMA


@pytest.mark.parametrize("shape", NARROW_CASES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("scatter", [False, True])
def test_cgemm_narrow_tiles(tnc, shape, scatter):
    """Narrow nodes on every narrow kernel that takes the shape (tile 0
    unrolled, 1 one row per thread, 2 tiled with the output staged in address
    order, 3 A tiles staged in shared memory by TMA: ranges of tiles per CTA
    that cross batches, M not a power of two), identity and shuffled output bit
    orders, element by element against NumPy.  All of them compute per
    component the same FP32 FMAs in the same order, so they agree bit for bit."""
    batch, M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 7 * K + batch)
    A = _crand(batch * M * K, rng)
    B = _crand(batch * K * N, rng)
    ref = _ref(A, B, batch, M, N, K, 0, 1)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c_pos, addr = None, None
    if scatter and not batch & (batch - 1) and not M & (M - 1):
        nN, nM, nB = N.bit_length() - 1, M.bit_length() - 1, batch.bit_length() - 1
        c_pos = rng.permutation(nN + nM + nB)
        b, m, n = np.meshgrid(np.arange(batch), np.arange(M), np.arange(N), indexing="ij")
        addr = np.zeros(b.shape, np.int64)
        for i in range(nN):
            addr |= ((n >> i) & 1) << int(c_pos[i])
        for i in range(nM):
            addr |= ((m >> i) & 1) << int(c_pos[nN + i])
        for i in range(nB):
            addr |= ((b >> i) & 1) << int(c_pos[nN + nM + i])
    elif scatter:
        pytest.skip("scattered output needs power-of-two batch and M")
    outs = {}
    for tile in NARROW_TILES:
        try:
            got = tnc.cgemm(dA, dB, batch, M, N, K, 0, 1, "fp32", kernel="narrow", tile=tile, c_pos=c_pos)
        except tnc.TncError as e:
            assert e.status == tnc.TNC_EINVAL  # the tile does not take this shape
            continue
        got = got.reshape(-1).cpu().numpy()
        got = got[addr] if addr is not None else got.reshape(batch, M, N)
        _assert_close(got, ref, "fp32", f"{shape} tile {tile}")
        outs[tile] = got
    assert 0 in outs and 1 in outs
    if K in (8, 16) and N >= 2 and M % 256 == 0:
        assert 3 in outs, "the TMA-staged kernel takes this shape"
    for tile, got in outs.items():
        assert np.array_equal(got.view(np.uint64), outs[0].view(np.uint64)), f"tile {tile} differs from tile 0 in bits"
