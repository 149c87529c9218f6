// CUDA kernels of the executor (sm_103a), CUDA-core forms:
//   gather   -- derived leaves (bit projection / fixed slice bits);
//   permute  -- tiled bit permutation of a 2^r complex64 tensor through
//               shared memory, coalesced on both the read and the write side;
//   cgemm    -- FP32 complex GEMM on CUDA cores (the reference form), a
//               register-tiled kernel, a one-row-per-thread kernel for narrow
//               N, K and a split-K warp-shuffle reduction for tiny outputs;
//   accum    -- FP64 accumulation of the root into complex128 amplitudes.
// Every pairwise contraction computes C[b][m][n] = sum_k A[b][m][k] B[b][k][n]
// (the node cost 2 M of Eq. 3 with M = batch * M * N * K).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <cstdio>

#include "devonce.cuh"
#include "outmap.cuh"
#include "tnc_kernels.h"

namespace tnc {

namespace {

__device__ __forceinline__ float2 cmul_add(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}

// ------------------------------------------------------------------ counter
__global__ void set_counter_kernel(uint64_t* ctr, uint64_t v) { *ctr = v; }

// ------------------------------------------------------------------ gather
__global__ void gather_kernel(const GatherDesc* __restrict__ descs, const float2* __restrict__ base,
                              float2* __restrict__ ws, const uint8_t* __restrict__ bits, int n_qubits,
                              const uint64_t* __restrict__ ctr) {
  const GatherDesc& g = descs[blockIdx.y];
  const uint64_t n = (uint64_t)1 << g.out_rank;
  const uint64_t slice = *ctr;
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n;
       o += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t src = 0, beta = 0;
    for (int j = 0; j < g.out_rank; ++j) {
      uint64_t bit = (o >> j) & 1;
      int s = g.out_src[j];
      if (s >= 0)
        src |= bit << s;
      else
        beta |= bit << (-1 - s);
    }
    for (int f = 0; f < g.n_fixed; ++f)
      src |= (uint64_t)(bits[beta * n_qubits + g.fixed_qubit[f]] & 1) << g.fixed_pos[f];
    for (int f = 0; f < g.n_sliced; ++f) src |= ((slice >> g.sliced_bit[f]) & 1) << g.sliced_pos[f];
    ws[g.dst + o] = base[g.src + src];
  }
}

// ------------------------------------------------------------------ permute
struct PermArgs {
  uint64_t src, dst;
  int nU, a, b, n_outer;
  int8_t t_in_pos[16];   // t bit i (i >= a) -> input bit position
  int8_t s_t_bit[16];    // s bit i -> t bit
  int8_t s_out_pos[16];  // s bit i (i >= b) -> output bit position
  int8_t outer_in[kMaxRank], outer_out[kMaxRank];
};

constexpr int kPermThreads = 256;

__global__ void __launch_bounds__(kPermThreads) permute_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                             PermArgs p) {
  extern __shared__ float2 tile[];
  uint64_t o = blockIdx.x + (uint64_t)blockIdx.y * gridDim.x;
  uint64_t in_base = 0, out_base = 0;
  for (int k = 0; k < p.n_outer; ++k) {
    uint64_t bit = (o >> k) & 1;
    in_base |= bit << p.outer_in[k];
    out_base |= bit << p.outer_out[k];
  }
  const int nT = 1 << p.nU;
  const uint32_t amask = (1u << p.a) - 1, bmask = (1u << p.b) - 1;
  const int sw = p.a;  // swizzle: low 5 bits of the slot xor the bits above a
  for (int t = threadIdx.x; t < nT; t += blockDim.x) {
    uint64_t off = in_base | (t & amask);
    for (int i = p.a; i < p.nU; ++i) off |= (uint64_t)((t >> i) & 1) << p.t_in_pos[i];
    int slot = t ^ ((t >> sw) & 31);
    tile[slot] = in[p.src + off];
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nT; s += blockDim.x) {
    int t = 0;
    for (int i = 0; i < p.nU; ++i) t |= ((s >> i) & 1) << p.s_t_bit[i];
    uint64_t off = out_base | (s & bmask);
    for (int i = p.b; i < p.nU; ++i) off |= (uint64_t)((s >> i) & 1) << p.s_out_pos[i];
    int slot = t ^ ((t >> sw) & 31);
    out[p.dst + off] = tile[slot];
  }
}

// ------------------------------------------------------------------ SIMT GEMM
// Staged epilogue of a full BM x BN tile whose output is scattered into the
// consumer's layout: the tile's log2(BM) + log2(BN) index bits land on as
// many output bit positions; the tile is written into shared memory at the
// rank of each element's output offset among the tile's (a bit compression)
// and read back in that order, so consecutive threads store consecutive
// output addresses wherever the tile's bits cover the low positions.  The
// ranks are computed on the host (TileRank: m bits first, then n bits); each
// block builds its row, column and offset tables in shared memory once.
struct TileRank {
  int8_t rank[kMaxRank];
};

__device__ __forceinline__ uint32_t tile_swz(uint32_t x) { return x ^ ((x >> 4) & 15u); }

// One BM x BN output tile of batch entry bz (tile index `tile`, m-tiles
// fastest) over the K range of split `split`: the body of the CUDA-core
// cGEMM, shared by the per-node kernel and the grouped kernel.
template <int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void simt_tile(const float2* __restrict__ A, const float2* __restrict__ B,
                                          float2* __restrict__ C, int64_t M, int64_t N, int64_t K, int transA,
                                          int transB, int64_t bz, int64_t tile, int64_t split, int64_t kchunk,
                                          int64_t part_stride, int staged, const OutMap& om, const TileRank& tr) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  // rows padded by 16 bytes: the transposing tile stores spread over banks
  __shared__ __align__(16) float2 As[BK][BM + 2];
  __shared__ __align__(16) float2 Bs[BK][BN + 2];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  A += bz * M * K;
  B += bz * K * N;
  C += split * part_stride;
  const int64_t kbeg = split * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  const int64_t mt = (M + BM - 1) / BM;
  const int64_t m0 = (tile % mt) * BM, n0 = (tile / mt) * BN;
  float2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (!transA) {
        kk = e % BK, mm = e / BK;
      } else {
        mm = e % BM, kk = e / BM;
      }
      int64_t m = m0 + mm, k = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (m < M && k < kend) v = transA ? A[k * M + m] : A[m * K + k];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int e = tid; e < BN * BK; e += NT) {
      int nn, kk;
      if (!transB) {
        nn = e % BN, kk = e / BN;
      } else {
        kk = e % BK, nn = e / BK;
      }
      int64_t n = n0 + nn, k = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (n < N && k < kend) v = transB ? B[n * K + k] : B[k * N + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = cmul_add(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  if (staged) {
    // full tile (M % BM == N % BN == 0), scattered output, no split-K
    constexpr int kMB = __builtin_ctz(BM), kNB = __builtin_ctz(BN), kBits = kMB + kNB;
    extern __shared__ __align__(16) uint8_t simt_dyn[];
    float2* S = (float2*)simt_dyn;                        // [BM * BN]
    uint64_t* hi = (uint64_t*)(S + BM * BN);              // [BM * BN / 32] offsets of staging bits 5..
    uint32_t* rowidx = (uint32_t*)(hi + BM * BN / 32);    // [BM]
    uint32_t* colidx = rowidx + BM;                       // [BN]
    // output bit position of tile bit b
    auto pos_of = [&](int b) -> int { return b < kMB ? om.pos[om.nN + b] : om.pos[b - kMB]; };
    auto offset_of = [&](uint32_t x) -> uint64_t {
      uint64_t o = 0;
#pragma unroll
      for (int b = 0; b < kBits; ++b) o |= (uint64_t)((x >> tr.rank[b]) & 1u) << pos_of(b);
      return o;
    };
    for (int e = tid; e < BM * BN / 32; e += NT) hi[e] = offset_of((uint32_t)e << 5);
    for (int r = tid; r < BM; r += NT) {
      uint32_t x = 0;
#pragma unroll
      for (int b = 0; b < kMB; ++b) x |= (uint32_t)((r >> b) & 1) << tr.rank[b];
      rowidx[r] = x;
    }
    for (int c = tid; c < BN; c += NT) {
      uint32_t x = 0;
#pragma unroll
      for (int b = 0; b < kNB; ++b) x |= (uint32_t)((c >> b) & 1) << tr.rank[kMB + b];
      colidx[c] = x;
    }
    const uint64_t lo = offset_of((uint32_t)(tid & 31));
    __syncthreads();
    uint32_t ci[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) ci[j] = colidx[tx * TN + j];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const uint32_t ri = rowidx[ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) S[tile_swz(ri | ci[j])] = acc[i][j];
    }
    __syncthreads();
    float2* dst = C + om.row(bz, m0, M, N) + om.col(n0) + lo;
#pragma unroll 4
    for (int e = tid; e < BM * BN; e += NT) dst[hi[e >> 5]] = S[tile_swz((uint32_t)e)];
    return;
  }
  uint64_t coff[TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    int64_t n = n0 + tx * TN + j;
    coff[j] = n < N ? om.col(n) : 0;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty * TM + i;
    if (m >= M) continue;
    const uint64_t roff = om.row(bz, m, M, N);
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx * TN + j;
      if (n < N) C[roff + coff[j]] = acc[i][j];
    }
  }
}

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN),
                                  (BM * BN >= 8192) ? 1 : ((BM / TM) * (BN / TN) >= 256 ? 3 : 4))
    cgemm_simt_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
                      int64_t M, int64_t N, int64_t K, int transA, int transB, int64_t b0, int64_t kchunk,
                      int64_t part_stride, int staged, const __grid_constant__ OutMap om,
                      const __grid_constant__ TileRank tr) {
  simt_tile<BM, BN, BK, TM, TN>(A, B, C, M, N, K, transA, transB, b0 + blockIdx.z, blockIdx.x, blockIdx.y, kchunk,
                                part_stride, staged, om, tr);
}

// Many CUDA-core cGEMM problems in one launch (nodes of different requests,
// each with its own operands and output layout): block -> (problem, batch
// entry, tile) by binary search over the problems' first blocks; the
// problem's descriptor is read into shared memory once per block.
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN),
                                  (BM * BN >= 8192) ? 1 : ((BM / TM) * (BN / TN) >= 256 ? 3 : 4))
    grouped_simt_kernel(const SimtProblem* __restrict__ probs, int n) {
  __shared__ SimtProblem p;
  __shared__ OutMap om;
  __shared__ TileRank tr;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    const int64_t blk = blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].first_block <= blk)
        lo = mid;
      else
        hi = mid - 1;
    }
    p = probs[lo];
    om.ident = p.ident, om.nN = p.nN, om.nM = p.nM, om.nB = p.nB;
    for (int i = 0; i < kMaxRank; ++i) om.pos[i] = p.c_pos[i], tr.rank[i] = p.rank[i];
  }
  __syncthreads();
  const int64_t local = (int64_t)blockIdx.x - p.first_block;
  const int64_t tiles = ((p.M + BM - 1) / BM) * ((p.N + BN - 1) / BN);
  simt_tile<BM, BN, BK, TM, TN>((const float2*)p.A, (const float2*)p.B, (float2*)p.C, p.M, p.N, p.K, p.transA,
                                p.transB, local / tiles, local % tiles, 0, p.K, 0, p.staged, om, tr);
}

// ------------------------------------------------------------------ narrow
// one output row per thread; N, K <= 16; B of the batch in shared memory
__global__ void __launch_bounds__(256)
    cgemm_narrow_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
                        int64_t M, int N, int K, int transA, int transB, int64_t b0,
                        const __grid_constant__ OutMap om) {
  __shared__ float2 Bs[16 * 16];
  __shared__ uint64_t coff[16];
  const int64_t bz = b0 + blockIdx.y;
  A += bz * M * K;
  B += bz * (int64_t)K * N;
  if (threadIdx.x < N) coff[threadIdx.x] = om.col(threadIdx.x);
  for (int e = threadIdx.x; e < K * N; e += blockDim.x) {
    int k = e / N, n = e % N;
    Bs[e] = transB ? B[(int64_t)n * K + k] : B[(int64_t)k * N + n];
  }
  __syncthreads();
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    float2 a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < K) a[k] = transA ? A[(int64_t)k * M + m] : A[m * K + k];
    const uint64_t roff = om.row(bz, m, M, N);
    for (int n = 0; n < N; ++n) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < K) acc = cmul_add(acc, a[k], Bs[k * N + n]);
      C[roff + coff[n]] = acc;
    }
  }
}

// ------------------------------------------------------------------ narrow, unrolled
// The narrow node with K and N known at compile time (powers of two <= 16), A
// K-major: one row per thread, its A row read with 16-byte loads and kept in
// registers as the packed pairs (a.x, a.x), (a.y, a.y) and (-a.y, -a.y); B in
// shared memory with two columns in each 16-byte word as (b0.x, b1.x, b0.y,
// b1.y), so that one broadcast per (k, column pair) feeds both columns and the
// packed FP32 FMAs (__ffma2_rn) take their pairs straight from the loaded
// word: the real parts of the two columns in one register pair, the imaginary
// parts in another.  Per component these are exactly the two FMAs of cmul_add
// in its order.  Fully unrolled over K: no index arithmetic or predicates in
// the inner loop.  (N = 1: one column, the second slot of each pair zero.)
template <int K, int N>
__global__ void __launch_bounds__(256)
    cgemm_narrow_unrolled_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
                                 int64_t M, int64_t b0, const __grid_constant__ OutMap om) {
  constexpr int NP = N >= 2 ? N / 2 : 1;  // column pairs
  __shared__ float4 Bq[K * NP];           // Bq[k][p] = (b[2p][k].x, b[2p+1][k].x, b[2p][k].y, b[2p+1][k].y)
  __shared__ uint64_t coff[N];
  const int64_t bz = b0 + blockIdx.y;
  A += bz * M * K;
  B += bz * (int64_t)K * N;
  for (int e = threadIdx.x; e < K * NP; e += blockDim.x) {
    const int k = e / NP, p = e % NP;
    const float2 x = B[(int64_t)(2 * p) * K + k];  // B stored [N][K]
    const float2 y = N >= 2 ? B[(int64_t)(2 * p + 1) * K + k] : make_float2(0.f, 0.f);
    Bq[e] = make_float4(x.x, y.x, x.y, y.y);
  }
  if (threadIdx.x < N) coff[threadIdx.x] = om.col(threadIdx.x);
  __syncthreads();
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    float2 ax[K], ay[K], an[K];
    if constexpr (K >= 2) {
      const float4* row = (const float4*)(A + m * K);
#pragma unroll
      for (int k = 0; k < K / 2; ++k) {
        const float4 v = row[k];
        ax[2 * k] = make_float2(v.x, v.x);
        ay[2 * k] = make_float2(v.y, v.y);
        an[2 * k] = make_float2(-v.y, -v.y);
        ax[2 * k + 1] = make_float2(v.z, v.z);
        ay[2 * k + 1] = make_float2(v.w, v.w);
        an[2 * k + 1] = make_float2(-v.w, -v.w);
      }
    } else {
      const float2 v = A[m];
      ax[0] = make_float2(v.x, v.x);
      ay[0] = make_float2(v.y, v.y);
      an[0] = make_float2(-v.y, -v.y);
    }
    const uint64_t roff = om.row(bz, m, M, N);
#pragma unroll 1
    for (int p = 0; p < NP; ++p) {
      float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);  // columns 2p, 2p + 1
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float4 b = Bq[k * NP + p];
        const float2 bx = make_float2(b.x, b.y), by = make_float2(b.z, b.w);
        re = __ffma2_rn(ax[k], bx, re);
        re = __ffma2_rn(an[k], by, re);
        im = __ffma2_rn(ax[k], by, im);
        im = __ffma2_rn(ay[k], bx, im);
      }
      C[roff + coff[2 * p]] = make_float2(re.x, im.x);
      if constexpr (N >= 2) C[roff + coff[2 * p + 1]] = make_float2(re.y, im.y);
    }
  }
}

template <int K, int N>
void launch_narrow_unrolled(const float2* A, const float2* B, float2* C, int64_t M, int64_t batch, const OutMap& om,
                            cudaStream_t st) {
  int64_t blocks = (M + 255) / 256;
  if (blocks > (int64_t)sm_count() * 16) blocks = (int64_t)sm_count() * 16;
  for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
    const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
    cgemm_narrow_unrolled_kernel<K, N><<<dim3((unsigned)blocks, (unsigned)nb), 256, 0, st>>>(A, B, C, M, b0, om);
  }
}

template <int K>
bool launch_narrow_unrolled_n(int N, const float2* A, const float2* B, float2* C, int64_t M, int64_t batch,
                              const OutMap& om, cudaStream_t st) {
  switch (N) {
    case 1: launch_narrow_unrolled<K, 1>(A, B, C, M, batch, om, st); return true;
    case 2: launch_narrow_unrolled<K, 2>(A, B, C, M, batch, om, st); return true;
    case 4: launch_narrow_unrolled<K, 4>(A, B, C, M, batch, om, st); return true;
    case 8: launch_narrow_unrolled<K, 8>(A, B, C, M, batch, om, st); return true;
    case 16: launch_narrow_unrolled<K, 16>(A, B, C, M, batch, om, st); return true;
    default: return false;
  }
}

template <int K>
void narrow_unrolled_fns_n(const void** out) {
  out[0] = (const void*)cgemm_narrow_unrolled_kernel<K, 1>;
  out[1] = (const void*)cgemm_narrow_unrolled_kernel<K, 2>;
  out[2] = (const void*)cgemm_narrow_unrolled_kernel<K, 4>;
  out[3] = (const void*)cgemm_narrow_unrolled_kernel<K, 8>;
  out[4] = (const void*)cgemm_narrow_unrolled_kernel<K, 16>;
}

// the 25 instances (for preloading)
void narrow_unrolled_fns(const void** out) {
  narrow_unrolled_fns_n<1>(out);
  narrow_unrolled_fns_n<2>(out + 5);
  narrow_unrolled_fns_n<4>(out + 10);
  narrow_unrolled_fns_n<8>(out + 15);
  narrow_unrolled_fns_n<16>(out + 20);
}

// false if (K, N) has no unrolled instance
bool launch_narrow_unrolled_kn(int K, int N, const float2* A, const float2* B, float2* C, int64_t M, int64_t batch,
                               const OutMap& om, cudaStream_t st) {
  switch (K) {
    case 1: return launch_narrow_unrolled_n<1>(N, A, B, C, M, batch, om, st);
    case 2: return launch_narrow_unrolled_n<2>(N, A, B, C, M, batch, om, st);
    case 4: return launch_narrow_unrolled_n<4>(N, A, B, C, M, batch, om, st);
    case 8: return launch_narrow_unrolled_n<8>(N, A, B, C, M, batch, om, st);
    case 16: return launch_narrow_unrolled_n<16>(N, A, B, C, M, batch, om, st);
    default: return false;
  }
}

// ------------------------------------------------------------------ narrow, tiled
// The narrow node again (N, K <= 16), for powers of two and a K-major A: one
// CTA per tile of R = 2^r rows of one batch entry.  The tile's A rows are one
// contiguous block of R K complex values, loaded with 16-byte coalesced loads
// into shared memory (rows padded by one element, so that threads of a warp
// reading different rows hit different banks).  Thread t takes row t mod R
// and a contiguous share of its N outputs: its A row goes to registers once,
// B is read as broadcasts.  A scattered output tile is staged in shared
// memory in the order of its output addresses (each tile bit at the rank of
// its output position among the tile's; row and column parts from tables)
// and stored by consecutive threads to increasing addresses (offsets from a
// table of the high staging bits plus one of the low five), so every run of
// consecutive output positions that the tile covers is written by
// consecutive threads; an identity layout is stored directly.
constexpr int kNarrowTile = 1024;     // R * N outputs and R * K inputs per CTA at most
constexpr int kNarrowThreads = 256;

__global__ void __launch_bounds__(kNarrowThreads)
    cgemm_narrow_tile_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
                             int64_t M, int N, int K, int r, int nN, int64_t b0,
                             const __grid_constant__ OutMap om, const __grid_constant__ TileRank tr) {
  __shared__ __align__(16) float2 As[kNarrowTile + kNarrowTile / 2];  // R rows of K + 1 (K >= 2), or R (K = 1)
  __shared__ float2 Bs[16 * 16];
  __shared__ float2 S[kNarrowTile];
  __shared__ uint16_t rowx[kNarrowTile], colx[16];
  __shared__ uint64_t hi_off[kNarrowTile / 32], lo_off[32];
  const int R = 1 << r;
  const int64_t bz = b0 + blockIdx.y;
  const int64_t m0 = (int64_t)blockIdx.x << r;
  const float2* Ab = A + (bz * M + m0) * K;
  const float2* Bb = B + bz * (int64_t)K * N;
  for (int e = threadIdx.x; e < K * N; e += blockDim.x) Bs[(e % K) * N + e / K] = Bb[e];  // B stored [N][K]
  const int kp = K >= 2 ? K + 1 : 1;
  if (K >= 2) {
    const float4* A4 = (const float4*)Ab;
    for (int i = threadIdx.x; i < (R * K) >> 1; i += blockDim.x) {
      const float4 v = A4[i];
      const int row = (2 * i) / K, k = (2 * i) % K;
      As[row * kp + k] = make_float2(v.x, v.y);
      As[row * kp + k + 1] = make_float2(v.z, v.w);
    }
  } else {
    for (int i = threadIdx.x; i < R; i += blockDim.x) As[i] = Ab[i];
  }
  const int bits = nN + r, total = R << nN;
  if (!om.ident) {
    // staging index of (m, n) = rowx[m] | colx[n]: tile bit b (n bits, then m
    // bits) at bit rank[b]; output offset of staging index x = hi_off[x >> 5]
    // + lo_off[x & 31] (tile bit b is output bit om.pos[b])
    for (int m = threadIdx.x; m < R; m += blockDim.x) {
      uint32_t x = 0;
      for (int b = 0; b < r; ++b) x |= ((uint32_t)(m >> b) & 1u) << tr.rank[nN + b];
      rowx[m] = (uint16_t)x;
    }
    if (threadIdx.x < N) {
      uint32_t x = 0;
      for (int b = 0; b < nN; ++b) x |= ((uint32_t)(threadIdx.x >> b) & 1u) << tr.rank[b];
      colx[threadIdx.x] = (uint16_t)x;
    }
    auto offset_of = [&](uint32_t x) {
      uint64_t o = 0;
      for (int b = 0; b < bits; ++b) o |= (uint64_t)((x >> tr.rank[b]) & 1u) << om.pos[b];
      return o;
    };
    for (int h = threadIdx.x; h < (total + 31) / 32; h += blockDim.x) hi_off[h] = offset_of((uint32_t)h << 5);
    if (threadIdx.x < 32) lo_off[threadIdx.x] = offset_of(threadIdx.x & (total - 1) & 31);
  }
  __syncthreads();
  // thread -> (row, share of the columns)
  const int per_row = blockDim.x / R > 0 ? blockDim.x / R : 1;  // threads per row
  const int share = (N + per_row - 1) / per_row;
  for (int t = threadIdx.x; t < R * per_row; t += blockDim.x) {
    const int m = t % R, n0 = (t / R) * share;
    if (n0 >= N) continue;
    float2 a[16];
    const float2* ar = As + m * kp;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < K) a[k] = ar[k];
    const int n1 = n0 + share < N ? n0 + share : N;
    for (int n = n0; n < n1; ++n) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < K) acc = cmul_add(acc, a[k], Bs[k * N + n]);
      if (om.ident)
        C[(bz * M + m0 + m) * N + n] = acc;
      else
        S[tile_swz((uint32_t)rowx[m] | colx[n])] = acc;
    }
  }
  if (om.ident) return;
  __syncthreads();
  float2* dst = C + om.row(bz, m0, M, N);
  for (int x = threadIdx.x; x < total; x += blockDim.x) dst[hi_off[x >> 5] + lo_off[x & 31]] = S[tile_swz((uint32_t)x)];
}

// ------------------------------------------------------------------ grouped narrow
// Many independent narrow nodes in one launch: block -> (problem, batch,
// row chunk) by binary search over the problems' first blocks.
constexpr int kGroupThreads = 128;

__global__ void __launch_bounds__(kGroupThreads)
    grouped_narrow_kernel(const GroupedDesc* __restrict__ descs, int n, const float2* __restrict__ base,
                          float2* __restrict__ ws) {
  __shared__ float2 Bs[16 * 16];
  __shared__ uint64_t coff[16];
  int lo = 0, hi = n - 1;
  const int64_t blk = blockIdx.x;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (descs[mid].first_block <= blk)
      lo = mid;
    else
      hi = mid - 1;
  }
  const GroupedDesc& d = descs[lo];
  const int64_t local = blk - d.first_block;
  const int64_t bz = local / d.blocks_per_batch;
  const int64_t chunk = local % d.blocks_per_batch;
  const int N = d.N, K = d.K;
  // a problem of another request carries its own buffers
  const float2* bb = d.base_ptr ? (const float2*)d.base_ptr : base;
  float2* wb = d.ws_ptr ? (float2*)d.ws_ptr : ws;
  const float2* A = (d.a_buf ? bb : wb) + d.a + bz * d.M * K;
  const float2* B = (d.b_buf ? bb : wb) + d.b + bz * (int64_t)K * N;
  float2* C = wb + d.c;
  for (int e = threadIdx.x; e < K * N; e += blockDim.x) {
    int kk = e / N, nn = e % N;
    Bs[e] = B[(int64_t)nn * K + kk];  // B stored [N][K]
  }
  OutMap om;
  om.ident = d.c_ident, om.nN = d.nN, om.nM = d.nM, om.nB = d.nB;
  for (int i = 0; i < kMaxRank; ++i) om.pos[i] = d.c_pos[i];
  if (threadIdx.x < N) coff[threadIdx.x] = om.col(threadIdx.x);
  __syncthreads();
  const int64_t m = chunk * kGroupThreads + threadIdx.x;
  if (m >= d.M) return;
  float2 a[16];
#pragma unroll
  for (int kk = 0; kk < 16; ++kk)
    if (kk < K) a[kk] = A[m * K + kk];
  const uint64_t roff = om.row(bz, m, d.M, N);
  for (int nn = 0; nn < N; ++nn) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
      if (kk < K) acc = cmul_add(acc, a[kk], Bs[kk * N + nn]);
    C[roff + coff[nn]] = acc;
  }
}

// ------------------------------------------------------------------ dot
// split-K for M*N <= 16: FP32 products summed in runs of 32, runs summed in
// FP64; per-block partials reduced by a second pass.
constexpr int kDotThreads = 256;

// VEC: both operands K-major ([m][K], [n][K]), K even, 16-byte aligned: each
// thread takes two consecutive k per 16-byte load of every row.
template <bool VEC>
__global__ void __launch_bounds__(kDotThreads)
    cgemm_dot_kernel(const float2* __restrict__ A, const float2* __restrict__ B, double2* __restrict__ part,
                     int M, int N, int64_t K, int transA, int transB, int64_t b0) {
  const int64_t bz = b0 + blockIdx.y;
  A += bz * (int64_t)M * K;
  B += bz * K * (int64_t)N;
  const int MN = M * N;
  double2 acc64[16];
  float2 acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc64[i] = make_double2(0, 0), acc[i] = make_float2(0.f, 0.f);
  int run = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (VEC) {
    // FP32 over the thread's k (16 products; more only when K exceeds the
    // 1024 blocks of 4096 k), an FP32 tree over the warp's 32 lanes, FP64
    // over the warps and blocks; accumulators indexed statically (registers)
    const float4* A4 = (const float4*)A;
    const float4* B4 = (const float4*)B;
    const int64_t K2 = K >> 1;
    float2 c[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n) c[m][n] = make_float2(0.f, 0.f);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K2; j += stride) {
      float4 a[4], b[4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (m < M) a[m] = A4[(int64_t)m * K2 + j];
#pragma unroll
      for (int n = 0; n < 4; ++n)
        if (n < N) b[n] = B4[(int64_t)n * K2 + j];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n)
          if (m < M && n < N) {
            const float2 t = cmul_add(c[m][n], make_float2(a[m].x, a[m].y), make_float2(b[n].x, b[n].y));
            c[m][n] = cmul_add(t, make_float2(a[m].z, a[m].w), make_float2(b[n].z, b[n].w));
          }
    }
    __shared__ float2 red32[kDotThreads / 32][16];
    const int lane32 = threadIdx.x & 31, wid32 = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        if (m >= M || n >= N) continue;  // uniform over the block
        float x = c[m][n].x, y = c[m][n].y;
        for (int off = 16; off; off >>= 1) {
          x += __shfl_xor_sync(0xffffffffu, x, off);
          y += __shfl_xor_sync(0xffffffffu, y, off);
        }
        if (lane32 == 0) red32[wid32][m * N + n] = make_float2(x, y);
      }
    __syncthreads();
    if (threadIdx.x < MN) {
      double2 sum = make_double2(0, 0);
      for (int w = 0; w < kDotThreads / 32; ++w) sum.x += red32[w][threadIdx.x].x, sum.y += red32[w][threadIdx.x].y;
      part[(bz * gridDim.x + blockIdx.x) * MN + threadIdx.x] = sum;
    }
    return;
  } else
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += stride) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (m >= M) break;
      float2 a = transA ? A[k * M + m] : A[(int64_t)m * K + k];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        if (n >= N || m * N + n >= 16) break;
        float2 b = transB ? B[(int64_t)n * K + k] : B[k * N + n];
        acc[m * N + n] = cmul_add(acc[m * N + n], a, b);
      }
    }
    if (++run == 32) {
      run = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        acc64[i].x += acc[i].x, acc64[i].y += acc[i].y;
        acc[i] = make_float2(0.f, 0.f);
      }
    }
  }
  __shared__ double2 red[kDotThreads / 32][16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (i >= MN) break;  // uniform over the block
    double x = acc64[i].x + acc[i].x, y = acc64[i].y + acc[i].y;
    for (int off = 16; off; off >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, off);
      y += __shfl_xor_sync(0xffffffffu, y, off);
    }
    if (lane == 0) red[wid][i] = make_double2(x, y);
  }
  __syncthreads();
  if (threadIdx.x < MN) {
    double2 s = make_double2(0, 0);
    for (int w = 0; w < kDotThreads / 32; ++w) s.x += red[w][threadIdx.x].x, s.y += red[w][threadIdx.x].y;
    part[(bz * gridDim.x + blockIdx.x) * MN + threadIdx.x] = s;
  }
}

// M = N = 1 (an inner product per batch entry, e.g. the root of a tree):
// 16-byte loads of two complex values from each operand, four independent
// loads in flight per thread, FP32 runs of up to 32 products summed in FP64.
__global__ void __launch_bounds__(kDotThreads)
    cgemm_dot11_kernel(const float4* __restrict__ A, const float4* __restrict__ B, double2* __restrict__ part,
                       int64_t K2, int64_t b0) {
  const int64_t bz = b0 + blockIdx.y;
  A += bz * K2;
  B += bz * K2;
  double2 acc64 = make_double2(0, 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  while (k < K2) {
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < 4 && k < K2; ++r) {
      float4 a[4], b[4];
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t kk = k + u * stride;
        if (kk < K2) {
          a[u] = A[kk];
          b[u] = B[kk];
          cnt = u + 1;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u < cnt) {
          acc = cmul_add(acc, make_float2(a[u].x, a[u].y), make_float2(b[u].x, b[u].y));
          acc = cmul_add(acc, make_float2(a[u].z, a[u].w), make_float2(b[u].z, b[u].w));
        }
      }
      k += 4 * stride;
    }
    acc64.x += acc.x, acc64.y += acc.y;
  }
  __shared__ double2 red[kDotThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double x = acc64.x, y = acc64.y;
  for (int off = 16; off; off >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, off);
    y += __shfl_xor_sync(0xffffffffu, y, off);
  }
  if (lane == 0) red[wid] = make_double2(x, y);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0, 0);
    for (int w = 0; w < kDotThreads / 32; ++w) t.x += red[w].x, t.y += red[w].y;
    part[bz * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void dot_finish_kernel(const double2* __restrict__ part, float2* __restrict__ C, int nblk, int M, int N,
                                  int64_t batch, const __grid_constant__ OutMap om) {
  const int MN = M * N;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= batch * MN) return;
  int64_t bz = i / MN, e = i % MN;
  double x = 0, y = 0;
  for (int b = 0; b < nblk; ++b) {
    double2 v = part[(bz * nblk + b) * MN + e];
    x += v.x, y += v.y;
  }
  C[om.row(bz, e / N, M, N) + om.col(e % N)] = make_float2((float)x, (float)y);
}

// ------------------------------------------------------------------ accum
__global__ void accum_kernel(const float2* __restrict__ root, double2* __restrict__ out, AccumDesc d, int batch) {
  const int64_t nopen = (int64_t)1 << d.n_open;
  const int64_t total = (int64_t)batch * nopen;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t beta = i / nopen, j = i % nopen;
    uint64_t base = 0;
    for (int k = 0; k < d.rank; ++k) {
      if (d.role[k] == 0)
        base |= (uint64_t)((beta >> d.idx[k]) & 1) << k;
      else if (d.role[k] == 1)
        base |= (uint64_t)((j >> d.idx[k]) & 1) << k;
    }
    double x = 0, y = 0;
    const int64_t npar = (int64_t)1 << d.n_par;
    for (int64_t p = 0; p < npar; ++p) {
      uint64_t off = base;
      for (int k = 0; k < d.rank; ++k)
        if (d.role[k] == 2) off |= (uint64_t)((p >> d.idx[k]) & 1) << k;
      float2 v = root[d.src + off];
      x += v.x, y += v.y;
    }
    double2 o = out[i];
    o.x += x, o.y += y;
    out[i] = o;
  }
}

__global__ void splitk_reduce_kernel(const float2* __restrict__ part, float2* __restrict__ C, int splits,
                                     int64_t n, int64_t M, int64_t N,
                                     const __grid_constant__ OutMap om) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = 0, y = 0;
    for (int s = 0; s < splits; ++s) {
      float2 v = part[(int64_t)s * n + i];
      x += v.x, y += v.y;
    }
    const int64_t nn = i % N, bm = i / N;
    C[om.row(bm / M, bm % M, M, N) + om.col(nn)] = make_float2((float)x, (float)y);
  }
}

}  // namespace

void launch_splitk_reduce(const float2* part, float2* C, int splits, int64_t n, int64_t M, int64_t N, const OutMap& om,
                          cudaStream_t st) {
  const int64_t cap = (int64_t)sm_count() * 16;
  const unsigned blocks = (unsigned)((n + 255) / 256 < cap ? (n + 255) / 256 : cap);
  if (blocks) splitk_reduce_kernel<<<blocks, 256, 0, st>>>(part, C, splits, n, M, N, om);
}

namespace {

template <int BM, int BN, int BK, int TM, int TN>
int run_simt(const GemmDesc& d, const float2* A, const float2* B, float2* C, float2* ws, cudaStream_t st) {
  constexpr int NT = (BM / TM) * (BN / TN);
  const int64_t mt = (d.M + BM - 1) / BM, nt = (d.N + BN - 1) / BN;
  if (mt * nt > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  const int splits = d.splitk > 1 ? d.splitk : 1;
  const int64_t nout = d.batch * d.M * d.N;
  float2* dst = C;
  if (splits > 1) {
    if ((uint64_t)splits * nout > d.scratch_elems) return (int)cudaErrorInvalidValue;
    dst = ws;
  }
  const int64_t kchunk = (d.K + splits - 1) / splits;
  const OutMap om = out_map(d);
  OutMap ident = om;
  ident.ident = 1;
  // staged epilogue for full tiles of a scattered output
  const int staged = (splits == 1 && !d.c_ident && d.M % BM == 0 && d.N % BN == 0) ? 1 : 0;
  const size_t dyn = staged ? (size_t)BM * BN * 8 + (size_t)BM * BN / 32 * 8 + (size_t)(BM + BN) * 4 : 0;
  TileRank tr;
  std::memset(&tr, 0, sizeof(tr));
  if (staged) {
    // rank of each tile bit's output position among the tile's positions
    constexpr int kMB = __builtin_ctz(BM), kNB = __builtin_ctz(BN);
    int pos[kMaxRank];
    for (int b = 0; b < kMB; ++b) pos[b] = d.c_pos[d.nN + b];
    for (int b = 0; b < kNB; ++b) pos[kMB + b] = d.c_pos[b];
    for (int b = 0; b < kMB + kNB; ++b) {
      int r = 0;
      for (int k = 0; k < kMB + kNB; ++k) r += pos[k] < pos[b];
      tr.rank[b] = (int8_t)r;
    }
  }
  static std::atomic<int> attr_done[kMaxDevices];
  if (staged) {
    int e = smem_attr_once(attr_done, cgemm_simt_kernel<BM, BN, BK, TM, TN>, (int)dyn);
    if (e) return e;
  }
  for (int64_t b0 = 0; b0 < d.batch; b0 += 65535) {
    int64_t nb = d.batch - b0 < 65535 ? d.batch - b0 : 65535;
    dim3 grid((unsigned)(mt * nt), (unsigned)splits, (unsigned)nb);
    cgemm_simt_kernel<BM, BN, BK, TM, TN><<<grid, NT, dyn, st>>>(A, B, dst, d.M, d.N, d.K, d.transA, d.transB,
                                                                  b0, kchunk, nout, staged, splits > 1 ? ident : om,
                                                                  tr);
  }
  if (splits > 1) {
    const int64_t cap = (int64_t)sm_count() * 16;
    unsigned blocks = (unsigned)((nout + 255) / 256 < cap ? (nout + 255) / 256 : cap);
    splitk_reduce_kernel<<<blocks, 256, 0, st>>>(dst, C, splits, nout, d.M, d.N, om);
  }
  return (int)cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- launchers
// SM count of the current device, cached per device (152 without one)
int sm_count() {
  static std::atomic<int> n[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;  // no device: a GB300's count
  }
  if (dev < 0 || dev >= kMaxDevices) return 152;
  int v = n[dev].load(std::memory_order_acquire);
  if (!v) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    n[dev].store(v, std::memory_order_release);
  }
  return v;
}

int launch_set_counter(uint64_t* d_ctr, uint64_t value, void* stream) {
  set_counter_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_ctr, value);
  return (int)cudaGetLastError();
}

int launch_zero(void* ptr, size_t bytes, void* stream) {
  return (int)cudaMemsetAsync(ptr, 0, bytes, (cudaStream_t)stream);
}

int launch_gather(const GatherDesc* d_descs, int n_descs, int max_out_rank, const void* base, void* ws,
                  const uint8_t* d_bits, int n_qubits, const uint64_t* d_slice_ctr, void* stream) {
  if (n_descs <= 0) return 0;
  if (n_descs > 65535) return (int)cudaErrorInvalidConfiguration;
  uint64_t n = (uint64_t)1 << max_out_rank;
  unsigned gx = (unsigned)((n + 255) / 256);
  if (gx > 4096) gx = 4096;
  dim3 grid(gx, (unsigned)n_descs);
  gather_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_descs, (const float2*)base, (float2*)ws, d_bits,
                                                         n_qubits, d_slice_ctr);
  return (int)cudaGetLastError();
}

int launch_permute(const PermDesc& d, void* ws, void* stream) {
  return launch_permute_ptr(d, (const float2*)ws + d.src, (float2*)ws + d.dst, stream);
}

int launch_permute_ptr(const PermDesc& d, const void* in, void* out, void* stream) {
  const int r = d.rank;
  PermArgs p;
  memset(&p, 0, sizeof(p));
  p.src = 0;
  p.dst = 0;
  int dst_of[kMaxRank];
  for (int j = 0; j < r; ++j) dst_of[(int)d.src_bit[j]] = j;
  int a = r < 5 ? r : 5, b = r < 5 ? r : 5;
  bool inU[kMaxRank];
  auto build_u = [&]() {
    int cnt = 0;
    for (int i = 0; i < r; ++i) inU[i] = false;
    for (int i = 0; i < a; ++i) inU[i] = true;
    for (int j = 0; j < b; ++j) inU[(int)d.src_bit[j]] = true;
    for (int i = 0; i < r; ++i) cnt += inU[i];
    return cnt;
  };
  int nU = build_u();
  while (nU < 10 && a < r) {
    ++a;
    nU = build_u();
  }
  if (nU > 12) return (int)cudaErrorInvalidValue;
  // t bits: 0..a-1 = input bits 0..a-1, then the extra input bits ascending
  int tpos_of_in[kMaxRank];
  for (int i = 0; i < r; ++i) tpos_of_in[i] = -1;
  for (int i = 0; i < a; ++i) tpos_of_in[i] = i, p.t_in_pos[i] = (int8_t)i;
  int t = a;
  for (int i = a; i < r; ++i)
    if (inU[i]) tpos_of_in[i] = t, p.t_in_pos[t] = (int8_t)i, ++t;
  // s bits: 0..b-1 = output bits 0..b-1, then the other tile bits
  int s = 0;
  for (int j = 0; j < b; ++j) p.s_t_bit[s] = (int8_t)tpos_of_in[(int)d.src_bit[j]], p.s_out_pos[s] = (int8_t)j, ++s;
  for (int i = 0; i < r; ++i)
    if (inU[i] && dst_of[i] >= b) p.s_t_bit[s] = (int8_t)tpos_of_in[i], p.s_out_pos[s] = (int8_t)dst_of[i], ++s;
  int k = 0;
  for (int i = 0; i < r; ++i)
    if (!inU[i]) p.outer_in[k] = (int8_t)i, p.outer_out[k] = (int8_t)dst_of[i], ++k;
  p.nU = nU;
  p.a = a;
  p.b = b;
  p.n_outer = k;
  uint64_t nblocks = (uint64_t)1 << k;
  unsigned gx = nblocks > 65536 ? 65536 : (unsigned)nblocks;
  unsigned gy = (unsigned)(nblocks / gx);
  dim3 grid(gx, gy);
  size_t smem = ((size_t)1 << nU) * sizeof(float2);
  permute_kernel<<<grid, kPermThreads, smem, (cudaStream_t)stream>>>((const float2*)in, (float2*)out, p);
  return (int)cudaGetLastError();
}

int launch_tc_gemm(const GemmDesc& d, const float2* A, const float2* B, float2* C, void* scratch, cudaStream_t st);
int launch_narrow_tma(const GemmDesc& d, const float2* A, const float2* B, float2* C, cudaStream_t st);

int launch_gemm(const GemmDesc& d, const void* base, void* ws, void* stream) {
  const float2* A = (const float2*)(d.a_buf ? base : ws) + d.a;
  const float2* B = (const float2*)(d.b_buf ? base : ws) + d.b;
  float2* C = (float2*)ws + d.c;
  return launch_gemm_ptr(d, A, B, C, d.scratch_elems ? (float2*)ws + d.scratch : nullptr, stream);
}

int launch_gemm_ptr(const GemmDesc& d, const void* Ap, const void* Bp, void* Cp, void* scratch, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const float2* A = (const float2*)Ap;
  const float2* B = (const float2*)Bp;
  float2* C = (float2*)Cp;
  float2* ws = (float2*)scratch;  // per-node scratch (d.scratch_elems complex64 slots)
  switch (d.kernel) {
    case KG_SIMT_128x64:
      return run_simt<128, 64, 8, 8, 4>(d, A, B, C, (float2*)ws, st);
    case KG_SIMT_64x32:
      return run_simt<64, 32, 8, 4, 4>(d, A, B, C, (float2*)ws, st);
    case KG_SIMT_32x128:
      return run_simt<32, 128, 8, 4, 4>(d, A, B, C, (float2*)ws, st);
    case KG_NARROW: {
      if (d.N > 16 || d.K > 16) return (int)cudaErrorInvalidValue;
      auto lg = [](int64_t v) { int r = 0; while (((int64_t)1 << r) < v) ++r; return ((int64_t)1 << r) == v ? r : -1; };
      const int lM = lg(d.M), lN = lg(d.N), lK = lg(d.K);
      const bool kmajor = !d.transA && d.transB && ((uintptr_t)A & 15) == 0;
      if (d.tile == 3) {
        const int r = launch_narrow_tma(d, A, B, C, st);
        if (r >= 0) return r;  // else (shape not eligible) as tile 0
      }
      if ((d.tile == 0 || d.tile == 3) && kmajor && lN >= 0 && lK >= 0 &&
          launch_narrow_unrolled_kn((int)d.K, (int)d.N, A, B, C, d.M, d.batch, out_map(d), st))
        return (int)cudaGetLastError();
      if (d.tile == 2 && lM >= 0 && lN >= 0 && lK >= 0 && kmajor && (d.c_ident || (d.nN == lN && d.nM == lM))) {
        // R rows: R * max(K, N) <= kNarrowTile, R <= M
        int r = 0;
        const int wide = lK > lN ? lK : lN;
        while (r < lM && ((1 << (r + 1)) << wide) <= kNarrowTile) ++r;
        TileRank tr;
        std::memset(&tr, 0, sizeof(tr));
        if (!d.c_ident)
          for (int b = 0; b < lN + r; ++b) {
            int rk = 0;
            for (int q = 0; q < lN + r; ++q) rk += d.c_pos[q] < d.c_pos[b];
            tr.rank[b] = (int8_t)rk;
          }
        const OutMap om = out_map(d);
        for (int64_t b0 = 0; b0 < d.batch; b0 += 65535) {
          int64_t nb = d.batch - b0 < 65535 ? d.batch - b0 : 65535;
          dim3 grid((unsigned)(d.M >> r), (unsigned)nb);
          cgemm_narrow_tile_kernel<<<grid, kNarrowThreads, 0, st>>>(A, B, C, d.M, (int)d.N, (int)d.K, r, lN, b0, om,
                                                                   tr);
        }
        return (int)cudaGetLastError();
      }
      int64_t blocks = (d.M + 255) / 256;
      if (blocks > (int64_t)sm_count() * 16) blocks = (int64_t)sm_count() * 16;
      for (int64_t b0 = 0; b0 < d.batch; b0 += 65535) {
        int64_t nb = d.batch - b0 < 65535 ? d.batch - b0 : 65535;
        dim3 grid((unsigned)blocks, (unsigned)nb);
        cgemm_narrow_kernel<<<grid, 256, 0, st>>>(A, B, C, d.M, (int)d.N, (int)d.K, d.transA, d.transB, b0,
                                                   out_map(d));
      }
      return (int)cudaGetLastError();
    }
    case KG_DOT: {
      if (d.M * d.N > 16 || d.M > 4 || d.N > 4) return run_simt<64, 32, 8, 4, 4>(d, A, B, C, (float2*)ws, st);
      double2* part = (double2*)ws;
      const int MN = (int)(d.M * d.N);
      const bool vec = MN > 1 && !d.transA && d.transB && d.K % 2 == 0 && ((uintptr_t)A & 15) == 0 &&
                       ((uintptr_t)B & 15) == 0;
      // vectorised: 16 k per thread (FP32), else about 32 (FP32 runs of 32 summed in FP64)
      const int64_t per_blk = vec ? kDotThreads * 16 : kDotThreads * 32;
      int64_t nblk = (d.K + per_blk - 1) / per_blk;
      if (nblk > 1024) nblk = 1024;
      if (nblk < 1) nblk = 1;
      if ((uint64_t)d.batch * nblk * MN * 2 > d.scratch_elems) return (int)cudaErrorInvalidValue;
      const bool vec11 = MN == 1 && d.K % 2 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0;
      for (int64_t b0 = 0; b0 < d.batch && vec11; b0 += 65535) {
        int64_t nb = d.batch - b0 < 65535 ? d.batch - b0 : 65535;
        dim3 grid((unsigned)nblk, (unsigned)nb);
        cgemm_dot11_kernel<<<grid, kDotThreads, 0, st>>>((const float4*)A, (const float4*)B, part, d.K / 2, b0);
      }
      for (int64_t b0 = 0; b0 < d.batch && !vec11; b0 += 65535) {
        int64_t nb = d.batch - b0 < 65535 ? d.batch - b0 : 65535;
        dim3 grid((unsigned)nblk, (unsigned)nb);
        if (vec)
          cgemm_dot_kernel<true><<<grid, kDotThreads, 0, st>>>(A, B, part, (int)d.M, (int)d.N, d.K, d.transA,
                                                                d.transB, b0);
        else
          cgemm_dot_kernel<false><<<grid, kDotThreads, 0, st>>>(A, B, part, (int)d.M, (int)d.N, d.K, d.transA,
                                                                 d.transB, b0);
      }
      int64_t tot = d.batch * MN;
      dot_finish_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, C, (int)nblk, (int)d.M, (int)d.N,
                                                                          d.batch, out_map(d));
      return (int)cudaGetLastError();
    }
    case KG_TC:
      return launch_tc_gemm(d, A, B, C, scratch, st);
    default:
      return (int)cudaErrorInvalidValue;
  }
}

int launch_grouped_narrow(const GroupedDesc* d_descs, int n, int64_t total_blocks, const void* base, void* ws,
                          void* stream) {
  if (n <= 0 || total_blocks <= 0) return 0;
  if (total_blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  grouped_narrow_kernel<<<(unsigned)total_blocks, kGroupThreads, 0, (cudaStream_t)stream>>>(
      d_descs, n, (const float2*)base, (float2*)ws);
  return (int)cudaGetLastError();
}

// tile shapes of the CUDA-core cGEMM by kernel variant
template <int V>
struct SimtShape;
template <>
struct SimtShape<KG_SIMT_128x64> {
  static constexpr int BM = 128, BN = 64, BK = 8, TM = 8, TN = 4;
};
template <>
struct SimtShape<KG_SIMT_64x32> {
  static constexpr int BM = 64, BN = 32, BK = 8, TM = 4, TN = 4;
};
template <>
struct SimtShape<KG_SIMT_32x128> {
  static constexpr int BM = 32, BN = 128, BK = 8, TM = 4, TN = 4;
};

template <int V>
int launch_grouped_simt_v(const SimtProblem* d_probs, int n, int64_t total_blocks, cudaStream_t st) {
  using S = SimtShape<V>;
  constexpr int NT = (S::BM / S::TM) * (S::BN / S::TN);
  const size_t dyn = (size_t)S::BM * S::BN * 8 + (size_t)S::BM * S::BN / 32 * 8 + (size_t)(S::BM + S::BN) * 4;
  static std::atomic<int> attr_done[kMaxDevices];
  if (int e = smem_attr_once(attr_done, grouped_simt_kernel<S::BM, S::BN, S::BK, S::TM, S::TN>, (int)dyn)) return e;
  grouped_simt_kernel<S::BM, S::BN, S::BK, S::TM, S::TN><<<(unsigned)total_blocks, NT, dyn, st>>>(d_probs, n);
  return (int)cudaGetLastError();
}

int simt_tile_shape(int kernel, int* bm, int* bn) {
  switch (kernel) {
    case KG_SIMT_128x64: *bm = 128, *bn = 64; return 0;
    case KG_SIMT_64x32: *bm = 64, *bn = 32; return 0;
    case KG_SIMT_32x128: *bm = 32, *bn = 128; return 0;
    default: return -1;
  }
}

int launch_grouped_simt(const SimtProblem* d_probs, int n, int64_t total_blocks, int kernel, void* stream) {
  if (n <= 0 || total_blocks <= 0) return 0;
  if (total_blocks > 0x7fffffff) return (int)cudaErrorInvalidConfiguration;
  cudaStream_t st = (cudaStream_t)stream;
  switch (kernel) {
    case KG_SIMT_128x64: return launch_grouped_simt_v<KG_SIMT_128x64>(d_probs, n, total_blocks, st);
    case KG_SIMT_64x32: return launch_grouped_simt_v<KG_SIMT_64x32>(d_probs, n, total_blocks, st);
    case KG_SIMT_32x128: return launch_grouped_simt_v<KG_SIMT_32x128>(d_probs, n, total_blocks, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_accum(const AccumDesc& d, const void* ws, void* d_out, int batch, void* stream) {
  int64_t total = (int64_t)batch << d.n_open;
  unsigned blocks = (unsigned)((total + 255) / 256);
  if (blocks > 65535) blocks = 65535;
  accum_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const float2*)ws, (double2*)d_out, d, batch);
  return (int)cudaGetLastError();
}

// Loads every kernel of this file onto the current device.  With lazy module
// loading (the CUDA default) a kernel is otherwise loaded, and device memory
// taken for its code and the module's data, at its first launch.
int preload_kernels_core() {
  const void* fns[] = {
      (const void*)set_counter_kernel,
      (const void*)gather_kernel,
      (const void*)permute_kernel,
      (const void*)cgemm_simt_kernel<128, 64, 8, 8, 4>,
      (const void*)cgemm_simt_kernel<64, 32, 8, 4, 4>,
      (const void*)cgemm_simt_kernel<32, 128, 8, 4, 4>,
      (const void*)cgemm_narrow_kernel,
      (const void*)cgemm_narrow_tile_kernel,
      (const void*)grouped_narrow_kernel,
      (const void*)cgemm_dot_kernel<false>,
      (const void*)cgemm_dot_kernel<true>,
      (const void*)cgemm_dot11_kernel,
      (const void*)dot_finish_kernel,
      (const void*)accum_kernel,
      (const void*)splitk_reduce_kernel,
      (const void*)grouped_simt_kernel<128, 64, 8, 8, 4>,
      (const void*)grouped_simt_kernel<64, 32, 8, 4, 4>,
      (const void*)grouped_simt_kernel<32, 128, 8, 4, 4>,
  };
  cudaFuncAttributes fa;
  for (const void* f : fns) {
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return (int)e;
  }
  const void* unrolled[25];
  narrow_unrolled_fns(unrolled);
  for (const void* f : unrolled) {
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

}  // namespace tnc
