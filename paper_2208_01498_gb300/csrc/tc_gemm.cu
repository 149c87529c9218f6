// Tensor-core complex GEMM on sm_103a (tcgen05 + TMEM + TMA) for the 3xTF32
// and split-BF16 forms of a pairwise contraction C[b] = A[b] B[b] (Eq. 3).
//
// Complex products become one real GEMM (the "4M" form):
//     [Ar | Ai] (M x 2K, interleaved along k)  x  B' (2K x 2N)  =  [Cr | Ci]
// with B'[2k][2n] = Br, B'[2k+1][2n] = -Bi, B'[2k][2n+1] = Bi,
// B'[2k+1][2n+1] = Br, so the real output (M x 2N, interleaved) is the complex
// C itself.  Each real operand x is split into x_hi + x_lo (x_hi = x rounded to
// bf16 or tf32, x_lo = x - x_hi rounded again) and the product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in tensor memory.
//
// prep kernels write the hi/lo planes K-major into the node's workspace
// scratch: A' as [b][M][2K], B'^T as [b][2N][2K].  The GEMM kernel computes one
// 128 x BN output tile per CTA: warp 0 issues TMA loads (128B-swizzled boxes
// of 128-byte rows) into a STAGES-deep shared-memory ring guarded by
// mbarriers, warp 1 (one lane) issues tcgen05.mma into one of two 128 x BN FP32
// accumulators in TMEM (alternating every 512 k' for bf16, 32 k' for tf32),
// and warps 2..5 add each finished accumulator into FP32 registers with
// tcgen05.ld, then store C.
// Every wait is bounded by a time limit; a timeout sets tc_error_flag and the
// CTA skips to teardown (waiting, bounded, for its own TMA copies and MMAs,
// then freeing its TMEM).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/tnc.h"
#include "devonce.cuh"
#include "outmap.cuh"
#include "tnc_kernels.h"

namespace tnc {

__device__ int tc_error_flag = 0;

// sum of FP32 split-K partials [splits][n] (FP64 sums) into C in the
// consumer's layout (kernels.cu)
void launch_splitk_reduce(const float2* part, float2* C, int splits, int64_t n, int64_t M, int64_t N, const OutMap& om,
                          cudaStream_t st);

namespace {

constexpr int BM = 128;
constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on a phase of an mbarrier: false after limit_ns
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

// The kernels' bounded wait on an mbarrier that nothing arrives at: result
// 1 when the wait gave up after limit_ns (the expected outcome), 0 if the
// phase completed.  One thread; no other state is touched.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int* result) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  *result = mbar_wait(&bar, 0, limit_ns) ? 0 : 1;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

template <bool kTF32>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (kTF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout a 128B-swizzled TMA box of 128-byte rows
// leaves in shared memory)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// the same for 64-byte rows with 64-byte swizzle (8-row groups 512 bytes
// apart; 16-byte chunk c of row r at r * 64 + ((c ^ ((r / 2) % 4)) * 16))
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // 64-byte swizzle
  return d;
}

// instruction descriptor: D FP32, A/B BF16 (format 1) or TF32 (format 2),
// both K-major, M = 128, N = BN
template <bool kTF32, int BN>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | ((kTF32 ? 2u : 1u) << 7) | ((kTF32 ? 2u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive TMEM columns of this thread's lane, loaded and waited for
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "{\n\ttcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t}"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ GEMM kernel
// D[b][m][n'] = sum_k' A'[b][m][k'] B'^T[b][n'][k'], 3 products per k-step.
// Warp 0: TMA producer; warp 1: MMA issuer; the remaining warps: accumulation
// and epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31; with BN = 256 two
// warps share each lane quarter, one per half of the columns, so that a
// thread keeps at most 128 FP32 partial sums in registers).  The K range is cut
// into chunks of CHUNK k-blocks; chunk c accumulates in TMEM slot c % 2 and
// the epilogue warps add each finished slot into FP32 registers while the
// other slot fills, so no tensor-core accumulation chain is longer than one
// chunk.
template <int BN>
struct TcShape {
  static constexpr int kEpiCols = BN > 128 ? 128 : BN;      // columns per accumulation thread
  static constexpr int kEpiWarps = 4 * BN / kEpiCols;        // 4 or 8
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
};

template <bool kTF32, int BN, int STAGES>
__global__ void __launch_bounds__(TcShape<BN>::kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
                   const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
                   float* __restrict__ C, int M, int N2, int K2, int b0, const __grid_constant__ OutMap om,
                   int ksplit, int64_t c_split) {
  constexpr int ES = kTF32 ? 4 : 2;
  constexpr int BK = 128 / ES;            // elements per 128-byte row
  constexpr int KSTEP = kTF32 ? 8 : 16;   // K of one MMA instruction
  // k-blocks per accumulation chunk: 512 k' for bf16; 32 k' (one k-block)
  // for tf32, whose three-product error budget leaves less room for the
  // tensor core's accumulation (on a 36-qubit depth-16 circuit: relative
  // error 1.4e-5 with 128 k' chunks, 9.7e-6 with 64, 5.2e-6 with 32)
  constexpr int CHUNK = (kTF32 ? 32 : 512) / BK;
  constexpr uint32_t A_BYTES = BM * 128, B_BYTES = BN * 128;
  constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t IDESC = instr_desc<kTF32, BN>();

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  uint64_t* coltab = (uint64_t*)(tmem_slot + 4);  // [BN/2] column offsets of this tile (8-aligned)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = M / BM;
  const int m0 = (blockIdx.x % tiles_m) * BM;
  const int n0 = (blockIdx.x / tiles_m) * BN;
  const int bz = b0 + blockIdx.z;
  // K split over gridDim.y (ksplit > 1): this CTA's k-blocks [kb0, kb0 + nk),
  // its FP32 partial tile written (plain layout) at C + blockIdx.y * c_split
  const int nk_all = K2 / BK;
  const int per = (nk_all + ksplit - 1) / ksplit;
  const int kb0 = (int)blockIdx.y * per;
  const int nk = kb0 >= nk_all ? 0 : (nk_all - kb0 < per ? nk_all - kb0 : per);
  const int nchunks = (nk + CHUNK - 1) / CHUNK;
  C += (int64_t)blockIdx.y * c_split;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], 32 * TcShape<BN>::kEpiWarps);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // producer: k-blocks whose loads were issued
  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) + 1) & 1)) {
          atomicExch(&tc_error_flag, 1);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        const int kx = (kb0 + kb) * BK;
        tma_load_3d(st, &mA_hi, &full[s], kx, m0, bz);
        tma_load_3d(st + A_BYTES, &mA_lo, &full[s], kx, m0, bz);
        tma_load_3d(st + 2 * A_BYTES, &mB_hi, &full[s], kx, n0, bz);
        tma_load_3d(st + 2 * A_BYTES + B_BYTES, &mB_lo, &full[s], kx, n0, bz);
        issued = kb + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int slot = c & 1;
        if (c >= 2 && !mbar_wait(&acc_empty[slot], ((c >> 1) + 1) & 1)) {
          atomicExch(&tc_error_flag, 4);
          *(volatile int*)abort_flag = 1;
          break;
        }
        const uint32_t dtm = tmem + slot * BN;
        const int kb_end = (c + 1) * CHUNK < nk ? (c + 1) * CHUNK : nk;
        for (int kb = c * CHUNK; kb < kb_end; ++kb) {
          const int s = kb % STAGES;
          if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
            atomicExch(&tc_error_flag, 2);
            *(volatile int*)abort_flag = 1;
            ok = false;
            break;
          }
          if (*(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t dAh = sw128_desc(sa), dAl = sw128_desc(sa + A_BYTES);
          const uint64_t dBh = sw128_desc(sa + 2 * A_BYTES), dBl = sw128_desc(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / KSTEP; ++kk) {
            const uint64_t adv = (uint64_t)((kk * KSTEP * ES) >> 4);
            const uint32_t first = (kb == c * CHUNK && kk == 0) ? 0u : 1u;
            mma<kTF32>(dtm, dAh + adv, dBh + adv, IDESC, first);
            mma<kTF32>(dtm, dAh + adv, dBl + adv, IDESC, 1u);
            mma<kTF32>(dtm, dAl + adv, dBh + adv, IDESC, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[slot]);
      }
      // completion of every MMA issued so far
      mma_commit(done);
    }
  } else {
    // accumulation warps: row 32 (warp % 4) + lane of the tile, columns
    // [half * EC, half * EC + EC)
    constexpr int EC = TcShape<BN>::kEpiCols;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;
    if (!om.ident && et < BN / 2) coltab[et] = om.col(n0 / 2 + et);
    asm volatile("bar.sync 1, %0;" ::"n"(32 * TcShape<BN>::kEpiWarps) : "memory");  // accumulation warps only
    float acc[EC];
#pragma unroll
    for (int i = 0; i < EC; ++i) acc[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int slot = c & 1;
      if (!mbar_wait(&acc_full[slot], (c >> 1) & 1)) {
        atomicExch(&tc_error_flag, 3);
        *(volatile int*)abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + slot * BN + half * EC;
#pragma unroll
      for (int col = 0; col < EC; col += 16) {
        float v[16];
        tmem_ld16(taddr + col, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[col + i] += v[i];
      }
      tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[slot])) : "memory");
    }
    if (ok && !*(volatile int*)abort_flag) {
      const int row = m0 + quarter * 32 + lane;
      if (om.ident) {
        float4* dst = (float4*)(C + ((int64_t)bz * M + row) * N2 + n0 + half * EC);
#pragma unroll
        for (int i = 0; i < EC / 4; ++i)
          dst[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
      } else {
        // complex column n0/2 + i of row `row`, placed in the consumer's layout
        float2* C2 = (float2*)C;
        const uint64_t roff = om.row(bz, row, M, N2 / 2);
        const uint64_t* ct = coltab + half * (EC / 2);
#pragma unroll
        for (int i = 0; i < EC / 2; ++i) C2[roff + ct[i]] = make_float2(acc[2 * i], acc[2 * i + 1]);
      }
    }
  }
  // all MMAs retired before TMEM is freed
  if (threadIdx.x == 0 && !mbar_wait(done, 0)) atomicExch(&tc_error_flag, 5);
  tc_fence_before();
  __syncthreads();
  // teardown after an abort: wait (bounded) for TMA copies still in flight
  if (warp == 0 && lane == 0 && *(volatile int*)abort_flag) {
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// ------------------------------------------------------------ fused split-BF16 kernel
// The same 4M product, but without hi/lo planes in global memory: converter
// warps read the complex64 operands (A [b][M][K], B [b][N][K]) straight from
// global memory, split each value into bf16 hi + lo in registers and store
// the A' and B'^T tiles into shared memory in the swizzled layout the MMA
// descriptors read (128-byte rows: 16-byte chunk c of tile row r at
// r * 128 + ((c ^ (r % 8)) * 16) within each 1024-byte group of 8 rows;
// 64-byte rows: at r * 64 + ((c ^ ((r / 2) % 4)) * 16)).
// Each operand byte then crosses HBM once instead of three times (read,
// planes written, planes read back).
//
// Warps 0..E-1: accumulation and epilogue (TMEM lane quarter = warp % 4;
// E = 4, or 8 with two warps per quarter, half of the columns each, for the
// epilogue-bound 256-column and plane-fed tiles); warp E: TMEM allocation and
// the MMA issuer (one lane); warps E+1 and up: converters (12 for BN = 128
// real output columns per CTA, 10 for BN = 64, 8 for BN = 256, whose 64-byte
// rows halve the converter work per k-block; 16 with one task each in the
// hybrid tile, whose converters handle A only) or the TMA producer.
// Finished accumulation chunks are added into a third TMEM region (the
// running sum) instead of registers, so no thread holds a whole row.  The
// register file is split between the SM's four sub-partitions (16K 32-bit
// registers each); the 17-warp blocks (BN = 128, 256) put 5 warps on one of
// them, which caps a thread at 96 registers (the 15-warp BN = 64 block: 128),
// and the converters are sized to fit that (one k-block of loads in
// registers; the PREFETCH variant also sends the k-block after next towards
// L2).  Two stages keep the block's shared memory under 196 KB: the SM's
// unified L1/shared storage then leaves about 90 KB of L1
// for the converters' loads in flight (with three stages the carve-out rose
// to 228 KB, L1 fell to 28 KB and the kernel ran 10-25 % slower).
// The epilogue re-orders each warp's 32 x 8 complex block through shared
// memory into output order (BlockOrder) before storing.
// Every wait is bounded as in tc_gemm_kernel; no asynchronous copies are in
// flight at teardown (the converters' stores are synchronous).
constexpr int kFzStages = 2;

// BN real output columns per CTA (BN / 2 complex): 64 or 128 with 128-byte
// rows (64 k' per k-block) and a TMEM running sum; 256 with 64-byte rows
// (32 k' per k-block, 64-byte swizzle), for K <= 256 only: one accumulation
// chunk per tile, so two 256-column slots fill TMEM without a running sum.
template <int BN>
struct FzCfg {
  static constexpr int kBN = BN;
  static constexpr bool kPlanes = false;
  static constexpr bool kHybrid = false;
  static constexpr bool kF32 = false;  // operands loaded by the converters themselves
  static constexpr int kSlots = 2;  // TMEM accumulator slots (alternating chunks / tiles)
  static constexpr int kRowBytes = BN == 256 ? 64 : 128;
  static constexpr int kChunks = kRowBytes / 16;              // 16-byte chunks per row
  static constexpr int kKC = kRowBytes / 4;                   // complex k per k-block
  static constexpr int kKSteps = kRowBytes / 32;              // MMAs of K = 16 per k-block
  static constexpr int kChunkKB = 512 / (kRowBytes / 2);      // k-blocks per 512 k' accumulation chunk
  static constexpr int kATasks = 128 * kChunks;
  static constexpr int kTasks = kATasks + (BN / 2) * kChunks;  // A 128 rows, B BN/2 complex rows
  static constexpr int kTPT = 4;                              // tasks per converter thread
  static constexpr int kConvWarps = kTasks / 128;             // 4 tasks per converter thread: 12, 10 or 8 warps
  static constexpr int kConvThreads = 32 * kConvWarps;
  static constexpr int kEpiWarps = BN == 256 ? 8 : 4;         // the short-K 256-column tiles are epilogue-bound
  static constexpr int kStageBlocks = BN == 128 ? 1 : 2;      // BN = 128: no registers to spare at 96
  static constexpr int kThreads = 32 * (kEpiWarps + 1 + kConvWarps);
  static constexpr int kFullArrivals = kConvThreads;          // arrivals completing a stage
  static constexpr uint32_t kATileBytes = 128 * kRowBytes;    // one A plane tile
  static constexpr uint32_t kBTileBytes = BN * kRowBytes;     // one B' plane tile
  static constexpr uint32_t kStageBytes = 2 * kATileBytes + 2 * kBTileBytes;  // A hi, A lo, B' hi, B' lo
  static constexpr bool kSum = BN != 256;                     // TMEM running sum region
  static constexpr int kTmemCols = BN == 256 ? 512 : (3 * BN <= 256 ? 256 : 512);
  __device__ static uint32_t swz(int row, int chunk) {
    if (kRowBytes == 128) return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
    return (uint32_t)(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4));
  }
  __device__ static uint64_t desc(uint32_t saddr) { return kRowBytes == 128 ? sw128_desc(saddr) : sw64_desc(saddr); }
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}

// bf16 hi/lo words of 8 consecutive reals: word j packs elements 2j (low
// half) and 2j + 1 (high half)
__device__ __forceinline__ void split_words(const float4& p, const float4& q, uint32_t* h, uint32_t* l) {
  const float x[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
    h[j] = *(const uint32_t*)&hb;
    l[j] = *(const uint32_t*)&lb;
  }
}

__device__ __forceinline__ void sts128(uint32_t addr, const uint32_t* w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}

// The same persistent pipeline fed by TMA from pre-split hi/lo planes
// (written by prep_a_vec / prep_b_vec): 128-byte rows (64 k' per k-block),
// one producer warp instead of the converters.  BN = 256 has no running sum
// (one accumulation chunk per tile: K <= 256).
template <int BN, int ROW = 128>
struct PlCfg {
  static constexpr int kBN = BN;
  static constexpr bool kPlanes = true;
  static constexpr bool kHybrid = false;
  static constexpr bool kF32 = false;
  static constexpr int kSlots = 2;
  static constexpr int kRowBytes = ROW;  // 64-byte rows keep BN = 256 at two stages of 48 KB
  // staging blocks per epilogue step: two unless the shared memory is full
  static constexpr int kStageBlocks = (BN == 256 && ROW == 128) ? 1 : 2;
  static constexpr int kKC = kRowBytes / 4;               // complex k per k-block
  static constexpr int kKSteps = kRowBytes / 32;
  static constexpr int kChunkKB = 512 / (kRowBytes / 2);
  static constexpr int kEpiWarps = 8;      // two per TMEM lane quarter, half of the columns each
  static constexpr int kThreads = 32 * (kEpiWarps + 2);
  static constexpr int kFullArrivals = 1;  // the producer's expect_tx arrival; the bytes complete it
  static constexpr int kTPT = 4;           // (no converters)
  static constexpr uint32_t kATileBytes = 128 * kRowBytes;
  static constexpr uint32_t kBTileBytes = BN * kRowBytes;
  static constexpr uint32_t kStageBytes = 2 * kATileBytes + 2 * kBTileBytes;
  static constexpr bool kSum = BN != 256;
  static constexpr int kTmemCols = BN == 256 ? 512 : (3 * BN <= 256 ? 256 : 512);
  __device__ static uint64_t desc(uint32_t saddr) { return kRowBytes == 128 ? sw128_desc(saddr) : sw64_desc(saddr); }
};

// Hybrid: A split on chip by converter warps (as FzCfg), B' streamed by TMA
// from its pre-split planes (as PlCfg).  For nodes whose B is small and
// re-read by many row tiles while A is large and read by few column tiles,
// this drops the A plane pass (write + read back) of the plane kernels.
// 256 columns, 64-byte rows (two 48 KB stages), K <= 256 (no running sum).
struct HyCfg {
  static constexpr int kBN = 256;
  static constexpr bool kPlanes = true;
  static constexpr bool kHybrid = true;
  static constexpr bool kF32 = false;
  static constexpr int kSlots = 2;
  static constexpr int kRowBytes = 64;
  static constexpr int kChunks = kRowBytes / 16;
  static constexpr int kKC = kRowBytes / 4;
  static constexpr int kKSteps = kRowBytes / 32;
  static constexpr int kChunkKB = 512 / (kRowBytes / 2);
  static constexpr int kATasks = 128 * kChunks;               // all converter tasks are A tasks
  // 1 task per thread: 16 warps (26 in the block, 72 registers), four times
  // the loads in flight of 4 warps with 4 tasks each (the A conversion of a
  // tile is load-latency bound: 4 -> 8 -> 16 warps took an M 4096 N 256
  // K 128 node from 1.03 to 0.94 to 0.90 ms)
  static constexpr int kTPT = 1;
  static constexpr int kConvWarps = kATasks / (32 * kTPT);
  static constexpr int kConvThreads = 32 * kConvWarps;
  static constexpr int kEpiWarps = 8;
  static constexpr int kStageBlocks = 2;
  static constexpr int kThreads = 32 * (kEpiWarps + 2 + kConvWarps);
  static constexpr int kFullArrivals = kConvThreads + 1;      // converters + the producer's expect_tx
  static constexpr uint32_t kATileBytes = 128 * kRowBytes;
  static constexpr uint32_t kBTileBytes = 256 * kRowBytes;
  static constexpr uint32_t kStageBytes = 2 * kATileBytes + 2 * kBTileBytes;
  static constexpr bool kSum = false;
  static constexpr int kTmemCols = 512;
  __device__ static uint32_t swz(int row, int chunk) { return (uint32_t)(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4)); }
  __device__ static uint64_t desc(uint32_t saddr) { return sw64_desc(saddr); }
};

// 256 columns split on chip for any K: one TMEM accumulator slot plus the
// running sum (256 + 256 columns).  The MMA waits while the epilogue folds
// each chunk into the sum; the converters, which set the pace on long-K
// nodes, run on meanwhile, and each A tile is converted for half as many
// column tiles as with 128 columns.  Chunks of 1024 k' halve the folds of
// 512 (3 % faster on a K = 4096 node; relative error 5.6e-6 against 4.8e-6:
// each chunk's sum stays inside the tensor core, whose accumulation error
// grows with the chain length).
struct FzWideCfg : FzCfg<256> {
  static constexpr bool kSum = true;
  static constexpr int kSlots = 1;
  static constexpr int kTmemCols = 512;
  static constexpr int kChunkKB = 1024 / (kRowBytes / 2);
};

// Split on chip from FP32 tiles that TMA brings into shared memory: a
// producer warp streams each k-block's A tile (128 rows) and B tile (BN / 2
// complex rows) of 16 complex k (128-byte rows, 128-byte swizzle) into a ring
// of kF32Stages stages, several k-blocks ahead; the converters read their
// tasks from there instead of from global memory, split them and store the
// 64-byte-row A' and B'^T tiles as FzCfg does.  The converters of FzCfg hold
// one k-block of loads in registers, so a CTA has about one k-block of DRAM
// reads in flight and the short-K, output-heavy nodes ran at half the HBM
// rate; the ring keeps several in flight without registers.  BN = 256 takes
// K <= 256 (one accumulation chunk per tile, no running sum).
template <int BN>
struct FtCfg {
  static constexpr int kBN = BN;
  static constexpr bool kPlanes = false;
  static constexpr bool kHybrid = false;
  static constexpr bool kF32 = true;
  static constexpr int kSlots = 2;
  static constexpr int kRowBytes = 64;
  static constexpr int kChunks = 4;
  static constexpr int kKC = 16;
  static constexpr int kKSteps = 2;
  static constexpr int kChunkKB = 512 / (kRowBytes / 2);
  static constexpr int kATasks = 128 * kChunks;
  static constexpr int kTasks = kATasks + (BN / 2) * kChunks;
  // Converters only read shared memory here, so 4 tasks a thread keep up;
  // the epilogue sets the pace of these output-heavy nodes, so 8 warps (two
  // per TMEM lane quarter, half of the columns each) drain it: 4 -> 8 took
  // the batch 256, M 2048, N 64, K 32 node from 0.157 to 0.114 ms.  15, 16
  // or 18 warps: 128, 128 and 96 registers a thread.
  static constexpr int kTPT = 4;
  static constexpr int kConvWarps = kTasks / (32 * kTPT);  // 5, 6 or 8
  static constexpr int kConvThreads = 32 * kConvWarps;
  static constexpr int kEpiWarps = 8;
  static constexpr int kStageBlocks = 2;
  static constexpr int kThreads = 32 * (kEpiWarps + 2 + kConvWarps);
  static constexpr int kFullArrivals = kConvThreads;
  static constexpr uint32_t kATileBytes = 128 * kRowBytes;
  static constexpr uint32_t kBTileBytes = BN * kRowBytes;
  static constexpr uint32_t kStageBytes = 2 * kATileBytes + 2 * kBTileBytes;
  static constexpr bool kSum = BN != 256;
  static constexpr int kTmemCols = BN == 256 ? 512 : (3 * BN <= 256 ? 256 : 512);
  static constexpr int kF32Stages = BN == 256 ? 2 : 4;
  static constexpr uint32_t kF32ABytes = 128 * 128;                 // 128 rows x 16 complex
  static constexpr uint32_t kF32StageBytes = kF32ABytes + (BN / 2) * 128;
  __device__ static uint32_t swz(int row, int chunk) { return (uint32_t)(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4)); }
  __device__ static uint64_t desc(uint32_t saddr) { return sw64_desc(saddr); }
};

// shared-memory bytes and stages of the FP32 ring (0 without one)
template <class Cf>
__host__ __device__ constexpr uint32_t f32_ring_bytes() {
  if constexpr (Cf::kF32)
    return Cf::kF32Stages * Cf::kF32StageBytes;
  else
    return 0;
}
template <class Cf>
__host__ __device__ constexpr int f32_stages() {
  if constexpr (Cf::kF32)
    return Cf::kF32Stages;
  else
    return 0;
}

struct PlMaps {
  CUtensorMap ah, al, bh, bl;
};

// Output order of one warp's epilogue block: 32 rows (m bits 0..4, from the
// lane) x 8 complex columns (n bits 0..2).  The consumer's layout puts these
// 8 index bits at 8 output bit positions; ranking the positions gives a
// staging index whose increasing order is increasing output address, so a
// block written into shared memory by (row, column) and read back by staging
// index stores runs of consecutive addresses (a whole 2 KB block when the 8
// positions are the lowest 8).  Requires nM >= 5 and nN >= 3.
struct BlockOrder {
  int pos[8];   // output bit position of block bit b (0..4 rows, 5..7 columns)
  int rank[8];  // rank of pos[b] among the 8
  __device__ explicit BlockOrder(const OutMap& om) {
#pragma unroll
    for (int b = 0; b < 5; ++b) pos[b] = om.pos[om.nN + b];
#pragma unroll
    for (int b = 0; b < 3; ++b) pos[5 + b] = om.pos[b];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      int r = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) r += pos[k] < pos[b];
      rank[b] = r;
    }
  }
  __device__ uint32_t index_row(uint32_t lane) const {
    uint32_t x = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) x |= ((lane >> b) & 1u) << rank[b];
    return x;
  }
  __device__ uint32_t index_col(uint32_t j) const {
    uint32_t x = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) x |= ((j >> b) & 1u) << rank[5 + b];
    return x;
  }
  // output offset (relative to the block's origin) of staging-index bits x
  __device__ uint64_t offset_of(uint32_t x) const {
    uint64_t o = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) o |= (uint64_t)((x >> rank[b]) & 1u) << pos[b];
    return o;
  }
};

// Direct epilogue stores of one warp's column blocks (v: NB blocks of 8
// complex columns, real and imaginary parts interleaved; ctc: the output
// offsets of those columns) when output bit 0 is column bit CB: the column
// pair (j, j | 2^CB) is 16 contiguous bytes.
template <int CB, int NB>
__device__ __forceinline__ void store_pairs(float2* base, const uint64_t* ctc, const float* v) {
#pragma unroll
  for (int h = 0; h < NB; ++h)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j & (1 << CB)) continue;
      const int k = j | (1 << CB);
      *(float4*)(base + ctc[8 * h + j]) =
          make_float4(v[16 * h + 2 * j], v[16 * h + 2 * j + 1], v[16 * h + 2 * k], v[16 * h + 2 * k + 1]);
    }
}

// bank spread of the staging block (8-byte elements): low 4 index bits XOR
// the high 4, a bijection on 0..255
__device__ __forceinline__ uint32_t stage_swz(uint32_t x) { return x ^ ((x >> 4) & 15u); }

// One k-block of a converter thread: its kTPT tasks (4; 1 in the hybrid
// tile), j = ct + T i with T the converter thread count (a multiple of 32
// and of the chunks per row C), of 2 x 16 bytes each.  Task j < 128 C: A tile row j / C; otherwise complex
// column (j - 128 C) / C of B, giving B' rows 2n and 2n + 1.  Chunk j % C =
// ct % C in both cases.  128 C is a multiple of 32, so A/B tasks never mix in
// a warp.
template <int TPT>
struct FzRegs {
  float4 v[TPT][2];
};

struct FzGeom {
  int M, N, K, tiles_m, tiles_n, nk;
  int64_t tiles;  // tiles_m * tiles_n * batch
};

// tile t -> (batch, first row, first real column); m-tiles fastest
template <int BN>
__device__ __forceinline__ void fz_tile(const FzGeom& g, int64_t t, int& bz, int& m0, int& n0) {
  const int64_t per_b = (int64_t)g.tiles_m * g.tiles_n;
  bz = (int)(t / per_b);
  const int r = (int)(t - (int64_t)bz * per_b);
  m0 = (r % g.tiles_m) * BM;
  n0 = (r / g.tiles_m) * BN;
}

template <class Cf>
__device__ __forceinline__ void fz_load(FzRegs<Cf::kTPT>& R, const float2* __restrict__ A, const float2* __restrict__ B,
                                        const FzGeom& g, int bz, int m0, int n0, int kb, int ct) {
  const int64_t koff = (int64_t)kb * Cf::kKC + 4 * (ct % Cf::kChunks);
#pragma unroll
  for (int i = 0; i < Cf::kTPT; ++i) {
    const int j = ct + Cf::kConvThreads * i;
    const float2* p = j < Cf::kATasks ? A + ((int64_t)bz * g.M + m0 + j / Cf::kChunks) * g.K + koff
                                      : B + ((int64_t)bz * g.N + n0 / 2 + (j - Cf::kATasks) / Cf::kChunks) * g.K + koff;
    R.v[i][0] = __ldg((const float4*)p);
    R.v[i][1] = __ldg((const float4*)p + 1);
  }
}

// L2 prefetch of a k-block's lines (one thread per 128-byte line), so that
// a second k-block of loads is on its way without holding registers
template <class Cf>
__device__ __forceinline__ void fz_prefetch(const float2* __restrict__ A, const float2* __restrict__ B,
                                            const FzGeom& g, int bz, int m0, int n0, int kb, int ct) {
  if (ct & 3) return;
  const int64_t koff = (int64_t)kb * Cf::kKC + 4 * (ct % Cf::kChunks);
#pragma unroll
  for (int i = 0; i < Cf::kTPT; ++i) {
    const int j = ct + Cf::kConvThreads * i;
    const float2* p = j < Cf::kATasks ? A + ((int64_t)bz * g.M + m0 + j / Cf::kChunks) * g.K + koff
                                      : B + ((int64_t)bz * g.N + n0 / 2 + (j - Cf::kATasks) / Cf::kChunks) * g.K + koff;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
}

// A converter thread's tasks of one k-block from the FP32 ring stage at
// `stage` (A tile, then B tile; 128-byte rows, 16-byte chunk c of row r at
// r * 128 + ((c ^ (r % 8)) * 16)): the same registers fz_load fills
template <class Cf>
__device__ __forceinline__ void ft_load(FzRegs<Cf::kTPT>& R, const uint8_t* stage, int ct) {
  const int cc = ct % Cf::kChunks;
#pragma unroll
  for (int i = 0; i < Cf::kTPT; ++i) {
    const int j = ct + Cf::kConvThreads * i;
    const bool a = j < Cf::kATasks;
    const int r = a ? j / Cf::kChunks : (j - Cf::kATasks) / Cf::kChunks;
    const uint8_t* row = stage + (a ? 0u : Cf::kF32ABytes) + r * 128;
    R.v[i][0] = *(const float4*)(row + (((2 * cc) ^ (r & 7)) << 4));
    R.v[i][1] = *(const float4*)(row + (((2 * cc + 1) ^ (r & 7)) << 4));
  }
}

template <class Cf>
__device__ __forceinline__ void fz_store(const FzRegs<Cf::kTPT>& R, uint32_t st, int ct) {
  constexpr uint32_t kAl = Cf::kATileBytes, kB = 2 * Cf::kATileBytes, kBl = kB + Cf::kBTileBytes;
  const int cc = ct % Cf::kChunks;
#pragma unroll
  for (int i = 0; i < Cf::kTPT; ++i) {
    const int j = ct + Cf::kConvThreads * i;
    uint32_t h[4], l[4];
    split_words(R.v[i][0], R.v[i][1], h, l);
    if (j < Cf::kATasks) {
      const uint32_t o = Cf::swz(j / Cf::kChunks, cc);
      sts128(st + o, h);
      sts128(st + kAl + o, l);
    } else {
      // words (br, bi) -> row 2n: (br, -bi), row 2n + 1: (bi, br)
      uint32_t h0[4], l0[4], h1[4], l1[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        h0[q] = h[q] ^ 0x80000000u;
        l0[q] = l[q] ^ 0x80000000u;
        h1[q] = __byte_perm(h[q], 0, 0x1032);
        l1[q] = __byte_perm(l[q], 0, 0x1032);
      }
      const int r0 = 2 * ((j - Cf::kATasks) / Cf::kChunks);
      if constexpr (Cf::kRowBytes == 64) {
        // rows 2n and 2n + 1 are the two halves of one 128-byte line: odd
        // chunks store row 2n + 1 first, so that each instruction fills both
        // halves of every line it touches (no bank conflicts)
        const bool odd = cc & 1;
        uint32_t ah[4], al[4], bh[4], bl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ah[q] = odd ? h1[q] : h0[q];
          al[q] = odd ? l1[q] : l0[q];
          bh[q] = odd ? h0[q] : h1[q];
          bl[q] = odd ? l0[q] : l1[q];
        }
        const int ra = r0 + (odd ? 1 : 0), rb = r0 + (odd ? 0 : 1);
        sts128(st + kB + Cf::swz(ra, cc), ah);
        sts128(st + kBl + Cf::swz(ra, cc), al);
        sts128(st + kB + Cf::swz(rb, cc), bh);
        sts128(st + kBl + Cf::swz(rb, cc), bl);
      } else {
        sts128(st + kB + Cf::swz(r0, cc), h0);
        sts128(st + kBl + Cf::swz(r0, cc), l0);
        sts128(st + kB + Cf::swz(r0 + 1, cc), h1);
        sts128(st + kBl + Cf::swz(r0 + 1, cc), l1);
      }
    }
  }
}

// Persistent: CTA c computes tiles c, c + gridDim.x, ...; the shared-memory
// ring, the two TMEM accumulator slots and their barriers run on across tile
// boundaries, so a tile's epilogue overlaps the next tile's MMAs and the
// converters keep two k-blocks of loads in flight through tile changes.
template <class Cf, bool PREFETCH>
__global__ void __launch_bounds__(Cf::kThreads, 1)
    tc_fused_bf16_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float* __restrict__ C,
                         const FzGeom geo, const __grid_constant__ OutMap om, const __grid_constant__ PlMaps maps) {
  constexpr int BN = Cf::kBN;
  // k-blocks per accumulation chunk (all of a tile's k-blocks without a
  // running sum; the launcher admits only K <= 256 then)
  constexpr int CHUNK = Cf::kSum ? Cf::kChunkKB : (1 << 30);
  constexpr uint32_t IDESC = instr_desc<false, BN>();
  constexpr uint32_t kStageBytes = Cf::kStageBytes;
  constexpr bool kProducer = Cf::kPlanes || Cf::kF32;  // warp E + 1 issues TMA loads
  constexpr int SF = f32_stages<Cf>();                   // FP32 ring stages (kF32)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* ring = smem + kFzStages * kStageBytes;        // FP32 ring (kF32), 1024-byte aligned
  uint64_t* full = (uint64_t*)(ring + f32_ring_bytes<Cf>());
  uint64_t* empty = full + kFzStages;
  uint64_t* acc_full = empty + kFzStages;  // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  uint64_t* coltab = (uint64_t*)(tmem_slot + 4);  // [4 warps][BN / 2]
  uint32_t* blk_col = (uint32_t*)(coltab + 4 * (BN / 2));  // [8] staging index of block column j
                                                            // (coltab: [E warps][CW / 2], 4 BN / 2 in all)
  uint64_t* blk_dep = (uint64_t*)(blk_col + 8);               // [8] output offset of staging index bits 5..7
  float2* stage_out = (float2*)(blk_dep + 8);                 // [E warps][2][256]
  uint64_t* ffull = (uint64_t*)(stage_out + Cf::kEpiWarps * Cf::kStageBlocks * 256);  // [SF] (kF32)
  uint64_t* fempty = ffull + SF;                                                       // [SF]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int E = Cf::kEpiWarps;        // warps 0..E-1: epilogue; E: MMA; E+1..: producer / converters
  constexpr int CW = BN * 4 / E;          // real columns per epilogue warp
  const int nk = geo.nk;
  const int nchunks = (nk + CHUNK - 1) / CHUNK;  // per tile
  const int64_t my_tiles = blockIdx.x < geo.tiles ? (geo.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int N2 = 2 * geo.N;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFzStages; ++s) {
      mbar_init(&full[s], Cf::kFullArrivals);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], 32 * E);
    }
    mbar_init(done, 1);
    if constexpr (Cf::kF32)
      for (int f = 0; f < SF; ++f) {
        mbar_init(&ffull[f], 1);
        mbar_init(&fempty[f], Cf::kConvThreads);
      }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == E) tmem_alloc(tmem_slot, Cf::kTmemCols);  // slot 0, slot 1, running sum (BN columns each)
  if (!om.ident && threadIdx.x < 8) {
    const BlockOrder bo(om);
    blk_col[threadIdx.x] = bo.index_col(threadIdx.x);
    blk_dep[threadIdx.x] = bo.offset_of((uint32_t)threadIdx.x << 5);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int64_t tma_issued = 0;  // planes: k-blocks whose TMA loads were issued
  if (Cf::kF32 && warp == E + 1) {
    // producer: TMA loads of the FP32 A and B tiles of every k-block into the ring
    if constexpr (Cf::kF32) {
      if (lane == 0) {
        int f = 0;
        uint32_t fph = 0;
        for (int64_t lt = 0; lt < my_tiles; ++lt) {
          int bz, m0, n0;
          fz_tile<BN>(geo, (int64_t)blockIdx.x + lt * gridDim.x, bz, m0, n0);
          bool ok = true;
          for (int kb = 0; kb < nk; ++kb) {
            if (tma_issued >= SF && !mbar_wait(&fempty[f], fph ^ 1u)) {
              atomicExch(&tc_error_flag, 10);
              *(volatile int*)abort_flag = 1;
              ok = false;
              break;
            }
            if (*(volatile int*)abort_flag) {
              ok = false;
              break;
            }
            uint8_t* st = ring + f * Cf::kF32StageBytes;
            const int kx = kb * (2 * Cf::kKC);  // first float of the k-block
            mbar_expect_tx(&ffull[f], Cf::kF32StageBytes);
            tma_load_3d(st, &maps.ah, &ffull[f], kx, m0, bz);
            tma_load_3d(st + Cf::kF32ABytes, &maps.bh, &ffull[f], kx, n0 / 2, bz);
            ++tma_issued;
            if (++f == SF) {
              f = 0;
              fph ^= 1u;
            }
          }
          if (!ok) break;
        }
      }
    }
  } else if (Cf::kPlanes && warp == E + 1) {
    // producer: TMA loads of the hi/lo plane tiles of every k-block
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      for (int64_t lt = 0; lt < my_tiles; ++lt) {
        int bz, m0, n0;
        fz_tile<BN>(geo, (int64_t)blockIdx.x + lt * gridDim.x, bz, m0, n0);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
          if (tma_issued >= kFzStages && !mbar_wait(&empty[s], ph ^ 1u)) {
            atomicExch(&tc_error_flag, 7);
            *(volatile int*)abort_flag = 1;
            ok = false;
            break;
          }
          if (*(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * kStageBytes;
          const int kx = kb * (Cf::kKC * 2);  // first bf16 column of the k-block
          if (Cf::kHybrid) {
            mbar_expect_tx(&full[s], 2 * Cf::kBTileBytes);  // the converters fill the A tiles
          } else {
            mbar_expect_tx(&full[s], kStageBytes);
            tma_load_3d(st, &maps.ah, &full[s], kx, m0, bz);
            tma_load_3d(st + Cf::kATileBytes, &maps.al, &full[s], kx, m0, bz);
          }
          tma_load_3d(st + 2 * Cf::kATileBytes, &maps.bh, &full[s], kx, n0, bz);
          tma_load_3d(st + 2 * Cf::kATileBytes + Cf::kBTileBytes, &maps.bl, &full[s], kx, n0, bz);
          ++tma_issued;
          if (++s == kFzStages) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp >= E + 1 + (kProducer ? 1 : 0)) {
   if constexpr (Cf::kF32) {
    // converters fed by the FP32 ring: k-block q in ring stage q % SF
    const int ct = threadIdx.x - 32 * (E + 2);
    const int64_t total = my_tiles * nk;
    FzRegs<Cf::kTPT> R;
    int s = 0, f = 0;
    uint32_t ph = 0, fph = 0;
    for (int64_t q = 0; q < total; ++q) {
      if (!mbar_wait(&ffull[f], fph)) {
        atomicExch(&tc_error_flag, 11);
        *(volatile int*)abort_flag = 1;
        break;
      }
      ft_load<Cf>(R, ring + f * Cf::kF32StageBytes, ct);
      // reads of the ring stage ordered before the producer's next TMA write into it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&fempty[f])) : "memory");
      if (++f == SF) {
        f = 0;
        fph ^= 1u;
      }
      if (q >= kFzStages && !mbar_wait(&empty[s], ph ^ 1u)) {
        atomicExch(&tc_error_flag, 6);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      fz_store<Cf>(R, smem_u32(smem + s * kStageBytes), ct);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s])) : "memory");
      if (++s == kFzStages) {
        s = 0;
        ph ^= 1u;
      }
    }
   } else if constexpr (!Cf::kPlanes || Cf::kHybrid) {
    // converters: global k-block q = (local tile) * nk + kb
    const int ct = threadIdx.x - 32 * (E + 1 + (Cf::kHybrid ? 1 : 0));
    const int64_t total = my_tiles * nk;
    FzRegs<Cf::kTPT> R0;
    // load cursor: local tile lt_ld (coordinates bz, m0, n0), k-block kb_ld
    int64_t lt_ld = 0;
    int kb_ld = 0, bz = 0, m0 = 0, n0 = 0;
    if (my_tiles > 0) fz_tile<BN>(geo, blockIdx.x, bz, m0, n0);
    auto load_next = [&](FzRegs<Cf::kTPT>& R) {
      fz_load<Cf>(R, A, B, geo, bz, m0, n0, kb_ld, ct);
      if (++kb_ld == nk) {
        kb_ld = 0;
        if (++lt_ld < my_tiles) fz_tile<BN>(geo, (int64_t)blockIdx.x + lt_ld * gridDim.x, bz, m0, n0);
      }
    };
    if (total > 0) load_next(R0);
    int s = 0;         // stage of k-block q
    uint32_t ph = 0;   // number of ring wraps before q, mod 2
    // one k-block from registers R into stage s, then the loads of k-block
    // q + 1 into R; false after a timeout or an abort.  (Two register sets
    // for two k-blocks in flight need more than the 96 registers a thread
    // of this 17-warp block can have, and spill.)
    auto step = [&](FzRegs<Cf::kTPT>& R, int64_t q) -> bool {
      if (q >= kFzStages && !mbar_wait(&empty[s], ph ^ 1u)) {
        atomicExch(&tc_error_flag, 6);
        *(volatile int*)abort_flag = 1;
        return false;
      }
      if (*(volatile int*)abort_flag) return false;
      fz_store<Cf>(R, smem_u32(smem + s * kStageBytes), ct);
      // make the generic-proxy stores visible to the tensor core, then signal
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s])) : "memory");
      if (++s == kFzStages) {
        s = 0;
        ph ^= 1u;
      }
      if (q + 1 < total) load_next(R);
      if (PREFETCH && q + 2 < total) fz_prefetch<Cf>(A, B, geo, bz, m0, n0, kb_ld, ct);  // cursor is at q + 2
      return true;
    };
    for (int64_t q = 0; q < total; ++q)
      if (!step(R0, q)) break;
   }
  } else if (warp == E) {
    if (lane == 0) {
      bool ok = true;
      int64_t gc = 0;       // global chunk counter
      int s = 0;            // stage of the next k-block
      uint32_t ph = 0;      // ring wraps before it, mod 2
      for (int64_t lt = 0; lt < my_tiles && ok; ++lt) {
        for (int c = 0; c < nchunks && ok; ++c, ++gc) {
          const int slot = (int)(gc % Cf::kSlots);
          if (gc >= Cf::kSlots && !mbar_wait(&acc_empty[slot], (uint32_t)(((gc / Cf::kSlots) + 1) & 1))) {
            atomicExch(&tc_error_flag, 4);
            *(volatile int*)abort_flag = 1;
            ok = false;
            break;
          }
          const uint32_t dtm = tmem + slot * BN;
          const int kb_end = (c + 1) * CHUNK < nk ? (c + 1) * CHUNK : nk;
          for (int kb = c * CHUNK; kb < kb_end; ++kb) {
            if (!mbar_wait(&full[s], ph)) {
              atomicExch(&tc_error_flag, 2);
              *(volatile int*)abort_flag = 1;
              ok = false;
              break;
            }
            if (*(volatile int*)abort_flag) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * kStageBytes);
            const uint64_t dAh = Cf::desc(sa), dAl = Cf::desc(sa + Cf::kATileBytes);
            const uint64_t dBh = Cf::desc(sa + 2 * Cf::kATileBytes);
            const uint64_t dBl = Cf::desc(sa + 2 * Cf::kATileBytes + Cf::kBTileBytes);
#pragma unroll
            for (int kk = 0; kk < Cf::kKSteps; ++kk) {
              const uint64_t adv = (uint64_t)((kk * 16 * 2) >> 4);
              const uint32_t first = (kb == c * CHUNK && kk == 0) ? 0u : 1u;
              mma<false>(dtm, dAh + adv, dBh + adv, IDESC, first);
              mma<false>(dtm, dAh + adv, dBl + adv, IDESC, 1u);
              mma<false>(dtm, dAl + adv, dBh + adv, IDESC, 1u);
            }
            mma_commit(&empty[s]);
            if (++s == kFzStages) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (ok) mma_commit(&acc_full[slot]);
        }
      }
      mma_commit(done);
    }
  } else {
    // accumulation: row 32 (warp % 4) + lane of each tile, real columns
    // [half * CW, half * CW + CW)
    const int quarter = warp & 3, half = warp >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const uint32_t tsum = tmem + lane_base + Cf::kSlots * BN;
    uint64_t* ct = coltab + warp * (CW / 2);
    float2* so = stage_out + warp * 256 * Cf::kStageBlocks;
    uint32_t idx_row = 0;
    uint64_t dep_lane = 0;
    // Direct stores, without the staging block, when the lowest output
    // address bits are bits of this warp's 32 x 8 block (rows 0..4 from the
    // lane, columns 0..2 from the register index): every store then fills
    // whole 32-byte sectors or halves that the same thread completes next,
    // and the re-ordering through shared memory would only add latency.
    //   direct 1: positions 0 and 1 both row bits: 8-byte stores, aligned
    //             groups of four lanes cover a sector;
    //   direct 2: position 0 a column bit c: 16-byte stores of the column
    //             pairs (j, j | 2^c).
    // (A row bit at 0 and a column bit at 1, the pair exchanged between two
    // lanes by a shuffle, was slower than the staging block: 0.101 -> 0.108 ms
    // on batch 256, M 512, N 256, K 64.)
    int direct = 0, dbit_c = 0;
    uint64_t lane_off = 0;
    if (!om.ident) {
      const BlockOrder bo(om);
      idx_row = bo.index_row(lane);
      dep_lane = bo.offset_of((uint32_t)lane);
      int r0 = -1, r1 = -1, c0 = -1;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        if (om.pos[om.nN + b] == 0) r0 = b;
        if (om.pos[om.nN + b] == 1) r1 = b;
      }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (om.pos[b] == 0) c0 = b;
      }
      if (r0 >= 0 && r1 >= 0) {
        direct = 1;
      } else if (c0 >= 0) {
        direct = 2;
        dbit_c = c0;
      }
      lane_off = om.row(0, lane, geo.M, geo.N);
    }
    int64_t gc = 0;
    bool ok = true;
    for (int64_t lt = 0; lt < my_tiles && ok; ++lt) {
      int bz, m0, n0;
      fz_tile<BN>(geo, (int64_t)blockIdx.x + lt * gridDim.x, bz, m0, n0);
      const int row = m0 + quarter * 32 + lane;
      const uint64_t roff = om.ident ? 0 : om.row(bz, m0 + quarter * 32, geo.M, geo.N);  // lane bits clear
      if (!om.ident)
        for (int i = lane; i < CW / 2; i += 32) ct[i] = om.col(n0 / 2 + half * (CW / 2) + i);
      __syncwarp();
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int slot = (int)(gc % Cf::kSlots);
        if (!mbar_wait(&acc_full[slot], (uint32_t)((gc / Cf::kSlots) & 1))) {
          atomicExch(&tc_error_flag, 3);
          *(volatile int*)abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const bool last = c == nchunks - 1;
        const uint32_t tslot = tmem + lane_base + slot * BN;
        const bool write_out = last && !*(volatile int*)abort_flag;
        // NB staging blocks of 8 complex columns (16 real) per step
        constexpr int NB = Cf::kStageBlocks;
#pragma unroll 1
        for (int col = half * CW; col < half * CW + CW; col += 16 * NB) {
          float v[16 * NB];
          if constexpr (NB == 2)
            tmem_ld32(tslot + col, v);
          else
            tmem_ld16(tslot + col, v);
          if (c > 0) {
#pragma unroll
            for (int h = 0; h < NB; ++h) {
              float w[16];
              tmem_ld16(tsum + col + 16 * h, w);
#pragma unroll
              for (int i = 0; i < 16; ++i) v[16 * h + i] += w[i];
            }
          }
          if (!last) {
#pragma unroll
            for (int h = 0; h < NB; ++h) tmem_st16(tsum + col + 16 * h, v + 16 * h);
          } else if (write_out) {
            if (om.ident) {
              float4* dst = (float4*)(C + ((int64_t)bz * geo.M + row) * N2 + n0 + col);
#pragma unroll
              for (int i = 0; i < 4 * NB; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            } else if (direct) {
              float2* base = (float2*)C + roff + lane_off;
              const uint64_t* ctc = ct + (col - half * CW) / 2;
              if (direct == 1) {
#pragma unroll
                for (int h = 0; h < NB; ++h)
#pragma unroll
                  for (int j = 0; j < 8; ++j) base[ctc[8 * h + j]] = make_float2(v[16 * h + 2 * j], v[16 * h + 2 * j + 1]);
              } else {
                if (dbit_c == 0) store_pairs<0, NB>(base, ctc, v);
                else if (dbit_c == 1) store_pairs<1, NB>(base, ctc, v);
                else store_pairs<2, NB>(base, ctc, v);
              }
            } else {
              // through the warp's staging blocks: written by (row, column),
              // read back in output order, so that each store covers the
              // block's runs of consecutive output addresses
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const uint32_t x = stage_swz(idx_row | blk_col[j]);
#pragma unroll
                for (int h = 0; h < NB; ++h) so[256 * h + x] = make_float2(v[16 * h + 2 * j], v[16 * h + 2 * j + 1]);
              }
              __syncwarp();
              const int cc = (col - half * CW) / 2;
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const uint32_t x = stage_swz((uint32_t)(t * 32 + lane));
#pragma unroll
                for (int h = 0; h < NB; ++h) ((float2*)C + roff + ct[cc + 8 * h] + dep_lane)[blk_dep[t]] = so[256 * h + x];
              }
              __syncwarp();
            }
          }
        }
        if (!last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[slot])) : "memory");
      }
      __syncwarp();  // coltab entries of this tile read by every lane before the next tile's
    }
  }
  if (threadIdx.x == 0 && !mbar_wait(done, 0)) atomicExch(&tc_error_flag, 5);
  tc_fence_before();
  __syncthreads();
  // planes, after an abort: wait (bounded) for the TMA copies still in flight
  if (Cf::kPlanes && warp == E + 1 && lane == 0 && *(volatile int*)abort_flag) {
    for (int64_t q = (tma_issued > kFzStages ? tma_issued - kFzStages : 0); q < tma_issued; ++q)
      mbar_wait(&full[q % kFzStages], (uint32_t)((q / kFzStages) & 1));
  }
  if (Cf::kF32 && warp == E + 1 && lane == 0 && *(volatile int*)abort_flag) {
    for (int64_t q = (tma_issued > SF ? tma_issued - SF : 0); q < tma_issued; ++q)
      mbar_wait(&ffull[q % SF], (uint32_t)((q / SF) & 1));
  }
  __syncthreads();
  if (warp == E) {
    tc_fence_after();
    tmem_dealloc(tmem, Cf::kTmemCols);
  }
}


// the kernel's register count times its block size fits the SM (checked
// once per process; otherwise the tile runs through the planes)
template <int BN>
bool fused_launchable() {
  static std::atomic<int> ok{-1};
  int v = ok.load(std::memory_order_acquire);
  if (v < 0) {
    cudaFuncAttributes fa;
    v = cudaFuncGetAttributes(&fa, tc_fused_bf16_kernel<FzCfg<BN>, false>) == cudaSuccess &&
        fa.maxThreadsPerBlock >= FzCfg<BN>::kThreads;
    ok.store(v, std::memory_order_release);
  }
  return v == 1;
}

template <class Cf, bool PREFETCH>
int launch_persistent(const GemmDesc& d, const float2* A, const float2* B, float* C, const PlMaps& maps,
                      cudaStream_t st) {
  constexpr int BN = Cf::kBN;
  // at least 117 KB so that one CTA (and one TMEM allocation) holds an SM
  const size_t need = 1024 + kFzStages * Cf::kStageBytes + f32_ring_bytes<Cf>() + (2 * kFzStages + 5) * 8 + 16 +
                      4 * BN / 2 * 8 + 8 * 4 + 8 * 8 + Cf::kEpiWarps * Cf::kStageBlocks * 256 * 8 +
                      2 * f32_stages<Cf>() * 8;
  const size_t smem = need > 117 * 1024 ? need : 117 * 1024;
  static std::atomic<int> attr_done[kMaxDevices];
  if (int e = smem_attr_once(attr_done, tc_fused_bf16_kernel<Cf, PREFETCH>, (int)smem)) return e;
  FzGeom g;
  g.M = (int)d.M, g.N = (int)d.N, g.K = (int)d.K;
  g.tiles_m = (int)(d.M / BM), g.tiles_n = (int)(2 * d.N / BN), g.nk = (int)((d.K + Cf::kKC - 1) / Cf::kKC);
  g.tiles = (int64_t)g.tiles_m * g.tiles_n * d.batch;
  const int64_t grid = g.tiles < sm_count() ? g.tiles : sm_count();
  tc_fused_bf16_kernel<Cf, PREFETCH><<<(unsigned)grid, Cf::kThreads, smem, st>>>(A, B, C, g, out_map(d), maps);
  return (int)cudaGetLastError();
}

template <int BN, bool PREFETCH>
int run_tc_fused(const GemmDesc& d, const float2* A, const float2* B, float* C, cudaStream_t st) {
  PlMaps none;
  std::memset(&none, 0, sizeof(none));
  return launch_persistent<FzCfg<BN>, PREFETCH>(d, A, B, C, none, st);
}

// ------------------------------------------------------------ prep kernels
template <bool kTF32>
__device__ __forceinline__ void split_val(float x, void* hi, void* lo, int64_t i) {
  if constexpr (kTF32) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    float hf = __uint_as_float(h);
    uint32_t l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hf));
    ((uint32_t*)hi)[i] = h;
    ((uint32_t*)lo)[i] = l;
  } else {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    ((__nv_bfloat16*)hi)[i] = h;
    ((__nv_bfloat16*)lo)[i] = l;
  }
}

// A (complex [b][M][K] or [b][K][M]) -> A' planes [b][M][2K]
template <bool kTF32>
__global__ void prep_a_kernel(const float2* __restrict__ A, void* hi, void* lo, int64_t M, int64_t K, int64_t total,
                              int transA) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    // i enumerates output complex positions (b, m, k) in [b][M][K] order
    const int64_t k = i % K, bm = i / K, m = bm % M, b = bm / M;
    const float2 v = transA ? A[(b * K + k) * M + m] : A[i];
    split_val<kTF32>(v.x, hi, lo, 2 * i);
    split_val<kTF32>(v.y, hi, lo, 2 * i + 1);
  }
}

// B (complex [b][K][N] or [b][N][K]) -> B'^T planes [b][2N][2K]:
// row 2n = (Br, -Bi) over k, row 2n+1 = (Bi, Br)
template <bool kTF32>
__global__ void prep_b_kernel(const float2* __restrict__ B, void* hi, void* lo, int64_t N, int64_t K, int64_t total,
                              int transB) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    // i enumerates (b, n, k) in [b][N][K] order
    const int64_t k = i % K, bn = i / K, n = bn % N, b = bn / N;
    const float2 v = transB ? B[i] : B[(b * K + k) * N + n];
    const int64_t r0 = (b * 2 * N + 2 * n) * (2 * K) + 2 * k;
    const int64_t r1 = r0 + 2 * K;
    split_val<kTF32>(v.x, hi, lo, r0);
    split_val<kTF32>(-v.y, hi, lo, r0 + 1);
    split_val<kTF32>(v.y, hi, lo, r1);
    split_val<kTF32>(v.x, hi, lo, r1 + 1);
  }
}

// Vectorised forms for the K-major operands every compiled program passes
// (A as [b][M][K], B as [b][N][K]).  A thread splits 4 consecutive complex
// values (two 16-byte loads) and writes 8 consecutive elements of each plane
// row it touches (16-byte stores for bf16, 32 bytes for tf32).
template <bool kTF32>
__device__ __forceinline__ void store8(void* plane, int64_t off, const float* v) {
  if constexpr (kTF32) {
    uint4* p = (uint4*)((uint32_t*)plane + off);
    p[0] = make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
    p[1] = make_uint4(__float_as_uint(v[4]), __float_as_uint(v[5]), __float_as_uint(v[6]), __float_as_uint(v[7]));
  } else {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      w[j] = *(uint32_t*)&h2;
    }
    *(uint4*)((__nv_bfloat16*)plane + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// hi = x rounded to the plane format, lo = (x - hi) rounded (values already
// representable in the format come out of store8's rounding unchanged)
template <bool kTF32>
__device__ __forceinline__ void split8(const float* x, float* hi, float* lo) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float h;
    if constexpr (kTF32) {
      uint32_t u;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x[j]));
      h = __uint_as_float(u);
      uint32_t l;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x[j] - h));
      lo[j] = __uint_as_float(l);
    } else {
      h = __bfloat162float(__float2bfloat16_rn(x[j]));
      lo[j] = x[j] - h;
    }
    hi[j] = h;
  }
}

// A [b][M][K] complex is already A' [b][M][2K] real: a plain split
template <bool kTF32>
__global__ void prep_a_vec_kernel(const float4* __restrict__ A, void* hi, void* lo, int64_t n8) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n8; t += (int64_t)gridDim.x * blockDim.x) {
    const float4 p = A[2 * t], q = A[2 * t + 1];
    const float x[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
    float h[8], l[8];
    split8<kTF32>(x, h, l);
    store8<kTF32>(hi, 8 * t, h);
    store8<kTF32>(lo, 8 * t, l);
  }
}

// B [b][N][K] complex -> B'^T [b][2N][2K]; log2k = log2(K)
template <bool kTF32>
__global__ void prep_b_vec_kernel(const float4* __restrict__ B, void* hi, void* lo, int64_t n4, int log2k) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 4 * t;  // first complex element (b, n, k..k+3)
    const int64_t bn = i >> log2k, k = i & ((1ll << log2k) - 1);
    const int64_t r0 = (bn << (log2k + 2)) + 2 * k, r1 = r0 + (2ll << log2k);
    const float4 p = B[2 * t], q = B[2 * t + 1];
    const float x0[8] = {p.x, -p.y, p.z, -p.w, q.x, -q.y, q.z, -q.w};
    const float x1[8] = {p.y, p.x, p.w, p.z, q.y, q.x, q.w, q.z};
    float h[8], l[8];
    split8<kTF32>(x0, h, l);
    store8<kTF32>(hi, r0, h);
    store8<kTF32>(lo, r0, l);
    split8<kTF32>(x1, h, l);
    store8<kTF32>(hi, r1, h);
    store8<kTF32>(lo, r1, l);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 3D map over a plane [batch][rows][cols], box (128-byte row, box_rows, 1)
int make_map(CUtensorMap* m, void* base, bool tf32, int64_t cols, int64_t rows, int64_t batch, int box_rows,
             int row_bytes = 128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return (int)cudaErrorNotSupported;
  const int es = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(cols * es), (cuuint64_t)(cols * rows * es)};
  cuuint32_t box[3] = {(cuuint32_t)(row_bytes / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

// split on chip from FP32 tiles brought by TMA (FtCfg): maps over A [b][M][K]
// and B [b][N][K] as FP32 rows of 2K floats, boxes of 16 complex k x 128
// (A) or BN / 2 (B) rows, 128-byte swizzle
template <int BN>
int run_tc_ft(const GemmDesc& d, const float2* A, const float2* B, float* C, cudaStream_t st) {
  PlMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  if (int e = make_map(&maps.ah, (void*)A, true, 2 * d.K, d.M, d.batch, BM, 128)) return e;
  if (int e = make_map(&maps.bh, (void*)B, true, 2 * d.K, d.N, d.batch, BN / 2, 128)) return e;
  return launch_persistent<FtCfg<BN>, false>(d, A, B, C, maps, st);
}

template <int BN>
bool ft_launchable() {
  static std::atomic<int> ok{-1};
  int v = ok.load(std::memory_order_acquire);
  if (v < 0) {
    cudaFuncAttributes fa;
    v = cudaFuncGetAttributes(&fa, tc_fused_bf16_kernel<FtCfg<BN>, false>) == cudaSuccess &&
        fa.maxThreadsPerBlock >= FtCfg<BN>::kThreads;
    ok.store(v, std::memory_order_release);
  }
  return v == 1;
}

// hi/lo planes of A' and B'^T in the scratch and TMA maps over them (boxes
// of 128-byte rows x 128 (A) or box_n (B) rows)
template <bool kTF32>
int prep_planes(const GemmDesc& d, const float2* A, const float2* B, uint8_t* scratch, int box_n, PlMaps& maps,
                cudaStream_t st, int row_bytes = 128, bool with_a = true) {
  const int64_t M = d.M, N2 = 2 * d.N, K2 = 2 * d.K, nb = d.batch;
  const int es = kTF32 ? 4 : 2;
  uint8_t* a_hi = scratch;
  uint8_t* a_lo = a_hi + nb * M * K2 * es;
  uint8_t* b_hi = a_lo + nb * M * K2 * es;
  uint8_t* b_lo = b_hi + nb * N2 * K2 * es;
  const int64_t na = nb * M * d.K, nbb = nb * d.N * d.K;
  const int64_t cap = (int64_t)sm_count() * 32;
  auto blocks = [cap](int64_t n) { return (unsigned)(n / 256 + 1 < cap ? n / 256 + 1 : cap); };
  const bool kpow2 = (d.K & (d.K - 1)) == 0;
  if (!with_a) {
    // A is split on chip by the kernel
  } else if (!d.transA && ((uintptr_t)A & 15) == 0)
    prep_a_vec_kernel<kTF32><<<blocks(na / 4), 256, 0, st>>>((const float4*)A, a_hi, a_lo, na / 4);
  else
    prep_a_kernel<kTF32><<<blocks(na), 256, 0, st>>>(A, a_hi, a_lo, M, d.K, na, d.transA);
  if (d.transB && kpow2 && ((uintptr_t)B & 15) == 0)
    prep_b_vec_kernel<kTF32><<<blocks(nbb / 4), 256, 0, st>>>((const float4*)B, b_hi, b_lo, nbb / 4,
                                                             __builtin_ctzll((unsigned long long)d.K));
  else
    prep_b_kernel<kTF32><<<blocks(nbb), 256, 0, st>>>(B, b_hi, b_lo, d.N, d.K, nbb, d.transB);
  int r;
  if (with_a && (r = make_map(&maps.ah, a_hi, kTF32, K2, M, nb, BM, row_bytes))) return r;
  if (with_a && (r = make_map(&maps.al, a_lo, kTF32, K2, M, nb, BM, row_bytes))) return r;
  if ((r = make_map(&maps.bh, b_hi, kTF32, K2, N2, nb, box_n, row_bytes))) return r;
  if ((r = make_map(&maps.bl, b_lo, kTF32, K2, N2, nb, box_n, row_bytes))) return r;
  return 0;
}

// persistent TMA-fed variant (split-BF16)
template <int BN, int ROW>
int run_tc_planes(const GemmDesc& d, const float2* A, const float2* B, float* C, uint8_t* scratch, cudaStream_t st) {
  PlMaps maps;
  int r = prep_planes<false>(d, A, B, scratch, BN, maps, st, ROW);
  if (r) return r;
  return launch_persistent<PlCfg<BN, ROW>, false>(d, A, B, C, maps, st);
}

// hybrid: B' planes through TMA, A split on chip
int run_tc_hybrid(const GemmDesc& d, const float2* A, const float2* B, float* C, uint8_t* scratch, cudaStream_t st) {
  PlMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  int r = prep_planes<false>(d, A, B, scratch, 256, maps, st, HyCfg::kRowBytes, false);
  if (r) return r;
  return launch_persistent<HyCfg, false>(d, A, B, C, maps, st);
}

template <bool kTF32, int BN, int STAGES>
int run_tc(const GemmDesc& d, const float2* A, const float2* B, float* C, uint8_t* scratch, cudaStream_t st,
           int ksplit = 1) {
  const int64_t M = d.M, N2 = 2 * d.N, K2 = 2 * d.K, nb = d.batch;
  PlMaps maps;
  int r = prep_planes<kTF32>(d, A, B, scratch, BN, maps, st);
  if (r) return r;
  // K split over CTAs: FP32 partial tiles after the planes in the scratch,
  // summed (in FP64) into C in the consumer's layout by splitk_reduce
  float* part = nullptr;
  OutMap om = out_map(d);
  const int64_t nout = nb * M * d.N;  // complex outputs
  if (ksplit > 1) {
    const uint64_t es = kTF32 ? 4 : 2;
    const uint64_t planes = (uint64_t)nb * (M * K2 * 2 + N2 * K2 * 2) * es;
    const uint64_t off = (planes + 255) / 256 * 256;
    if (off + (uint64_t)ksplit * nout * 8 > d.scratch_elems * 8) return (int)cudaErrorInvalidValue;
    part = (float*)(scratch + off);
    om.ident = 1;
  }
  const CUtensorMap &mAh = maps.ah, &mAl = maps.al, &mBh = maps.bh, &mBl = maps.bl;
  constexpr uint32_t STAGE_BYTES = 2 * BM * 128 + 2 * BN * 128;
  const size_t smem = 1024 + STAGES * STAGE_BYTES + (2 * STAGES + 5) * 8 + 16 + BN / 2 * 8;
  static std::atomic<int> attr_done[kMaxDevices];
  if (int e = smem_attr_once(attr_done, tc_gemm_kernel<kTF32, BN, STAGES>, (int)smem)) return e;
  const int64_t tiles = (M / BM) * (N2 / BN);
  for (int64_t b0 = 0; b0 < nb; b0 += 65535) {
    int64_t cnt = nb - b0 < 65535 ? nb - b0 : 65535;
    dim3 grid((unsigned)tiles, 1, (unsigned)cnt);
    grid.y = (unsigned)ksplit;
    tc_gemm_kernel<kTF32, BN, STAGES><<<grid, TcShape<BN>::kThreads, smem, st>>>(
        mAh, mAl, mBh, mBl, part ? part : C, (int)M, (int)N2, (int)K2, (int)b0, om, ksplit, 2 * nout);
  }
  if (ksplit > 1) launch_splitk_reduce((const float2*)part, (float2*)C, ksplit, nout, M, d.N, out_map(d), st);
  return (int)cudaGetLastError();
}

}  // namespace

// Shapes reaching here are powers of two with M >= 128, N >= 32, K >= 32
// (checked again below); the scratch holds the four planes.
int launch_tc_gemm(const GemmDesc& d, const float2* A, const float2* B, float2* C, void* scratch_ptr,
                   cudaStream_t st) {
  // every epilogue may store 16 bytes at a time (plain layouts, column pairs):
  // the output must be 16-byte aligned (the plans' workspace offsets are
  // 256-byte aligned; a caller's misaligned buffer is refused, not faulted)
  if ((uintptr_t)C & 15) return (int)cudaErrorInvalidValue;
  // the persistent plane tiles (9, 10) also take short K (a power of two
  // >= 4): TMA fills the k-block beyond the plane rows with zeros
  const bool short_k = (((d.tile >= 9 && d.tile <= 12) || (d.tile == 13 && d.K >= 16)) && d.K >= 4 && d.K < 32 &&
                        !(d.K & (d.K - 1))) ||
                       (d.tile >= 16 && d.tile <= 18 && d.K >= 2 && d.K < 32 && !(d.K & 1));
  if (d.M < BM || d.N < 32 || (d.K < 32 && !short_k) || (d.M % BM) || (d.N % 32) || (d.K % 32 && !short_k) ||
      d.M > (1 << 30) || 2 * d.N > (1 << 30) || 2 * d.K > (1 << 30))
    return (int)cudaErrorInvalidValue;
  const bool tf32 = d.form == TNC_3XTF32;
  const int tile = d.tile ? d.tile : (d.N >= 64 ? 2 : 1);
  if (tile >= 16 && tile <= 18) {  // no scratch
    // split on chip from FP32 tiles by TMA: K-major, 16-byte aligned, K even;
    // 18: 256 columns, K <= 256
    const int bn = tile == 16 ? 64 : (tile == 17 ? 128 : 256);
    if (tf32 || d.transA || !d.transB || 2 * d.N < bn || (2 * d.N) % bn || (d.K & 1) || (tile == 18 && d.K > 256) ||
        ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
      return (int)cudaErrorInvalidValue;
    if (tile == 16 && ft_launchable<64>()) return run_tc_ft<64>(d, A, B, (float*)C, st);
    if (tile == 17 && ft_launchable<128>()) return run_tc_ft<128>(d, A, B, (float*)C, st);
    if (tile == 18 && ft_launchable<256>()) return run_tc_ft<256>(d, A, B, (float*)C, st);
    return (int)cudaErrorInvalidValue;
  }
  const uint64_t es = tf32 ? 4 : 2;
  const uint64_t need = (uint64_t)d.batch * (d.M * 2 * d.K * 2 + 2 * d.N * 2 * d.K * 2) * es;
  if (need > d.scratch_elems * 8) return (int)cudaErrorInvalidValue;
  uint8_t* scratch = (uint8_t*)scratch_ptr;
  if (!scratch) return (int)cudaErrorInvalidValue;
  // tile 1: 128 x 64 real outputs per CTA, 2: 128 x 128, 3: 128 x 256;
  // 4, 5: 128 x 128, 6, 7: 128 x 64 and 8: 128 x 256 (K <= 256) with the
  // split done on chip (split-BF16, K-major operands), 5 and 7 with an L2
  // prefetch of the k-block after next; 9: 128 x 256 (K <= 256) and
  // 10: 128 x 128, persistent from the planes (split-BF16); 11: as 9 with
  // 64-byte rows and two staging blocks per epilogue step; 12: 128 x 64;
  // 13: 128 x 256 (K <= 256) with A split on chip and B' from its planes;
  // 14, 15: 128 x 256 split on chip for any K (one TMEM slot + running sum),
  // 15 with the L2 prefetch
  if (tile == 19) {
    // plane tiles with K split over CTAs, for nodes with few output tiles
    // and long K (K a multiple of 32)
    if (d.K < 32 || d.K % 32 || d.M % BM || d.N < 32) return (int)cudaErrorInvalidValue;
    const int bn = d.N >= 64 ? 128 : 64;
    const int64_t tiles = (d.M / BM) * (2 * d.N / bn) * d.batch;
    const int64_t nk = 2 * d.K / (tf32 ? 32 : 64);
    int64_t ks = 2 * (int64_t)sm_count() / (tiles > 0 ? tiles : 1);
    if (ks > nk) ks = nk;
    if (ks > 65535) ks = 65535;
    if (ks < 1) ks = 1;
    if (tf32) return bn == 128 ? run_tc<true, 128, 3>(d, A, B, (float*)C, scratch, st, (int)ks)
                               : run_tc<true, 64, 4>(d, A, B, (float*)C, scratch, st, (int)ks);
    return bn == 128 ? run_tc<false, 128, 3>(d, A, B, (float*)C, scratch, st, (int)ks)
                     : run_tc<false, 64, 4>(d, A, B, (float*)C, scratch, st, (int)ks);
  }
  if (tile < 1 || tile > 15 || (tile == 2 && d.N < 64) || (tile == 3 && d.N < 128) ||
      (tile >= 4 && tile <= 8 && (d.transA || !d.transB)) || (tile >= 4 && tf32) ||
      ((tile == 4 || tile == 5 || tile == 10) && d.N < 64) ||
      ((tile == 8 || tile == 9 || tile == 11) && (d.N < 128 || d.K > 256)))
    return (int)cudaErrorInvalidValue;
  if (tile == 9) return run_tc_planes<256, 128>(d, A, B, (float*)C, scratch, st);
  if (tile == 10) return run_tc_planes<128, 128>(d, A, B, (float*)C, scratch, st);
  if (tile == 11) return run_tc_planes<256, 64>(d, A, B, (float*)C, scratch, st);
  if (tile == 12) return run_tc_planes<64, 128>(d, A, B, (float*)C, scratch, st);
  if (tile == 14 || tile == 15) {
    // 256 columns split on chip, any K (a multiple of 16)
    if (tf32 || d.transA || !d.transB || d.N < 128 || d.K % 16) return (int)cudaErrorInvalidValue;
    if (((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0 && fused_launchable<256>()) {
      PlMaps none;
      std::memset(&none, 0, sizeof(none));
      return tile == 15 ? launch_persistent<FzWideCfg, true>(d, A, B, (float*)C, none, st)
                        : launch_persistent<FzWideCfg, false>(d, A, B, (float*)C, none, st);
    }
    return run_tc<false, 128, 3>(d, A, B, (float*)C, scratch, st);
  }
  if (tile == 13) {
    // A split on chip: K-major, 16-byte aligned, K a multiple of 16
    if (tf32 || d.transA || d.N < 128 || d.K > 256 || d.K % 16 || ((uintptr_t)A & 15))
      return (int)cudaErrorInvalidValue;
    return run_tc_hybrid(d, A, B, (float*)C, scratch, st);
  }
  if (tile >= 4) {
    const bool aligned = ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0;
    if (aligned && tile <= 5 && fused_launchable<128>())
      return tile == 5 ? run_tc_fused<128, true>(d, A, B, (float*)C, st)
                       : run_tc_fused<128, false>(d, A, B, (float*)C, st);
    if (aligned && (tile == 6 || tile == 7) && fused_launchable<64>())
      return tile == 7 ? run_tc_fused<64, true>(d, A, B, (float*)C, st)
                       : run_tc_fused<64, false>(d, A, B, (float*)C, st);
    if (aligned && tile == 8 && fused_launchable<256>()) return run_tc_fused<256, false>(d, A, B, (float*)C, st);
    // unaligned operands: through the planes
    return d.N >= 64 ? run_tc<false, 128, 3>(d, A, B, (float*)C, scratch, st)
                     : run_tc<false, 64, 4>(d, A, B, (float*)C, scratch, st);
  }
  if (tf32) {
    if (tile == 3) return run_tc<true, 256, 2>(d, A, B, (float*)C, scratch, st);
    if (tile == 2) return run_tc<true, 128, 3>(d, A, B, (float*)C, scratch, st);
    return run_tc<true, 64, 4>(d, A, B, (float*)C, scratch, st);
  }
  if (tile == 3) return run_tc<false, 256, 2>(d, A, B, (float*)C, scratch, st);
  if (tile == 2) return run_tc<false, 128, 3>(d, A, B, (float*)C, scratch, st);
  return run_tc<false, 64, 4>(d, A, B, (float*)C, scratch, st);
}

// ------------------------------------------------------------------ narrow nodes staged by TMA
// The narrow node (N <= 16 complex columns, K = 8 or 16, A K-major [b][M][K],
// B [b][N][K], FP32 on the CUDA cores) with its A rows brought into shared
// memory by TMA: one 256-row tile (64 or 128 bytes a row) per box, swizzled
// (64- or 128-byte pattern) so that each thread's 16-byte reads of its own row
// are free of bank conflicts, in a ring of stages refilled as soon as every
// thread holds its row.  The loads of a warp then move whole contiguous tiles
// instead of one scattered 16-byte piece of 32 rows each, which set the pace
// of the kernel that reads its rows from global memory.  One thread a row; B
// in shared memory with two columns per 16-byte word as (b0.x, b1.x, b0.y,
// b1.y), so the packed FP32 FMAs take both column pairs straight from the
// loaded word: per component they are exactly the FMAs of cmul_add in its
// order (bit-identical to the other CUDA-core kernels).  Each CTA takes a
// contiguous range of tiles (B reloaded when the batch changes); every wait is
// bounded (a timeout sets tc_error_flag, all threads leave together after
// thread 0 has waited, bounded, for the copies still in flight).
constexpr int kNtRows = 256;  // rows per tile = threads per CTA

template <int K>
struct NtCfg {
  static constexpr int kRowBytes = K * 8;  // 64 or 128
  static constexpr int kStages = K == 16 ? 3 : 4;
  static constexpr uint32_t kTileBytes = kNtRows * kRowBytes;
  static constexpr int kSmem = kStages * (int)kTileBytes + 1024;  // + slack to align the swizzle atoms
  static constexpr int kCtasPerSm = K == 16 ? 2 : 3;               // by shared memory (97 / 65 KB a CTA)
};

template <int K>
__device__ __forceinline__ int nt_chunk(int row, int c) {
  return K == 16 ? (c ^ (row & 7)) : (c ^ ((row >> 1) & 3));
}

template <int K, int N>
__global__ void __launch_bounds__(kNtRows, 2)
    cgemm_narrow_tma_kernel(const __grid_constant__ CUtensorMap mA, const float2* __restrict__ B,
                            float2* __restrict__ C, int64_t M, int64_t n_tiles, const __grid_constant__ OutMap om) {
  static_assert(K == 8 || K == 16, "K");
  static_assert(N >= 2 && N <= 16, "N");
  using Cfg = NtCfg<K>;
  constexpr int NP = N / 2;
  constexpr int S = Cfg::kStages;
  extern __shared__ uint8_t nt_dyn[];
  __shared__ float4 Bq[K * NP];  // Bq[k][p] = (b[2p][k].x, b[2p+1][k].x, b[2p][k].y, b[2p+1][k].y)
  __shared__ uint64_t coff[N];
  __shared__ __align__(8) uint64_t full[S];
  uint8_t* tiles = nt_dyn + ((1024u - (smem_u32(nt_dyn) & 1023u)) & 1023u);
  const int tid = threadIdx.x;
  const int64_t tiles_m = M / kNtRows;
  const int64_t per = n_tiles / gridDim.x, extra = n_tiles % gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per + ((int64_t)blockIdx.x < extra ? blockIdx.x : extra);
  const int64_t nt = per + ((int64_t)blockIdx.x < extra ? 1 : 0);
  if (tid < N) coff[tid] = om.col(tid);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int j = 0; j < S && j < nt; ++j) {
      const int64_t t = t0 + j;
      mbar_expect_tx(&full[j], Cfg::kTileBytes);
      tma_load_3d(tiles + j * Cfg::kTileBytes, &mA, &full[j], 0, (int)((t % tiles_m) * kNtRows), (int)(t / tiles_m));
    }
  }
  int64_t cur_b = -1;
  int64_t failed_at = -1;
  for (int64_t j = 0; j < nt; ++j) {
    const int64_t t = t0 + j;
    const int64_t bz = t / tiles_m;
    if (bz != cur_b) {  // the same for every thread of the CTA
      __syncthreads();  // (also orders the barrier set-up before the first waits)
      const float2* Bb = B + bz * (int64_t)K * N;
      for (int e = tid; e < K * NP; e += kNtRows) {
        const int k = e / NP, p = e % NP;
        const float2 x = Bb[(int64_t)(2 * p) * K + k];
        const float2 y = Bb[(int64_t)(2 * p + 1) * K + k];
        Bq[e] = make_float4(x.x, y.x, x.y, y.y);
      }
      __syncthreads();
      cur_b = bz;
    }
    const int s = (int)(j % S);
    const bool ok = mbar_wait(&full[s], (uint32_t)((j / S) & 1));
    float2 ax[K], ay[K], an[K];  // (a.x, a.x), (a.y, a.y), (-a.y, -a.y)
    if (ok) {
      const uint8_t* rowp = tiles + s * Cfg::kTileBytes + tid * Cfg::kRowBytes;
#pragma unroll
      for (int c = 0; c < K / 2; ++c) {
        const float4 v = *(const float4*)(rowp + (nt_chunk<K>(tid, c) << 4));
        ax[2 * c] = make_float2(v.x, v.x);
        ay[2 * c] = make_float2(v.y, v.y);
        an[2 * c] = make_float2(-v.y, -v.y);
        ax[2 * c + 1] = make_float2(v.z, v.z);
        ay[2 * c + 1] = make_float2(v.w, v.w);
        an[2 * c + 1] = make_float2(-v.w, -v.w);
      }
    }
    // the stage is rewritten next by TMA (the async proxy): order this
    // thread's reads of it before that write, then meet at the barrier
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
      failed_at = j;
      break;
    }
    // every thread holds its row: refill the stage
    if (tid == 0 && j + S < nt) {
      const int64_t tn = t + S;
      mbar_expect_tx(&full[s], Cfg::kTileBytes);
      tma_load_3d(tiles + s * Cfg::kTileBytes, &mA, &full[s], 0, (int)((tn % tiles_m) * kNtRows), (int)(tn / tiles_m));
    }
    const int64_t m = (t % tiles_m) * kNtRows + tid;
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
      C[roff + coff[2 * p + 1]] = make_float2(re.y, im.y);
    }
  }
  if (failed_at >= 0 && tid == 0) {
    atomicExch(&tc_error_flag, 9);
    // tiles failed_at .. failed_at + S - 1 were issued and not consumed
    for (int64_t j = failed_at; j < failed_at + S && j < nt; ++j)
      mbar_wait(&full[j % S], (uint32_t)((j / S) & 1));
  }
}

// The TMA-staged narrow kernel for this node, or kNtNotEligible when its
// shape or layout does not fit (A K-major and 16-byte aligned, B [b][N][K],
// K in {8, 16}, N in {2, 4, 8, 16}, M a multiple of 256).
constexpr int kNtNotEligible = -1;

template <int K, int N>
int launch_narrow_tma_kn(const GemmDesc& d, const float2* A, const float2* B, float2* C, cudaStream_t st) {
  using Cfg = NtCfg<K>;
  static std::atomic<int> attr_done[kMaxDevices];
  if (int e = smem_attr_once(attr_done, cgemm_narrow_tma_kernel<K, N>, Cfg::kSmem)) return e;
  CUtensorMap m;
  if (int e = make_map(&m, (void*)A, true, 2 * K, d.M, d.batch, kNtRows, Cfg::kRowBytes)) return e;
  const int64_t n_tiles = d.batch * (d.M / kNtRows);
  int64_t grid = (int64_t)sm_count() * Cfg::kCtasPerSm;
  if (grid > n_tiles) grid = n_tiles;
  cgemm_narrow_tma_kernel<K, N><<<(unsigned)grid, kNtRows, Cfg::kSmem, st>>>(m, B, C, d.M, n_tiles, out_map(d));
  return (int)cudaGetLastError();
}

template <int K>
int launch_narrow_tma_k(const GemmDesc& d, const float2* A, const float2* B, float2* C, cudaStream_t st) {
  switch (d.N) {
    case 2: return launch_narrow_tma_kn<K, 2>(d, A, B, C, st);
    case 4: return launch_narrow_tma_kn<K, 4>(d, A, B, C, st);
    case 8: return launch_narrow_tma_kn<K, 8>(d, A, B, C, st);
    case 16: return launch_narrow_tma_kn<K, 16>(d, A, B, C, st);
    default: return kNtNotEligible;
  }
}

int launch_narrow_tma(const GemmDesc& d, const float2* A, const float2* B, float2* C, cudaStream_t st) {
  if (d.transA || !d.transB || ((uintptr_t)A & 15) || d.M < kNtRows || d.M % kNtRows || d.batch < 1 ||
      d.M > ((int64_t)1 << 31) || d.batch > ((int64_t)1 << 31))
    return kNtNotEligible;
  if (d.K == 16) return launch_narrow_tma_k<16>(d, A, B, C, st);
  if (d.K == 8) return launch_narrow_tma_k<8>(d, A, B, C, st);
  return kNtNotEligible;
}

int read_tc_error(int* flag) {
  return (int)cudaMemcpyFromSymbol(flag, tc_error_flag, sizeof(int));
}

int bounded_wait_selftest(uint64_t limit_ns, int* timed_out) {
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  bounded_wait_selftest_kernel<<<1, 1>>>(limit_ns, d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(timed_out, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return (int)e;
}

// Loads every kernel of this file onto the current device (see
// preload_kernels_core in kernels.cu).
int preload_kernels_tc() {
  const void* fns[] = {
      (const void*)tc_gemm_kernel<true, 256, 2>,
      (const void*)tc_gemm_kernel<true, 128, 3>,
      (const void*)tc_gemm_kernel<true, 64, 4>,
      (const void*)tc_gemm_kernel<false, 256, 2>,
      (const void*)tc_gemm_kernel<false, 128, 3>,
      (const void*)tc_gemm_kernel<false, 64, 4>,
      (const void*)tc_fused_bf16_kernel<FzCfg<128>, false>,
      (const void*)tc_fused_bf16_kernel<FzCfg<128>, true>,
      (const void*)tc_fused_bf16_kernel<FzCfg<64>, false>,
      (const void*)tc_fused_bf16_kernel<FzCfg<64>, true>,
      (const void*)tc_fused_bf16_kernel<FzCfg<256>, false>,
      (const void*)tc_fused_bf16_kernel<FzWideCfg, false>,
      (const void*)tc_fused_bf16_kernel<FzWideCfg, true>,
      (const void*)tc_fused_bf16_kernel<HyCfg, false>,
      (const void*)tc_fused_bf16_kernel<PlCfg<256, 128>, false>,
      (const void*)tc_fused_bf16_kernel<PlCfg<128, 128>, false>,
      (const void*)tc_fused_bf16_kernel<PlCfg<256, 64>, false>,
      (const void*)tc_fused_bf16_kernel<PlCfg<64, 128>, false>,
      (const void*)tc_fused_bf16_kernel<FtCfg<64>, false>,
      (const void*)tc_fused_bf16_kernel<FtCfg<128>, false>,
      (const void*)tc_fused_bf16_kernel<FtCfg<256>, false>,
      (const void*)prep_a_kernel<false>,
      (const void*)prep_a_kernel<true>,
      (const void*)prep_b_kernel<false>,
      (const void*)prep_b_kernel<true>,
      (const void*)prep_a_vec_kernel<false>,
      (const void*)prep_a_vec_kernel<true>,
      (const void*)prep_b_vec_kernel<false>,
      (const void*)prep_b_vec_kernel<true>,
      (const void*)cgemm_narrow_tma_kernel<16, 2>,
      (const void*)cgemm_narrow_tma_kernel<16, 4>,
      (const void*)cgemm_narrow_tma_kernel<16, 8>,
      (const void*)cgemm_narrow_tma_kernel<16, 16>,
      (const void*)cgemm_narrow_tma_kernel<8, 2>,
      (const void*)cgemm_narrow_tma_kernel<8, 4>,
      (const void*)cgemm_narrow_tma_kernel<8, 8>,
      (const void*)cgemm_narrow_tma_kernel<8, 16>,
  };
  cudaFuncAttributes fa;
  for (const void* f : fns) {
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

}  // namespace tnc
