// Plain descriptors passed from the host plan compiler to the CUDA kernels,
// and the host-callable launchers (implemented in kernels.cu / tc_gemm.cu).
//
// Every tensor is a dense row-major array of 2^rank complex64 values whose
// indices are all binary: a tensor index is a bit of the linear offset.  Bit
// j of an offset is counted from the least significant end (bit 0 = the last,
// fastest-varying index).
#pragma once
#include <cstddef>
#include <cstdint>

namespace tnc {

constexpr int kMaxRank = 48;

// Gather of one derived leaf from its base leaf: output bit j comes from
// base bit out_src[j] (>= 0), or is bit b of the bitstring index beta when
// out_src[j] = -1 - b.  Base bits not fed by an output bit are fixed: a final
// wire of qubit q takes bits[beta][q]; a sliced bond takes bit k of the
// slice-group counter.
struct GatherDesc {
  uint64_t src;          // element offset of the base leaf (plan buffer)
  uint64_t dst;          // element offset of the derived leaf (workspace)
  int out_rank;
  int n_fixed;
  int n_sliced;
  int src_rank;
  int8_t out_src[32];
  int8_t fixed_pos[4];
  int16_t fixed_qubit[4];
  int8_t sliced_pos[24];
  int8_t sliced_bit[24];
};

// out[j] = in[i] where bit k of i is bit src_bit^-1 ... stated directly:
// for every output offset j, input offset i has bit src_bit[k] equal to bit
// k of j (k < rank).
struct PermDesc {
  uint64_t src, dst;     // element offsets in the workspace
  int rank;
  int8_t src_bit[kMaxRank];
};

// C[b][m][n] = sum_k A[b][m][k] B[b][k][n]; A stored [b][K][M] if transA,
// B stored [b][N][K] if transB; C stored [b][M][N].  Buffers: 0 = workspace,
// 1 = plan leaf buffer.
struct GemmDesc {
  uint64_t a, b, c;
  int64_t batch, M, N, K;
  int transA, transB;
  int a_buf, b_buf;
  int kernel;            // kernel variant chosen by the compiler / autotuner
  int form;              // TNC_FP32 / TNC_3XTF32 / TNC_SPLIT_BF16
  uint64_t scratch;      // workspace element offset of per-node scratch (0 if none)
  uint64_t scratch_elems;
  int splitk;            // CUDA-core kernels: K split into this many FP32 chunks summed in FP64
  // Output layout.  c_ident: C stored [b][M][N].  Otherwise element (b, m, n)
  // is stored at sum_i bit_i(n) << c_pos[i] + sum_i bit_i(m) << c_pos[nN + i]
  // + sum_i bit_i(b) << c_pos[nN + nM + i] (M, N, batch powers of two with
  // nN = log2 N, nM = log2 M, nB = log2 batch): the layout the consumer reads.
  int c_ident;
  int nN, nM, nB;
  int8_t c_pos[kMaxRank];
  int tile;              // tensor-core tile width: 0 auto, 1 N = 64 real columns, 2 N = 128, 3 N = 256,
                        // 4, 5 N = 128, 6, 7 N = 64 and 8 N = 256 (K <= 256) with the
                        // split-BF16 split on chip (5, 7: with prefetch); 9 N = 256
                        // (K <= 256), 10 N = 128, 11 N = 256 with 64-byte rows, 12 N = 64:
                        // persistent from the planes (9-12 also for K = 4..16); 13 N = 256
                        // (K <= 256): A split on chip, B' from its planes; 14, 15 N = 256 split
                        // on chip for any K (one TMEM slot + running sum; 15: with prefetch);
                        // 16 N = 64, 17 N = 128, 18 N = 256 (K <= 256): split on chip from FP32
                        // tiles that TMA streams into a shared-memory ring (K even, also < 32);
                        // 19: the plane tiles (N = 128, or 64 when N < 64 complex) with K split
                        // over CTAs and an FP64 sum of the partials, for few tiles and long K.
                        // Narrow kernel: 0 unrolled for K, N in {1, 2, 4, 8, 16} with packed FP32
                        // FMAs (K-major A; else as 1), 1 one row per thread, 2 tiled with the output
                        // staged in address order (powers of two, K-major A; else as 1), 3 A tiles
                        // staged in shared memory by TMA (K in {8, 16}, N in {2, 4, 8, 16}, M a
                        // multiple of 256, K-major A; else as 0)
};

// One problem of a grouped launch of narrow nodes (N, K <= 16): the same
// contraction as a GemmDesc with the narrow kernel, A [b][M][K], B [b][N][K].
// first_block: prefix sum of the blocks of the earlier problems.
struct GroupedDesc {
  uint64_t a, b, c;      // element offsets (a_buf/b_buf: 0 workspace, 1 leaf buffer)
  int64_t M;
  int N, K, batch;
  int a_buf, b_buf;
  int c_ident, nN, nM, nB;
  int blocks_per_batch;
  int8_t c_pos[kMaxRank];
  int64_t first_block;
  // buffers of this problem when it belongs to another request than the
  // launch's (cross-request grouping); NULL: the launch's ws / leaf buffer
  const void* ws_ptr;
  const void* base_ptr;
};

// One problem of a grouped CUDA-core cGEMM launch (grouped_simt_kernel): a
// node of any request, by absolute pointers, without split-K.
// first_block: prefix sum of the blocks (tiles x batch) of the earlier problems.
struct SimtProblem {
  const void* A;
  const void* B;
  void* C;
  int64_t M, N, K;
  int transA, transB;
  int staged;            // full tiles of a scattered output: staged epilogue (rank below)
  int ident, nN, nM, nB;
  int8_t c_pos[kMaxRank];
  int8_t rank[kMaxRank]; // staged epilogue: rank of each tile bit's output position
  int64_t first_block;
};

// Final accumulation: out[beta][j] += sum over the bits of the grouped
// slices of root[...]; root bit k is beta bit (role 0, idx), open bit (role
// 1, idx) or a grouped-slice bit (role 2, idx).
struct AccumDesc {
  uint64_t src;
  int rank;
  int n_beta, n_open, n_par;
  int8_t role[kMaxRank];
  int8_t idx[kMaxRank];
};

// ---------------------------------------------------------------- launchers
// Each returns 0 on success or a cudaError_t value.
int launch_gather(const GatherDesc* d_descs, int n_descs, int max_out_rank, const void* base,
                  void* ws, const uint8_t* d_bits, int n_qubits, const uint64_t* d_slice_ctr,
                  void* stream);
int launch_permute(const PermDesc& d, void* ws, void* stream);
int launch_permute_ptr(const PermDesc& d, const void* in, void* out, void* stream);
int launch_gemm(const GemmDesc& d, const void* base, void* ws, void* stream);
int launch_gemm_ptr(const GemmDesc& d, const void* A, const void* B, void* C, void* scratch, void* stream);

// kernel variant, split-K and scratch size of a GEMM node (shared by the
// plan compiler and the kernel-level entry points)
void choose_gemm_kernel(GemmDesc& g);
uint64_t gemm_scratch_bytes(const GemmDesc& g);
// every kernel variant that can run this node (the default choice first)
void gemm_candidates(const GemmDesc& g, GemmDesc* out, int* n);
constexpr int kMaxCandidates = 24;
int launch_accum(const AccumDesc& d, const void* ws, void* d_out, int batch, void* stream);
int launch_grouped_narrow(const GroupedDesc* d_descs, int n, int64_t total_blocks, const void* base, void* ws,
                          void* stream);
int launch_zero(void* ptr, size_t bytes, void* stream);
// grouped CUDA-core cGEMM over problems of one tile shape (kernel = KG_SIMT_*)
int launch_grouped_simt(const SimtProblem* d_probs, int n, int64_t total_blocks, int kernel, void* stream);
// BM x BN tile of a CUDA-core kernel variant (-1 if not one)
int simt_tile_shape(int kernel, int* bm, int* bn);
// SM count of the current device (152, a GB300's, when there is none)
int sm_count();
int launch_set_counter(uint64_t* d_ctr, uint64_t value, void* stream);

// kernel variants of launch_gemm
enum GemmKernel {
  KG_SIMT_128x64 = 0,   // register-tiled CUDA-core cGEMM
  KG_SIMT_64x32 = 1,
  KG_NARROW = 2,        // one output row per thread, B in shared memory
  KG_DOT = 3,           // split-K reduction for tiny outputs (FP64 across threads)
  KG_TC = 4,            // tcgen05 tensor-core cGEMM (3xTF32 / split-BF16)
  KG_SIMT_32x128 = 5,
  KG_COUNT
};

}  // namespace tnc
