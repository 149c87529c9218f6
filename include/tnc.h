/*
 * tnc.h -- C ABI of the GB300 tensor-network amplitude executor.
 *
 * The executor computes quantum-circuit amplitudes <x| C |0...0> by
 * contracting the circuit's tensor network along a contraction tree found by
 * the separator method of Wahl & Strelchuk, "Simulating quantum circuits using
 * efficient tensor network contraction algorithms with subexponential upper
 * bound" (arXiv 2208.01498):
 *
 *   - the network is the one of the "Classical Simulation of Quantum
 *     Circuits" section: two-qubit gates are rank-4 tensors, single-qubit
 *     gates and the boundary vectors are absorbed into them, and each
 *     two-qubit gate is split by an SVD into two rank-3 tensors joined by a
 *     bond (proof of Thm. 2);
 *   - the tree is the separator hierarchy of the proof of Thm. 1, built with
 *     the Sphere Separator Algorithm (Algorithm 1, Supplemental Material),
 *     with greedy contraction of the bottom clusters ("Numerical
 *     implementation" section); index slicing (named as future work in the
 *     Conclusion) bounds its memory;
 *   - every tree node is a pairwise contraction costing 2 M scalar operations,
 *     M the product of the dimensions of all indices of both operands
 *     (Eq. 3); the executor runs each node on one GPU as a complex GEMM.
 *
 * Conventions.  Qubit q has coordinates coords[q*dim .. q*dim+dim).  A gate
 * matrix is row-major complex (interleaved re, im), rows = outputs; a
 * two-qubit gate on (a, b) acts on |x_a x_b> with x_a the most significant
 * bit.  A bitstring is n_qubits bytes, entry q = value (0/1) of qubit q.
 * Amplitudes are complex128 out[b][j] (interleaved re, im); bit i of j is the
 * value of open qubit open_qubits[i] after they are sorted ascending.
 *
 * Errors.  Every int-returning call returns TNC_OK (0) or a negative status;
 * tnc_last_error() describes the last failure of the calling thread.
 * Threading.  A plan may be used by one thread at a time; a server is
 * thread-safe.
 */
#ifndef TNC_H
#define TNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define TNC_OK 0
#define TNC_EINVAL (-1)   /* bad argument: qubit, gate shape, sizes, NULL */
#define TNC_ENOMEM (-2)   /* plan over mem_cap even after slicing, or ws too small */
#define TNC_ECUDA (-3)    /* a CUDA runtime call failed */
#define TNC_ETIMEOUT (-4) /* a bounded device or host wait gave up */
#define TNC_EBUSY (-5)    /* admission refused: server full */
#define TNC_ESTATE (-6)   /* call not valid in the object's current state */
#define TNC_ENOTFOUND (-7)/* unknown server ticket */

/* contraction forms (precision of the pairwise contractions) */
#define TNC_FP32 0        /* complex64 in/out, FP32 CUDA-core products  */
#define TNC_3XTF32 1      /* hi/lo TF32 split, 3 products, tensor cores */
#define TNC_SPLIT_BF16 2  /* hi/lo BF16 split, 3 products, tensor cores */

typedef struct tnc_network tnc_network_t;
typedef struct tnc_plan tnc_plan_t;
typedef struct tnc_server tnc_server_t;

/* A circuit as plain data.  The library copies everything it needs. */
typedef struct {
  int n_qubits;          /* >= 1 */
  int dim;               /* embedding dimension of the qubit layout, 1..3 */
  const double* coords;  /* [n_qubits][dim] */
  int n_gates;           /* >= 0, in time order */
  const int* arity;      /* [n_gates], each 1 or 2 */
  const int* qubits;     /* concatenated qubit lists, sum(arity) entries */
  const double* mats;    /* concatenated row-major 2x2 / 4x4 complex, FP64 */
} tnc_network_desc;

typedef struct {
  int n_open;               /* number of open output qubits (<= 20) */
  const int* open_qubits;   /* [n_open], any order, distinct */
  int max_batch;            /* bitstrings per call, 1..65536 (rounded up to 2^k) */
  size_t mem_cap_bytes;     /* cap on the workspace; 0 = no cap */
  int form;                 /* TNC_FP32, TNC_3XTF32 or TNC_SPLIT_BF16 */
  uint64_t seed;            /* seed of the randomised separator search */
  int ssa_trials;           /* great circles tried per separator (Alg. 1 step 7) */
  int leaf_size;            /* clusters of at most this many tensors are contracted greedily */
  int max_group_log2;       /* at most 2^k slices run together in one launch per node */
  int use_graph;            /* 1: replay each slice group as a captured CUDA graph */
  int embedding;            /* tensor positions given to the separator search: TNC_EMBED_AUTO (both
                               below, the tree with the smaller Eq. 3 cost is kept), TNC_EMBED_COLLAPSED
                               (time axis collapsed, the Thm. 2 proof) or TNC_EMBED_SPACETIME (the
                               (d+1)-dimensional network before the collapse, Fig. 1a; d <= 2 only) */
  int n_starts;             /* separator hierarchies built per embedding, with seeds seed, seed + 1, ...;
                               the one with the smallest Eq. 3 cost is kept (0 = 1) */
  int refine_window;        /* 0: the separator tree as built; 3..12: each tree is refined by exact
                               re-association of windows of up to this many subtrees (an addition to
                               the paper's method; it never raises the Eq. 3 cost nor enlarges the
                               largest intermediate) */
  int tree_only;            /* 1: build and report the contraction tree only (Eq. 3 cost in
                               tree_cost_log2 and paper_ops, n_leaves, max_rank; tnc_plan_export_json
                               gives the tree): no slicing and no device program, so networks whose
                               intermediates exceed the executor's 48 binary indices can be costed;
                               tnc_plan_upload and every contraction call return TNC_ESTATE */
} tnc_plan_opts;

#define TNC_EMBED_AUTO 0
#define TNC_EMBED_COLLAPSED 1
#define TNC_EMBED_SPACETIME 2

typedef struct {
  double paper_ops;     /* sum over nodes and slices of 2 M (Eq. 3) */
  double real_flops;    /* 8 M per node and slice: real FP32 flops of the complex products */
  double bytes;         /* sum over GEMM nodes and slices of 8 (|A| + |B| + |C|) */
  double peak_bytes;    /* largest live set of intermediates of one slice group */
  size_t ws_bytes;      /* workspace needed by tnc_contract_amplitudes */
  double n_slices;      /* total number of slices (2^|S|) */
  int n_slice_groups;   /* serial iterations (2^|S_serial|) */
  int n_sliced;         /* |S| */
  int n_nodes;          /* contraction steps per slice group */
  int n_leaves;         /* tensors of the network */
  int max_rank;         /* log2 of the largest intermediate (elements) */
  int n_launches;       /* kernel launches per slice group */
  double plan_ms;       /* host time spent planning */
  double tree_cost_log2;/* log2 of the unsliced tree's paper_ops */
  int embedding_used;   /* TNC_EMBED_COLLAPSED or TNC_EMBED_SPACETIME: the kept tree's embedding */
  int seed_used;        /* seed of the kept tree's separator search */
  double time_scale;    /* space-time embedding: distance between consecutive layers (lattice units) */
  double sep_cost_log2; /* log2 of the kept tree's paper_ops before refinement */
  int n_refined;        /* windows rebuilt by the refinement */
} tnc_plan_report;

/* Human-readable name of a status code. */
const char* tnc_status_string(int status);
/* Message of the last failure on the calling thread ("" if none). */
const char* tnc_last_error(void);

/* Build the tensor network of <x| C |0> (Classical Simulation section;
 * Thm. 2 proof for the SVD split).  desc and its arrays are only read during
 * the call.  *out is owned by the caller (tnc_free_network).
 * TNC_EINVAL for a qubit out of range, a repeated qubit in a gate, arity not
 * in {1, 2}, dim not in 1..3 or non-finite numbers. */
int tnc_load_network(const tnc_network_desc* desc, tnc_network_t** out);
void tnc_free_network(tnc_network_t* net);

/* Same as tnc_load_network, with build options.  TNC_NET_HYPEREDGES: every
 * gate that is diagonal in the computational basis (CZ, the Z and ZZ phases
 * of IQP circuits, any exactly diagonal 2x2 or 4x4 matrix) reads its wire
 * without changing it, D|z> = d(z)|z>, so it becomes a tensor of its diagonal
 * d on the wire labels (rank 1 or 2), and all diagonal gates between two
 * non-diagonal gates of a qubit share one wire label: a hyper-edge (copy
 * tensor) of the Classical Simulation section's network, as the bitstring
 * batch index is.  The pending non-diagonal single-qubit product of a qubit
 * becomes a rank-2 tensor of its own before such a label (or the vector
 * P|0> before the first one); non-diagonal two-qubit gates are split as in
 * tnc_load_network.  The amplitudes are the same; the plans differ.
 * TNC_EINVAL for unknown flags or an invalid desc. */
#define TNC_NET_HYPEREDGES 1
int tnc_load_network_opts(const tnc_network_desc* desc, int flags, tnc_network_t** out);

/* Fill *opts with defaults (no open qubits, batch 1, no cap, FP32, 32
 * trials, leaf size 8, group log2 6, CUDA graphs on, both embeddings, 4
 * starts per embedding, refinement windows of 8 subtrees). */
void tnc_plan_opts_default(tnc_plan_opts* opts);

/* ------------------------------------------------- planner primitives (host)
 * tnc_ssa_separate: one application of the Sphere Separator Algorithm
 * (Algorithm 1, Supplemental Material) to n spheres in R^dim (dim 1..3),
 * centres pos[n][dim], radii rad[n].  side[i] receives the class of sphere i
 * with respect to the separator kept: 0 inside (Gamma_I), 1 outside
 * (Gamma_E), 2 intersected (Gamma_O).  *valid = 1 if it satisfies Eqs. (1)
 * and (2) of the Sphere Separator Theorem (|Gamma_O| <= c_d k^(1/d)
 * n^(1-1/d), |Gamma_E|, |Gamma_I| <= (d+1)/(d+2) n), 0 if no trial did and a
 * fallback split was kept; *k receives the overlap number used in Eq. (1)
 * (most spheres containing one sphere centre). */
int tnc_ssa_separate(const double* pos, const double* rad, int n, int dim, uint64_t seed, int trials, int* side,
                     int* valid, int* k);

/* tnc_centerpoint: approximate centerpoint (Algorithm 1 step 2) of n points
 * in R^D (D <= 4), pts[n][D], by iterated Radon points; c[D] receives it. */
int tnc_centerpoint(const double* pts, int n, int D, uint64_t seed, double* c);

/* The paper's analytic cost bounds for a circuit (host only), all as log2
 * of a number of scalar operations for c = <0| U^dagger P U |0> (the doubled
 * network of the Classical Simulation section), beside which a plan's
 * tree_cost_log2 can be read.  From desc: N = n_qubits, d = dim, f(x_i) =
 * two-qubit gates on qubit i, F = max f, S = sum f, l = largest distance
 * between the qubits of a two-qubit gate, r = smallest distance between two
 * qubits, T = time steps (gates packed into layers as early as their qubits
 * allow).  Bounds that need d >= 2, a two-qubit gate or r > 0 are NaN
 * without them.  TNC_EINVAL for an invalid desc (as tnc_load_network). */
typedef struct {
  int n_qubits, dim, depth;   /* N, d, T */
  double sum_f, max_f;        /* S, F */
  double l, r;                /* gate range, qubit spacing */
  double n_tensors, k;        /* Thm. 2 proof: n = 2 S tensors, overlap k = 2 F (1 + l/r)^d */
  double a_d, a2_pst;         /* Thm. 1's a_d = c_d / (2 - 2 ((d+1)/(d+2))^(1-1/d)); a_2' with c_PST = 1.971 */
  double thm1_log2;           /* Thm. 1 at n, M = 16, k: 1 + log2(n) / log2((d+2)/(d+1)) + a_d k^(1/d) n^(1-1/d) log2 M */
  double thm2_log2;           /* Thm. 2: log2(2 S) / log2((d+2)/(d+1)) + 1 + 8 a_d (1 + l/r) F^(1/d) S^(1-1/d) */
  double thm2_pst_log2;       /* Thm. 2, d = 2 and l = r (PST): log2(W) / log2(3/2) + 1 + 4 a_2' sqrt(W),
                                 W = sum f (2 + f/2); NaN otherwise */
  double sidewise_log2;       /* left-to-right contraction: 1 + 4 F N^(1-1/d) + log2(N) / d */
  double explicit_log2;       /* explicit time evolution: log2(T N) + 2 + N */
} tnc_circuit_bounds;
int tnc_circuit_bounds_eval(const tnc_network_desc* desc, tnc_circuit_bounds* out);

/* Plan the contraction (host only, no GPU needed): separator hierarchies
 * (Thm. 1 proof, Algorithm 1) with greedy leaves over the embeddings and
 * seeds of opts, each refined if opts->refine_window asks, the cheapest tree
 * by Eq. 3 (with a cap: the cheapest after slicing among the four cheapest),
 * index slicing to meet mem_cap_bytes, and the compiled node program.  The
 * plan keeps what it needs from net; net may be freed afterwards.  rep may be
 * NULL.  TNC_ENOMEM if no slicing meets the cap, or an intermediate needs
 * more than the executor's 48 binary indices (set a cap to slice it);
 * TNC_EINVAL for bad options. */
int tnc_plan(const tnc_network_t* net, const tnc_plan_opts* opts, tnc_plan_t** out,
             tnc_plan_report* rep);
void tnc_free_plan(tnc_plan_t* plan);

/* Report of an existing plan. */
int tnc_plan_get_report(const tnc_plan_t* plan, tnc_plan_report* rep);

/* JSON description of the plan for host-side checks: leaves (labels and
 * FP64 values), tree nodes (children, output labels), sliced labels, batch
 * and open labels.  Writes at most cap bytes (NUL-terminated) into buf and
 * the full size (without NUL) into *needed.  buf may be NULL to query. */
int tnc_plan_export_json(const tnc_plan_t* plan, char* buf, size_t cap, size_t* needed);

/* Copy the plan's leaf tensors and node descriptors to the current CUDA
 * device (device memory owned by the plan, freed by tnc_free_plan).  Called
 * automatically by the first contraction if needed.  stream may be NULL.
 * For a plan whose workspace fits the static workspace of
 * tnc_contract_amplitudes_static (64 MiB), the first upload on a device also
 * loads every kernel of the library there and resolves that workspace's
 * address (the set-up that entry point relies on; a failure of it is not an
 * error of the upload). */
int tnc_plan_upload(tnc_plan_t* plan, void* cuda_stream);

/* Per-step CUDA-event profiling of the node program.  While enabled, every
 * contraction records one event before each slice group and one after each
 * step on the contraction's stream (no host synchronisation).  Disabling
 * drops the recorded events. */
int tnc_plan_set_profiling(tnc_plan_t* plan, int enable);

/* Aggregate of the recorded events (synchronises on them): for each of the
 * n = *n_steps steps of the program (n <= cap), the summed duration in ms
 * over all recorded runs, the number of runs, the kernel variant
 * (TNC_STEP_* below), and its algorithmic flops and bytes per launch
 * (8 M real flops per node, Eq. 3; 8 (|A|+|B|+|C|) bytes; a permutation
 * moves 16 bytes per element).  Arrays may be NULL to query n. */
#define TNC_STEP_PERMUTE 100
#define TNC_STEP_GROUPED 101
int tnc_plan_get_profile(tnc_plan_t* plan, int* n_steps, int cap, double* ms, int* runs, int* kind,
                         double* flops, double* bytes);

/* ------------------------------------------------- kernel-level entry points
 * The two steps of one tree node, callable on their own (for unit tests and
 * micro-benchmarks of the kernels).  All pointers DEVICE; enqueued on
 * cuda_stream; the device is the one owning the output pointer.
 *
 * tnc_permute: the index permutation of a node operand.  A dense complex64
 * tensor of 2^rank elements with binary indices (rank <= 40); out[j] = in[i]
 * where bit src_bit[k] of i equals bit k of j (bits counted from the least
 * significant end; src_bit a permutation of 0..rank-1).  d_in and d_out must
 * not overlap.  TNC_EINVAL for a bad permutation. */
int tnc_permute(const void* d_in, void* d_out, int rank, const int* src_bit, void* cuda_stream);

/* Scratch bytes tnc_cgemm (and tnc_cgemm_variant, any variant) needs for
 * this shape and form (0 if none). */
size_t tnc_cgemm_scratch_bytes(int64_t batch, int64_t M, int64_t N, int64_t K, int form);

/* tnc_cgemm: one pairwise contraction (Eq. 3: M_paper = batch*M*N*K
 * multiplications) as a batched complex GEMM,
 * C[b][m][n] = sum_k A[b][m][k] B[b][k][n], complex64 in and out; A stored
 * [b][M][K] ([b][K][M] if transA), B stored [b][K][N] ([b][N][K] if transB),
 * C stored [b][M][N].  form as in tnc_plan_opts; the kernel variant is chosen
 * by shape exactly as in a plan (tensor cores only for power-of-two shapes with
 * M >= 128, N >= 32, K >= 32).  d_scratch: scratch_bytes >=
 * tnc_cgemm_scratch_bytes(), 256-byte aligned (may be NULL if that is 0). */
int tnc_cgemm(const void* d_A, const void* d_B, void* d_C, int64_t batch, int64_t M, int64_t N, int64_t K,
              int transA, int transB, int form, void* d_scratch, size_t scratch_bytes, void* cuda_stream);

/* tnc_cgemm with the kernel variant named: kernel = TNC_KG_* below (-1: by
 * shape, as tnc_cgemm), tile = tensor-core tile width (1: 128 x 64 real
 * outputs per CTA, 2: 128 x 128, 3: 128 x 256; 4 and 5: 128 x 128, 6 and
 * 7: 128 x 64, 8: 128 x 256 (K <= 256), with the split-BF16 split done on
 * chip, persistent, for
 * K-major operands (transA = 0, transB = 1), 5 and 7 also prefetching the
 * k-block after next; these run through the hi/lo planes instead when an
 * operand is not 16-byte aligned; 9: 128 x 256 (K <= 256), 10: 128 x 128,
 * 11: 128 x 256 (K <= 256, 64-byte rows) and 12: 128 x 64, split-BF16 from
 * the hi/lo planes in a persistent kernel, also for K = 4, 8 or 16;
 * 13: 128 x 256 (K <= 256, transA = 0) with A split on chip and B' from its
 * planes; 14 and 15: 128 x 256 split on chip for any K (15 with prefetch),
 * K-major operands; -1: any; 0 for the other kernels).  The variants are those a plan's autotuner may pick for the
 * shape; TNC_EINVAL for one that cannot run it.  c_pos (HOST, may be NULL):
 * C stored in a consumer's bit order, as in a plan: with nN = log2 N,
 * nM = log2 M, nB = log2 batch (all powers of two), bit i of n goes to output
 * bit c_pos[i], bit i of m to c_pos[nN + i], bit i of b to c_pos[nN + nM + i];
 * c_pos must be a permutation of 0 .. nN + nM + nB - 1 (TNC_EINVAL otherwise).
 * NULL = [b][M][N]. */
#define TNC_KG_SIMT_128x64 0
#define TNC_KG_SIMT_64x32 1
#define TNC_KG_NARROW 2
#define TNC_KG_DOT 3
#define TNC_KG_TC 4
#define TNC_KG_SIMT_32x128 5
int tnc_cgemm_variant(const void* d_A, const void* d_B, void* d_C, int64_t batch, int64_t M, int64_t N, int64_t K,
                      int transA, int transB, int form, int kernel, int tile, const int* c_pos, void* d_scratch,
                      size_t scratch_bytes, void* cuda_stream);

/* Device-side error flag of the kernels with bounded waits (the tcgen05
 * pipeline): 0 if no wait has timed out on the current device since load,
 * else the code of the first timeout.  Synchronising read; *flag receives the
 * value; returns TNC_ETIMEOUT when it is set.  A set flag means the affected
 * contraction results are invalid. */
int tnc_device_error(int* flag);

/* Self-test of the bounded device wait the tcgen05 kernels use: one thread
 * waits on an mbarrier phase that nothing completes, for limit_us
 * microseconds (1 .. 10^6).  *timed_out receives 1 when the wait gave up (the
 * expected outcome; returns TNC_ETIMEOUT), 0 otherwise (TNC_OK).  Touches no
 * other state; the device stays usable.  Synchronous, on the current device.
 * The paper has no counterpart. */
int tnc_selftest_bounded_wait(unsigned limit_us, int* timed_out);

/* Autotuner: for every contraction step of the plan, time each kernel
 * variant that can run it on this GPU (tile shapes of the CUDA-core cGEMM,
 * the narrow and split-K kernels, the tensor-core tile widths of the 3xTF32
 * and split-BF16 forms), keep the fastest, and drop captured graphs.  Runs one
 * slice group on d_ws (contents are scratch; ws_bytes >= report.ws_bytes);
 * reps timed launches per variant (>= 1); synchronous.  *n_changed (may be
 * NULL) receives the number of steps whose kernel changed. */
int tnc_plan_autotune(tnc_plan_t* plan, void* d_ws, size_t ws_bytes, void* cuda_stream, int reps, int* n_changed);

/* Kernel choice of every step (for saving and restoring autotuner results):
 * choices[2 i] = kernel variant, choices[2 i + 1] = tensor-core tile width
 * of step i (grouped and permute steps report -1).  get: cap >= 2 * n_steps,
 * *n_steps receives the step count.  set: exactly the array get returns for
 * the same plan; TNC_EINVAL if a choice cannot run its step.  Setting drops
 * captured graphs. */
int tnc_plan_get_kernels(const tnc_plan_t* plan, int* choices, int cap, int* n_steps);
int tnc_plan_set_kernels(tnc_plan_t* plan, const int* choices, int n_steps);

/* Amplitudes for `batch` bitstrings (1 <= batch <= max_batch).
 * bits: HOST uint8 [batch][n_qubits]; entries of open qubits are ignored.
 * d_out: DEVICE complex128 [batch][2^n_open], caller-owned, overwritten.
 * d_ws: DEVICE workspace of ws_bytes >= report.ws_bytes, caller-owned,
 *       256-byte aligned; its contents are scratch.
 * Enqueued on cuda_stream (NULL = legacy default stream); asynchronous with
 * respect to the host except for the staging of bits, which is copied before
 * the call returns.  TNC_ENOMEM if ws_bytes is too small. */
int tnc_contract_amplitudes(tnc_plan_t* plan, const uint8_t* bits, int batch, void* d_out,
                            void* d_ws, size_t ws_bytes, void* cuda_stream);

/* Same, with bits already in DEVICE memory (uint8 [batch][n_qubits]). */
int tnc_contract_amplitudes_dbits(tnc_plan_t* plan, const uint8_t* d_bits, int batch,
                                  void* d_out, void* d_ws, size_t ws_bytes, void* cuda_stream);

/* Same as tnc_contract_amplitudes, for callers that cannot allocate device
 * memory when they need amplitudes (a host framework whose allocator owns all
 * device memory, a latency-bound request handler that may not call
 * cudaMalloc/cudaFree because they can synchronise the device, a plugin whose
 * host forbids allocation after start-up).  The paper has no
 * counterpart: this is a deployment variant of the same contraction.
 * The workspace is a 64 MiB array that the library holds statically on every
 * GPU that loads it, until exit; nothing is allocated by the call.
 * - The plan must already be resident on d_out's device (tnc_plan_upload),
 *   else TNC_ESTATE; profiling must be off, else TNC_ESTATE.
 * - A plan whose workspace (report.ws_bytes) exceeds 64 MiB: TNC_ENOMEM.
 * - Its set-up is done by tnc_plan_upload (which allocates anyway): for a
 *   plan whose workspace fits the array, the upload loads every kernel of
 *   the library onto the device and resolves the array's device address
 *   there, once per device.  Without it (with lazy module loading, the CUDA
 *   default) the first call would take device memory for the array and the
 *   kernels.  If that set-up failed, this call returns TNC_ESTATE with the
 *   reason.
 * - All calls share the array and it keeps the last call's contents; each
 *   call re-initialises what must start at zero.  Calls whose GPU work
 *   overlaps (several streams or threads) race on it: serialise them.
 * bits: HOST uint8 [batch][n_qubits]; d_out: DEVICE complex128
 * [batch][2^n_open]; enqueued on cuda_stream like tnc_contract_amplitudes. */
int tnc_contract_amplitudes_static(tnc_plan_t* plan, const uint8_t* bits, int batch, void* d_out,
                                   void* cuda_stream);

/* Several requests, possibly on different circuits, contracted together in
 * one stream, so that many small requests share launches.  Their
 * node programs advance in lockstep, in waves (wave w = step w of every
 * request that has one); in each wave the narrow nodes of all requests run as
 * one grouped launch and their CUDA-core cGEMM nodes as one grouped launch
 * per tile shape, each problem with its own operands and output layout; the
 * tensor-core, split-K and split-K-dot nodes run as launches of their own.
 * Every node does the same arithmetic as when its request runs alone, so the
 * results are those of tnc_contract_amplitudes per request.
 * plans[n]: plans with one serial slice group each (else TNC_EINVAL), made
 *   resident on the workspace's device by the call if needed; profiling off.
 * bits[i]: HOST uint8 [batches[i]][n_qubits of plan i]; d_outs[i]: DEVICE
 *   complex128 [batches[i]][2^n_open of plan i], caller-owned.
 * d_ws: DEVICE workspace of ws_bytes >= tnc_batch_ws_bytes(n, plans),
 *   256-byte aligned (descriptor tables, then one workspace per request).
 * Enqueued on cuda_stream; the bitstrings and descriptor tables are copied
 * before the call returns. */
int tnc_contract_batch(int n, tnc_plan_t* const* plans, const uint8_t* const* bits, const int* batches,
                       void* const* d_outs, void* d_ws, size_t ws_bytes, void* cuda_stream);
/* Workspace bytes tnc_contract_batch needs for these n plans (0 on a NULL). */
size_t tnc_batch_ws_bytes(int n, tnc_plan_t* const* plans);

/* Partial sum over the serial slice groups [group_begin, group_end) only
 * (0 <= begin <= end <= n_slice_groups): the slice-sharded form used when
 * several processes each own a range of slices; the partial results add up
 * (FP64) to the amplitudes.  d_bits in DEVICE memory. */
int tnc_contract_partial(tnc_plan_t* plan, const uint8_t* d_bits, int batch, int group_begin,
                         int group_end, void* d_out, void* d_ws, size_t ws_bytes,
                         void* cuda_stream);

/* ------------------------------------------------------------- serving --
 * A server owns a host thread and a pool of CUDA streams.  Requests
 * (plan, bitstrings) are admitted in arrival order while the sum of their
 * planned workspace bytes fits in the caller-provided device arena; admitted
 * requests run concurrently on separate streams (continuous batching), and a
 * finished request frees its bytes for the next.  d_arena (DEVICE,
 * arena_bytes, 256-byte aligned) stays owned by the caller and must outlive
 * the server. */
int tnc_server_create(void* d_arena, size_t arena_bytes, int n_streams, tnc_server_t** out);
/* Batching of admitted requests: with max_requests >= 2, whenever a stream is
 * free and at least two small requests wait at the head of the queue, up to
 * max_requests of them (in arrival order, as many as fit the arena together,
 * tnc_batch_ws_bytes) are admitted as one batch of tnc_contract_batch on that
 * stream: their nodes run in grouped launches across requests, wave by wave.
 * Small: one serial slice group, and planned real flops and bytes (report
 * real_flops, bytes) at most max_request_flops and max_request_bytes (0: no
 * limit) -- a batch finishes with its slowest request, so large requests run
 * alone.  max_requests 1 (the default): every request runs its own launches.
 * A request's result does not depend on the setting.  TNC_EINVAL for
 * max_requests outside 1..1024 or a negative limit. */
int tnc_server_set_batching(tnc_server_t* srv, int max_requests, double max_request_flops,
                            double max_request_bytes);
/* Submit a request.  bits (HOST, [batch][n_qubits]) are copied before
 * returning.  d_out (DEVICE complex128 [batch][2^n_open]) must stay valid
 * until the request is done.  TNC_EBUSY if the request can never fit the
 * arena or the queue holds max_queue requests. */
int tnc_server_submit(tnc_server_t* srv, tnc_plan_t* plan, const uint8_t* bits, int batch,
                      void* d_out, uint64_t* ticket);
/* *done = 1 when the result is in d_out (0 otherwise); also returns the
 * request's status once done.  TNC_ENOTFOUND for an unknown ticket. */
int tnc_server_poll(tnc_server_t* srv, uint64_t ticket, int* done);
/* Wait (bounded by timeout_ms) for a ticket; TNC_ETIMEOUT on expiry.
 * latency_ms (may be NULL) receives submit-to-completion time. */
int tnc_server_wait(tnc_server_t* srv, uint64_t ticket, int timeout_ms, double* latency_ms);
/* Cancel a queued (not yet admitted) request: TNC_ESTATE if already running. */
int tnc_server_cancel(tnc_server_t* srv, uint64_t ticket);
/* Finish the running requests, drop the queued ones, join the thread. */
int tnc_server_destroy(tnc_server_t* srv);

#ifdef __cplusplus
}
#endif
#endif /* TNC_H */
