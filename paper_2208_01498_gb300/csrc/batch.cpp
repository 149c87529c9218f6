// Several requests, possibly on different circuits, contracted together.
//
// Small requests are launch-bound: each is tens of small kernels.  Here their
// programs advance in lockstep, in waves (wave w runs step w of every request
// that has one): in each wave the narrow nodes of all requests (grouped
// narrow steps and single narrow nodes) run as one grouped launch, and their
// CUDA-core cGEMM nodes as one grouped launch per tile shape, each problem
// carrying its own operands and output layout by absolute pointers; only the
// tensor-core, split-K and split-K-dot nodes (and permutes) are launched per
// request.  Steps of one request stay in order (waves run in stream order);
// the steps of a wave belong to different requests and are independent.  The
// arithmetic of every node is the same as in its own launch, so each result
// equals the one of the request contracted alone.
//
// Workspace layout: the descriptor tables of all waves (copied once from the
// host), then one workspace per request (each 256-byte aligned).
#include <cuda_runtime_api.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tnc_internal.h"

namespace tnc {

namespace {

constexpr uint64_t kAl = 256;
uint64_t al(uint64_t x) { return (x + kAl - 1) & ~(kAl - 1); }

int fail(cudaError_t e, const char* what) {
  set_error("tnc_contract_batch: %s: %s", what, cudaGetErrorString(e));
  return TNC_ECUDA;
}

bool is_simt(int k) { return k == KG_SIMT_128x64 || k == KG_SIMT_64x32 || k == KG_SIMT_32x128; }

// a narrow node that the grouped narrow kernel runs (A [b][M][K], B [b][N][K])
bool groupable_narrow(const GemmDesc& g) { return g.kernel == KG_NARROW && !g.transA && g.transB && g.N <= 16 && g.K <= 16; }

bool groupable_simt(const GemmDesc& g) { return is_simt(g.kernel) && g.splitk <= 1; }

// descriptor table bytes for these plans (an upper bound: every step grouped)
uint64_t table_bytes(int n, tnc_plan_t* const* plans) {
  uint64_t narrow = 0, simt = 0;
  for (int i = 0; i < n; ++i)
    for (const Step& s : plans[i]->p.prog.steps) {
      if (s.kind == ST_GROUPED) narrow += s.g_count;
      if (s.kind == ST_GEMM && groupable_narrow(s.gemm)) narrow += 1;
      if (s.kind == ST_GEMM && groupable_simt(s.gemm)) simt += 1;
    }
  return al(narrow * sizeof(GroupedDesc)) + al(simt * sizeof(SimtProblem));
}

}  // namespace

uint64_t batch_ws_bytes(int n, tnc_plan_t* const* plans) {
  uint64_t b = table_bytes(n, plans);
  for (int i = 0; i < n; ++i) b += al(plans[i]->p.prog.ws_bytes);
  return b;
}

int run_batch(int n, tnc_plan_t* const* plans, const uint8_t* const* bits, const int* batches, void* const* d_outs,
              void* d_ws, size_t ws_bytes, void* stream) {
  if (n < 1 || !plans || !bits || !batches || !d_outs || !d_ws) {
    set_error("tnc_contract_batch: invalid argument");
    return TNC_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !bits[i] || !d_outs[i]) {
      set_error("tnc_contract_batch: request %d: NULL argument", i);
      return TNC_EINVAL;
    }
    const Plan& p = plans[i]->p;
    if (p.rep.n_slice_groups != 1) {
      set_error("tnc_contract_batch: request %d: a plan with %d serial slice groups runs alone", i,
                p.rep.n_slice_groups);
      return TNC_EINVAL;
    }
    if (batches[i] < 1 || batches[i] > std::max(1, p.opts.max_batch)) {
      set_error("tnc_contract_batch: request %d: batch %d outside 1..%d", i, batches[i], p.opts.max_batch);
      return TNC_EINVAL;
    }
    if (p.profiling) {
      set_error("tnc_contract_batch: request %d: profiling is on", i);
      return TNC_ESTATE;
    }
  }
  const uint64_t need = batch_ws_bytes(n, plans);
  if (ws_bytes < need) {
    set_error("tnc_contract_batch: workspace of %zu bytes < required %llu", ws_bytes, (unsigned long long)need);
    return TNC_ENOMEM;
  }
  if (((uintptr_t)d_ws & 255) != 0) {
    set_error("tnc_contract_batch: workspace not 256-byte aligned");
    return TNC_EINVAL;
  }
  {
    cudaPointerAttributes attr;
    cudaError_t e0 = cudaPointerGetAttributes(&attr, d_ws);
    if (e0 != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      set_error("tnc_contract_batch: workspace is not device memory");
      return TNC_EINVAL;
    }
    if ((e0 = cudaSetDevice(attr.device)) != cudaSuccess) return fail(e0, "cudaSetDevice");
  }
  for (int i = 0; i < n; ++i) {
    int rc = tnc_plan_upload(plans[i], stream);
    if (rc != TNC_OK) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* base_ws = (char*)d_ws;
  const uint64_t tb = table_bytes(n, plans);
  std::vector<char*> ws(n);
  {
    uint64_t off = tb;
    for (int i = 0; i < n; ++i) {
      ws[i] = base_ws + off;
      off += al(plans[i]->p.prog.ws_bytes);
    }
  }

  // ---- descriptor tables of every wave, built on the host
  size_t max_steps = 0;
  for (int i = 0; i < n; ++i) max_steps = std::max(max_steps, plans[i]->p.prog.steps.size());
  struct Wave {
    size_t narrow_first = 0, narrow_count = 0;
    int64_t narrow_blocks = 0;
    size_t simt_first[3] = {0, 0, 0}, simt_count[3] = {0, 0, 0};
    int64_t simt_blocks[3] = {0, 0, 0};
  };
  std::vector<Wave> waves(max_steps);
  std::vector<GroupedDesc> narrow;
  std::vector<SimtProblem> simt[3];
  const int simt_kernels[3] = {KG_SIMT_128x64, KG_SIMT_64x32, KG_SIMT_32x128};
  auto simt_slot = [&](int k) { return k == KG_SIMT_128x64 ? 0 : k == KG_SIMT_64x32 ? 1 : 2; };
  for (size_t w = 0; w < max_steps; ++w) {
    Wave& wv = waves[w];
    wv.narrow_first = narrow.size();
    for (int q = 0; q < 3; ++q) wv.simt_first[q] = simt[q].size();
    for (int i = 0; i < n; ++i) {
      const Plan& p = plans[i]->p;
      if (w >= p.prog.steps.size()) continue;
      const Step& s = p.prog.steps[w];
      if (s.kind == ST_GROUPED) {
        for (int q = 0; q < s.g_count; ++q) {
          GroupedDesc gd = p.prog.grouped[s.g_first + q];
          gd.ws_ptr = ws[i];
          gd.base_ptr = p.d_base;
          gd.first_block = wv.narrow_blocks;
          wv.narrow_blocks += (int64_t)gd.blocks_per_batch * gd.batch;
          narrow.push_back(gd);
        }
      } else if (s.kind == ST_GEMM && groupable_narrow(s.gemm)) {
        const GemmDesc& g = s.gemm;
        GroupedDesc gd;
        std::memset(&gd, 0, sizeof(gd));
        gd.a = g.a, gd.b = g.b, gd.c = g.c;
        gd.a_buf = g.a_buf, gd.b_buf = g.b_buf;
        gd.M = g.M, gd.N = (int)g.N, gd.K = (int)g.K, gd.batch = (int)g.batch;
        gd.c_ident = g.c_ident, gd.nN = g.nN, gd.nM = g.nM, gd.nB = g.nB;
        std::memcpy(gd.c_pos, g.c_pos, sizeof(gd.c_pos));
        gd.blocks_per_batch = (int)((g.M + 127) / 128);
        gd.ws_ptr = ws[i];
        gd.base_ptr = p.d_base;
        gd.first_block = wv.narrow_blocks;
        wv.narrow_blocks += (int64_t)gd.blocks_per_batch * gd.batch;
        narrow.push_back(gd);
      } else if (s.kind == ST_GEMM && groupable_simt(s.gemm)) {
        const GemmDesc& g = s.gemm;
        int bm = 0, bn = 0;
        simt_tile_shape(g.kernel, &bm, &bn);
        SimtProblem sp;
        std::memset(&sp, 0, sizeof(sp));
        sp.A = (const std::complex<float>*)(g.a_buf ? p.d_base : (void*)ws[i]) + g.a;
        sp.B = (const std::complex<float>*)(g.b_buf ? p.d_base : (void*)ws[i]) + g.b;
        sp.C = (std::complex<float>*)ws[i] + g.c;
        sp.M = g.M, sp.N = g.N, sp.K = g.K;
        sp.transA = g.transA, sp.transB = g.transB;
        sp.ident = g.c_ident, sp.nN = g.nN, sp.nM = g.nM, sp.nB = g.nB;
        std::memcpy(sp.c_pos, g.c_pos, sizeof(sp.c_pos));
        // staged epilogue for full tiles of a scattered output (as run_simt)
        sp.staged = (!g.c_ident && g.M % bm == 0 && g.N % bn == 0) ? 1 : 0;
        if (sp.staged) {
          const int kMB = __builtin_ctz(bm), kNB = __builtin_ctz(bn);
          int pos[kMaxRank];
          for (int b = 0; b < kMB; ++b) pos[b] = g.c_pos[g.nN + b];
          for (int b = 0; b < kNB; ++b) pos[kMB + b] = g.c_pos[b];
          for (int b = 0; b < kMB + kNB; ++b) {
            int r = 0;
            for (int k = 0; k < kMB + kNB; ++k) r += pos[k] < pos[b];
            sp.rank[b] = (int8_t)r;
          }
        }
        const int q = simt_slot(g.kernel);
        sp.first_block = wv.simt_blocks[q];
        wv.simt_blocks[q] += ((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * g.batch;
        simt[q].push_back(sp);
      }
    }
    wv.narrow_count = narrow.size() - wv.narrow_first;
    for (int q = 0; q < 3; ++q) wv.simt_count[q] = simt[q].size() - wv.simt_first[q];
  }
  // one copy of all tables (pageable host memory: staged by the driver before
  // the call returns, so the host vectors may go)
  GroupedDesc* d_narrow = (GroupedDesc*)base_ws;
  SimtProblem* d_simt = (SimtProblem*)(base_ws + al(narrow.size() * sizeof(GroupedDesc)));
  size_t simt_off[3] = {0, simt[0].size(), simt[0].size() + simt[1].size()};
  cudaError_t e;
  if (!narrow.empty() &&
      (e = cudaMemcpyAsync(d_narrow, narrow.data(), narrow.size() * sizeof(GroupedDesc), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return fail(e, "copy narrow descriptors");
  {
    std::vector<SimtProblem> all;
    for (int q = 0; q < 3; ++q) all.insert(all.end(), simt[q].begin(), simt[q].end());
    if (!all.empty() && (e = cudaMemcpyAsync(d_simt, all.data(), all.size() * sizeof(SimtProblem),
                                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return fail(e, "copy cGEMM descriptors");
  }

  // ---- per request: bitstrings, accumulator, slice counter, derived leaves
  for (int i = 0; i < n; ++i) {
    const Plan& p = plans[i]->p;
    const int maxb = 1 << p.beta_bits, nq = p.net.n_qubits;
    char* w_ = ws[i];
    if ((e = cudaMemsetAsync(w_ + p.prog.off_bits, 0, (size_t)maxb * nq, st)) != cudaSuccess)
      return fail(e, "memset bits");
    if ((e = cudaMemcpyAsync(w_ + p.prog.off_bits, bits[i], (size_t)batches[i] * nq, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return fail(e, "copy bits");
    const size_t out_bytes = (size_t)batches[i] * ((size_t)16 << p.open_qubits.size());
    if ((e = cudaMemsetAsync(w_ + p.prog.off_acc, 0, out_bytes, st)) != cudaSuccess) return fail(e, "memset acc");
    if ((e = cudaMemsetAsync(w_ + p.prog.off_ctr, 0, sizeof(uint64_t), st)) != cudaSuccess)
      return fail(e, "memset counter");
    if (!p.prog.gathers.empty()) {
      int r = launch_gather((const GatherDesc*)p.d_gathers, (int)p.prog.gathers.size(), p.prog.max_gather_rank,
                            p.d_base, w_, (const uint8_t*)(w_ + p.prog.off_bits), nq,
                            (const uint64_t*)(w_ + p.prog.off_ctr), st);
      if (r) return fail((cudaError_t)r, "gather");
    }
  }
  // ---- the waves
  for (size_t w = 0; w < max_steps; ++w) {
    const Wave& wv = waves[w];
    int r;
    if (wv.narrow_count &&
        (r = launch_grouped_narrow(d_narrow + wv.narrow_first, (int)wv.narrow_count, wv.narrow_blocks, nullptr,
                                   ws[0], st)))
      return fail((cudaError_t)r, "grouped narrow");
    for (int q = 0; q < 3; ++q)
      if (wv.simt_count[q] && (r = launch_grouped_simt(d_simt + simt_off[q] + wv.simt_first[q], (int)wv.simt_count[q],
                                                       wv.simt_blocks[q], simt_kernels[q], st)))
        return fail((cudaError_t)r, "grouped cGEMM");
    for (int i = 0; i < n; ++i) {
      const Plan& p = plans[i]->p;
      if (w >= p.prog.steps.size()) continue;
      const Step& s = p.prog.steps[w];
      if (s.kind == ST_PERMUTE)
        r = launch_permute(s.perm, ws[i], st);
      else if (s.kind == ST_GEMM && !groupable_narrow(s.gemm) && !groupable_simt(s.gemm))
        r = launch_gemm(s.gemm, p.d_base, ws[i], st);
      else
        r = 0;
      if (r) return fail((cudaError_t)r, "node");
    }
  }
  // ---- FP64 accumulation and results
  for (int i = 0; i < n; ++i) {
    const Plan& p = plans[i]->p;
    double2* acc = (double2*)(ws[i] + p.prog.off_acc);
    int r = launch_accum(p.prog.accum, ws[i], acc, batches[i], st);
    if (r) return fail((cudaError_t)r, "accum");
    const size_t out_bytes = (size_t)batches[i] * ((size_t)16 << p.open_qubits.size());
    if ((e = cudaMemcpyAsync(d_outs[i], acc, out_bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return fail(e, "copy out");
  }
  return TNC_OK;
}

}  // namespace tnc

extern "C" {

size_t tnc_batch_ws_bytes(int n, tnc_plan_t* const* plans) {
  if (n < 1 || !plans) return 0;
  for (int i = 0; i < n; ++i)
    if (!plans[i]) return 0;
  return (size_t)tnc::batch_ws_bytes(n, plans);
}

int tnc_contract_batch(int n, tnc_plan_t* const* plans, const uint8_t* const* bits, const int* batches,
                       void* const* d_outs, void* d_ws, size_t ws_bytes, void* stream) {
  return tnc::run_batch(n, plans, bits, batches, d_outs, d_ws, ws_bytes, stream);
}

}  // extern "C"
