// Index slicing and the compiled node program.
//
// Slicing (the index-slicing approach the paper's Conclusion names as future
// work): a set S of contracted labels is fixed to each of its 2^|S| value
// combinations; each combination is an independent network with the same
// tree, and the amplitudes are the sum over all of them.  Labels are added
// greedily -- the one that gives the smallest total work among those that
// lower the peak -- until the live intermediates of one slice fit the cap.
// Up to 2^max_group_log2 slices then run together ("grouped"): their labels
// are not fixed but carried as batch indices up to the root, where the final
// FP64 accumulation sums over them; the rest ("serial") loop on the host.
//
// The program of one slice group, in execution order:
//   gather  -- derived leaves: final wires projected onto the requested bits
//              (the bitstring index beta becomes a batch index), serial
//              sliced labels fixed to the group's values;
//   per tree node (post-order, larger subtree first):
//     permute -- only when an operand cannot be read as [batch][M][K] or
//                [batch][K][M] (leaves are stored in whatever order their
//                consumer wants, so only intermediates are ever permuted);
//     gemm    -- C[b][m][n] = sum_k A[b][m][k] B[b][k][n] (Eq. 3 node);
//   accum   -- FP64 sum of the root over the grouped slice labels into the
//              caller's complex128 output.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <set>

#include "tnc_internal.h"

namespace tnc {

namespace {

constexpr uint64_t kAlign = 256;
uint64_t align_up(uint64_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// first-fit allocator over [0, inf) used to lay out the arena
struct Arena {
  std::map<uint64_t, uint64_t> used;  // offset -> size
  uint64_t peak = 0;
  uint64_t alloc(uint64_t bytes) {
    bytes = align_up(std::max<uint64_t>(bytes, 16));
    uint64_t cur = 0;
    for (auto& kv : used) {
      if (kv.first - cur >= bytes) break;
      cur = std::max(cur, kv.first + kv.second);
    }
    used[cur] = bytes;
    peak = std::max(peak, cur + bytes);
    return cur;
  }
  void release(uint64_t off) { used.erase(off); }
};

// Can layout L (labels, most significant first) be read as consecutive
// blocks g[0], g[1], g[2] (label sets)?  Fills the block-internal orders.
bool view_as(const std::vector<int>& L, const std::vector<std::set<int>>& g,
             std::vector<std::vector<int>>& ord) {
  ord.assign(g.size(), {});
  size_t pos = 0;
  for (size_t b = 0; b < g.size(); ++b) {
    for (size_t k = 0; k < g[b].size(); ++k, ++pos) {
      if (pos >= L.size() || !g[b].count(L[pos])) return false;
      ord[b].push_back(L[pos]);
    }
  }
  return pos == L.size();
}

std::vector<int> concat(std::initializer_list<const std::vector<int>*> parts) {
  std::vector<int> r;
  for (auto* p : parts) r.insert(r.end(), p->begin(), p->end());
  return r;
}

std::vector<int> sorted_vec(const std::set<int>& s) { return std::vector<int>(s.begin(), s.end()); }

// bit position (from the least significant end) of label x in layout L
int bitpos(const std::vector<int>& L, int x) {
  for (size_t i = 0; i < L.size(); ++i)
    if (L[i] == x) return (int)(L.size() - 1 - i);
  return -1;
}

}  // namespace

static void set_splitk(GemmDesc& g);

// Kernel variant by shape: tiny outputs with long K -> split-K dot; narrow
// N and K -> one row per thread; dense enough nodes of the tensor-core forms
// -> tcgen05; otherwise the register-tiled CUDA-core kernel.  Long FP32 sums
// over K are cut into chunks summed in FP64 (split-K) when the output is small
// enough for the partials.
void choose_gemm_kernel(GemmDesc& g) {
  const double MN = (double)g.M * g.N;
  const bool pow2 = !(g.M & (g.M - 1)) && !(g.N & (g.N - 1)) && !(g.K & (g.K - 1));
  if (MN <= 16 && g.K >= 512)
    g.kernel = KG_DOT;
  else if (g.N <= 16 && g.K <= 16)
    g.kernel = KG_NARROW;
  else if (g.form != TNC_FP32 && pow2 && g.M >= 128 && g.N >= 32 && g.K >= 32) {
    g.kernel = KG_TC;
    // split-BF16 nodes with K-major operands and moderate M N split on chip
    // (the operands cross HBM once; long K prefetches the k-block after
    // next); very large M N re-read the operands from many tiles and run
    // faster from pre-split planes
    if (g.form == TNC_SPLIT_BF16 && !g.transA && g.transB && MN <= (double)(1 << 22))
      g.tile = g.N >= 64 ? (g.K >= 512 ? 5 : 4) : (g.K >= 512 ? 7 : 6);
  }
  else if (g.N <= 32)
    g.kernel = KG_SIMT_64x32;
  else
    g.kernel = KG_SIMT_128x64;
  set_splitk(g);
}

static void set_splitk(GemmDesc& g) {
  g.splitk = 1;
  const bool simt = g.kernel == KG_SIMT_128x64 || g.kernel == KG_SIMT_64x32 || g.kernel == KG_SIMT_32x128 ||
                    (g.kernel == KG_DOT && (g.M > 4 || g.N > 4));
  if (simt && g.K >= 8192 && (double)g.batch * g.M * g.N <= (double)(1 << 20)) {
    int64_t s = g.K / 2048;
    while (s > 1 && (double)s * g.batch * g.M * g.N * 8 > (double)(256u << 20)) s >>= 1;
    g.splitk = (int)std::min<int64_t>(s, 4096);
  } else if (simt && g.kernel != KG_DOT && g.K >= 512) {
    // fewer output tiles than SMs (e.g. batch 1, M = N = 64, K = 4096: one
    // block would run the whole sum): split K until about two tiles per SM,
    // each split keeping at least 64 k
    const int bm = g.kernel == KG_SIMT_128x64 ? 128 : g.kernel == KG_SIMT_64x32 ? 64 : 32;
    const int bn = g.kernel == KG_SIMT_128x64 ? 64 : g.kernel == KG_SIMT_64x32 ? 32 : 128;
    const double tiles = (double)g.batch * (double)((g.M + bm - 1) / bm) * (double)((g.N + bn - 1) / bn);
    const double sms = (double)sm_count();  // of the current device (152 without one)
    if (tiles < sms) {
      int64_t s = 1;
      while (tiles * (double)(2 * s) <= 2.0 * sms && g.K / (2 * s) >= 64 &&
             (double)(2 * s) * g.batch * g.M * g.N * 8 <= (double)(256u << 20))
        s *= 2;
      g.splitk = (int)s;
    } else if (tiles < 4.0 * sms && g.K >= 2048) {
      // one or two waves of tiles, each a long serial sum (e.g. batch 256,
      // M 32, N 16, K 4096: 1.16 ms on 256 tiles): split K until about four
      // tiles per SM, each split keeping at least 512 k
      int64_t s = 1;
      while (tiles * (double)s < 4.0 * sms && g.K / (2 * s) >= 512 &&
             (double)(2 * s) * g.batch * g.M * g.N * 8 <= (double)(256u << 20))
        s *= 2;
      g.splitk = (int)s;
    }
  }
}

void gemm_candidates(const GemmDesc& g0, GemmDesc* out, int* n) {
  int k = 0;
  out[k++] = g0;
  auto add = [&](int kernel, int tile) {
    GemmDesc g = g0;
    g.kernel = kernel;
    g.tile = tile;
    set_splitk(g);
    for (int i = 0; i < k; ++i)
      if (out[i].kernel == g.kernel && out[i].tile == g.tile) return;
    if (k < kMaxCandidates) out[k++] = g;
  };
  add(KG_SIMT_128x64, 0);
  add(KG_SIMT_64x32, 0);
  add(KG_SIMT_32x128, 0);
  if (g0.N <= 16 && g0.K <= 16) {
    add(KG_NARROW, 0);  // unrolled for K, N in {1, 2, 4, 8, 16} (K-major A), else one row per thread
    add(KG_NARROW, 1);  // one row per thread
    add(KG_NARROW, 2);  // tiled, output staged in address order (powers of two, K-major A)
    if (!g0.transA && g0.transB && (g0.K == 8 || g0.K == 16) && g0.N >= 2 && !(g0.N & (g0.N - 1)) &&
        g0.M >= 256 && g0.M % 256 == 0)
      add(KG_NARROW, 3);  // A tiles staged in shared memory by TMA
  }
  if (g0.M <= 4 && g0.N <= 4 && g0.K >= 512) add(KG_DOT, 0);
  const bool pow2 = !(g0.M & (g0.M - 1)) && !(g0.N & (g0.N - 1)) && !(g0.K & (g0.K - 1));
  if (g0.form != TNC_FP32 && pow2 && g0.M >= 128 && g0.N >= 32 && g0.K >= 32) {
    add(KG_TC, 1);
    if (g0.N >= 64) add(KG_TC, 2);
    if (g0.N >= 128) add(KG_TC, 3);
    if (g0.form == TNC_SPLIT_BF16 && !g0.transA && g0.transB) {
      if (g0.N >= 64) {
        add(KG_TC, 4);
        add(KG_TC, 5);
      }
      add(KG_TC, 6);
      add(KG_TC, 7);
      if (g0.N >= 128 && g0.K <= 256) add(KG_TC, 8);
      if (g0.N >= 128) {
        add(KG_TC, 14);
        add(KG_TC, 15);
      }
      add(KG_TC, 16);  // split on chip from FP32 tiles brought by TMA
      if (g0.N >= 64) add(KG_TC, 17);
      if (g0.N >= 128 && g0.K <= 256) add(KG_TC, 18);
    }
    if (g0.form == TNC_SPLIT_BF16 && g0.N >= 64) add(KG_TC, 10);
    if (g0.form == TNC_SPLIT_BF16) add(KG_TC, 12);
    if (g0.form == TNC_SPLIT_BF16 && g0.N >= 128 && g0.K <= 256) {
      add(KG_TC, 9);
      add(KG_TC, 11);
      if (!g0.transA) add(KG_TC, 13);
    }
  } else if (g0.form == TNC_SPLIT_BF16 && pow2 && g0.M >= 128 && g0.N >= 32 && g0.K >= 4 && g0.K < 32) {
    // short K: the persistent plane tiles (k-block zero-filled by TMA)
    add(KG_TC, 12);
    if (g0.N >= 64) add(KG_TC, 10);
    if (g0.N >= 128) {
      add(KG_TC, 9);
      add(KG_TC, 11);
      if (g0.K >= 16 && !g0.transA) add(KG_TC, 13);
    }
  }
  if (g0.form == TNC_SPLIT_BF16 && pow2 && g0.M >= 128 && g0.N >= 32 && g0.K >= 2 && g0.K < 32 && !g0.transA &&
      g0.transB) {
    add(KG_TC, 16);
    if (g0.N >= 64) add(KG_TC, 17);
    if (g0.N >= 128) add(KG_TC, 18);
  }
  // few output tiles and long K: the plane tiles with K split over CTAs
  if (g0.form != TNC_FP32 && pow2 && g0.M >= 128 && g0.N >= 32 && g0.K >= 1024 &&
      (double)(g0.M / 128) * (2.0 * g0.N / (g0.N >= 64 ? 128 : 64)) * g0.batch < (double)sm_count())
    add(KG_TC, 19);
  *n = k;
}

uint64_t gemm_scratch_bytes(const GemmDesc& g) {
  uint64_t bytes = 0;
  if (g.kernel == KG_DOT) bytes = (uint64_t)g.batch * g.M * g.N * 16 * 1024;
  if (g.kernel == KG_TC && !(g.tile >= 16 && g.tile <= 18)) {  // 16-18 split on chip: no planes
    // hi/lo planes of A' (batch x M x 2K) and B'^T (batch x 2N x 2K), 2 or 4 bytes each
    const uint64_t es = g.form == TNC_SPLIT_BF16 ? 2 : 4;
    bytes = (uint64_t)g.batch * (g.M * 2 * g.K * 2 + 2 * g.N * 2 * g.K * 2) * es + 4096;
    // tile 19 (K split over CTAs): partial tiles after the planes, splits x
    // tiles <= 2 x SMs, each 128 rows x 64 complex columns at most
    if (g.tile == 19) bytes += 256 + (uint64_t)2 * sm_count() * 128 * 64 * 8;
  }
  if (g.splitk > 1) bytes = std::max<uint64_t>(bytes, (uint64_t)g.splitk * g.batch * g.M * g.N * 8);
  return bytes;
}

// ----------------------------------------------------------------- slicing
namespace {

struct Eval {
  double peak_bytes = 0;
  double cost_log2 = 0;   // log2 of paper ops of one group (all nodes)
  int peak_node = -1;
};

// live-memory model of one slice group: post-order, larger subtree first;
// a node holds its operands, its output and operand copies for a permute
// (plus the split planes of the tensor-core forms).
Eval evaluate(const PlanNet& pn, Tree& t, int form) {
  annotate_tree(pn, t);
  Eval ev;
  ev.cost_log2 = tree_cost_log2(t);
  std::function<double(int, int*)> peak = [&](int v, int* at) -> double {
    const TreeNode& nd = t.nodes[v];
    double self = std::exp2((double)nd.out.size()) * 8;
    if (nd.left < 0) {
      *at = v;
      return self;
    }
    int al, ar;
    double pl = peak(nd.left, &al), pr = peak(nd.right, &ar);
    double sl = std::exp2((double)t.nodes[nd.left].out.size()) * 8;
    double sr = std::exp2((double)t.nodes[nd.right].out.size()) * 8;
    double p1 = std::max(pl, sl + pr), p2 = std::max(pr, sr + pl);
    double first = std::min(p1, p2);
    int fat = (p1 <= p2) ? (pl >= sl + pr ? al : ar) : (pr >= sr + pl ? ar : al);
    double work = sl + sr + self + std::max(sl, sr);
    if (form != TNC_FP32) work += sl + sr + 2 * std::min(sl, sr);
    if (work >= first) {
      *at = v;
      return work;
    }
    *at = fat;
    return first;
  };
  int at = -1;
  ev.peak_bytes = peak(t.root, &at);
  ev.peak_node = at;
  return ev;
}

PlanNet exec_net(const PlanNet& base, const std::vector<int>& ser, const std::vector<int>& par) {
  PlanNet pn = base;
  std::vector<char> drop(pn.n_labels, 0);
  for (int x : ser) drop[x] = 1;
  for (auto& L : pn.leaf_labels) {
    std::vector<int> r;
    for (int x : L)
      if (!drop[x]) r.push_back(x);
    L.swap(r);
  }
  for (int x : ser) pn.holders[x].clear();
  for (int x : par) pn.global_out[x] = 1;
  return pn;
}

// Fast model of the sliced tree: node output labels and operand labels of
// the unsliced tree; a set S of sliced labels removes its labels from every
// node.  Cost of all slices (log2 paper ops): |S| + log2 sum_v 2 M_v / 2^|L_v n S|
// (L_v: the distinct labels of v's operands, M_v = 2^|L_v|, Eq. 3); peak: the
// live-memory recursion of evaluate() with the sliced sizes.
class SliceModel {
 public:
  SliceModel(const PlanNet& pn, Tree& t, int form) : t_(t), form_(form) {
    annotate_tree(pn, t);
    const size_t n = t.nodes.size();
    out_.resize(n);
    ops_.resize(n);
    for (size_t v = 0; v < n; ++v) out_[v] = t.nodes[v].out;
    for (size_t v = 0; v < n; ++v) {
      const TreeNode& nd = t.nodes[v];
      if (nd.left < 0) continue;
      std::vector<int>& L = ops_[v];
      std::set_union(out_[nd.left].begin(), out_[nd.left].end(), out_[nd.right].begin(), out_[nd.right].end(),
                     std::back_inserter(L));
    }
  }

  double cost_log2(const std::vector<char>& inS, int nS) const {
    double mx = -1e300;
    std::vector<double> c(t_.nodes.size(), -1e300);
    for (size_t v = 0; v < t_.nodes.size(); ++v) {
      if (t_.nodes[v].left < 0) continue;
      int k = 0;
      for (int x : ops_[v]) k += inS[x];
      c[v] = (double)ops_[v].size() - k;
      mx = std::max(mx, c[v]);
    }
    if (mx < -1e299) return 0;
    double sum = 0;
    for (double cv : c)
      if (cv > -1e299) sum += std::exp2(cv - mx);
    return nS + mx + std::log2(sum) + 1;
  }

  // peak live bytes of one slice; *big receives every node whose output
  // alone exceeds `over` bytes
  double peak(const std::vector<char>& inS, double over = -1, std::vector<int>* big = nullptr) const {
    std::function<double(int)> rec = [&](int v) -> double {
      const TreeNode& nd = t_.nodes[v];
      const double self = size(v, inS);
      if (big && over >= 0 && self > over) big->push_back(v);
      if (nd.left < 0) return self;
      const double pl = rec(nd.left), pr = rec(nd.right);
      const double sl = size(nd.left, inS), sr = size(nd.right, inS);
      const double first = std::min(std::max(pl, sl + pr), std::max(pr, sr + pl));
      double work = sl + sr + self + std::max(sl, sr);
      if (form_ != TNC_FP32) work += sl + sr + 2 * std::min(sl, sr);
      return std::max(first, work);
    };
    return rec(t_.root);
  }

  const std::vector<int>& out(int v) const { return out_[v]; }

 private:
  double size(int v, const std::vector<char>& inS) const {
    int k = 0;
    for (int x : out_[v]) k += inS[x];
    return std::exp2((double)out_[v].size() - k) * 8;
  }
  const Tree& t_;
  int form_;
  std::vector<std::vector<int>> out_, ops_;
};

}  // namespace

// Sliced labels for one tree under a memory cap: greedy additions scored by
// the added work per halving of the peak, over the contracted labels of every
// intermediate larger than the cap; then labels are dropped while the peak
// stays under the cap, and single swaps are tried that keep it there and
// lower the total work.  Returns TNC_ENOMEM when no set reaches the cap.
int choose_slices(const PlanNet& base, Tree& t, int form, size_t cap_bytes, std::vector<int>& S,
                  double* total_log2) {
  S.clear();
  SliceModel m(base, t, form);
  std::vector<char> inS(base.n_labels, 0);
  const double cap = (double)cap_bytes;
  double peak = m.peak(inS);
  double cost = m.cost_log2(inS, 0);
  if (cap_bytes == 0 || peak <= cap) {
    if (total_log2) *total_log2 = cost;
    return TNC_OK;
  }
  auto sliceable = [&](int x) { return !base.global_out[x] && base.holders[x].size() >= 2; };
  while (peak > cap) {
    // candidates: contracted labels of every intermediate above the cap
    std::vector<int> big;
    m.peak(inS, cap / 2, &big);
    std::set<int> cand;
    for (int v : big)
      for (int x : m.out(v))
        if (!inS[x] && sliceable(x)) cand.insert(x);
    if (cand.empty())
      for (size_t v = 0; v < t.nodes.size(); ++v)
        for (int x : m.out((int)v))
          if (!inS[x] && sliceable(x)) cand.insert(x);
    if (cand.empty() || S.size() >= 40) {
      set_error("tnc_plan: cannot slice the plan under mem_cap_bytes = %zu (peak %.3g bytes)", cap_bytes, peak);
      return TNC_ENOMEM;
    }
    int best = -1;
    double best_score = 1e300, best_peak = 0, best_cost = 0;
    for (int x : cand) {
      inS[x] = 1;
      const double p2 = m.peak(inS);
      const double c2 = m.cost_log2(inS, (int)S.size() + 1);
      inS[x] = 0;
      if (!(p2 < peak)) continue;
      // added log2 work per halving of the peak (fewer bits first on ties)
      const double score = (c2 - cost) / std::log2(peak / p2);
      if (score < best_score - 1e-12 || (std::fabs(score - best_score) <= 1e-12 && p2 < best_peak)) {
        best_score = score;
        best = x;
        best_peak = p2;
        best_cost = c2;
      }
    }
    if (best < 0) {
      set_error("tnc_plan: slicing does not lower the peak under mem_cap_bytes = %zu", cap_bytes);
      return TNC_ENOMEM;
    }
    S.push_back(best);
    inS[best] = 1;
    peak = best_peak;
    cost = best_cost;
  }
  // drop labels that are no longer needed (the costliest first)
  for (bool again = true; again;) {
    again = false;
    int drop = -1;
    double drop_cost = cost;
    for (size_t i = 0; i < S.size(); ++i) {
      inS[S[i]] = 0;
      if (m.peak(inS) <= cap) {
        const double c2 = m.cost_log2(inS, (int)S.size() - 1);
        if (c2 < drop_cost) drop_cost = c2, drop = (int)i;
      }
      inS[S[i]] = 1;
    }
    if (drop >= 0) {
      inS[S[drop]] = 0;
      S.erase(S.begin() + drop);
      cost = drop_cost;
      again = true;
    }
  }
  // single swaps that keep the cap and lower the work
  std::set<int> pool;
  {
    std::vector<int> big;
    std::vector<char> none(base.n_labels, 0);
    m.peak(none, cap / 2, &big);
    for (int v : big)
      for (int x : m.out(v))
        if (sliceable(x)) pool.insert(x);
  }
  for (int round = 0; round < 4; ++round) {
    bool improved = false;
    for (size_t i = 0; i < S.size(); ++i) {
      int best_y = -1;
      double best_c = cost;
      inS[S[i]] = 0;
      for (int y : pool) {
        if (inS[y] || y == S[i]) continue;
        inS[y] = 1;
        if (m.peak(inS) <= cap) {
          const double c2 = m.cost_log2(inS, (int)S.size());
          if (c2 < best_c - 1e-9) best_c = c2, best_y = y;
        }
        inS[y] = 0;
      }
      if (best_y >= 0) {
        S[i] = best_y;
        cost = best_c;
        improved = true;
      }
      inS[S[i]] = 1;
    }
    if (!improved) break;
  }
  if (total_log2) *total_log2 = cost;
  return TNC_OK;
}

int plan_slices(Plan& p, size_t cap_bytes) {
  const PlanNet& base = p.pn;
  p.sliced_serial.clear();
  p.sliced_par.clear();
  const int form = p.opts.form;
  std::vector<int> S;
  Tree t = p.tree;
  int rc = choose_slices(base, t, form, cap_bytes, S, nullptr);
  if (rc != TNC_OK) return rc;
  if (S.empty()) return TNC_OK;
  // group sliced labels while the group still fits the cap: each time the
  // serial label whose grouping raises the peak the least
  std::vector<int> ser = S, par;
  while (!ser.empty() && (int)par.size() < p.opts.max_group_log2) {
    int best = -1;
    double best_peak = (double)cap_bytes;
    for (size_t i = 0; i < ser.size(); ++i) {
      std::vector<int> ser2 = ser, par2 = par;
      ser2.erase(ser2.begin() + i);
      par2.push_back(ser[i]);
      PlanNet pn2 = exec_net(base, ser2, par2);
      Tree t2 = p.tree;
      Eval e2 = evaluate(pn2, t2, form);
      if (e2.peak_bytes <= best_peak) best_peak = e2.peak_bytes, best = (int)i;
    }
    if (best < 0) break;
    par.push_back(ser[best]);
    ser.erase(ser.begin() + best);
  }
  if (ser.size() > 30) {
    set_error("tnc_plan: %zu serial sliced labels (2^%zu slice groups) exceed the executor's 2^30", ser.size(),
              ser.size());
    return TNC_ENOMEM;
  }
  p.sliced_serial = ser;
  p.sliced_par = par;
  return TNC_OK;
}

// ----------------------------------------------------------------- compile
int compile_program(Plan& p) {
  Program& pr = p.prog;
  pr = Program();
  const Network& net = p.net;
  // execution view: serial sliced labels removed, grouped ones kept to the root
  PlanNet pn = exec_net(p.pn, p.sliced_serial, p.sliced_par);
  Tree& t = p.tree;
  annotate_tree(pn, t);
  const int form = p.opts.form;
  // the kernels address a tensor by at most kMaxRank binary indices (and a
  // node's operands and output by at most kMaxRank bits each)
  for (const TreeNode& nd : t.nodes) {
    const int r = (int)nd.out.size();
    if (r > kMaxRank) {
      set_error("tnc_plan: an intermediate of rank %d exceeds the executor's %d binary indices; "
                "set mem_cap_bytes to slice it",
                r, kMaxRank);
      return TNC_ENOMEM;
    }
  }

  std::vector<char> is_open(net.n_qubits, 0);
  for (int q : p.open_qubits) is_open[q] = 1;
  std::vector<int> ser_index(pn.n_labels, -1), par_index(pn.n_labels, -1), beta_index(pn.n_labels, -1);
  for (size_t i = 0; i < p.sliced_serial.size(); ++i) ser_index[p.sliced_serial[i]] = (int)i;
  for (size_t i = 0; i < p.sliced_par.size(); ++i) par_index[p.sliced_par[i]] = (int)i;
  for (int b = 0; b < p.beta_bits; ++b) beta_index[p.beta_labels[b]] = b;

  // which leaves need a gather (fixed final wire or serial sliced label)
  const int nL = pn.n_leaves;
  std::vector<char> derived(nL, 0);
  for (int l = 0; l < nL; ++l) {
    for (int x : net.leaves[l].labels) {
      if (net.label_kind[x] == LK_FINAL) {
        int q = net.leaves[l].qubit;
        // the final label belongs to the qubit whose final wire it is
        for (int qq = 0; qq < net.n_qubits; ++qq)
          if (net.final_label[qq] == x) q = qq;
        if (!is_open[q]) derived[l] = 1;
      }
      if (ser_index[x] >= 0) derived[l] = 1;
    }
  }
  if (t.nodes[t.root].left < 0) derived[t.nodes[t.root].leaf] = 1;

  // ws layout: bits | counter | derived leaves | arena
  const int batch_pad = 1 << p.beta_bits;
  pr.off_bits = 0;
  uint64_t off = align_up((uint64_t)batch_pad * net.n_qubits);
  pr.off_ctr = off;
  off += kAlign;
  pr.off_acc = off;
  off += align_up((uint64_t)batch_pad * 16 << p.open_qubits.size());
  const uint64_t leaf_area = off;

  // execution order: post-order, the child with the larger subtree peak first
  std::vector<double> sub_peak(t.nodes.size(), 0);
  std::function<double(int)> speak = [&](int v) -> double {
    const TreeNode& nd = t.nodes[v];
    double self = std::exp2((double)nd.out.size());
    if (nd.left < 0) return sub_peak[v] = self;
    double a = speak(nd.left), b = speak(nd.right);
    double sa = std::exp2((double)t.nodes[nd.left].out.size());
    double sb = std::exp2((double)t.nodes[nd.right].out.size());
    return sub_peak[v] = std::max({std::min(std::max(a, sa + b), std::max(b, sb + a)), sa + sb + self});
  };
  speak(t.root);
  std::vector<int> order;
  std::function<void(int)> post = [&](int v) {
    const TreeNode& nd = t.nodes[v];
    if (nd.left < 0) return;
    int a = nd.left, b = nd.right;
    double sa = std::exp2((double)t.nodes[a].out.size()), sb = std::exp2((double)t.nodes[b].out.size());
    if (std::max(sub_peak[a], sa + sub_peak[b]) > std::max(sub_peak[b], sb + sub_peak[a])) std::swap(a, b);
    post(a);
    post(b);
    order.push_back(v);
  };
  post(t.root);

  // ---- layouts, top down: every tensor is stored in the order its consumer
  // reads.  A node reads both operands K-major, [batch][free][K]; its GEMM
  // writes its output through the epilogue's scatter directly into the order
  // its own consumer asked for, so no tensor is ever permuted.
  std::vector<std::vector<int>> want(t.nodes.size());
  {
    std::vector<int> ro = t.nodes[t.root].out;
    std::sort(ro.begin(), ro.end());
    want[t.root] = ro;
    std::function<void(int)> down = [&](int v) {
      const TreeNode& nd = t.nodes[v];
      if (nd.left < 0) return;
      const int x = nd.left, y = nd.right;
      std::set<int> Lx(t.nodes[x].out.begin(), t.nodes[x].out.end());
      std::set<int> Ly(t.nodes[y].out.begin(), t.nodes[y].out.end());
      std::set<int> Lv(nd.out.begin(), nd.out.end());
      std::vector<int> b, fx, fy, K;
      for (int a : want[v]) {
        if (Lx.count(a) && Ly.count(a))
          b.push_back(a);
        else if (Lx.count(a))
          fx.push_back(a);
        else
          fy.push_back(a);
      }
      for (int a : Lx)
        if (Ly.count(a) && !Lv.count(a)) K.push_back(a);
      want[x] = concat({&b, &fx, &K});
      want[y] = concat({&b, &fy, &K});
      down(x);
      down(y);
    };
    down(t.root);
  }

  // per-node storage
  std::vector<int> buf(t.nodes.size(), -1);        // 0 leaf area, 1 leaf buffer, 2 arena
  std::vector<uint64_t> loc(t.nodes.size(), 0);    // element offset
  std::vector<char> placed(t.nodes.size(), 0);
  Arena arena;
  std::vector<Step> steps;
  std::vector<std::pair<size_t, int>> fix_b;  // (step, operand buffer tags)

  auto nsize = [&](int v) { return (uint64_t)1 << t.nodes[v].out.size(); };

  // place a leaf in the order its consumer reads
  uint64_t leaf_ws_off = 0;   // elements, relative to leaf_area
  std::vector<cd> base_data;  // assembled leaf buffer (FP64, converted at the end)
  auto place_leaf = [&](int v) {
    const std::vector<int>& ord = want[v];
    int l = t.nodes[v].leaf;
    placed[v] = 1;
    const Leaf& L = net.leaves[l];
    if (derived[l]) {
      GatherDesc g;
      std::memset(&g, 0, sizeof(g));
      // base data stored in the original order
      g.src = base_data.size();
      base_data.insert(base_data.end(), L.data.begin(), L.data.end());
      while (base_data.size() % 4) base_data.push_back(0);
      g.dst = leaf_ws_off;  // relative, fixed below
      g.out_rank = (int)ord.size();
      g.src_rank = (int)L.labels.size();
      for (int j = 0; j < g.out_rank; ++j) {
        int x = ord[ord.size() - 1 - j];
        if (beta_index[x] >= 0)
          g.out_src[j] = (int8_t)(-1 - beta_index[x]);
        else
          g.out_src[j] = (int8_t)bitpos(L.labels, x);
      }
      for (int x : L.labels) {
        if (net.label_kind[x] == LK_FINAL) {
          int q = -1;
          for (int qq = 0; qq < net.n_qubits; ++qq)
            if (net.final_label[qq] == x) q = qq;
          if (!is_open[q]) {
            g.fixed_pos[g.n_fixed] = (int8_t)bitpos(L.labels, x);
            g.fixed_qubit[g.n_fixed] = (int16_t)q;
            g.n_fixed++;
          }
        }
        if (ser_index[x] >= 0) {
          g.sliced_pos[g.n_sliced] = (int8_t)bitpos(L.labels, x);
          g.sliced_bit[g.n_sliced] = (int8_t)ser_index[x];
          g.n_sliced++;
        }
      }
      pr.gathers.push_back(g);
      pr.max_gather_rank = std::max(pr.max_gather_rank, g.out_rank);
      buf[v] = 0;
      loc[v] = leaf_ws_off;  // relative to the leaf area
      leaf_ws_off += align_up(((uint64_t)1 << ord.size()) * 8) / 8;
    } else {
      const int r = (int)ord.size();
      std::vector<int> srcbit(r);
      for (int j = 0; j < r; ++j) srcbit[j] = bitpos(L.labels, ord[r - 1 - j]);
      uint64_t start = base_data.size();
      base_data.resize(start + ((uint64_t)1 << r));
      for (uint64_t o = 0; o < ((uint64_t)1 << r); ++o) {
        uint64_t i = 0;
        for (int j = 0; j < r; ++j)
          if ((o >> j) & 1) i |= (uint64_t)1 << srcbit[j];
        base_data[start + o] = L.data[i];
      }
      while (base_data.size() % 4) base_data.push_back(0);  // keep 32-byte alignment
      buf[v] = 1;
      loc[v] = start;
    }
  };

  constexpr int BUF_ARENA = 2;
  double flops = 0, bytes = 0, pops = 0;

  // shape of every node: batch, M (larger free side), N, K; operands are
  // [b][free][K], so either child can play A
  struct Shape {
    int A, B, nb, nk, nM, nN;
    GemmDesc g;
  };
  std::vector<Shape> shp(t.nodes.size());
  for (int v : order) {
    const TreeNode& nd = t.nodes[v];
    const int x = nd.left, y = nd.right;
    std::set<int> Lx(t.nodes[x].out.begin(), t.nodes[x].out.end());
    std::set<int> Ly(t.nodes[y].out.begin(), t.nodes[y].out.end());
    int nb = 0, nk = 0, nfx = 0, nfy = 0;
    for (int a : Lx) {
      if (Ly.count(a))
        (std::find(nd.out.begin(), nd.out.end(), a) != nd.out.end() ? nb : nk)++;
      else
        ++nfx;
    }
    for (int a : Ly)
      if (!Lx.count(a)) ++nfy;
    Shape& s = shp[v];
    s.A = nfx >= nfy ? x : y;
    s.B = nfx >= nfy ? y : x;
    s.nM = nfx >= nfy ? nfx : nfy;
    s.nN = nfx >= nfy ? nfy : nfx;
    s.nb = nb;
    s.nk = nk;
    GemmDesc& g = s.g;
    std::memset(&g, 0, sizeof(g));
    g.batch = (int64_t)1 << nb;
    g.M = (int64_t)1 << s.nM;
    g.N = (int64_t)1 << s.nN;
    g.K = (int64_t)1 << nk;
    g.transA = 0;
    g.transB = 1;
    g.form = form;
    // output scatter: n bits (B's free labels, least significant first), then
    // m bits (A's free labels), then batch bits, to their places in want[v]
    const std::vector<int>& LA = want[s.A];
    const std::vector<int>& LB = want[s.B];
    const std::vector<int>& LC = want[v];
    g.nN = s.nN, g.nM = s.nM, g.nB = nb;
    int i = 0;
    for (int j = s.nN - 1; j >= 0; --j) g.c_pos[i++] = (int8_t)bitpos(LC, LB[nb + j]);
    for (int j = s.nM - 1; j >= 0; --j) g.c_pos[i++] = (int8_t)bitpos(LC, LA[nb + j]);
    for (int j = nb - 1; j >= 0; --j) g.c_pos[i++] = (int8_t)bitpos(LC, LA[j]);
    bool ident = true;
    for (int q = 0; q < i; ++q) ident &= g.c_pos[q] == q;
    g.c_ident = ident ? 1 : 0;
    choose_gemm_kernel(g);
    double work = (double)g.batch * g.M * g.N * g.K;
    flops += 8 * work;
    pops += 2 * work;
    bytes += 8.0 * ((double)g.batch * (g.M * g.K + g.K * g.N + g.M * g.N));
  }

  // nodes whose whole subtree is made of small narrow contractions run first,
  // level by level, each level as one grouped launch
  std::vector<char> small(t.nodes.size(), 0);
  std::vector<int> lvl(t.nodes.size(), 0);
  int max_lvl = 0;
  for (int v : order) {
    const TreeNode& nd = t.nodes[v];
    const GemmDesc& g = shp[v].g;
    bool ok = g.kernel == KG_NARROW && (double)g.batch * g.M * g.N <= (double)(1 << 20);
    for (int c : {nd.left, nd.right})
      if (t.nodes[c].left >= 0 && !small[c]) ok = false;
    small[v] = ok ? 1 : 0;
    lvl[v] = 1 + std::max(t.nodes[nd.left].left >= 0 ? lvl[nd.left] : 0,
                          t.nodes[nd.right].left >= 0 ? lvl[nd.right] : 0);
    if (small[v]) max_lvl = std::max(max_lvl, lvl[v]);
  }
  for (int L = 1; L <= max_lvl; ++L) {
    std::vector<int> members;
    for (int v : order)
      if (small[v] && lvl[v] == L) members.push_back(v);
    if (members.empty()) continue;
    Step s;
    std::memset(&s, 0, sizeof(s));
    s.kind = ST_GROUPED;
    s.node = -1;
    s.g_first = (int)pr.grouped.size();
    s.g_count = (int)members.size();
    int64_t blocks = 0;
    std::vector<uint64_t> to_free;
    for (int v : members) {
      const Shape& sh = shp[v];
      for (int c : {sh.A, sh.B})
        if (!placed[c]) place_leaf(c);
      uint64_t coff = arena.alloc(nsize(v) * 8);
      GroupedDesc gd;
      std::memset(&gd, 0, sizeof(gd));
      gd.a = loc[sh.A];
      gd.b = loc[sh.B];
      gd.a_buf = buf[sh.A];  // tag, fixed below
      gd.b_buf = buf[sh.B];
      gd.c = coff / 8;
      gd.M = sh.g.M;
      gd.N = (int)sh.g.N;
      gd.K = (int)sh.g.K;
      gd.batch = (int)sh.g.batch;
      gd.c_ident = sh.g.c_ident;
      gd.nN = sh.g.nN, gd.nM = sh.g.nM, gd.nB = sh.g.nB;
      for (int q = 0; q < kMaxRank; ++q) gd.c_pos[q] = sh.g.c_pos[q];
      gd.blocks_per_batch = (int)((sh.g.M + 127) / 128);
      gd.first_block = blocks;
      blocks += (int64_t)gd.blocks_per_batch * gd.batch;
      pr.grouped.push_back(gd);
      for (int c : {sh.A, sh.B})
        if (buf[c] == BUF_ARENA) to_free.push_back(loc[c] * 8);
      buf[v] = BUF_ARENA;
      loc[v] = coff / 8;
      placed[v] = 1;
    }
    s.g_blocks = blocks;
    steps.push_back(s);
    for (uint64_t f : to_free) arena.release(f);
  }

  for (int v : order) {
    if (small[v]) continue;
    const Shape& sh = shp[v];
    for (int c : {sh.A, sh.B})
      if (!placed[c]) place_leaf(c);
    uint64_t coff = arena.alloc(nsize(v) * 8);
    Step s;
    std::memset(&s, 0, sizeof(s));
    s.kind = ST_GEMM;
    s.node = v;
    s.gemm = sh.g;
    GemmDesc& g = s.gemm;
    g.a = loc[sh.A];
    g.b = loc[sh.B];
    g.a_buf = buf[sh.A];
    g.b_buf = buf[sh.B];
    g.c = coff / 8;
    uint64_t scratch_bytes = 0;  // room for any candidate the autotuner may pick
    {
      GemmDesc cand[kMaxCandidates];
      int nc = 0;
      gemm_candidates(g, cand, &nc);
      for (int q = 0; q < nc; ++q) scratch_bytes = std::max(scratch_bytes, gemm_scratch_bytes(cand[q]));
    }
    uint64_t soff = scratch_bytes ? arena.alloc(scratch_bytes) : 0;
    g.scratch = soff / 8;
    g.scratch_elems = scratch_bytes / 8;
    steps.push_back(s);
    fix_b.push_back({steps.size() - 1, 0});
    if (scratch_bytes) arena.release(soff);
    for (int c : {sh.A, sh.B})
      if (buf[c] == BUF_ARENA) arena.release(loc[c] * 8);
    buf[v] = BUF_ARENA;
    loc[v] = coff / 8;
    placed[v] = 1;
  }
  if (!placed[t.root]) place_leaf(t.root);  // single-leaf network
  const std::vector<std::vector<int>>& layout = want;

  // fix up offsets: leaf area size known now
  const uint64_t leaf_bytes = align_up(leaf_ws_off * 8);
  const uint64_t arena_base = leaf_area + leaf_bytes;  // bytes
  for (auto& gd : pr.gathers) gd.dst = leaf_area / 8 + gd.dst;
  auto abs_off = [&](int b, uint64_t rel) -> uint64_t {
    if (b == BUF_ARENA) return arena_base / 8 + rel;
    if (b == 0) return leaf_area / 8 + rel;
    return rel;
  };
  for (auto& gd : pr.grouped) {
    gd.a = abs_off(gd.a_buf, gd.a);
    gd.b = abs_off(gd.b_buf, gd.b);
    gd.c = abs_off(BUF_ARENA, gd.c);
    gd.a_buf = gd.a_buf == 1 ? 1 : 0;
    gd.b_buf = gd.b_buf == 1 ? 1 : 0;
  }
  for (auto& f : fix_b) {
    Step& s = steps[f.first];
    s.gemm.a = abs_off(s.gemm.a_buf, s.gemm.a);
    s.gemm.b = abs_off(s.gemm.b_buf, s.gemm.b);
    s.gemm.a_buf = s.gemm.a_buf == 1 ? 1 : 0;
    s.gemm.b_buf = s.gemm.b_buf == 1 ? 1 : 0;
    s.gemm.c = abs_off(BUF_ARENA, s.gemm.c);
    if (s.gemm.scratch_elems) s.gemm.scratch = abs_off(BUF_ARENA, s.gemm.scratch);
  }
  pr.steps = std::move(steps);

  // final accumulation from the root
  AccumDesc& ad = pr.accum;
  std::memset(&ad, 0, sizeof(ad));
  const int root = t.root;
  ad.src = abs_off(buf[root] == BUF_ARENA ? BUF_ARENA : 0, loc[root]);
  ad.rank = (int)layout[root].size();
  ad.n_beta = p.beta_bits;
  ad.n_open = (int)p.open_qubits.size();
  ad.n_par = (int)p.sliced_par.size();
  for (int j = 0; j < ad.rank; ++j) {
    int x = layout[root][ad.rank - 1 - j];
    if (beta_index[x] >= 0) {
      ad.role[j] = 0, ad.idx[j] = (int8_t)beta_index[x];
    } else if (par_index[x] >= 0) {
      ad.role[j] = 2, ad.idx[j] = (int8_t)par_index[x];
    } else {
      int oi = -1;
      for (size_t i = 0; i < p.open_qubits.size(); ++i)
        if (net.final_label[p.open_qubits[i]] == x) oi = (int)i;
      if (oi < 0) {
        set_error("tnc_plan: internal error: unexpected root label %d", x);
        return TNC_EINVAL;
      }
      ad.role[j] = 1, ad.idx[j] = (int8_t)oi;
    }
  }

  pr.ws_bytes = arena_base + align_up(arena.peak);
  pr.peak_bytes = (double)arena.peak;
  pr.base_elems = base_data.size();
  pr.base_host.resize(base_data.size());
  for (size_t i = 0; i < base_data.size(); ++i)
    pr.base_host[i] = std::complex<float>((float)base_data[i].real(), (float)base_data[i].imag());
  pr.flops_per_group = flops;
  pr.bytes_per_group = bytes;
  pr.paper_ops_per_group = pops;
  pr.max_rank = tree_max_rank(t);
  return TNC_OK;
}

}  // namespace tnc
