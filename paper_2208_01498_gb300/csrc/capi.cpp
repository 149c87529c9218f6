// C ABI entry points (include/tnc.h): network loading, planning, device
// upload and the executor loop over slice groups.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>

#include "tnc_internal.h"


namespace tnc {

int read_tc_error(int* flag);
int bounded_wait_selftest(uint64_t limit_ns, int* timed_out);
size_t static_workspace_bytes();
int prepare_static_workspace(int dev);

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

static int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return TNC_ECUDA;
}

// Planning view: fixed final wires are replaced by the beta bits of the
// bitstring batch; open final wires and beta bits survive to the root.
// time_scale > 0 places the tensors in (dim + 1)-dimensional space-time, the
// extra coordinate being the gate's layer times time_scale (the network
// before the collapse of the Thm. 2 proof, Fig. 1a); 0 keeps the time axis
// collapsed.
static void make_plan_net(const Network& net, const std::vector<int>& open_q, int beta_bits,
                          PlanNet& pn, std::vector<int>& beta_labels, double time_scale = 0) {
  pn = PlanNet();
  pn.dim = time_scale > 0 ? net.dim + 1 : net.dim;
  pn.n_leaves = (int)net.leaves.size();
  int nlab = (int)net.label_kind.size();
  beta_labels.clear();
  for (int b = 0; b < beta_bits; ++b) beta_labels.push_back(nlab + b);
  pn.n_labels = nlab + beta_bits;
  std::vector<char> is_open(net.n_qubits, 0);
  for (int q : open_q) is_open[q] = 1;
  std::vector<char> fixed_final(nlab, 0);
  for (int q = 0; q < net.n_qubits; ++q)
    if (!is_open[q]) fixed_final[net.final_label[q]] = 1;
  pn.leaf_labels.resize(pn.n_leaves);
  pn.pos.resize(pn.n_leaves);
  pn.radius.resize(pn.n_leaves);
  for (int l = 0; l < pn.n_leaves; ++l) {
    const Leaf& L = net.leaves[l];
    bool has_fixed = false;
    for (int x : L.labels) {
      if (fixed_final[x])
        has_fixed = true;
      else
        pn.leaf_labels[l].push_back(x);
    }
    if (has_fixed)
      for (int x : beta_labels) pn.leaf_labels[l].push_back(x);
    for (int k = 0; k < 3; ++k) pn.pos[l][k] = L.pos[k];
    if (time_scale > 0) pn.pos[l][net.dim] = L.layer * time_scale;
    pn.radius[l] = L.radius;
  }
  pn.holders.assign(pn.n_labels, {});
  for (int l = 0; l < pn.n_leaves; ++l)
    for (int x : pn.leaf_labels[l]) pn.holders[x].push_back(l);
  pn.global_out.assign(pn.n_labels, 0);
  for (int x : beta_labels) pn.global_out[x] = 1;
  for (int q : open_q) pn.global_out[net.final_label[q]] = 1;
}

// kernels of this library launched per slice group: the counter, the
// gather and the accumulation, plus every step's launches
static int launches_per_group(const Plan& p) {
  int per_group = 2 + (p.prog.gathers.empty() ? 0 : 1);
  for (auto& s : p.prog.steps) {
    if (s.kind == ST_PERMUTE || s.kind == ST_GROUPED) {
      per_group += 1;
      continue;
    }
    const GemmDesc& g = s.gemm;
    int chunks = (int)((g.batch + 65534) / 65535);
    if (g.kernel == KG_DOT && g.M <= 4 && g.N <= 4)
      per_group += chunks + 1;
    else if (g.splitk > 1)
      per_group += chunks + 1;
    else if (g.kernel == KG_TC)
      per_group += 3;
    else
      per_group += chunks;
  }
  return per_group;
}

// distances between consecutive layers tried by the space-time embedding
// (lattice units; the qubit spacing is 1)
static const double kTimeScales[] = {0.25, 0.5, 1.0, 2.0};

static void fill_report(Plan& p, double plan_ms) {
  tnc_plan_report& r = p.rep;
  const double groups = std::exp2((double)p.sliced_serial.size());
  r.paper_ops = p.prog.paper_ops_per_group * groups;
  r.real_flops = p.prog.flops_per_group * groups;
  r.bytes = p.prog.bytes_per_group * groups;
  r.peak_bytes = p.prog.peak_bytes;
  r.ws_bytes = p.prog.ws_bytes;
  r.n_sliced = (int)(p.sliced_serial.size() + p.sliced_par.size());
  r.n_slices = std::exp2((double)r.n_sliced);
  r.n_slice_groups = (int)groups;
  int nodes = 0;
  for (auto& s : p.prog.steps) nodes += s.kind == ST_GEMM ? 1 : s.kind == ST_GROUPED ? s.g_count : 0;
  r.n_nodes = nodes;
  r.n_leaves = (int)p.net.leaves.size();
  r.max_rank = p.prog.max_rank;
  const int per_group = launches_per_group(p);
  r.n_launches = (int)(per_group * groups);
  r.plan_ms = plan_ms;
}

}  // namespace tnc

using namespace tnc;

extern "C" {

const char* tnc_status_string(int s) {
  switch (s) {
    case TNC_OK: return "ok";
    case TNC_EINVAL: return "invalid argument";
    case TNC_ENOMEM: return "out of memory / workspace too small";
    case TNC_ECUDA: return "CUDA error";
    case TNC_ETIMEOUT: return "timed out";
    case TNC_EBUSY: return "busy";
    case TNC_ESTATE: return "invalid state";
    case TNC_ENOTFOUND: return "not found";
    default: return "unknown status";
  }
}

const char* tnc_last_error(void) { return g_err.c_str(); }

int tnc_load_network(const tnc_network_desc* desc, tnc_network_t** out) {
  return tnc_load_network_opts(desc, 0, out);
}

int tnc_load_network_opts(const tnc_network_desc* desc, int flags, tnc_network_t** out) {
  if (!out) {
    set_error("tnc_load_network: out is NULL");
    return TNC_EINVAL;
  }
  *out = nullptr;
  if (flags & ~TNC_NET_HYPEREDGES) {
    set_error("tnc_load_network_opts: unknown flags 0x%x", flags);
    return TNC_EINVAL;
  }
  auto* n = new tnc_network();
  int rc = build_network(desc, &n->net, flags);
  if (rc != TNC_OK) {
    delete n;
    return rc;
  }
  *out = n;
  return TNC_OK;
}

void tnc_free_network(tnc_network_t* net) { delete net; }

int tnc_ssa_separate(const double* pos, const double* rad, int n, int dim, uint64_t seed, int trials, int* side,
                     int* valid, int* k) {
  if (!pos || !rad || !side || !valid || !k || n < 2 || dim < 1 || dim > 3 || trials < 1) {
    set_error("tnc_ssa_separate: invalid argument");
    return TNC_EINVAL;
  }
  return ssa_separate_points(pos, rad, n, dim, seed, trials, side, valid, k);
}

int tnc_centerpoint(const double* pts, int n, int D, uint64_t seed, double* c) {
  if (!pts || !c || n < 1 || D < 1 || D > 4) {
    set_error("tnc_centerpoint: invalid argument");
    return TNC_EINVAL;
  }
  return centerpoint_points(pts, n, D, seed, c);
}

void tnc_plan_opts_default(tnc_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_batch = 1;
  o->form = TNC_FP32;
  o->seed = 1;
  o->ssa_trials = 32;
  o->leaf_size = 8;
  o->max_group_log2 = 6;
  o->use_graph = 1;
  o->embedding = TNC_EMBED_AUTO;
  o->n_starts = 4;
  o->refine_window = 8;
}

int tnc_plan(const tnc_network_t* net, const tnc_plan_opts* opts, tnc_plan_t** out, tnc_plan_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  if (!net || !opts || !out) {
    set_error("tnc_plan: NULL argument");
    return TNC_EINVAL;
  }
  *out = nullptr;
  const Network& N = net->net;
  if (opts->n_open < 0 || opts->n_open > 20 || (opts->n_open > 0 && !opts->open_qubits) ||
      opts->max_batch < 1 || opts->max_batch > 65536 || opts->form < 0 || opts->form > 2 ||
      opts->ssa_trials < 0 || opts->leaf_size < 0 || opts->max_group_log2 < 0 ||
      opts->max_group_log2 > 16 || opts->embedding < 0 || opts->embedding > 2 || opts->n_starts < 0 ||
      opts->n_starts > 64 || (opts->embedding == TNC_EMBED_SPACETIME && N.dim > 2) || opts->refine_window < 0 ||
      (opts->refine_window > 0 && opts->refine_window < 3) || opts->refine_window > 12) {
    set_error("tnc_plan: invalid options");
    return TNC_EINVAL;
  }
  std::vector<int> oq(opts->open_qubits, opts->open_qubits + opts->n_open);
  std::sort(oq.begin(), oq.end());
  for (size_t i = 0; i < oq.size(); ++i)
    if (oq[i] < 0 || oq[i] >= N.n_qubits || (i && oq[i] == oq[i - 1])) {
      set_error("tnc_plan: invalid open qubit list");
      return TNC_EINVAL;
    }
  auto* tp = new struct tnc_plan();
  Plan& p = tp->p;
  p.net = N;
  p.opts = *opts;
  p.opts.open_qubits = nullptr;
  p.open_qubits = oq;
  if (p.opts.ssa_trials == 0) p.opts.ssa_trials = 32;
  if (p.opts.leaf_size == 0) p.opts.leaf_size = 8;
  int bb = 0;
  while ((1 << bb) < opts->max_batch) ++bb;
  p.beta_bits = bb;
  // separator hierarchies over the embeddings and seeds asked for (each
  // refined if asked); without a cap the cheapest tree by Eq. 3 whose
  // intermediates the executor can address is kept, with a cap the cheapest
  // after slicing among the four cheapest trees (ties: the earlier candidate)
  struct Cand {
    Tree tree;
    PlanNet pn;
    std::vector<int> beta_labels;
    double cost, sep_cost, time_scale;
    int n_refined, embedding, seed, max_rank;
  };
  std::vector<Cand> cands;
  std::vector<double> scales;
  if (opts->embedding != TNC_EMBED_SPACETIME) scales.push_back(0.0);
  if (opts->embedding != TNC_EMBED_COLLAPSED && N.dim <= 2)
    for (double h : kTimeScales) scales.push_back(h);
  const int starts = std::max(1, opts->n_starts);
  for (double h : scales) {
    PlanNet pn;
    std::vector<int> bl;
    make_plan_net(p.net, p.open_qubits, bb, pn, bl, h);
    for (int k = 0; k < starts; ++k) {
      PlannerOpts po;
      po.seed = opts->seed + (uint64_t)k;
      po.trials = p.opts.ssa_trials;
      po.leaf_size = p.opts.leaf_size;
      PlannerStats st;
      Cand c;
      c.tree = plan_tree(pn, po, &st);
      c.sep_cost = tree_cost_log2(c.tree);
      c.n_refined = opts->refine_window ? refine_tree(pn, c.tree, opts->refine_window, 4) : 0;
      c.cost = tree_cost_log2(c.tree);
      c.max_rank = tree_max_rank(c.tree);
      c.pn = pn;
      c.beta_labels = bl;
      c.time_scale = h;
      c.embedding = h > 0 ? TNC_EMBED_SPACETIME : TNC_EMBED_COLLAPSED;
      c.seed = (int)po.seed;
      cands.push_back(std::move(c));
    }
  }
  std::vector<int> idx(cands.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cands[a].cost < cands[b].cost - 1e-9; });
  int pick = -1;
  if (opts->tree_only) {
    pick = idx[0];  // nothing is compiled: the cheapest tree whatever its largest intermediate
  } else if (!opts->mem_cap_bytes) {
    for (int i : idx)
      if (cands[i].max_rank <= kMaxRank) {
        pick = i;
        break;
      }
    if (pick < 0) pick = idx[0];  // compile_program reports the rank limit
  } else {
    double best_total = 1e300;
    for (size_t r = 0; r < idx.size() && r < 4; ++r) {
      Cand& c = cands[idx[r]];
      std::vector<int> S;
      double total = 0;
      Tree t = c.tree;
      if (choose_slices(c.pn, t, p.opts.form, opts->mem_cap_bytes, S, &total) != TNC_OK) continue;
      if (total < best_total - 1e-9) best_total = total, pick = idx[r];
    }
    if (pick < 0) pick = idx[0];  // plan_slices reports why it cannot slice
  }
  {
    Cand& c = cands[pick];
    p.tree = std::move(c.tree);
    p.pn = std::move(c.pn);
    p.beta_labels = c.beta_labels;
    p.rep.embedding_used = c.embedding;
    p.rep.seed_used = c.seed;
    p.rep.time_scale = c.time_scale;
    p.rep.sep_cost_log2 = c.sep_cost;
    p.rep.n_refined = c.n_refined;
  }
  p.rep.tree_cost_log2 = tree_cost_log2(p.tree);
  if (opts->tree_only) {
    // the tree and its Eq. 3 cost only: no slicing, no device program
    p.tree_only = true;
    p.rep.paper_ops = std::exp2(p.rep.tree_cost_log2);
    p.rep.n_leaves = (int)p.net.leaves.size();
    p.rep.max_rank = tree_max_rank(p.tree);
    p.rep.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = p.rep;
    *out = tp;
    return TNC_OK;
  }
  int rc = plan_slices(p, opts->mem_cap_bytes);
  if (rc == TNC_OK) rc = compile_program(p);
  if (rc == TNC_OK && opts->mem_cap_bytes && p.prog.ws_bytes > opts->mem_cap_bytes * 1.5 + (1 << 20)) {
    // the compiled arena can exceed the model by fragmentation; stay honest
    set_error("tnc_plan: compiled workspace %.3g B exceeds mem_cap_bytes", (double)p.prog.ws_bytes);
    rc = TNC_ENOMEM;
  }
  if (rc != TNC_OK) {
    delete tp;
    return rc;
  }
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  fill_report(p, ms);
  if (rep) *rep = p.rep;
  *out = tp;
  return TNC_OK;
}

int tnc_plan_get_report(const tnc_plan_t* plan, tnc_plan_report* rep) {
  if (!plan || !rep) {
    set_error("tnc_plan_get_report: NULL argument");
    return TNC_EINVAL;
  }
  *rep = plan->p.rep;
  return TNC_OK;
}

void tnc_free_plan(tnc_plan_t* plan) {
  if (!plan) return;
  Plan& p = plan->p;
  for (auto& r : p.prof) cudaEventDestroy((cudaEvent_t)r.ev);
  p.prof.clear();
  for (auto& ge : p.graphs) cudaGraphExecDestroy((cudaGraphExec_t)ge.exec);
  p.graphs.clear();
  if (p.d_base || p.d_gathers) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (p.device >= 0) cudaSetDevice(p.device);
    if (p.d_base) cudaFree(p.d_base);
    if (p.d_gathers) cudaFree(p.d_gathers);
    if (p.d_grouped) cudaFree(p.d_grouped);
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete plan;
}

int tnc_plan_export_json(const tnc_plan_t* plan, char* buf, size_t cap, size_t* needed) {
  if (!plan) {
    set_error("tnc_plan_export_json: NULL plan");
    return TNC_EINVAL;
  }
  const Plan& p = plan->p;
  std::ostringstream o;
  o.precision(17);
  auto vec = [&](const std::vector<int>& v) {
    o << "[";
    for (size_t i = 0; i < v.size(); ++i) o << (i ? "," : "") << v[i];
    o << "]";
  };
  o << "{\"n_qubits\":" << p.net.n_qubits << ",\"beta_bits\":" << p.beta_bits;
  o << ",\"beta_labels\":";
  vec(p.beta_labels);
  o << ",\"open_qubits\":";
  vec(p.open_qubits);
  o << ",\"final_label\":";
  vec(p.net.final_label);
  o << ",\"sliced_serial\":";
  vec(p.sliced_serial);
  o << ",\"sliced_par\":";
  vec(p.sliced_par);
  o << ",\"leaves\":[";
  for (size_t l = 0; l < p.net.leaves.size(); ++l) {
    const Leaf& L = p.net.leaves[l];
    o << (l ? "," : "") << "{\"labels\":";
    vec(L.labels);
    o << ",\"qubit\":" << L.qubit << ",\"re\":[";
    for (size_t i = 0; i < L.data.size(); ++i) o << (i ? "," : "") << L.data[i].real();
    o << "],\"im\":[";
    for (size_t i = 0; i < L.data.size(); ++i) o << (i ? "," : "") << L.data[i].imag();
    o << "]}";
  }
  o << "],\"nodes\":[";
  for (size_t v = 0; v < p.tree.nodes.size(); ++v) {
    const TreeNode& nd = p.tree.nodes[v];
    o << (v ? "," : "") << "{\"left\":" << nd.left << ",\"right\":" << nd.right
      << ",\"leaf\":" << nd.leaf << ",\"cost_log2\":" << nd.cost_log2 << ",\"out\":";
    vec(nd.out);
    o << "}";
  }
  o << "],\"root\":" << p.tree.root;
  // the compiled program, for host-side emulation
  const Program& pr = p.prog;
  o << ",\"program\":{\"ws_bytes\":" << pr.ws_bytes << ",\"off_bits\":" << pr.off_bits
    << ",\"off_ctr\":" << pr.off_ctr << ",\"n_groups\":" << p.rep.n_slice_groups << ",\"base_re\":[";
  for (size_t i = 0; i < pr.base_host.size(); ++i) o << (i ? "," : "") << pr.base_host[i].real();
  o << "],\"base_im\":[";
  for (size_t i = 0; i < pr.base_host.size(); ++i) o << (i ? "," : "") << pr.base_host[i].imag();
  o << "],\"gathers\":[";
  for (size_t i = 0; i < pr.gathers.size(); ++i) {
    const GatherDesc& g = pr.gathers[i];
    o << (i ? "," : "") << "{\"src\":" << g.src << ",\"dst\":" << g.dst << ",\"out_src\":[";
    for (int j = 0; j < g.out_rank; ++j) o << (j ? "," : "") << (int)g.out_src[j];
    o << "],\"fixed_pos\":[";
    for (int j = 0; j < g.n_fixed; ++j) o << (j ? "," : "") << (int)g.fixed_pos[j];
    o << "],\"fixed_qubit\":[";
    for (int j = 0; j < g.n_fixed; ++j) o << (j ? "," : "") << (int)g.fixed_qubit[j];
    o << "],\"sliced_pos\":[";
    for (int j = 0; j < g.n_sliced; ++j) o << (j ? "," : "") << (int)g.sliced_pos[j];
    o << "],\"sliced_bit\":[";
    for (int j = 0; j < g.n_sliced; ++j) o << (j ? "," : "") << (int)g.sliced_bit[j];
    o << "]}";
  }
  o << "],\"accum\":{\"src\":" << pr.accum.src << ",\"n_open\":" << pr.accum.n_open
    << ",\"n_beta\":" << pr.accum.n_beta << ",\"n_par\":" << pr.accum.n_par << ",\"role\":[";
  for (int j = 0; j < pr.accum.rank; ++j) o << (j ? "," : "") << (int)pr.accum.role[j];
  o << "],\"idx\":[";
  for (int j = 0; j < pr.accum.rank; ++j) o << (j ? "," : "") << (int)pr.accum.idx[j];
  o << "]}}";
  o << ",\"steps\":[";
  for (size_t i = 0; i < p.prog.steps.size(); ++i) {
    const Step& s = p.prog.steps[i];
    o << (i ? "," : "") << "{\"kind\":" << s.kind << ",\"node\":" << s.node;
    if (s.kind == ST_GROUPED) {
      o << ",\"problems\":[";
      for (int q = 0; q < s.g_count; ++q) {
        const GroupedDesc& gd = p.prog.grouped[s.g_first + q];
        o << (q ? "," : "") << "{\"batch\":" << gd.batch << ",\"M\":" << gd.M << ",\"N\":" << gd.N
          << ",\"K\":" << gd.K << ",\"tA\":0,\"tB\":1,\"kernel\":2,\"a\":" << gd.a << ",\"b\":" << gd.b
          << ",\"c\":" << gd.c << ",\"a_buf\":" << gd.a_buf << ",\"b_buf\":" << gd.b_buf
          << ",\"c_ident\":" << gd.c_ident << ",\"c_pos\":[";
        for (int j = 0; j < gd.nN + gd.nM + gd.nB; ++j) o << (j ? "," : "") << (int)gd.c_pos[j];
        o << "]}";
      }
      o << "]";
    } else if (s.kind == ST_GEMM) {
      o << ",\"batch\":" << s.gemm.batch << ",\"M\":" << s.gemm.M << ",\"N\":" << s.gemm.N
        << ",\"K\":" << s.gemm.K << ",\"kernel\":" << s.gemm.kernel << ",\"tA\":" << s.gemm.transA
        << ",\"tB\":" << s.gemm.transB << ",\"a\":" << s.gemm.a << ",\"b\":" << s.gemm.b
        << ",\"c\":" << s.gemm.c << ",\"a_buf\":" << s.gemm.a_buf << ",\"b_buf\":" << s.gemm.b_buf
        << ",\"c_ident\":" << s.gemm.c_ident << ",\"c_pos\":[";
      for (int j = 0; j < s.gemm.nN + s.gemm.nM + s.gemm.nB; ++j) o << (j ? "," : "") << (int)s.gemm.c_pos[j];
      o << "]";
    } else {
      o << ",\"rank\":" << s.perm.rank << ",\"src\":" << s.perm.src << ",\"dst\":" << s.perm.dst
        << ",\"src_bit\":[";
      for (int j = 0; j < s.perm.rank; ++j) o << (j ? "," : "") << (int)s.perm.src_bit[j];
      o << "]";
    }
    o << "}";
  }
  o << "]}";
  std::string s = o.str();
  if (needed) *needed = s.size();
  if (buf && cap) {
    size_t n = std::min(cap - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return TNC_OK;
}

int tnc_plan_upload(tnc_plan_t* plan, void* stream) {
  if (!plan) {
    set_error("tnc_plan_upload: NULL plan");
    return TNC_EINVAL;
  }
  Plan& p = plan->p;
  if (p.tree_only) {
    set_error("tnc_plan_upload: the plan was built with tree_only and has no device program");
    return TNC_ESTATE;
  }
  std::lock_guard<std::mutex> lk(p.mu);
  int dev = 0;
  cudaError_t e;
  if (stream) {
    e = cudaStreamGetDevice((cudaStream_t)stream, &dev);
    if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: cudaStreamGetDevice");
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: cudaSetDevice");
  }
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: cudaGetDevice");
  if (p.d_base && p.device == dev) return TNC_OK;
  if (p.d_base) {
    set_error("tnc_plan_upload: plan already resident on device %d", p.device);
    return TNC_ESTATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  size_t bb = std::max<size_t>(p.prog.base_elems * 8, 256);
  e = cudaMalloc(&p.d_base, bb);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: cudaMalloc");
  size_t gb = std::max<size_t>(p.prog.gathers.size() * sizeof(GatherDesc), 256);
  e = cudaMalloc(&p.d_gathers, gb);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: cudaMalloc");
  if (p.prog.base_elems) {
    e = cudaMemcpyAsync(p.d_base, p.prog.base_host.data(), p.prog.base_elems * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: copy leaves");
  }
  if (!p.prog.gathers.empty()) {
    e = cudaMemcpyAsync(p.d_gathers, p.prog.gathers.data(), p.prog.gathers.size() * sizeof(GatherDesc),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: copy descriptors");
  }
  size_t grb = std::max<size_t>(p.prog.grouped.size() * sizeof(GroupedDesc), 256);
  e = cudaMalloc(&p.d_grouped, grb);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: cudaMalloc");
  if (!p.prog.grouped.empty()) {
    e = cudaMemcpyAsync(p.d_grouped, p.prog.grouped.data(), p.prog.grouped.size() * sizeof(GroupedDesc),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: copy grouped descriptors");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_upload: sync");
  p.device = dev;
  // a plan that fits the static workspace may be contracted by
  // tnc_contract_amplitudes_static, which allocates nothing: its set-up
  // (kernels loaded, the array's address resolved) is done here, where
  // allocating is allowed.  A failure only disables that entry point.
  if (p.prog.ws_bytes <= static_workspace_bytes()) {
    std::string keep = tnc_last_error();
    if (prepare_static_workspace(dev) != TNC_OK) cudaGetLastError();
    set_error("%s", keep.c_str());
  }
  return TNC_OK;
}

// The executor: per serial slice group set the counter, gather the derived
// leaves, run the node program, accumulate the root in FP64.
static int run(tnc_plan_t* tp, const uint8_t* bits, bool bits_on_device, int batch, int g0, int g1, void* d_out,
               void* d_ws, size_t ws_bytes, void* stream, bool allow_graph = true) {
  Plan& p = tp->p;
  if (!d_out || !d_ws || !bits) {
    set_error("tnc_contract: NULL pointer argument");
    return TNC_EINVAL;
  }
  const int maxb = 1 << p.beta_bits;
  if (batch < 1 || batch > maxb || batch > std::max(1, p.opts.max_batch)) {
    set_error("tnc_contract: batch %d outside 1..%d", batch, p.opts.max_batch);
    return TNC_EINVAL;
  }
  if (ws_bytes < p.prog.ws_bytes) {
    set_error("tnc_contract: workspace of %zu bytes < required %llu", ws_bytes,
              (unsigned long long)p.prog.ws_bytes);
    return TNC_ENOMEM;
  }
  if (((uintptr_t)d_ws & 255) != 0) {
    set_error("tnc_contract: workspace not 256-byte aligned");
    return TNC_EINVAL;
  }
  const int ngroups = p.rep.n_slice_groups;
  if (g0 < 0 || g1 < g0 || g1 > ngroups) {
    set_error("tnc_contract: slice groups [%d, %d) outside [0, %d)", g0, g1, ngroups);
    return TNC_EINVAL;
  }
  // the device is the one owning the workspace (this library keeps its own
  // CUDA runtime state, so it follows the caller's memory, not a global)
  {
    cudaPointerAttributes attr;
    cudaError_t e0 = cudaPointerGetAttributes(&attr, d_ws);
    if (e0 != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      set_error("tnc_contract: workspace is not device memory");
      return TNC_EINVAL;
    }
    e0 = cudaSetDevice(attr.device);
    if (e0 != cudaSuccess) return cuda_fail(e0, "tnc_contract: cudaSetDevice");
  }
  int rc = tnc_plan_upload(tp, stream);
  if (rc != TNC_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  const int nq = p.net.n_qubits;
  cudaError_t e;
  // stage the bitstrings (zero-padded to the padded batch)
  e = cudaMemsetAsync(ws + p.prog.off_bits, 0, (size_t)maxb * nq, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_contract: memset");
  e = cudaMemcpyAsync(ws + p.prog.off_bits, bits, (size_t)batch * nq,
                      bits_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_contract: copy bits");
  const size_t out_bytes = (size_t)batch * ((size_t)16 << p.open_qubits.size());
  double2* acc = (double2*)(ws + p.prog.off_acc);
  e = cudaMemsetAsync(acc, 0, out_bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_contract: memset accumulator");
  uint64_t* d_ctr = (uint64_t*)(ws + p.prog.off_ctr);
  auto mark = [&](int step) -> int {
    if (!p.profiling) return TNC_OK;
    cudaEvent_t ev;
    cudaError_t ee = cudaEventCreate(&ev);
    if (ee != cudaSuccess) return cuda_fail(ee, "profiling: cudaEventCreate");
    ee = cudaEventRecord(ev, st);
    if (ee != cudaSuccess) return cuda_fail(ee, "profiling: cudaEventRecord");
    p.prof.push_back({step, (void*)ev});
    return TNC_OK;
  };
  // one slice group's program: gather, node steps, FP64 accumulation
  auto program = [&](cudaStream_t s, bool marks) -> int {
    int r;
    if (!p.prog.gathers.empty()) {
      r = launch_gather((const GatherDesc*)p.d_gathers, (int)p.prog.gathers.size(), p.prog.max_gather_rank,
                        p.d_base, ws, (const uint8_t*)(ws + p.prog.off_bits), nq, d_ctr, s);
      if (r) return cuda_fail((cudaError_t)r, "gather");
    }
    if (marks && (r = mark(-2)) != TNC_OK) return r;
    for (size_t si = 0; si < p.prog.steps.size(); ++si) {
      const Step& sp = p.prog.steps[si];
      if (sp.kind == ST_PERMUTE)
        r = launch_permute(sp.perm, ws, s);
      else if (sp.kind == ST_GROUPED)
        r = launch_grouped_narrow((const GroupedDesc*)p.d_grouped + sp.g_first, sp.g_count, sp.g_blocks,
                                  p.d_base, ws, s);
      else
        r = launch_gemm(sp.gemm, p.d_base, ws, s);
      if (r)
        return cuda_fail((cudaError_t)r,
                         sp.kind == ST_PERMUTE ? "permute" : sp.kind == ST_GROUPED ? "grouped" : "gemm");
      if (marks && (r = mark((int)si)) != TNC_OK) return r;
    }
    r = launch_accum(p.prog.accum, ws, acc, batch, s);
    if (r) return cuda_fail((cudaError_t)r, "accum");
    return TNC_OK;
  };
  cudaGraphExec_t gexec = nullptr;
  if (allow_graph && p.opts.use_graph && !p.profiling && g1 > g0) {
    for (auto& ge : p.graphs)
      if (ge.ws == d_ws && ge.batch == batch) gexec = (cudaGraphExec_t)ge.exec;
    if (!gexec) {
      // capture on a private stream (the caller's may be the legacy stream)
      cudaStream_t cs;
      e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "graph: cudaStreamCreate");
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(e, "graph: cudaStreamBeginCapture");
      }
      int rc2 = program(cs, false);
      cudaGraph_t graph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      cudaStreamDestroy(cs);
      if (rc2 != TNC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc2;
      }
      if (e2 != cudaSuccess) return cuda_fail(e2, "graph: cudaStreamEndCapture");
      e2 = cudaGraphInstantiate(&gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e2 != cudaSuccess) return cuda_fail(e2, "graph: cudaGraphInstantiate");
      if (p.graphs.size() >= 4) {
        cudaGraphExecDestroy((cudaGraphExec_t)p.graphs.front().exec);
        p.graphs.erase(p.graphs.begin());
      }
      p.graphs.push_back({d_ws, batch, (void*)gexec});
    }
  }
  for (int g = g0; g < g1; ++g) {
    int r;
    if ((r = mark(-1)) != TNC_OK) return r;
    if ((r = launch_set_counter(d_ctr, (uint64_t)g, st))) return cuda_fail((cudaError_t)r, "set counter");
    if (gexec) {
      e = cudaGraphLaunch(gexec, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    } else if ((r = program(st, true)) != TNC_OK) {
      return r;
    }
  }
  e = cudaMemcpyAsync(d_out, acc, out_bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_contract: copy out");
  return TNC_OK;
}

}  // extern "C"

namespace tnc {
// Host-bitstring contraction without CUDA-graph capture (used by the server,
// whose workspace differs per request, and by the static-workspace entry
// point, which must not take driver resources).
int run_request(tnc_plan_t* plan, const uint8_t* host_bits, int batch, void* d_out, void* d_ws, size_t ws_bytes,
                void* stream) {
  return run(plan, host_bits, false, batch, 0, plan->p.rep.n_slice_groups, d_out, d_ws, ws_bytes, stream, false);
}
}  // namespace tnc

extern "C" {

static int device_of(const void* p, const char* who) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("%s: pointer is not device memory", who);
    return TNC_EINVAL;
  }
  cudaError_t e = cudaSetDevice(attr.device);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return TNC_OK;
}

int tnc_permute(const void* d_in, void* d_out, int rank, const int* src_bit, void* stream) {
  if (!d_in || !d_out || rank < 0 || rank > 40 || (rank > 0 && !src_bit)) {
    set_error("tnc_permute: invalid argument");
    return TNC_EINVAL;
  }
  PermDesc d;
  std::memset(&d, 0, sizeof(d));
  d.rank = rank;
  unsigned long long seen = 0;
  for (int j = 0; j < rank; ++j) {
    if (src_bit[j] < 0 || src_bit[j] >= rank || ((seen >> src_bit[j]) & 1)) {
      set_error("tnc_permute: src_bit is not a permutation of 0..%d", rank - 1);
      return TNC_EINVAL;
    }
    seen |= 1ull << src_bit[j];
    d.src_bit[j] = (int8_t)src_bit[j];
  }
  int rc = device_of(d_out, "tnc_permute");
  if (rc != TNC_OK) return rc;
  int r = launch_permute_ptr(d, d_in, d_out, stream);
  return r ? cuda_fail((cudaError_t)r, "tnc_permute") : TNC_OK;
}

static GemmDesc make_gemm(int64_t batch, int64_t M, int64_t N, int64_t K, int tA, int tB, int form) {
  GemmDesc g;
  std::memset(&g, 0, sizeof(g));
  g.batch = batch, g.M = M, g.N = N, g.K = K, g.transA = tA, g.transB = tB, g.form = form;
  g.c_ident = 1;  // C stored [b][M][N]
  choose_gemm_kernel(g);
  return g;
}

size_t tnc_cgemm_scratch_bytes(int64_t batch, int64_t M, int64_t N, int64_t K, int form) {
  if (batch < 1 || M < 1 || N < 1 || K < 1 || form < 0 || form > 2) return 0;
  // enough for every variant tnc_cgemm_variant accepts for this shape
  GemmDesc cand[kMaxCandidates];
  int n = 0;
  gemm_candidates(make_gemm(batch, M, N, K, 0, 0, form), cand, &n);
  uint64_t need = 0;
  for (int i = 0; i < n; ++i) need = std::max<uint64_t>(need, gemm_scratch_bytes(cand[i]));
  return (size_t)need;
}

int tnc_cgemm_variant(const void* A, const void* B, void* Cp, int64_t batch, int64_t M, int64_t N, int64_t K,
                      int tA, int tB, int form, int kernel, int tile, const int* c_pos, void* scratch,
                      size_t scratch_bytes, void* stream) {
  if (!A || !B || !Cp || batch < 1 || M < 1 || N < 1 || K < 1 || form < 0 || form > 2 || (tA & ~1) ||
      (tB & ~1)) {
    set_error("tnc_cgemm: invalid argument");
    return TNC_EINVAL;
  }
  GemmDesc g = make_gemm(batch, M, N, K, tA, tB, form);
  if (c_pos) {
    // C stored as a permutation of the bits of [b][M][N] (powers of two)
    auto lg = [](int64_t v) { int r = 0; while (((int64_t)1 << r) < v) ++r; return ((int64_t)1 << r) == v ? r : -1; };
    const int nN = lg(N), nM = lg(M), nB = lg(batch);
    const int nb = nN + nM + nB;
    if (nN < 0 || nM < 0 || nB < 0 || nb > kMaxRank) {
      set_error("tnc_cgemm_variant: c_pos needs power-of-two batch, M, N");
      return TNC_EINVAL;
    }
    uint64_t seen = 0;
    for (int i = 0; i < nb; ++i) {
      if (c_pos[i] < 0 || c_pos[i] >= nb || ((seen >> c_pos[i]) & 1)) {
        set_error("tnc_cgemm_variant: c_pos is not a permutation of 0..%d", nb - 1);
        return TNC_EINVAL;
      }
      seen |= (uint64_t)1 << c_pos[i];
    }
    g.c_ident = 1;
    for (int i = 0; i < nb; ++i) {
      g.c_pos[i] = (int8_t)c_pos[i];
      if (c_pos[i] != i) g.c_ident = 0;
    }
    g.nN = nN, g.nM = nM, g.nB = nB;
  }
  if (kernel >= 0) {
    GemmDesc cand[kMaxCandidates];
    int n = 0, hit = -1;
    gemm_candidates(g, cand, &n);
    for (int i = 0; i < n && hit < 0; ++i)
      if (cand[i].kernel == kernel && (tile < 0 || cand[i].tile == tile)) hit = i;
    if (hit < 0) {
      set_error("tnc_cgemm_variant: kernel %d tile %d cannot run this shape", kernel, tile);
      return TNC_EINVAL;
    }
    g = cand[hit];
  }
  const uint64_t need = gemm_scratch_bytes(g);
  if (need > scratch_bytes || (need && !scratch)) {
    set_error("tnc_cgemm: scratch of %zu bytes < required %llu", scratch_bytes, (unsigned long long)need);
    return TNC_ENOMEM;
  }
  if (need && ((uintptr_t)scratch & 255)) {
    set_error("tnc_cgemm: scratch not 256-byte aligned");
    return TNC_EINVAL;
  }
  g.scratch_elems = need / 8;
  int rc = device_of(Cp, "tnc_cgemm");
  if (rc != TNC_OK) return rc;
  int r = launch_gemm_ptr(g, A, B, Cp, scratch, stream);
  return r ? cuda_fail((cudaError_t)r, "tnc_cgemm") : TNC_OK;
}

int tnc_cgemm(const void* A, const void* B, void* Cp, int64_t batch, int64_t M, int64_t N, int64_t K, int tA,
              int tB, int form, void* scratch, size_t scratch_bytes, void* stream) {
  return tnc_cgemm_variant(A, B, Cp, batch, M, N, K, tA, tB, form, -1, -1, nullptr, scratch, scratch_bytes, stream);
}

int tnc_plan_autotune(tnc_plan_t* plan, void* d_ws, size_t ws_bytes, void* stream, int reps, int* n_changed) {
  if (!plan || !d_ws || reps < 1) {
    set_error("tnc_plan_autotune: invalid argument");
    return TNC_EINVAL;
  }
  Plan& p = plan->p;
  if (p.tree_only) {
    set_error("tnc_plan_autotune: the plan was built with tree_only and has no device program");
    return TNC_ESTATE;
  }
  if (ws_bytes < p.prog.ws_bytes || ((uintptr_t)d_ws & 255)) {
    set_error("tnc_plan_autotune: workspace too small or not 256-byte aligned");
    return ws_bytes < p.prog.ws_bytes ? TNC_ENOMEM : TNC_EINVAL;
  }
  int rc = device_of(d_ws, "tnc_plan_autotune");
  if (rc != TNC_OK) return rc;
  if ((rc = tnc_plan_upload(plan, stream)) != TNC_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  const int nq = p.net.n_qubits;
  cudaError_t e = cudaMemsetAsync(ws + p.prog.off_bits, 0, ((size_t)1 << p.beta_bits) * nq, st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_autotune: memset");
  uint64_t* d_ctr = (uint64_t*)(ws + p.prog.off_ctr);
  int r = launch_set_counter(d_ctr, 0, st);
  if (!r && !p.prog.gathers.empty())
    r = launch_gather((const GatherDesc*)p.d_gathers, (int)p.prog.gathers.size(), p.prog.max_gather_rank, p.d_base,
                      ws, (const uint8_t*)(ws + p.prog.off_bits), nq, d_ctr, st);
  if (r) return cuda_fail((cudaError_t)r, "tnc_plan_autotune: gather");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int changed = 0;
  for (Step& s : p.prog.steps) {
    if (s.kind == ST_GROUPED) {
      r = launch_grouped_narrow((const GroupedDesc*)p.d_grouped + s.g_first, s.g_count, s.g_blocks, p.d_base, ws, st);
      if (r) break;
      continue;
    }
    if (s.kind != ST_GEMM) continue;
    GemmDesc cand[kMaxCandidates];
    int nc = 0;
    gemm_candidates(s.gemm, cand, &nc);
    int best = 0;
    float best_ms = 3.4e38f;
    for (int q = 0; q < nc; ++q) {
      GemmDesc g = cand[q];
      g.scratch = s.gemm.scratch;
      g.scratch_elems = s.gemm.scratch_elems;
      if (gemm_scratch_bytes(g) > g.scratch_elems * 8) continue;
      if (launch_gemm(g, p.d_base, ws, st)) {
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, st);
      for (int i = 0; i < reps; ++i) launch_gemm(g, p.d_base, ws, st);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "tnc_plan_autotune: timing");
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) best_ms = ms, best = q;
    }
    GemmDesc g = cand[best];
    g.scratch = s.gemm.scratch;
    g.scratch_elems = s.gemm.scratch_elems;
    if (g.kernel != s.gemm.kernel || g.tile != s.gemm.tile) ++changed;
    s.gemm = g;
    if ((r = launch_gemm(s.gemm, p.d_base, ws, st))) break;  // leave real data for the next steps
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r) return cuda_fail((cudaError_t)r, "tnc_plan_autotune: launch");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_autotune: sync");
  for (auto& ge : p.graphs) cudaGraphExecDestroy((cudaGraphExec_t)ge.exec);
  p.graphs.clear();
  p.rep.n_launches = launches_per_group(p) * p.rep.n_slice_groups;
  if (n_changed) *n_changed = changed;
  return TNC_OK;
}

int tnc_plan_get_kernels(const tnc_plan_t* plan, int* choices, int cap, int* n_steps) {
  if (!plan || !n_steps) {
    set_error("tnc_plan_get_kernels: NULL argument");
    return TNC_EINVAL;
  }
  const Plan& p = plan->p;
  const int n = (int)p.prog.steps.size();
  *n_steps = n;
  if (!choices) return TNC_OK;
  if (cap < 2 * n) {
    set_error("tnc_plan_get_kernels: cap %d < %d", cap, 2 * n);
    return TNC_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    const Step& s = p.prog.steps[i];
    choices[2 * i] = s.kind == ST_GEMM ? s.gemm.kernel : -1;
    choices[2 * i + 1] = s.kind == ST_GEMM ? s.gemm.tile : -1;
  }
  return TNC_OK;
}

int tnc_plan_set_kernels(tnc_plan_t* plan, const int* choices, int n_steps) {
  if (!plan || !choices) {
    set_error("tnc_plan_set_kernels: NULL argument");
    return TNC_EINVAL;
  }
  Plan& p = plan->p;
  if (n_steps != (int)p.prog.steps.size()) {
    set_error("tnc_plan_set_kernels: %d choices for %zu steps", n_steps, p.prog.steps.size());
    return TNC_EINVAL;
  }
  std::vector<GemmDesc> chosen(n_steps);
  for (int i = 0; i < n_steps; ++i) {
    const Step& s = p.prog.steps[i];
    if (s.kind != ST_GEMM) continue;
    GemmDesc cand[kMaxCandidates];
    int nc = 0, hit = -1;
    gemm_candidates(s.gemm, cand, &nc);
    for (int q = 0; q < nc; ++q)
      if (cand[q].kernel == choices[2 * i] && cand[q].tile == choices[2 * i + 1]) hit = q;
    if (hit < 0) {
      set_error("tnc_plan_set_kernels: step %d cannot run kernel %d tile %d", i, choices[2 * i], choices[2 * i + 1]);
      return TNC_EINVAL;
    }
    chosen[i] = cand[hit];
    chosen[i].scratch = s.gemm.scratch;
    chosen[i].scratch_elems = s.gemm.scratch_elems;
    if (gemm_scratch_bytes(chosen[i]) > chosen[i].scratch_elems * 8) {
      set_error("tnc_plan_set_kernels: step %d: scratch too small for kernel %d", i, choices[2 * i]);
      return TNC_EINVAL;
    }
  }
  for (int i = 0; i < n_steps; ++i)
    if (p.prog.steps[i].kind == ST_GEMM) p.prog.steps[i].gemm = chosen[i];
  for (auto& ge : p.graphs) cudaGraphExecDestroy((cudaGraphExec_t)ge.exec);
  p.graphs.clear();
  p.rep.n_launches = launches_per_group(p) * p.rep.n_slice_groups;
  return TNC_OK;
}

int tnc_device_error(int* flag) {
  if (!flag) {
    set_error("tnc_device_error: NULL argument");
    return TNC_EINVAL;
  }
  int r = tnc::read_tc_error(flag);
  if (r) return cuda_fail((cudaError_t)r, "tnc_device_error");
  if (*flag) {
    set_error("tnc_device_error: a bounded device wait gave up (code %d)", *flag);
    return TNC_ETIMEOUT;
  }
  return TNC_OK;
}

int tnc_selftest_bounded_wait(unsigned limit_us, int* timed_out) {
  if (!timed_out || limit_us == 0 || limit_us > 1000000) {
    set_error("tnc_selftest_bounded_wait: invalid argument");
    return TNC_EINVAL;
  }
  int r = tnc::bounded_wait_selftest((uint64_t)limit_us * 1000, timed_out);
  if (r) return cuda_fail((cudaError_t)r, "tnc_selftest_bounded_wait");
  if (*timed_out) {
    set_error("tnc_selftest_bounded_wait: the wait gave up after %u us", limit_us);
    return TNC_ETIMEOUT;
  }
  return TNC_OK;
}

static void drop_profile(Plan& p) {
  for (auto& r : p.prof) cudaEventDestroy((cudaEvent_t)r.ev);
  p.prof.clear();
  p.prof_ms.assign(p.prog.steps.size(), 0.0);
  p.prof_runs.assign(p.prog.steps.size(), 0);
}

int tnc_plan_set_profiling(tnc_plan_t* plan, int enable) {
  if (!plan) {
    set_error("tnc_plan_set_profiling: NULL plan");
    return TNC_EINVAL;
  }
  Plan& p = plan->p;
  drop_profile(p);
  p.profiling = enable != 0;
  return TNC_OK;
}

int tnc_plan_get_profile(tnc_plan_t* plan, int* n_steps, int cap, double* ms, int* runs, int* kind, double* flops,
                         double* bytes) {
  if (!plan || !n_steps) {
    set_error("tnc_plan_get_profile: NULL argument");
    return TNC_EINVAL;
  }
  Plan& p = plan->p;
  const int n = (int)p.prog.steps.size();
  *n_steps = n;
  if (p.prof_ms.size() != (size_t)n) {
    p.prof_ms.assign(n, 0.0);
    p.prof_runs.assign(n, 0);
  }
  // fold the recorded events: each step's time is from the previous record
  cudaEvent_t prev = nullptr;
  for (auto& r : p.prof) {
    cudaEvent_t ev = (cudaEvent_t)r.ev;
    cudaError_t e = cudaEventSynchronize(ev);
    if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_get_profile: cudaEventSynchronize");
    if (r.step >= 0 && prev) {
      float t = 0;
      e = cudaEventElapsedTime(&t, prev, ev);
      if (e != cudaSuccess) return cuda_fail(e, "tnc_plan_get_profile: cudaEventElapsedTime");
      p.prof_ms[r.step] += t;
      p.prof_runs[r.step] += 1;
    }
    prev = (r.step == -1) ? nullptr : ev;
  }
  for (auto& r : p.prof) cudaEventDestroy((cudaEvent_t)r.ev);
  p.prof.clear();
  for (int i = 0; i < n && i < cap; ++i) {
    const Step& s = p.prog.steps[i];
    if (ms) ms[i] = p.prof_ms[i];
    if (runs) runs[i] = p.prof_runs[i];
    if (kind)
      kind[i] = s.kind == ST_PERMUTE ? TNC_STEP_PERMUTE : s.kind == ST_GROUPED ? TNC_STEP_GROUPED : s.gemm.kernel;
    double f = 0, b = 0;
    if (s.kind == ST_GROUPED) {
      for (int q = 0; q < s.g_count; ++q) {
        const GroupedDesc& gd = p.prog.grouped[s.g_first + q];
        f += 8.0 * gd.batch * gd.M * gd.N * gd.K;
        b += 8.0 * gd.batch * ((double)gd.M * gd.K + (double)gd.K * gd.N + (double)gd.M * gd.N);
      }
    } else if (s.kind == ST_GEMM) {
      const GemmDesc& g = s.gemm;
      f = 8.0 * g.batch * g.M * g.N * g.K;
      b = 8.0 * g.batch * ((double)g.M * g.K + (double)g.K * g.N + (double)g.M * g.N);
    } else {
      b = 16.0 * std::exp2((double)s.perm.rank);
    }
    if (flops) flops[i] = f;
    if (bytes) bytes[i] = b;
  }
  return TNC_OK;
}

int tnc_contract_amplitudes(tnc_plan_t* plan, const uint8_t* bits, int batch, void* d_out, void* d_ws,
                            size_t ws_bytes, void* stream) {
  if (!plan) {
    set_error("tnc_contract_amplitudes: NULL plan");
    return TNC_EINVAL;
  }
  return run(plan, bits, false, batch, 0, plan->p.rep.n_slice_groups, d_out, d_ws, ws_bytes, stream);
}

int tnc_contract_amplitudes_dbits(tnc_plan_t* plan, const uint8_t* d_bits, int batch, void* d_out, void* d_ws,
                                  size_t ws_bytes, void* stream) {
  if (!plan) {
    set_error("tnc_contract_amplitudes_dbits: NULL plan");
    return TNC_EINVAL;
  }
  return run(plan, d_bits, true, batch, 0, plan->p.rep.n_slice_groups, d_out, d_ws, ws_bytes, stream);
}

int tnc_contract_partial(tnc_plan_t* plan, const uint8_t* d_bits, int batch, int g0, int g1, void* d_out,
                         void* d_ws, size_t ws_bytes, void* stream) {
  if (!plan) {
    set_error("tnc_contract_partial: NULL plan");
    return TNC_EINVAL;
  }
  return run(plan, d_bits, true, batch, g0, g1, d_out, d_ws, ws_bytes, stream);
}

}  // extern "C"
