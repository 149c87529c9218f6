// Internal host-side structures of the executor: the tensor network, the
// contraction tree, the compiled node program and the plan.
#pragma once
#include <array>
#include <complex>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tnc.h"
#include "tnc_kernels.h"

namespace tnc {

using cd = std::complex<double>;

void set_error(const char* fmt, ...);

enum LabelKind { LK_WIRE = 0, LK_BOND = 1, LK_FINAL = 2, LK_BETA = 3 };

// One tensor of the network.  labels[0] is the most significant index of the
// row-major data (2^rank entries, all indices binary).
struct Leaf {
  std::vector<int> labels;
  std::vector<cd> data;
  double pos[3] = {0, 0, 0};
  double radius = 0;
  int qubit = -1;
  int time = 0;   // index of the 2q gate among the circuit's 2q gates
  int layer = 0;  // ASAP layer: 1 + the latest layer on either of its qubits (0 for a bare wire)
  bool diag = false;  // hyper-edge form: the diagonal of a diagonal gate on its wire labels
};

struct Network {
  int n_qubits = 0, dim = 2;
  std::vector<double> coords;
  std::vector<Leaf> leaves;
  std::vector<int> label_kind;    // per label
  std::vector<int> final_label;   // per qubit: label of its last wire
  std::vector<int> final_holder;  // per qubit: leaf holding that label
  double gate_range = 1.0;        // l: largest distance between the qubits of a gate
  int n_gates_2q = 0;
};

int build_network(const tnc_network_desc* desc, Network* net, int flags);

// ------------------------------------------------------------------ planning
// Planning view of the network: leaf label sets after the request-specific
// edits (fixed final wires replaced by the beta bits), and the labels that
// survive to the root.
struct PlanNet {
  int n_leaves = 0;
  int n_labels = 0;
  std::vector<std::vector<int>> leaf_labels;
  std::vector<std::array<double, 3>> pos;
  std::vector<double> radius;
  std::vector<std::vector<int>> holders;  // per label: leaves holding it
  std::vector<char> global_out;           // per label: kept to the root
  int dim = 2;
};

struct TreeNode {
  int left = -1, right = -1;  // children (node ids); -1 for a leaf node
  int leaf = -1;              // leaf id for leaf nodes
  std::vector<int> out;       // output labels (unordered set, sorted)
  double cost_log2 = -1;      // log2 of M (Eq. 3) for internal nodes
};

struct Tree {
  std::vector<TreeNode> nodes;
  int root = -1;
};

struct PlannerOpts {
  uint64_t seed = 1;
  int trials = 32;
  int leaf_size = 8;
};

// Separator hierarchy (Thm. 1 proof) with Algorithm 1 separators and greedy
// leaves.  Returns the tree; fills stats.
struct PlannerStats {
  int ssa_calls = 0, ssa_valid = 0, ssa_fallback = 0, greedy_clusters = 0;
};
Tree plan_tree(const PlanNet& pn, const PlannerOpts& o, PlannerStats* st);
int ssa_separate_points(const double* pos, const double* rad, int n, int dim, uint64_t seed, int trials,
                        int* cls_out, int* valid, int* k_out);
int centerpoint_points(const double* pts, int n, int D, uint64_t seed, double* c);

// Node output labels recomputed for a given set of labels that are kept to
// the root; cost and size in log2.
void annotate_tree(const PlanNet& pn, Tree& t);
double tree_cost_log2(const Tree& t);       // log2 sum_nodes 2 M
// exact re-association of windows of at most max_items subtrees (refine.cpp);
// returns the number of windows rebuilt
int refine_tree(const PlanNet& pn, Tree& t, int max_items, int max_passes);
int tree_max_rank(const Tree& t);

// ------------------------------------------------------------------ program
enum StepKind { ST_PERMUTE = 0, ST_GEMM = 1, ST_GROUPED = 2 };

struct Step {
  int kind;
  PermDesc perm;
  GemmDesc gemm;
  int node;  // tree node this step belongs to (-1 for a grouped step)
  // grouped step: problems [g_first, g_first + g_count) of Program::grouped
  int g_first, g_count;
  int64_t g_blocks;
};

struct Program {
  std::vector<GatherDesc> gathers;
  std::vector<GroupedDesc> grouped;
  int max_gather_rank = 0;
  std::vector<Step> steps;
  AccumDesc accum;
  uint64_t ws_bytes = 0;
  uint64_t off_bits = 0, off_ctr = 0;   // byte offsets in the workspace
  uint64_t off_acc = 0;                 // FP64 accumulator of the amplitudes
  uint64_t base_elems = 0;              // complex64 elements of the leaf buffer
  std::vector<std::complex<float>> base_host;
  double flops_per_group = 0, bytes_per_group = 0, paper_ops_per_group = 0;
  double peak_bytes = 0;
  int max_rank = 0;
};

struct Plan {
  Network net;           // copy of the network (leaf data, final wires)
  PlanNet pn;
  Tree tree;
  tnc_plan_opts opts;
  std::vector<int> open_qubits;  // sorted
  int beta_bits = 0;             // log2 of the padded batch
  std::vector<int> beta_labels;  // label id of beta bit b
  std::vector<int> sliced_serial, sliced_par;
  Program prog;
  tnc_plan_report rep{};
  bool tree_only = false;  // built with tnc_plan_opts.tree_only: no device program
  // per-step CUDA-event profiling
  bool profiling = false;
  struct ProfRec {
    int step;  // -1 marks the start of a slice group
    void* ev;
  };
  std::vector<ProfRec> prof;
  std::vector<void*> ev_pool;
  std::vector<double> prof_ms;
  std::vector<int> prof_runs;
  // captured CUDA graphs of one slice group, per (workspace, batch)
  struct GraphEntry {
    void* ws;
    int batch;
    void* exec;
  };
  std::vector<GraphEntry> graphs;
  // device state
  int device = -1;
  void* d_base = nullptr;        // leaf buffer (complex64)
  void* d_gathers = nullptr;
  void* d_grouped = nullptr;
  std::mutex mu;
};

int compile_program(Plan& p);
int plan_slices(Plan& p, size_t cap_bytes);
// sliced labels of one tree under a memory cap (compile.cpp); *total_log2 =
// log2 of the paper ops of all slices
int choose_slices(const PlanNet& base, Tree& t, int form, size_t cap_bytes, std::vector<int>& S,
                  double* total_log2);

}  // namespace tnc

struct tnc_network {
  tnc::Network net;
};
struct tnc_plan {
  tnc::Plan p;
};
