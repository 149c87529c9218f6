// Tree refinement: exact re-association of small windows of the separator
// tree.  This is an addition to the paper's method, which stops at the
// separator hierarchy with greedy leaves.
//
// A window is an internal node v together with the part of its subtree down
// to a frontier of at most W subtrees ("items"), found by repeatedly
// expanding the item whose own merge is the most expensive.  The items'
// output label sets fix everything the window can change: the way the items
// are combined into v's output.  The cheapest way, by the Eq. 3 cost
// (sum of 2 M over the window's merges, M = 2^(distinct labels of both
// operands)), is found exactly by dynamic programming over subsets of the
// items (the subset recursion of Pfeifer, Haegeman and Verstraete, Phys. Rev.
// E 90, 033315, 2014, restricted to the window).  The window is rebuilt when
// that is cheaper and no intermediate of the new window is larger than the
// largest one of the old window, so the refinement never raises the Eq. 3
// cost of the tree and never enlarges its largest intermediate.
#include <algorithm>
#include <array>
#include <cmath>
#include <functional>
#include <vector>

#include "tnc_internal.h"

namespace tnc {

namespace {

constexpr int kWords = 8;  // labels of one window: at most 512
using Bits = std::array<uint64_t, kWords>;

int popc(const Bits& b) {
  int c = 0;
  for (uint64_t w : b) c += __builtin_popcountll(w);
  return c;
}

class Refiner {
 public:
  Refiner(const PlanNet& pn, Tree& t) : pn_(pn), t_(t) {}

  // One pass over all internal nodes, children before parents; returns the
  // number of windows rebuilt.
  int pass(int max_items) {
    int changed = 0;
    std::vector<int> order;
    std::function<void(int)> post = [&](int v) {
      const TreeNode& nd = t_.nodes[v];
      if (nd.left < 0) return;
      post(nd.left);
      post(nd.right);
      order.push_back(v);
    };
    post(t_.root);
    for (int v : order) changed += window(v, max_items);
    return changed;
  }

 private:
  const PlanNet& pn_;
  Tree& t_;

  bool internal(int v) const { return t_.nodes[v].left >= 0; }

  int window(int v, int max_items) {
    std::vector<int> items = {t_.nodes[v].left, t_.nodes[v].right};
    std::vector<int> inner = {v};
    while ((int)items.size() < max_items) {
      int pick = -1;
      for (size_t i = 0; i < items.size(); ++i)
        if (internal(items[i]) &&
            (pick < 0 || t_.nodes[items[i]].cost_log2 > t_.nodes[items[pick]].cost_log2))
          pick = (int)i;
      if (pick < 0) break;
      const int u = items[pick];
      inner.push_back(u);
      items[pick] = t_.nodes[u].left;
      items.push_back(t_.nodes[u].right);
    }
    const int n = (int)items.size();
    if (n < 3) return 0;  // two items combine one way only
    // current cost and largest intermediate of the window
    double cur = 0;
    int guard = 0;
    for (int u : inner) {
      cur += std::exp2(t_.nodes[u].cost_log2);
      if (u != v) guard = std::max(guard, (int)t_.nodes[u].out.size());
    }
    for (int it : items) guard = std::max(guard, (int)t_.nodes[it].out.size());
    // label universe of the window
    std::vector<int> labels;
    for (int it : items) labels.insert(labels.end(), t_.nodes[it].out.begin(), t_.nodes[it].out.end());
    std::sort(labels.begin(), labels.end());
    labels.erase(std::unique(labels.begin(), labels.end()), labels.end());
    if (labels.size() > (size_t)kWords * 64) return 0;
    const int nl = (int)labels.size();
    std::vector<uint32_t> mask(nl, 0);
    std::vector<char> ext(nl, 0);  // kept beyond v
    for (int i = 0; i < n; ++i)
      for (int x : t_.nodes[items[i]].out)
        mask[std::lower_bound(labels.begin(), labels.end(), x) - labels.begin()] |= 1u << i;
    for (int x : t_.nodes[v].out) {
      auto itx = std::lower_bound(labels.begin(), labels.end(), x);
      if (itx != labels.end() && *itx == x) ext[itx - labels.begin()] = 1;
    }
    // output labels of every subset of items: a label stays open unless all
    // of the window's holders of it are in the subset and it is not kept
    // beyond v
    const uint32_t full = (1u << n) - 1;
    std::vector<Bits> out(full + 1);
    for (uint32_t S = 1; S <= full; ++S) {
      Bits b{};
      for (int j = 0; j < nl; ++j)
        if ((mask[j] & S) && (ext[j] || (mask[j] & ~S)))
          b[j >> 6] |= 1ull << (j & 63);
      out[S] = b;
    }
    // subset recursion
    std::vector<double> best(full + 1, HUGE_VAL);
    std::vector<uint32_t> split(full + 1, 0);
    for (int i = 0; i < n; ++i) best[1u << i] = 0;
    for (uint32_t S = 1; S <= full; ++S) {
      if (!(S & (S - 1))) continue;
      if (S != full && popc(out[S]) > guard) continue;  // would enlarge the window's largest intermediate
      const uint32_t low = S & (~S + 1);
      double b = HUGE_VAL;
      uint32_t bs = 0;
      // S1 ranges over the proper subsets of S holding its lowest item
      for (uint32_t S1 = (S - 1) & S; S1; S1 = (S1 - 1) & S) {
        if (!(S1 & low)) continue;
        const uint32_t S2 = S ^ S1;
        if (best[S1] == HUGE_VAL || best[S2] == HUGE_VAL) continue;
        Bits u;
        for (int w = 0; w < kWords; ++w) u[w] = out[S1][w] | out[S2][w];
        const double c = best[S1] + best[S2] + std::exp2((double)popc(u));
        if (c < b) b = c, bs = S1;
      }
      best[S] = b;
      split[S] = bs;
    }
    // exp2(cost_log2) sums the same M's as the subset costs
    if (!(best[full] < cur * (1 - 1e-9))) return 0;
    // rebuild: the window's internal node ids are reused, v stays the root
    size_t next = 1;
    std::function<int(uint32_t)> build = [&](uint32_t S) -> int {
      if (!(S & (S - 1))) return items[__builtin_ctz(S)];
      const int id = S == full ? v : inner[next++];
      const uint32_t S1 = split[S], S2 = S ^ S1;
      const int a = build(S1), b = build(S2);
      TreeNode& nd = t_.nodes[id];
      nd.left = a;
      nd.right = b;
      nd.leaf = -1;
      Bits u;
      for (int w = 0; w < kWords; ++w) u[w] = out[S1][w] | out[S2][w];
      nd.cost_log2 = popc(u);
      nd.out.clear();
      for (int j = 0; j < nl; ++j)
        if ((out[S][j >> 6] >> (j & 63)) & 1) nd.out.push_back(labels[j]);
      return id;
    };
    build(full);
    return 1;
  }
};

}  // namespace

int refine_tree(const PlanNet& pn, Tree& t, int max_items, int max_passes) {
  if (max_items < 3 || t.root < 0 || t.nodes[t.root].left < 0) return 0;
  max_items = std::min(max_items, 12);
  annotate_tree(pn, t);
  Refiner r(pn, t);
  int total = 0;
  for (int pass = 0; pass < max_passes; ++pass) {
    const int c = r.pass(max_items);
    total += c;
    if (!c) break;
  }
  annotate_tree(pn, t);
  return total;
}

}  // namespace tnc
