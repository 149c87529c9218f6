// Contraction-order planner: the separator hierarchy of the proof of Thm. 1,
// with separators found by the Sphere Separator Algorithm (Algorithm 1,
// Supplemental Material) and the bottom clusters contracted greedily
// ("Numerical implementation" section).
//
// Each tensor is a sphere (centre = its position with the time axis
// collapsed, radius l/4 + eps; Thm. 2 proof).  Algorithm 1:
//   1. lift the centres to the unit sphere S^d by stereographic projection Pi;
//   2. find a centerpoint c of the lifted points;
//   3. an orthogonal R with R c = (0, ..., 0, |c|);
//   4. the dilation D_alpha = Pi o (alpha 1) o Pi^-1, alpha = sqrt((1-|c|)/(1+|c|));
//   5. a random great circle C;
//   6. the separator S = Pi^-1 o R^T o D_alpha^-1 (C), a sphere (or plane) in R^d;
//   7. accept S if the classification of the tensor spheres into
//      Gamma_O (intersected by S), Gamma_I (inside), Gamma_E (outside)
//      satisfies Eqs. (1) and (2); otherwise draw another great circle.
// The tensors of Gamma_O join the side they share more bond dimension with
// (ties: the smaller side, then side 0), and both sides are split again
// until clusters of at most leaf_size tensors remain; those are contracted
// greedily (smallest output first, then smallest M, then lowest ids).
//
// Readings where the paper leaves a choice open:
//   - centerpoint (step 2): iterated Radon points instead of linear
//     programming on random subsets;
//   - step 7: among `trials` great circles the valid one with the fewest cut
//     bond bits is kept (the paper retries until one is valid);
//   - if no trial satisfies Eqs. (1)-(2) after 4 x trials, the best
//     trial satisfying Eq. (2) alone, else a median split along the principal
//     axis, is used (counted in PlannerStats::ssa_fallback).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "tnc_internal.h"

namespace tnc {

namespace {

struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull) {}
  uint64_t next() {  // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
  double normal() {
    double u1 = std::max(uniform(), 1e-300), u2 = uniform();
    return std::sqrt(-2 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  int below(int n) { return (int)(next() % (uint64_t)n); }
};

constexpr int kD = 4;  // max lifted dimension (d <= 3)
using P4 = std::array<double, kD>;

// Radon point of D+2 points in R^D: lambda with sum lambda_i p_i = 0,
// sum lambda_i = 0, then the convex combination of the positive part.
bool radon_point(const P4* pts, int D, P4& out) {
  const int rows = D + 1, cols = D + 2;
  double A[kD + 1][kD + 2];
  for (int j = 0; j < cols; ++j) {
    for (int i = 0; i < D; ++i) A[i][j] = pts[j][i];
    A[D][j] = 1.0;
  }
  int piv_col[kD + 1];
  int r = 0;
  for (int c = 0; c < cols && r < rows; ++c) {
    int best = r;
    for (int i = r + 1; i < rows; ++i)
      if (std::fabs(A[i][c]) > std::fabs(A[best][c])) best = i;
    if (std::fabs(A[best][c]) < 1e-12) continue;
    for (int j = 0; j < cols; ++j) std::swap(A[r][j], A[best][j]);
    double inv = 1.0 / A[r][c];
    for (int j = 0; j < cols; ++j) A[r][j] *= inv;
    for (int i = 0; i < rows; ++i)
      if (i != r && A[i][c] != 0) {
        double f = A[i][c];
        for (int j = 0; j < cols; ++j) A[i][j] -= f * A[r][j];
      }
    piv_col[r++] = c;
  }
  // first free column
  bool is_piv[kD + 2] = {false};
  for (int i = 0; i < r; ++i) is_piv[piv_col[i]] = true;
  int f = -1;
  for (int c = 0; c < cols; ++c)
    if (!is_piv[c]) {
      f = c;
      break;
    }
  if (f < 0) return false;
  double lam[kD + 2] = {0};
  lam[f] = 1.0;
  for (int i = 0; i < r; ++i) lam[piv_col[i]] = -A[i][f];
  double wsum = 0;
  P4 acc{};
  for (int j = 0; j < cols; ++j)
    if (lam[j] > 0) {
      wsum += lam[j];
      for (int i = 0; i < D; ++i) acc[i] += lam[j] * pts[j][i];
    }
  if (wsum <= 0) return false;
  for (int i = 0; i < D; ++i) out[i] = acc[i] / wsum;
  return true;
}

// Approximate centerpoint by iterated Radon points over a random sample
// (Clarkson, Eppstein, Miller, Sturtivant, Teng 1996).
P4 centerpoint(const std::vector<P4>& pts, int D, Rng& rng) {
  const int g = D + 2;
  int levels = D <= 2 ? 5 : 4;
  size_t m = 1;
  for (int i = 0; i < levels; ++i) m *= g;
  std::vector<P4> cur(m);
  for (size_t i = 0; i < m; ++i) cur[i] = pts[rng.below((int)pts.size())];
  while (cur.size() > 1) {
    std::vector<P4> nxt(cur.size() / g);
    for (size_t i = 0; i < nxt.size(); ++i) {
      if (!radon_point(&cur[i * g], D, nxt[i])) {
        P4 avg{};
        for (int j = 0; j < g; ++j)
          for (int k = 0; k < D; ++k) avg[k] += cur[i * g + j][k] / g;
        nxt[i] = avg;
      }
    }
    cur.swap(nxt);
  }
  return cur[0];
}

struct Sphere {
  bool plane = false;
  double c[3] = {0, 0, 0};  // centre, or normal for a plane
  double r = 0;             // radius, or offset (n.x = r) for a plane
};

// side of a tensor sphere (p, rad) w.r.t. separator S: 0 inside (I),
// 1 outside (E), 2 intersected (O)
int classify(const Sphere& S, const double* p, double rad, int d) {
  if (!S.plane) {
    double dd = 0;
    for (int k = 0; k < d; ++k) dd += (p[k] - S.c[k]) * (p[k] - S.c[k]);
    double dist = std::sqrt(dd);
    if (std::fabs(dist - S.r) < rad) return 2;
    return dist < S.r ? 0 : 1;
  }
  double nn = 0, dot = 0;
  for (int k = 0; k < d; ++k) {
    nn += S.c[k] * S.c[k];
    dot += S.c[k] * p[k];
  }
  double sd = (dot - S.r) / std::sqrt(nn);
  if (std::fabs(sd) < rad) return 2;
  return sd < 0 ? 0 : 1;
}

double sst_cd(int d) { return d == 1 ? 1.0 : d == 2 ? 2.0 : 2.135; }

class Builder {
 public:
  Builder(const PlanNet& pn, const PlannerOpts& o, PlannerStats* st)
      : pn_(pn), o_(o), st_(st), rng_(o.seed) {
    side_.assign(pn.n_leaves, -1);
  }

  int build(std::vector<int> set) {
    if (set.size() == 1) return leaf_node(set[0]);
    if ((int)set.size() <= std::max(2, o_.leaf_size)) return greedy(set);
    std::vector<int> s0, s1;
    separate(set, s0, s1);
    int a = build(s0);
    int b = build(s1);
    return internal(a, b);
  }

  Tree tree;
  // classification (0 inside, 1 outside, 2 intersected) of the separator
  // kept by the last call of separate(), whether it met Eqs. (1)-(2), and k
  std::vector<int> last_cls;
  bool last_valid = false;
  int last_k = 0;

  void separate_public(const std::vector<int>& set, std::vector<int>& s0, std::vector<int>& s1) {
    separate(set, s0, s1);
  }

 private:
  const PlanNet& pn_;
  PlannerOpts o_;
  PlannerStats* st_;
  Rng rng_;
  std::vector<int> side_;  // scratch: side of each leaf in the current split

  int leaf_node(int leaf) {
    TreeNode n;
    n.leaf = leaf;
    tree.nodes.push_back(n);
    return (int)tree.nodes.size() - 1;
  }
  int internal(int a, int b) {
    TreeNode n;
    n.left = a;
    n.right = b;
    tree.nodes.push_back(n);
    return (int)tree.nodes.size() - 1;
  }

  // Greedy contraction of a small cluster: repeatedly merge the pair with
  // the smallest output, then the smallest M, then the lowest ids; pairs that
  // share a contracted label are preferred over outer products.
  int greedy(const std::vector<int>& set) {
    if (st_) st_->greedy_clusters++;
    struct Item {
      int node;
      std::vector<std::pair<int, int>> labs;  // (label, holders inside)
    };
    std::vector<Item> items;
    for (int l : set) {
      Item it;
      it.node = leaf_node(l);
      for (int x : pn_.leaf_labels[l]) it.labs.push_back({x, 1});
      std::sort(it.labs.begin(), it.labs.end());
      items.push_back(std::move(it));
    }
    auto merge = [&](const Item& A, const Item& B, int* shared, int* out_bits, int* all_bits) {
      std::vector<std::pair<int, int>> r;
      size_t i = 0, j = 0;
      *shared = 0;
      *all_bits = 0;
      while (i < A.labs.size() || j < B.labs.size()) {
        std::pair<int, int> e;
        if (j >= B.labs.size() || (i < A.labs.size() && A.labs[i].first < B.labs[j].first)) {
          e = A.labs[i++];
        } else if (i >= A.labs.size() || B.labs[j].first < A.labs[i].first) {
          e = B.labs[j++];
        } else {
          e = {A.labs[i].first, A.labs[i].second + B.labs[j].second};
          ++i, ++j;
          if (!pn_.global_out[e.first]) (*shared)++;
        }
        (*all_bits)++;
        if (pn_.global_out[e.first] || e.second < (int)pn_.holders[e.first].size()) r.push_back(e);
      }
      *out_bits = (int)r.size();
      return r;
    };
    while (items.size() > 1) {
      int bi = -1, bj = -1, bo = 0, bm = 0;
      bool bshare = false;
      for (size_t i = 0; i < items.size(); ++i)
        for (size_t j = i + 1; j < items.size(); ++j) {
          int sh, ob, ab;
          merge(items[i], items[j], &sh, &ob, &ab);
          bool share = sh > 0;
          bool better = bi < 0 || (share && !bshare) ||
                        (share == bshare && (ob < bo || (ob == bo && ab < bm)));
          if (better) {
            bi = (int)i, bj = (int)j, bo = ob, bm = ab, bshare = share;
          }
        }
      int sh, ob, ab;
      Item m;
      m.labs = merge(items[bi], items[bj], &sh, &ob, &ab);
      m.node = internal(items[bi].node, items[bj].node);
      items.erase(items.begin() + bj);
      items[bi] = std::move(m);
    }
    return items[0].node;
  }

  // number of binary labels (not kept to the root) with holders on both sides
  int cut_bits(const std::vector<int>& set) {
    int cut = 0;
    for (int t : set)
      if (side_[t] == 0)
        for (int x : pn_.leaf_labels[t]) {
          if (pn_.global_out[x]) continue;
          for (int h : pn_.holders[x])
            if (h != t && side_[h] == 1) {
              ++cut;
              break;
            }
        }
    return cut;
  }

  // Gamma_O assignment: each intersected tensor joins the side it shares more
  // bond bits with (ties: smaller side, then side 0), in id order.
  void assign_overlap(const std::vector<int>& set, const std::vector<int>& cls) {
    int n0 = 0, n1 = 0;
    for (size_t i = 0; i < set.size(); ++i) {
      side_[set[i]] = cls[i] == 2 ? -2 : cls[i];
      if (cls[i] == 0) ++n0;
      if (cls[i] == 1) ++n1;
    }
    for (size_t i = 0; i < set.size(); ++i) {
      if (cls[i] != 2) continue;
      int t = set[i];
      int b0 = 0, b1 = 0;
      for (int x : pn_.leaf_labels[t]) {
        if (pn_.global_out[x]) continue;
        for (int h : pn_.holders[x]) {
          if (h == t) continue;
          if (side_[h] == 0) ++b0;
          if (side_[h] == 1) ++b1;
        }
      }
      int s = b0 > b1 ? 0 : b1 > b0 ? 1 : (n0 <= n1 ? 0 : 1);
      side_[t] = s;
      (s == 0 ? n0 : n1)++;
    }
  }

  void separate(const std::vector<int>& set, std::vector<int>& s0, std::vector<int>& s1) {
    if (st_) st_->ssa_calls++;
    const int n = (int)set.size();
    const int d = pn_.dim, D = d + 1;
    // normalise: centroid at the origin, RMS radius 1
    double cen[3] = {0, 0, 0};
    for (int t : set)
      for (int k = 0; k < d; ++k) cen[k] += pn_.pos[t][k] / n;
    double rms = 0;
    for (int t : set)
      for (int k = 0; k < d; ++k) rms += (pn_.pos[t][k] - cen[k]) * (pn_.pos[t][k] - cen[k]) / n;
    rms = std::sqrt(rms);
    if (rms < 1e-12) rms = 1;
    std::vector<std::array<double, 3>> p(n);
    std::vector<double> rad(n);
    std::vector<P4> lifted(n);
    for (int i = 0; i < n; ++i) {
      int t = set[i];
      double r2 = 0;
      for (int k = 0; k < d; ++k) {
        p[i][k] = (pn_.pos[t][k] - cen[k]) / rms;
        r2 += p[i][k] * p[i][k];
      }
      rad[i] = pn_.radius[t] / rms;
      // step 1: stereographic lift Pi(x) = (2x, |x|^2 - 1) / (|x|^2 + 1)
      for (int k = 0; k < d; ++k) lifted[i][k] = 2 * p[i][k] / (r2 + 1);
      lifted[i][d] = (r2 - 1) / (r2 + 1);
    }
    // overlap number k: most spheres containing one tensor centre
    int kmax = 1;
    for (int i = 0; i < n; ++i) {
      int cnt = 0;
      for (int j = 0; j < n; ++j) {
        double dd = 0;
        for (int k = 0; k < d; ++k) dd += (p[i][k] - p[j][k]) * (p[i][k] - p[j][k]);
        if (dd <= rad[j] * rad[j]) ++cnt;
      }
      kmax = std::max(kmax, cnt);
    }
    const double eq1 = sst_cd(d) * std::pow((double)kmax, 1.0 / d) * std::pow((double)n, 1.0 - 1.0 / d);
    const double eq2 = (d + 1.0) / (d + 2.0) * n;
    // step 2: centerpoint
    P4 c = centerpoint(lifted, D, rng_);
    double nc = 0;
    for (int k = 0; k < D; ++k) nc += c[k] * c[k];
    nc = std::sqrt(nc);
    if (nc >= 1 - 1e-9) {
      for (int k = 0; k < D; ++k) c[k] *= (1 - 1e-9) / nc;
      nc = 1 - 1e-9;
    }
    // step 3: Householder reflection R with R c = |c| e_D (R = R^T)
    double u[kD] = {0};
    double uu = 0;
    if (nc > 1e-12) {
      for (int k = 0; k < D; ++k) u[k] = c[k] / nc - (k == D - 1 ? 1.0 : 0.0);
      for (int k = 0; k < D; ++k) uu += u[k] * u[k];
    }
    auto applyR = [&](const double* x, double* y) {
      if (uu < 1e-24) {
        for (int k = 0; k < D; ++k) y[k] = x[k];
        return;
      }
      double dot = 0;
      for (int k = 0; k < D; ++k) dot += u[k] * x[k];
      for (int k = 0; k < D; ++k) y[k] = x[k] - 2 * dot / uu * u[k];
    };
    // step 4: dilation parameter
    const double alpha = std::sqrt((1 - nc) / (1 + nc));

    std::vector<int> cls(n), best_cls, best_raw, eq2_raw;
    int best_cut = 1 << 30, best_imb = 1 << 30;
    bool best_valid = false;
    std::vector<int> eq2_cls;
    int eq2_cut = 1 << 30;
    const int max_trials = 4 * std::max(1, o_.trials);
    int valid_found = 0;
    for (int trial = 0; trial < max_trials; ++trial) {
      if (valid_found > 0 && trial >= o_.trials) break;
      // step 5: random great circle {z : g.z = 0}
      double g[kD];
      double gn = 0;
      for (int k = 0; k < D; ++k) {
        g[k] = rng_.normal();
        gn += g[k] * g[k];
      }
      gn = std::sqrt(gn);
      for (int k = 0; k < D; ++k) g[k] /= gn;
      // step 6: D_alpha^-1 (C) is the section {y : w'.y = t'} of S^d with
      // w' = (2 alpha g_{1..d}, (alpha^2 + 1) g_D), t' = (1 - alpha^2) g_D;
      // R^T maps it to {y : (R w').y = t'}; Pi^-1 maps that to a sphere.
      double wp[kD], w[kD];
      for (int k = 0; k < d; ++k) wp[k] = 2 * alpha * g[k];
      wp[d] = (alpha * alpha + 1) * g[d];
      const double tp = (1 - alpha * alpha) * g[d];
      applyR(wp, w);
      Sphere S;
      const double a = w[d] - tp;
      double wn2 = 0;
      for (int k = 0; k < d; ++k) wn2 += w[k] * w[k];
      if (std::fabs(a) > 1e-9 * std::sqrt(wn2 + w[d] * w[d])) {
        double r2 = (w[d] + tp) / a + wn2 / (a * a);
        if (!(r2 > 0)) continue;
        for (int k = 0; k < d; ++k) S.c[k] = -w[k] / a;
        S.r = std::sqrt(r2);
      } else {
        S.plane = true;
        for (int k = 0; k < d; ++k) S.c[k] = 2 * w[k];
        S.r = w[d] + tp;
      }
      int nO = 0, nI = 0, nE = 0;
      for (int i = 0; i < n; ++i) {
        cls[i] = classify(S, p[i].data(), rad[i], d);
        (cls[i] == 0 ? nI : cls[i] == 1 ? nE : nO)++;
      }
      // step 7: Eqs. (1) and (2)
      const bool ok2 = nI <= eq2 && nE <= eq2;
      const bool ok1 = nO <= eq1;
      assign_overlap(set, cls);
      int n0 = 0;
      for (int t : set) n0 += side_[t] == 0;
      if (n0 == 0 || n0 == n) continue;
      int cut = cut_bits(set);
      int imb = std::abs(2 * n0 - n);
      std::vector<int> sides(n);
      for (int i = 0; i < n; ++i) sides[i] = side_[set[i]];
      if (ok1 && ok2) {
        ++valid_found;
        if (!best_valid || cut < best_cut || (cut == best_cut && imb < best_imb)) {
          best_valid = true;
          best_cut = cut;
          best_imb = imb;
          best_cls = sides;
          best_raw = cls;
        }
      } else if (ok2 && cut < eq2_cut) {
        eq2_cut = cut;
        eq2_cls = sides;
        eq2_raw = cls;
      }
    }
    std::vector<int> sides;
    last_k = kmax;
    last_valid = best_valid;
    last_cls.clear();
    if (best_valid) {
      if (st_) st_->ssa_valid++;
      sides = best_cls;
      last_cls = best_raw;
    } else {
      if (st_) st_->ssa_fallback++;
      if (!eq2_cls.empty()) {
        sides = eq2_cls;
        last_cls = eq2_raw;
      } else {
        // median split along the axis of largest spread
        int ax = 0;
        double best = -1;
        for (int k = 0; k < d; ++k) {
          double lo = 1e300, hi = -1e300;
          for (int i = 0; i < n; ++i) lo = std::min(lo, p[i][k]), hi = std::max(hi, p[i][k]);
          if (hi - lo > best) best = hi - lo, ax = k;
        }
        std::vector<int> idx(n);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return p[x][ax] < p[y][ax]; });
        sides.assign(n, 1);
        for (int i = 0; i < n / 2; ++i) sides[idx[i]] = 0;
      }
    }
    s0.clear();
    s1.clear();
    for (int i = 0; i < n; ++i) (sides[i] == 0 ? s0 : s1).push_back(set[i]);
    for (int t : set) side_[t] = -1;
  }
};

}  // namespace

// Algorithm 1 on a bare set of spheres (no bonds): the classification of the
// separator kept, whether it satisfies Eqs. (1)-(2), and the overlap number k.
int ssa_separate_points(const double* pos, const double* rad, int n, int dim, uint64_t seed, int trials,
                        int* cls_out, int* valid, int* k_out) {
  PlanNet pn;
  pn.dim = dim;
  pn.n_leaves = n;
  pn.leaf_labels.assign(n, {});
  pn.pos.resize(n);
  pn.radius.resize(n);
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) pn.pos[i][k] = k < dim ? pos[(size_t)i * dim + k] : 0.0;
    pn.radius[i] = rad[i];
  }
  PlannerOpts o;
  o.seed = seed;
  o.trials = trials;
  Builder b(pn, o, nullptr);
  std::vector<int> all(n), s0, s1;
  std::iota(all.begin(), all.end(), 0);
  b.separate_public(all, s0, s1);
  for (int i = 0; i < n; ++i) cls_out[i] = b.last_cls.empty() ? -1 : b.last_cls[i];
  *valid = b.last_valid ? 1 : 0;
  *k_out = b.last_k;
  return 0;
}

int centerpoint_points(const double* pts, int n, int D, uint64_t seed, double* c) {
  std::vector<P4> v(n);
  for (int i = 0; i < n; ++i) {
    v[i] = P4{};
    for (int k = 0; k < D; ++k) v[i][k] = pts[(size_t)i * D + k];
  }
  Rng rng(seed);
  P4 r = centerpoint(v, D, rng);
  for (int k = 0; k < D; ++k) c[k] = r[k];
  return 0;
}

Tree plan_tree(const PlanNet& pn, const PlannerOpts& o, PlannerStats* st) {
  Builder b(pn, o, st);
  std::vector<int> all(pn.n_leaves);
  std::iota(all.begin(), all.end(), 0);
  int root = b.build(all);
  Tree t = std::move(b.tree);
  t.root = root;
  annotate_tree(pn, t);
  return t;
}

// Output labels of every node: a label survives a node unless every tensor
// holding it lies in the node's subtree and it is not kept to the root.
// cost_log2 = log2 M, M = 2^(number of distinct labels of both children)
// (Eq. 3).
void annotate_tree(const PlanNet& pn, Tree& t) {
  std::vector<std::vector<std::pair<int, int>>> labs(t.nodes.size());
  std::function<void(int)> rec = [&](int v) {
    TreeNode& nd = t.nodes[v];
    if (nd.left < 0) {
      for (int x : pn.leaf_labels[nd.leaf]) labs[v].push_back({x, 1});
      std::sort(labs[v].begin(), labs[v].end());
    } else {
      rec(nd.left);
      rec(nd.right);
      auto& A = labs[nd.left];
      auto& B = labs[nd.right];
      size_t i = 0, j = 0;
      int all = 0;
      std::vector<std::pair<int, int>> r;
      while (i < A.size() || j < B.size()) {
        std::pair<int, int> e;
        if (j >= B.size() || (i < A.size() && A[i].first < B[j].first))
          e = A[i++];
        else if (i >= A.size() || B[j].first < A[i].first)
          e = B[j++];
        else {
          e = {A[i].first, A[i].second + B[j].second};
          ++i, ++j;
        }
        ++all;
        if (pn.global_out[e.first] || e.second < (int)pn.holders[e.first].size()) r.push_back(e);
      }
      labs[v] = std::move(r);
      nd.cost_log2 = all;
      std::vector<std::pair<int, int>>().swap(A);
      std::vector<std::pair<int, int>>().swap(B);
    }
    nd.out.clear();
    for (auto& e : labs[v]) nd.out.push_back(e.first);
  };
  // iterative depth is small (separator hierarchy); recursion is fine
  rec(t.root);
}

double tree_cost_log2(const Tree& t) {
  double mx = -1;
  for (auto& n : t.nodes)
    if (n.left >= 0) mx = std::max(mx, n.cost_log2);
  if (mx < 0) return 0;
  double s = 0;
  for (auto& n : t.nodes)
    if (n.left >= 0) s += std::exp2(n.cost_log2 - mx);
  return mx + std::log2(s) + 1;  // 2 M per node
}

int tree_max_rank(const Tree& t) {
  int r = 0;
  for (auto& n : t.nodes) r = std::max(r, (int)n.out.size());
  return r;
}

}  // namespace tnc
