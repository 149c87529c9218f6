// The paper's analytic cost bounds for a circuit (host only).
//
// Thm. 1 bounds the scalar operations of contracting a finite-ranged network
// of n tensors (at most M entries each, at most k spheres over any point) in
// R^d by 2 n^(1/log2((d+2)/(d+1))) M^(a_d k^(1/d) n^(1-1/d)).  Thm. 2 applies
// it to c = <0|U^dagger P U|0>: each two-qubit gate is split into two rank-3
// tensors (M = 16), U and U^dagger give n = 2 sum_i f(x_i) tensors, and the
// sphere overlap is at most k = 2 F (1 + l/r)^d; for d = 2 and
// nearest-neighbour gates the Planar Separator Theorem gives a tighter form.
// The text after Thm. 2 compares them with left-to-right contraction and
// explicit time evolution.  Every quantity below is evaluated in log2.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "tnc_internal.h"

namespace {

// c_d of the Sphere Separator Theorem (c_3 is given as an upper bound)
double sst_c(int d) { return d == 1 ? 1.0 : d == 2 ? 2.0 : 2.135; }
constexpr double kCPst = 1.971;  // Planar Separator Theorem constant (upper bound)

}  // namespace

extern "C" int tnc_circuit_bounds_eval(const tnc_network_desc* desc, tnc_circuit_bounds* out) {
  if (!out) {
    tnc::set_error("tnc_circuit_bounds_eval: NULL output");
    return TNC_EINVAL;
  }
  {
    tnc::Network check;  // same validation as tnc_load_network
    const int rc = tnc::build_network(desc, &check, 0);
    if (rc != TNC_OK) return rc;
  }
  const double nan = std::numeric_limits<double>::quiet_NaN();
  const int n = desc->n_qubits, d = desc->dim;
  auto x = [&](int q, int k) { return desc->coords[(size_t)q * d + k]; };
  auto dist = [&](int a, int b) {
    double s = 0;
    for (int k = 0; k < d; ++k) s += (x(a, k) - x(b, k)) * (x(a, k) - x(b, k));
    return std::sqrt(s);
  };
  // f(x_i), gate range l, depth T (each gate one layer after the latest
  // layer of its qubits)
  std::vector<double> f(n, 0.0);
  std::vector<int> layer(n, 0);
  double l = 0;
  int depth = 0;
  size_t qoff = 0;
  for (int g = 0; g < desc->n_gates; ++g) {
    const int a = desc->arity[g];
    int t = 0;
    for (int j = 0; j < a; ++j) t = std::max(t, layer[desc->qubits[qoff + j]]);
    ++t;
    for (int j = 0; j < a; ++j) layer[desc->qubits[qoff + j]] = t;
    depth = std::max(depth, t);
    if (a == 2) {
      const int qa = desc->qubits[qoff], qb = desc->qubits[qoff + 1];
      f[qa] += 1, f[qb] += 1;
      l = std::max(l, dist(qa, qb));
    }
    qoff += a;
  }
  double r = std::numeric_limits<double>::infinity();
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) r = std::min(r, dist(a, b));
  if (n < 2) r = nan;
  double S = 0, F = 0, W = 0;
  for (double fi : f) {
    S += fi;
    F = std::max(F, fi);
    W += fi * (2.0 + fi / 2.0);
  }
  tnc_circuit_bounds& b = *out;
  b.n_qubits = n, b.dim = d, b.depth = depth;
  b.sum_f = S, b.max_f = F, b.l = l, b.r = r;
  const bool ok = d >= 2 && S > 0 && r > 0;
  const double dd = d;
  b.a_d = d >= 2 ? sst_c(d) / (2.0 - 2.0 * std::pow((dd + 1) / (dd + 2), 1.0 - 1.0 / dd)) : nan;
  b.a2_pst = kCPst / (2.0 - 2.0 * std::sqrt(2.0 / 3.0));
  b.n_tensors = 2 * S;
  b.k = ok ? 2 * F * std::pow(1.0 + l / r, dd) : nan;
  const double lg = d >= 2 ? std::log2((dd + 2) / (dd + 1)) : nan;
  if (ok) {
    const double nt = b.n_tensors;
    b.thm1_log2 = 1.0 + std::log2(nt) / lg + b.a_d * std::pow(b.k, 1.0 / dd) * std::pow(nt, 1.0 - 1.0 / dd) * 4.0;
    b.thm2_log2 = std::log2(2 * S) / lg + 1.0 + 8.0 * b.a_d * (1.0 + l / r) * std::pow(F, 1.0 / dd) *
                                                      std::pow(S, 1.0 - 1.0 / dd);
  } else {
    b.thm1_log2 = b.thm2_log2 = nan;
  }
  const bool nn = ok && d == 2 && std::fabs(l - r) <= 1e-9 * r;
  b.thm2_pst_log2 = nn ? std::log2(W) / std::log2(1.5) + 1.0 + 4.0 * b.a2_pst * std::sqrt(W) : nan;
  b.sidewise_log2 = 1.0 + 4.0 * F * std::pow((double)n, 1.0 - 1.0 / dd) + std::log2((double)n) / dd;
  b.explicit_log2 = std::log2((double)std::max(depth, 1) * n) + 2.0 + n;
  return TNC_OK;
}
