// Circuit -> tensor network.
//
// Classical Simulation section of the paper: a circuit acting on |0...0> is a
// tensor network whose two-qubit gates are rank-4 tensors; single-qubit
// gates and the boundary vectors are absorbed into them, so only the
// two-qubit gates set the cost.  Following the proof of Thm. 2, each two-qubit
// gate is split by a singular value decomposition of its operator-Schmidt
// reshaping into two rank-3 tensors joined by a bond (dimension = Schmidt
// rank: 2 for CZ, 4 for fSim), and the two halves are placed a quarter of the
// way from each qubit towards the other, with the time axis collapsed.
//
// Here every index is binary: a bond of dimension 4 is two binary labels, a
// Schmidt rank of 3 would be padded with a zero singular value.  The final
// wire of every qubit is left as a label of kind LK_FINAL; the plan decides
// whether it stays open or is projected onto the requested bit values.
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "tnc_internal.h"

namespace tnc {

// One-sided (Hestenes) Jacobi SVD of a small complex matrix a (m x n,
// row-major): a = U diag(s) V^H.  On return w holds a V (orthogonal columns,
// norms s), v the n x n unitary V.  Columns are sorted by decreasing s.
static void jacobi_svd(int m, int n, std::vector<cd>& w, std::vector<cd>& v, std::vector<double>& s) {
  v.assign(n * n, cd(0));
  for (int i = 0; i < n; ++i) v[i * n + i] = 1;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double al = 0, be = 0;
        cd ga = 0;
        for (int i = 0; i < m; ++i) {
          al += std::norm(w[i * n + p]);
          be += std::norm(w[i * n + q]);
          ga += std::conj(w[i * n + p]) * w[i * n + q];
        }
        double g = std::abs(ga);
        if (g <= 1e-300 || g <= 1e-16 * std::sqrt(al * be)) continue;
        rotated = true;
        cd ph = ga / g;  // e^{i phi}
        double zeta = (be - al) / (2 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        double c = 1 / std::sqrt(1 + t * t), sn = c * t;
        for (int i = 0; i < m; ++i) {
          cd ap = w[i * n + p], aq = w[i * n + q] * std::conj(ph);
          w[i * n + p] = c * ap - sn * aq;
          w[i * n + q] = sn * ap + c * aq;
        }
        for (int i = 0; i < n; ++i) {
          cd vp = v[i * n + p], vq = v[i * n + q] * std::conj(ph);
          v[i * n + p] = c * vp - sn * vq;
          v[i * n + q] = sn * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  s.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int i = 0; i < m; ++i) acc += std::norm(w[i * n + j]);
    s[j] = std::sqrt(acc);
  }
  // sort columns by decreasing singular value
  for (int j = 0; j < n; ++j) {
    int best = j;
    for (int k = j + 1; k < n; ++k)
      if (s[k] > s[best]) best = k;
    if (best != j) {
      std::swap(s[j], s[best]);
      for (int i = 0; i < m; ++i) std::swap(w[i * n + j], w[i * n + best]);
      for (int i = 0; i < n; ++i) std::swap(v[i * n + j], v[i * n + best]);
    }
  }
}

// Multiply a 2x2 matrix P into the axis of `label` of leaf L:
// T'[.., w', ..] = sum_w P[w'][w] T[.., w, ..].
static void apply_on_axis(Leaf& L, int label, const cd P[4]) {
  int r = (int)L.labels.size(), ax = -1;
  for (int i = 0; i < r; ++i)
    if (L.labels[i] == label) ax = i;
  size_t bit = (size_t)1 << (r - 1 - ax);
  std::vector<cd> out(L.data.size());
  for (size_t i = 0; i < L.data.size(); ++i) {
    int wv = (i & bit) ? 1 : 0;
    size_t i0 = i & ~bit, i1 = i | bit;
    out[i] = P[wv * 2 + 0] * L.data[i0] + P[wv * 2 + 1] * L.data[i1];
  }
  L.data.swap(out);
}

static bool is_identity(const std::array<cd, 4>& P) {
  return P[0] == cd(1) && P[1] == cd(0) && P[2] == cd(0) && P[3] == cd(1);
}

// A gate matrix (dim x dim, interleaved re/im, row-major) that is diagonal in
// the computational basis, exactly: D|z> = d(z)|z>.
static bool is_diagonal(const double* m, int dim) {
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c)
      if (r != c && (m[2 * (r * dim + c)] != 0.0 || m[2 * (r * dim + c) + 1] != 0.0)) return false;
  return true;
}

// Hyper-edge form: diagonal tensors on the same wire labels commute and
// multiply elementwise, so they are merged on the host in FP64 (fewer
// tensors, and no long chains of FP32 products of phases on the device):
// all rank-2 diagonal tensors on one pair of labels become one, and every
// rank-1 diagonal tensor joins a rank-2 one on its label where there is one
// (otherwise all rank-1 ones on a label become one).  The merged tensor sits
// at the mean position and layer of its parts.
static void merge_diagonals(Network* net) {
  std::vector<Leaf>& L = net->leaves;
  std::map<std::pair<int, int>, int> pair_of;  // (x < y) -> merged leaf
  std::map<int, int> single_of;                  // x -> merged rank-1 leaf
  std::vector<Leaf> merged;
  std::vector<int> parts;
  std::vector<int> keep_index(L.size(), -1);
  std::vector<Leaf> out;
  for (size_t i = 0; i < L.size(); ++i) {
    if (!L[i].diag || L[i].labels.size() != 2) continue;
    int x = L[i].labels[0], y = L[i].labels[1];
    std::array<cd, 4> d = {L[i].data[0], L[i].data[1], L[i].data[2], L[i].data[3]};
    if (x > y) {  // transpose to (min, max) order
      std::swap(x, y);
      std::swap(d[1], d[2]);
    }
    auto it = pair_of.find({x, y});
    if (it == pair_of.end()) {
      Leaf m = L[i];
      m.labels = {x, y};
      m.data.assign(d.begin(), d.end());
      pair_of[{x, y}] = (int)merged.size();
      merged.push_back(std::move(m));
      parts.push_back(1);
    } else {
      Leaf& m = merged[it->second];
      for (int k = 0; k < 4; ++k) m.data[k] *= d[k];
      for (int k = 0; k < 3; ++k) m.pos[k] += L[i].pos[k];
      m.layer += L[i].layer;
      parts[it->second]++;
    }
  }
  // rank-1 diagonals: into a rank-2 diagonal on their label, else merged per label
  std::map<int, int> pair_with;  // label -> a merged rank-2 diagonal holding it
  for (size_t j = 0; j < merged.size(); ++j)
    for (int x : merged[j].labels) pair_with.emplace(x, (int)j);
  for (size_t i = 0; i < L.size(); ++i) {
    if (!L[i].diag || L[i].labels.size() != 1) continue;
    const int x = L[i].labels[0];
    auto pw = pair_with.find(x);
    if (pw != pair_with.end()) {
      Leaf& m = merged[pw->second];
      const bool first = m.labels[0] == x;  // the axis of x: bit 1 (first label) or bit 0
      for (int k = 0; k < 4; ++k) m.data[k] *= L[i].data[first ? (k >> 1) : (k & 1)];
      continue;
    }
    auto it = single_of.find(x);
    if (it == single_of.end()) {
      single_of[x] = (int)merged.size();
      merged.push_back(L[i]);
      parts.push_back(1);
    } else {
      Leaf& m = merged[it->second];
      m.data[0] *= L[i].data[0];
      m.data[1] *= L[i].data[1];
      for (int k = 0; k < 3; ++k) m.pos[k] += L[i].pos[k];
      m.layer += L[i].layer;
      parts[it->second]++;
    }
  }
  for (size_t j = 0; j < merged.size(); ++j) {
    for (int k = 0; k < 3; ++k) merged[j].pos[k] /= parts[j];
    merged[j].layer = (int)std::lround((double)merged[j].layer / parts[j]);
  }
  for (size_t i = 0; i < L.size(); ++i)
    if (!L[i].diag) {
      keep_index[i] = (int)out.size();
      out.push_back(std::move(L[i]));
    }
  for (auto& m : merged) out.push_back(std::move(m));
  for (int& h : net->final_holder)
    if (h >= 0) h = keep_index[h];  // final wires are never held by a diagonal tensor alone
  L.swap(out);
}

int build_network(const tnc_network_desc* d, Network* net, int flags) {
  if (!d || d->n_qubits < 1 || d->dim < 1 || d->dim > 3 || d->n_gates < 0 || !d->coords ||
      (d->n_gates > 0 && (!d->arity || !d->qubits || !d->mats))) {
    set_error("tnc_load_network: invalid descriptor");
    return TNC_EINVAL;
  }
  const int n = d->n_qubits, dim = d->dim;
  net->n_qubits = n;
  net->dim = dim;
  net->coords.assign(d->coords, d->coords + (size_t)n * dim);
  for (double x : net->coords)
    if (!std::isfinite(x)) {
      set_error("tnc_load_network: non-finite coordinate");
      return TNC_EINVAL;
    }
  auto xq = [&](int q, int k) { return k < dim ? net->coords[(size_t)q * dim + k] : 0.0; };

  // validate gates, find the gate range l
  double l = 0;
  size_t qoff = 0, moff = 0;
  int n2 = 0;
  for (int g = 0; g < d->n_gates; ++g) {
    int a = d->arity[g];
    if (a != 1 && a != 2) {
      set_error("tnc_load_network: gate %d has arity %d", g, a);
      return TNC_EINVAL;
    }
    for (int j = 0; j < a; ++j) {
      int q = d->qubits[qoff + j];
      if (q < 0 || q >= n) {
        set_error("tnc_load_network: gate %d acts on qubit %d (n = %d)", g, q, n);
        return TNC_EINVAL;
      }
    }
    if (a == 2) {
      int qa = d->qubits[qoff], qb = d->qubits[qoff + 1];
      if (qa == qb) {
        set_error("tnc_load_network: gate %d acts twice on qubit %d", g, qa);
        return TNC_EINVAL;
      }
      double dd = 0;
      for (int k = 0; k < dim; ++k) dd += (xq(qa, k) - xq(qb, k)) * (xq(qa, k) - xq(qb, k));
      l = std::max(l, std::sqrt(dd));
      ++n2;
    }
    size_t ne = (size_t)(1 << a) * (1 << a) * 2;
    for (size_t k = 0; k < ne; ++k)
      if (!std::isfinite(d->mats[moff + k])) {
        set_error("tnc_load_network: gate %d has a non-finite entry", g);
        return TNC_EINVAL;
      }
    qoff += a;
    moff += ne;
  }
  if (l <= 0) l = 1.0;
  net->gate_range = l;
  net->n_gates_2q = n2;
  const double eps = 0.05 * l;                 // sphere radius l/4 + eps (Thm. 2 proof)
  const double jit = 0.5 * eps / std::max(1, n2);  // time displacement eps' per gate
  const double jdir[3] = {0.6, 0.8, 0.0};

  auto new_label = [&](int kind) {
    net->label_kind.push_back(kind);
    return (int)net->label_kind.size() - 1;
  };

  std::vector<std::array<cd, 4>> pend(n, {cd(1), cd(0), cd(0), cd(1)});
  std::vector<int> cur_label(n, -1), cur_holder(n, -1);
  std::vector<int> qlayer(n, 0);  // ASAP layer of the latest 2q gate on each qubit
  std::vector<int> n_holders;     // per label (hyper-edge form)
  const bool hyper = (flags & TNC_NET_HYPEREDGES) != 0;
  auto hold = [&](int label) {
    if ((int)n_holders.size() <= label) n_holders.resize(label + 1, 0);
    n_holders[label]++;
  };
  qoff = moff = 0;
  int g2 = 0;
  // Hyper-edge form: the pending single-qubit product of qubit q becomes a
  // tensor of its own, from the current wire label to a fresh one (or the
  // vector P|0> on a fresh label when the qubit has none yet), so that the
  // next diagonal gates can share the wire label it leaves.
  auto flush = [&](int q, int layer) {
    const std::array<cd, 4>& P = pend[q];
    if (cur_label[q] >= 0 && is_identity(P)) return;
    Leaf L;
    const int nl = new_label(LK_WIRE);
    L.labels.push_back(nl);
    if (cur_label[q] >= 0) {
      L.labels.push_back(cur_label[q]);
      L.data = {P[0], P[1], P[2], P[3]};  // [w'][w]
      hold(cur_label[q]);
    } else {
      L.data = {P[0], P[2]};  // P |0>
    }
    hold(nl);
    for (int k = 0; k < dim; ++k) L.pos[k] = xq(q, k) + jdir[k] * jit * g2;
    L.radius = 0.25 * l + eps;
    L.qubit = q;
    L.time = g2;
    L.layer = layer;
    net->leaves.push_back(std::move(L));
    cur_label[q] = nl;
    cur_holder[q] = (int)net->leaves.size() - 1;
    pend[q] = {cd(1), cd(0), cd(0), cd(1)};
  };
  for (int g = 0; g < d->n_gates; ++g) {
    int a = d->arity[g];
    const double* m = d->mats + moff;
    if (hyper && a == 1 && is_diagonal(m, 2) && is_identity(pend[d->qubits[qoff]]) &&
        cur_label[d->qubits[qoff]] >= 0) {
      // a diagonal single-qubit gate right on a wire label: one more holder of it
      const int q = d->qubits[qoff];
      Leaf L;
      L.labels = {cur_label[q]};
      L.data = {cd(m[0], m[1]), cd(m[6], m[7])};
      L.diag = true;
      hold(cur_label[q]);
      for (int k = 0; k < dim; ++k) L.pos[k] = xq(q, k) + jdir[k] * jit * g2;
      L.radius = 0.25 * l + eps;
      L.qubit = q;
      L.time = g2;
      L.layer = qlayer[q];
      net->leaves.push_back(std::move(L));
      qoff += a;
      moff += 8;
      continue;
    }
    if (hyper && a == 2 && is_diagonal(m, 4)) {
      // a diagonal two-qubit gate: a rank-2 tensor d(z_a, z_b) on the two wire labels
      const int qa = d->qubits[qoff], qb = d->qubits[qoff + 1];
      const int layer = std::max(qlayer[qa], qlayer[qb]) + 1;
      flush(qa, qlayer[qa]);
      flush(qb, qlayer[qb]);
      Leaf L;
      L.labels = {cur_label[qa], cur_label[qb]};
      for (int r = 0; r < 4; ++r) L.data.push_back(cd(m[2 * (r * 4 + r)], m[2 * (r * 4 + r) + 1]));
      L.diag = true;
      hold(cur_label[qa]);
      hold(cur_label[qb]);
      for (int k = 0; k < dim; ++k) L.pos[k] = 0.5 * (xq(qa, k) + xq(qb, k)) + jdir[k] * jit * g2;
      L.radius = 0.5 * l + eps;
      L.qubit = qa;
      L.time = g2;
      L.layer = layer;
      net->leaves.push_back(std::move(L));
      qlayer[qa] = qlayer[qb] = layer;
      ++g2;
      qoff += a;
      moff += 32;
      continue;
    }
    if (a == 1) {
      int q = d->qubits[qoff];
      cd U[4] = {cd(m[0], m[1]), cd(m[2], m[3]), cd(m[4], m[5]), cd(m[6], m[7])};
      std::array<cd, 4> P = pend[q], R;
      R[0] = U[0] * P[0] + U[1] * P[2];
      R[1] = U[0] * P[1] + U[1] * P[3];
      R[2] = U[2] * P[0] + U[3] * P[2];
      R[3] = U[2] * P[1] + U[3] * P[3];
      pend[q] = R;
    } else {
      int qa = d->qubits[qoff], qb = d->qubits[qoff + 1];
      cd G[16];
      for (int k = 0; k < 16; ++k) G[k] = cd(m[2 * k], m[2 * k + 1]);
      // G' = G (P_a x P_b): absorb the pending single-qubit gates on the inputs
      cd Gp[16];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          cd acc = 0;
          int ca = c >> 1, cb = c & 1;
          for (int k = 0; k < 4; ++k) {
            int ka = k >> 1, kb = k & 1;
            acc += G[r * 4 + k] * pend[qa][ka * 2 + ca] * pend[qb][kb * 2 + cb];
          }
          Gp[r * 4 + c] = acc;
        }
      const bool sa = cur_label[qa] >= 0, sb = cur_label[qb] >= 0;  // input legs present
      const int ia = sa ? 2 : 1, ib = sb ? 2 : 1;
      const int rows = 2 * ia, cols = 2 * ib;
      // Mat[(out_a, in_a)][(out_b, in_b)]; an absent input leg is fixed to |0>
      std::vector<cd> W(rows * cols);
      for (int oa = 0; oa < 2; ++oa)
        for (int ina = 0; ina < ia; ++ina)
          for (int ob = 0; ob < 2; ++ob)
            for (int inb = 0; inb < ib; ++inb) {
              int rr = oa * ia + ina, cc = ob * ib + inb;
              W[rr * cols + cc] = Gp[(oa * 2 + ob) * 4 + (ina * 2 + inb)];
            }
      std::vector<cd> V;
      std::vector<double> s;
      jacobi_svd(rows, cols, W, V, s);
      int rank = 0;
      for (int k = 0; k < cols; ++k)
        if (s[k] > 1e-12 * std::max(s[0], 1e-300)) ++rank;
      if (rank == 0) rank = 1;
      const int rp = rank == 1 ? 1 : (rank == 2 ? 2 : 4);
      const int nb = rp == 1 ? 0 : (rp == 2 ? 1 : 2);
      Leaf A, B;
      const int la = new_label(LK_WIRE), lb = new_label(LK_WIRE);
      std::vector<int> bond;
      for (int k = 0; k < nb; ++k) bond.push_back(new_label(LK_BOND));
      A.labels.push_back(la);
      if (sa) A.labels.push_back(cur_label[qa]);
      for (int x : bond) A.labels.push_back(x);
      for (int x : bond) B.labels.push_back(x);
      B.labels.push_back(lb);
      if (sb) B.labels.push_back(cur_label[qb]);
      A.data.assign((size_t)rows << nb, cd(0));
      B.data.assign((size_t)cols << nb, cd(0));
      for (int k = 0; k < rank && k < rp; ++k) {
        double sq = std::sqrt(s[k]);
        for (int rr = 0; rr < rows; ++rr)
          A.data[((size_t)rr << nb) | k] = s[k] > 0 ? W[rr * cols + k] / sq : cd(0);
        for (int cc = 0; cc < cols; ++cc)
          B.data[((size_t)k * cols) + cc] = sq * std::conj(V[cc * cols + k]);
      }
      for (int k = 0; k < dim; ++k) {
        A.pos[k] = xq(qa, k) + 0.25 * (xq(qb, k) - xq(qa, k)) + jdir[k] * jit * g2;
        B.pos[k] = xq(qb, k) + 0.25 * (xq(qa, k) - xq(qb, k)) + jdir[k] * jit * g2;
      }
      A.radius = B.radius = 0.25 * l + eps;
      A.qubit = qa;
      B.qubit = qb;
      A.time = B.time = g2;
      A.layer = B.layer = std::max(qlayer[qa], qlayer[qb]) + 1;
      qlayer[qa] = qlayer[qb] = A.layer;
      for (int x : A.labels) hold(x);
      for (int x : B.labels) hold(x);
      net->leaves.push_back(std::move(A));
      net->leaves.push_back(std::move(B));
      const int ida = (int)net->leaves.size() - 2, idb = ida + 1;
      pend[qa] = {cd(1), cd(0), cd(0), cd(1)};
      pend[qb] = {cd(1), cd(0), cd(0), cd(1)};
      cur_label[qa] = la;
      cur_holder[qa] = ida;
      cur_label[qb] = lb;
      cur_holder[qb] = idb;
      ++g2;
    }
    qoff += a;
    moff += (size_t)(1 << a) * (1 << a) * 2;
  }
  net->final_label.assign(n, -1);
  net->final_holder.assign(n, -1);
  for (int q = 0; q < n; ++q) {
    // hyper-edge form: a wire label shared by several tensors cannot take the
    // pending product on one holder's axis; it gets a tensor of its own
    if (hyper && cur_holder[q] >= 0 && !is_identity(pend[q]) && n_holders[cur_label[q]] > 1)
      flush(q, qlayer[q]);
    if (cur_holder[q] >= 0) {
      Leaf& L = net->leaves[cur_holder[q]];
      cd P[4] = {pend[q][0], pend[q][1], pend[q][2], pend[q][3]};
      apply_on_axis(L, cur_label[q], P);
      net->label_kind[cur_label[q]] = LK_FINAL;
      net->final_label[q] = cur_label[q];
      net->final_holder[q] = cur_holder[q];
    } else {
      Leaf L;
      int lf = new_label(LK_FINAL);
      L.labels.push_back(lf);
      L.data = {pend[q][0], pend[q][2]};  // P |0>
      for (int k = 0; k < dim; ++k) L.pos[k] = xq(q, k);
      L.radius = eps;
      L.qubit = q;
      L.time = 0;
      net->leaves.push_back(std::move(L));
      net->final_label[q] = lf;
      net->final_holder[q] = (int)net->leaves.size() - 1;
    }
  }
  if (hyper) merge_diagonals(net);
  return TNC_OK;
}

}  // namespace tnc
