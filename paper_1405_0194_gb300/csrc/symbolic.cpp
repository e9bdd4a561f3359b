// Host-side ordering and symbolic analysis (Sec. II.B, steps 1 and 2).
//
// Pipeline: validate the CSC pattern -> group columns with identical row sets
// into supervariables (all orbitals of one atom) -> nested dissection of the
// supervariable graph with spectral bisection -> elimination tree (Eq.
// parent) and post-order -> row structures -> fundamental supernodes ->
// relaxed amalgamation -> front layout, relative-index maps and the map from
// the CSC entries of H to front positions.
#include "symbolic.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>

#include "../../include/pexsi_gb300.h"

namespace pexsi {
namespace {

struct Graph {
  int32_t nv = 0;
  std::vector<int64_t> xadj;
  std::vector<int32_t> adj;
  std::vector<int32_t> w;  // vertex weight (columns)
};

// Small deterministic generator (SplitMix64) for Lanczos start vectors.
struct SplitMix {
  uint64_t s;
  explicit SplitMix(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }
};

int validate(int64_t n, const int64_t* colptr, const int32_t* rowind, std::string& err) {
  if (n <= 0 || n > INT32_MAX - 1 || !colptr || !rowind) {
    err = "n must be in [1, 2^31-2] and colptr/rowind non-NULL";
    return PEXSI_ERR_INVALID_ARG;
  }
  if (colptr[0] != 0) { err = "colptr[0] != 0"; return PEXSI_ERR_INVALID_ARG; }
  for (int64_t j = 0; j < n; ++j) {
    if (colptr[j + 1] < colptr[j]) { err = "colptr not non-decreasing"; return PEXSI_ERR_INVALID_ARG; }
    bool diag = false;
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      int32_t i = rowind[e];
      if (i < 0 || i >= n) { err = "row index out of range in column " + std::to_string(j); return PEXSI_ERR_INVALID_ARG; }
      if (e > colptr[j] && rowind[e - 1] >= i) { err = "rows not strictly increasing in column " + std::to_string(j); return PEXSI_ERR_INVALID_ARG; }
      if (i == j) diag = true;
    }
    if (!diag) { err = "missing diagonal entry in column " + std::to_string(j); return PEXSI_ERR_INVALID_ARG; }
  }
  // structural symmetry: (i, j) present => (j, i) present
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      int32_t i = rowind[e];
      if (i == j) continue;
      const int32_t* b = rowind + colptr[i];
      const int32_t* en = rowind + colptr[i + 1];
      const int32_t* f = std::lower_bound(b, en, int32_t(j));
      if (f == en || *f != j) {
        err = "pattern not symmetric: (" + std::to_string(i) + "," + std::to_string(j) + ") without its transpose";
        return PEXSI_ERR_NOT_SYMMETRIC;
      }
    }
  }
  return PEXSI_OK;
}

// Columns with identical row sets (diagonal included) form one supervariable.
void supervariables(int64_t n, const int64_t* colptr, const int32_t* rowind, std::vector<int32_t>& sv_of,
                    std::vector<std::vector<int32_t>>& members) {
  std::vector<uint64_t> h(n);
  for (int64_t j = 0; j < n; ++j) {
    uint64_t a = 0, b = 0;
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      SplitMix m(uint64_t(rowind[e]) + 0x1234567ull);
      uint64_t v = m.next();
      a += v;
      b ^= v * 0x9E3779B97F4A7C15ull;
    }
    h[j] = a ^ (b << 1) ^ uint64_t(colptr[j + 1] - colptr[j]);
  }
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return h[x] < h[y]; });
  sv_of.assign(n, -1);
  members.clear();
  auto same = [&](int32_t x, int32_t y) {
    int64_t lx = colptr[x + 1] - colptr[x], ly = colptr[y + 1] - colptr[y];
    return lx == ly && std::memcmp(rowind + colptr[x], rowind + colptr[y], sizeof(int32_t) * lx) == 0;
  };
  // group equal hashes; within a group compare exactly against representatives
  int64_t g0 = 0;
  std::vector<std::pair<int32_t, int32_t>> assign;  // (col, sv)
  while (g0 < n) {
    int64_t g1 = g0;
    while (g1 < n && h[idx[g1]] == h[idx[g0]]) ++g1;
    std::vector<int32_t> reps;
    std::vector<int32_t> rep_sv;
    for (int64_t t = g0; t < g1; ++t) {
      int32_t c = idx[t];
      int32_t found = -1;
      for (size_t q = 0; q < reps.size(); ++q)
        if (same(reps[q], c)) { found = rep_sv[q]; break; }
      if (found < 0) {
        found = int32_t(members.size());
        members.emplace_back();
        reps.push_back(c);
        rep_sv.push_back(found);
      }
      assign.emplace_back(c, found);
    }
    g0 = g1;
  }
  for (auto& p : assign) sv_of[p.first] = p.second;
  // renumber supervariables by their smallest column so the result does not
  // depend on hash order, and list members ascending
  std::vector<int32_t> minc(members.size(), INT32_MAX);
  for (int64_t j = 0; j < n; ++j) minc[sv_of[j]] = std::min<int32_t>(minc[sv_of[j]], int32_t(j));
  std::vector<int32_t> order(members.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return minc[a] < minc[b]; });
  std::vector<int32_t> newid(members.size());
  for (size_t t = 0; t < order.size(); ++t) newid[order[t]] = int32_t(t);
  for (int64_t j = 0; j < n; ++j) sv_of[j] = newid[sv_of[j]];
  for (auto& mm : members) mm.clear();
  for (int64_t j = 0; j < n; ++j) members[sv_of[j]].push_back(int32_t(j));
}

Graph sv_graph(int64_t n, const int64_t* colptr, const int32_t* rowind, const std::vector<int32_t>& sv_of,
               const std::vector<std::vector<int32_t>>& members) {
  Graph g;
  g.nv = int32_t(members.size());
  g.xadj.assign(g.nv + 1, 0);
  g.w.resize(g.nv);
  std::vector<int32_t> mark(g.nv, -1);
  std::vector<int32_t> tmp;
  for (int32_t v = 0; v < g.nv; ++v) {
    g.w[v] = int32_t(members[v].size());
    int32_t c = members[v][0];
    tmp.clear();
    for (int64_t e = colptr[c]; e < colptr[c + 1]; ++e) {
      int32_t u = sv_of[rowind[e]];
      if (u != v && mark[u] != v) { mark[u] = v; tmp.push_back(u); }
    }
    std::sort(tmp.begin(), tmp.end());
    g.adj.insert(g.adj.end(), tmp.begin(), tmp.end());
    g.xadj[v + 1] = int64_t(g.adj.size());
  }
  (void)n;
  return g;
}

// The `which`-th smallest eigenpair (0-based) of a symmetric tridiagonal
// matrix (diag a, offdiag b): Sturm-sequence bisection for the eigenvalue,
// inverse iteration for the vector.
void tridiag_eigpair(const std::vector<double>& a, const std::vector<double>& b, int which, std::vector<double>& y) {
  int k = int(a.size());
  auto count_below = [&](double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      double bb = i ? b[i - 1] * b[i - 1] : 0.0;
      d = a[i] - x - (i ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++c;
    }
    return c;
  };
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= which + 1) hi = mid; else lo = mid;
  }
  double lam = 0.5 * (lo + hi);
  double shift = lam - 1e-10 * std::max(1.0, std::fabs(lam));
  y.assign(k, 0.0);
  for (int i = 0; i < k; ++i) y[i] = 1.0 + 0.01 * ((i * 7919) % 13);
  std::vector<double> c(k), d(k), x(k);
  for (int it = 0; it < 5; ++it) {
    // solve (T - shift I) x = y by the Thomas algorithm
    for (int i = 0; i < k; ++i) {
      double diag = a[i] - shift - (i ? b[i - 1] * c[i - 1] : 0.0);
      if (std::fabs(diag) < 1e-300) diag = 1e-300;
      c[i] = (i + 1 < k) ? b[i] / diag : 0.0;
      d[i] = (y[i] - (i ? b[i - 1] * d[i - 1] : 0.0)) / diag;
    }
    for (int i = k - 1; i >= 0; --i) x[i] = d[i] - (i + 1 < k ? c[i] * x[i + 1] : 0.0);
    double nrm = 0;
    for (double v : x) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (int i = 0; i < k; ++i) y[i] = x[i] / nrm;
  }
}

class NestedDissection {
 public:
  NestedDissection(const Graph& g, int leaf_w) : g_(g), leaf_w_(leaf_w), part_(g.nv, -1), loc_(g.nv, -1), rng_(0xC0FFEEull) {}

  std::vector<int32_t> run() {
    std::vector<int32_t> all(g_.nv);
    std::iota(all.begin(), all.end(), 0);
    order_.clear();
    recurse(all);
    return order_;
  }

 private:
  const Graph& g_;
  int leaf_w_;
  std::vector<int32_t> part_, loc_;
  std::vector<int32_t> order_;
  int32_t next_part_ = 0;
  SplitMix rng_;

  int64_t weight(const std::vector<int32_t>& vs) const {
    int64_t s = 0;
    for (int32_t v : vs) s += g_.w[v];
    return s;
  }

  void recurse(std::vector<int32_t>& vs) {
    if (vs.empty()) return;
    if (weight(vs) <= leaf_w_ || vs.size() <= 3) { leaf(vs); return; }
    int32_t pid = next_part_++;
    for (int32_t v : vs) part_[v] = pid;
    // connected components of the induced subgraph
    std::vector<std::vector<int32_t>> comps;
    {
      std::vector<int32_t> seen_tag(0);
      int32_t cid = next_part_++;
      for (int32_t s : vs) {
        if (part_[s] != pid) continue;
        comps.emplace_back();
        std::vector<int32_t>& cc = comps.back();
        std::queue<int32_t> q;
        q.push(s);
        part_[s] = cid;
        while (!q.empty()) {
          int32_t v = q.front(); q.pop();
          cc.push_back(v);
          for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
            int32_t u = g_.adj[e];
            if (part_[u] == pid) { part_[u] = cid; q.push(u); }
          }
        }
      }
    }
    if (comps.size() > 1) {
      for (auto& cc : comps) recurse(cc);
      return;
    }
    std::vector<int32_t> A, B, S;
    if (!bisect(comps[0], A, B, S)) { leaf(comps[0]); return; }
    recurse(A);
    recurse(B);
    leaf(S);
  }

  void leaf(const std::vector<int32_t>& vs) {
    std::vector<int32_t> s(vs);
    std::sort(s.begin(), s.end());
    order_.insert(order_.end(), s.begin(), s.end());
  }

  // Vertex separator from a two-way split: a greedy cover of the cut edges
  // (repeatedly the vertex with most cut edges per unit weight), then
  // thinning (a separator vertex with no neighbour on one side joins it).
  void separate(const std::vector<int32_t>& vs, int32_t pid, std::vector<int8_t>& side, std::vector<int32_t>& cut) {
    const int32_t nl = int32_t(vs.size());
    for (int32_t t = 0; t < nl; ++t) {
      cut[t] = 0;
      int32_t v = vs[t];
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
        int32_t u = g_.adj[e];
        if (part_[u] == pid && side[loc_[u]] != side[t]) ++cut[t];
      }
    }
    using Item = std::pair<double, int32_t>;
    std::priority_queue<Item> pq;
    for (int32_t t = 0; t < nl; ++t)
      if (cut[t] > 0) pq.push({double(cut[t]) / g_.w[vs[t]], t});
    while (!pq.empty()) {
      auto [score, t] = pq.top();
      pq.pop();
      if (side[t] == 2 || cut[t] == 0) continue;
      if (score != double(cut[t]) / g_.w[vs[t]]) { pq.push({double(cut[t]) / g_.w[vs[t]], t}); continue; }
      int8_t my = side[t];
      side[t] = 2;
      int32_t v = vs[t];
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
        int32_t u = g_.adj[e];
        if (part_[u] != pid) continue;
        int32_t lu = loc_[u];
        if (side[lu] != 2 && side[lu] != my) {
          --cut[lu];
          if (cut[lu] > 0) pq.push({double(cut[lu]) / g_.w[u], lu});
        }
      }
      cut[t] = 0;
    }
    for (int pass = 0; pass < 3; ++pass) {
      bool changed = false;
      for (int32_t t = 0; t < nl; ++t) {
        if (side[t] != 2) continue;
        bool hasA = false, hasB = false;
        int32_t v = vs[t];
        for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
          int32_t u = g_.adj[e];
          if (part_[u] != pid) continue;
          int8_t su = side[loc_[u]];
          if (su == 0) hasA = true;
          if (su == 1) hasB = true;
        }
        if (!hasB) { side[t] = 0; changed = true; }
        else if (!hasA) { side[t] = 1; changed = true; }
      }
      if (!changed) break;
    }
  }

  // Spectral bisection: the Fiedler vector of the induced Laplacian from a
  // fully reorthogonalised Lanczos run, a weighted median split, then a
  // greedy vertex cover of the cut edges as separator, thinned.
  bool bisect(const std::vector<int32_t>& vs, std::vector<int32_t>& A, std::vector<int32_t>& B, std::vector<int32_t>& S) {
    const int32_t nl = int32_t(vs.size());
    int32_t pid = next_part_++;
    for (int32_t t = 0; t < nl; ++t) { part_[vs[t]] = pid; loc_[vs[t]] = t; }
    std::vector<int32_t> deg(nl, 0);
    for (int32_t t = 0; t < nl; ++t) {
      int32_t v = vs[t];
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e)
        if (part_[g_.adj[e]] == pid) ++deg[t];
    }
    auto lap = [&](const double* x, double* y) {
      for (int32_t t = 0; t < nl; ++t) {
        int32_t v = vs[t];
        double acc = deg[t] * x[t];
        for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
          int32_t u = g_.adj[e];
          if (part_[u] == pid) acc -= x[loc_[u]];
        }
        y[t] = acc;
      }
    };
    const int k = std::min<int>(nl - 1, 200);
    std::vector<double> Q(size_t(k + 1) * nl);
    std::vector<double> alpha, beta;
    const double inv_sqrt_n = 1.0 / std::sqrt(double(nl));
    auto orth_ones = [&](double* x) {
      double s = 0;
      for (int32_t t = 0; t < nl; ++t) s += x[t];
      s *= inv_sqrt_n;
      for (int32_t t = 0; t < nl; ++t) x[t] -= s * inv_sqrt_n;
    };
    auto norm = [&](const double* x) {
      double s = 0;
      for (int32_t t = 0; t < nl; ++t) s += x[t] * x[t];
      return std::sqrt(s);
    };
    double* q0 = Q.data();
    for (int32_t t = 0; t < nl; ++t) q0[t] = rng_.uniform() - 0.5;
    orth_ones(q0);
    double n0 = norm(q0);
    if (n0 == 0) return false;
    for (int32_t t = 0; t < nl; ++t) q0[t] /= n0;
    std::vector<double> w(nl);
    int steps = 0;
    for (int j = 0; j < k; ++j) {
      double* qj = Q.data() + size_t(j) * nl;
      lap(qj, w.data());
      double a = 0;
      for (int32_t t = 0; t < nl; ++t) a += qj[t] * w[t];
      alpha.push_back(a);
      orth_ones(w.data());
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i <= j; ++i) {
          const double* qi = Q.data() + size_t(i) * nl;
          double d = 0;
          for (int32_t t = 0; t < nl; ++t) d += qi[t] * w[t];
          for (int32_t t = 0; t < nl; ++t) w[t] -= d * qi[t];
        }
      steps = j + 1;
      double bn = norm(w.data());
      if (bn < 1e-10 || j + 1 == k) break;
      beta.push_back(bn);
      double* qn = Q.data() + size_t(j + 1) * nl;
      for (int32_t t = 0; t < nl; ++t) qn[t] = w[t] / bn;
    }
    alpha.resize(steps);
    beta.resize(steps > 0 ? steps - 1 : 0);
    int64_t tot = 0;
    for (int32_t v : vs) tot += g_.w[v];

    // Candidate splits: the smallest Ritz vectors (low-frequency modes of the
    // graph), each cut at several weight fractions; keep the candidate with
    // the lightest separator among those with both sides >= 30% of the weight
    std::vector<int8_t> best_side;
    int64_t best_cost = INT64_MAX;
    const int nvec = std::min(steps, 3);
    std::vector<double> y, f(nl);
    std::vector<int32_t> idx(nl);
    std::vector<int8_t> side(nl);
    std::vector<int32_t> cut(nl);
    for (int vi = 0; vi < nvec; ++vi) {
      tridiag_eigpair(alpha, beta, vi, y);
      std::fill(f.begin(), f.end(), 0.0);
      for (int i = 0; i < steps; ++i) {
        const double* qi = Q.data() + size_t(i) * nl;
        for (int32_t t = 0; t < nl; ++t) f[t] += y[i] * qi[t];
      }
      std::iota(idx.begin(), idx.end(), 0);
      std::sort(idx.begin(), idx.end(), [&](int32_t x, int32_t z) { return f[x] < f[z] || (f[x] == f[z] && x < z); });
      for (int fi = 0; fi < 7; ++fi) {
        const double frac = 0.35 + 0.05 * fi;
        std::fill(side.begin(), side.end(), int8_t(1));  // 0 = A, 1 = B, 2 = S
        int64_t acc = 0;
        for (int32_t t = 0; t < nl; ++t) {
          if (double(acc) >= frac * double(tot)) break;
          side[idx[t]] = 0;
          acc += g_.w[vs[idx[t]]];
        }
        separate(vs, pid, side, cut);
        int64_t wa = 0, wb = 0, ws = 0;
        for (int32_t t = 0; t < nl; ++t) (side[t] == 0 ? wa : side[t] == 1 ? wb : ws) += g_.w[vs[t]];
        if (wa == 0 || wb == 0) continue;
        if (10 * std::min(wa, wb) < 3 * (wa + wb)) continue;
        // separator weight, with a mild preference for balance
        int64_t cost = 4 * ws + std::llabs(wa - wb) / 4;
        if (cost < best_cost) { best_cost = cost; best_side = side; }
      }
    }
    if (best_side.empty()) return false;
    side = best_side;
    A.clear(); B.clear(); S.clear();
    for (int32_t t = 0; t < nl; ++t) (side[t] == 0 ? A : side[t] == 1 ? B : S).push_back(vs[t]);
    if (A.empty() || B.empty()) return false;
    int64_t ws = 0;
    for (int32_t v : S) ws += g_.w[v];
    if (2 * ws > tot) return false;  // separator no better than the whole
    return true;
  }
};

}  // namespace

int analyse(int64_t n, const int64_t* colptr, const int32_t* rowind, const int32_t* perm_or_null, int leaf_cols,
            bool amalgamate, Symbolic& out, std::string& err) {
  int rc = validate(n, colptr, rowind, err);
  if (rc) return rc;
  out = Symbolic();
  out.n = n;
  out.nnz = colptr[n];

  std::vector<int32_t> sv_of;
  std::vector<std::vector<int32_t>> members;
  supervariables(n, colptr, rowind, sv_of, members);
  Graph g = sv_graph(n, colptr, rowind, sv_of, members);
  const int32_t nsv = g.nv;

  // ---- ordering of supervariables
  std::vector<int32_t> sv_order;  // position -> sv
  if (perm_or_null) {
    std::vector<int8_t> seen(n, 0);
    for (int64_t t = 0; t < n; ++t) {
      int32_t c = perm_or_null[t];
      if (c < 0 || c >= n || seen[c]) { err = "perm is not a permutation"; return PEXSI_ERR_INVALID_ARG; }
      seen[c] = 1;
    }
    // supervariables in the order of their first appearance
    std::vector<int8_t> svseen(nsv, 0);
    for (int64_t t = 0; t < n; ++t) {
      int32_t v = sv_of[perm_or_null[t]];
      if (!svseen[v]) { svseen[v] = 1; sv_order.push_back(v); }
    }
  } else {
    NestedDissection nd(g, std::max(1, leaf_cols));
    sv_order = nd.run();
  }
  if (int32_t(sv_order.size()) != nsv) { err = "ordering lost supervariables"; return PEXSI_ERR_INTERNAL; }
  std::vector<int32_t> pos_of(nsv);
  for (int32_t t = 0; t < nsv; ++t) pos_of[sv_order[t]] = t;

  // permuted supervariable graph (vertex t = sv_order[t])
  auto nbrs = [&](int32_t t, auto&& fn) {
    int32_t v = sv_order[t];
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) fn(pos_of[g.adj[e]]);
  };

  // ---- elimination tree (Liu's algorithm with path compression)
  std::vector<int32_t> par(nsv, -1), anc(nsv, -1);
  for (int32_t j = 0; j < nsv; ++j) {
    nbrs(j, [&](int32_t i) {
      if (i >= j) return;
      int32_t r = i;
      while (anc[r] != -1 && anc[r] != j) {
        int32_t t = anc[r];
        anc[r] = j;
        r = t;
      }
      if (anc[r] == -1) { anc[r] = j; par[r] = j; }
    });
  }
  // ---- post-order
  std::vector<std::vector<int32_t>> kids(nsv);
  std::vector<int32_t> roots;
  for (int32_t j = 0; j < nsv; ++j) (par[j] < 0 ? roots : kids[par[j]]).push_back(j);
  std::vector<int32_t> post;  // post-order position -> old position
  post.reserve(nsv);
  {
    std::vector<std::pair<int32_t, size_t>> st;
    for (int32_t r0 : roots) {
      st.push_back({r0, 0});
      while (!st.empty()) {
        auto& [v, ci] = st.back();
        if (ci < kids[v].size()) {
          int32_t c = kids[v][ci++];
          st.push_back({c, 0});
        } else {
          post.push_back(v);
          st.pop_back();
        }
      }
    }
  }
  // relabel: vertex p (post-order) = old position post[p]
  std::vector<int32_t> inv_post(nsv);
  for (int32_t p = 0; p < nsv; ++p) inv_post[post[p]] = p;
  std::vector<int32_t> sv_at(nsv), epar(nsv);
  for (int32_t p = 0; p < nsv; ++p) {
    sv_at[p] = sv_order[post[p]];
    epar[p] = par[post[p]] < 0 ? -1 : inv_post[par[post[p]]];
  }
  std::vector<int32_t> pos2(nsv);
  for (int32_t p = 0; p < nsv; ++p) pos2[sv_at[p]] = p;

  // ---- row structures at supervariable level: struct(j) = higher neighbours
  //      U (struct(children) \ {j})
  std::vector<std::vector<int32_t>> st(nsv);
  std::vector<std::vector<int32_t>> ekids(nsv);
  for (int32_t p = 0; p < nsv; ++p)
    if (epar[p] >= 0) ekids[epar[p]].push_back(p);
  std::vector<int32_t> mark(nsv, -1);
  for (int32_t j = 0; j < nsv; ++j) {
    std::vector<int32_t>& s = st[j];
    int32_t v = sv_at[j];
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
      int32_t i = pos2[g.adj[e]];
      if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
    }
    for (int32_t c : ekids[j]) {
      for (int32_t i : st[c])
        if (i != j && mark[i] != j) { mark[i] = j; s.push_back(i); }
    }
    std::sort(s.begin(), s.end());
    if (!s.empty() && epar[j] != s[0]) { err = "etree/structure mismatch"; return PEXSI_ERR_INTERNAL; }
    if (s.empty() && epar[j] != -1) { err = "etree/structure mismatch (root)"; return PEXSI_ERR_INTERNAL; }
  }

  // ---- fundamental supernodes over supervariables
  struct Node {
    std::vector<int32_t> svs;  // own supervariables, in column order
    std::vector<int32_t> strc; // structure (sv positions, post-order numbering)
    int32_t parent = -1;
    std::vector<int32_t> kids;
    int64_t s = 0, r = 0;
    double zeros = 0;
    bool alive = true;
  };
  std::vector<Node> nodes;
  std::vector<int32_t> node_of(nsv, -1);
  for (int32_t j = 0; j < nsv; ++j) {
    bool join = j > 0 && epar[j - 1] == j && ekids[j].size() == 1 && st[j - 1].size() == st[j].size() + 1;
    if (!join) nodes.emplace_back();
    Node& nd = nodes.back();
    nd.svs.push_back(j);
    nd.strc = st[j];
    node_of[j] = int32_t(nodes.size()) - 1;
  }
  for (size_t K = 0; K < nodes.size(); ++K) {
    Node& nd = nodes[K];
    int32_t last = nd.svs.back();
    nd.parent = epar[last] < 0 ? -1 : node_of[epar[last]];
    for (int32_t v : nd.svs) nd.s += g.w[sv_at[v]];
    for (int32_t v : nd.strc) nd.r += g.w[sv_at[v]];
  }
  for (size_t K = 0; K < nodes.size(); ++K)
    if (nodes[K].parent >= 0) nodes[nodes[K].parent].kids.push_back(int32_t(K));

  // ---- relaxed amalgamation (children before parents: node index order)
  if (amalgamate) {
    auto nz = [](const Node& a) { return double(a.s) * (a.s + 1) / 2 + double(a.s) * a.r - a.zeros; };
    for (size_t P = 0; P < nodes.size(); ++P) {
      Node& p = nodes[P];
      bool again = true;
      while (again) {
        again = false;
        std::vector<int32_t> kids = p.kids;
        // try large children last so small ones merge first
        std::sort(kids.begin(), kids.end(), [&](int32_t a, int32_t b) { return nodes[a].s < nodes[b].s; });
        for (int32_t C : kids) {
          Node& c = nodes[C];
          double s = double(c.s + p.s), r = double(p.r);
          double entries = s * (s + 1) / 2 + s * r;
          double z = entries - nz(c) - nz(p);
          double frac = z / entries;
          bool ok = (s <= 16) || (s <= 48 && frac < 0.6) || (s <= 128 && frac < 0.15) || (frac < 0.04);
          if (!ok) continue;
          // merge C into P: C's columns precede P's; C's children become P's
          std::vector<int32_t> svs = c.svs;
          svs.insert(svs.end(), p.svs.begin(), p.svs.end());
          p.svs.swap(svs);
          p.s += c.s;
          p.zeros = z;
          p.kids.erase(std::find(p.kids.begin(), p.kids.end(), C));
          for (int32_t gc : c.kids) { nodes[gc].parent = int32_t(P); p.kids.push_back(gc); }
          c.alive = false;
          c.kids.clear();
          again = true;
        }
      }
    }
  }

  // ---- final post-order of the (amalgamated) supernodal tree
  std::vector<int32_t> final_nodes;
  {
    std::vector<int32_t> rts;
    for (size_t K = 0; K < nodes.size(); ++K)
      if (nodes[K].alive && nodes[K].parent < 0) rts.push_back(int32_t(K));
    std::vector<std::pair<int32_t, size_t>> stk;
    for (int32_t r0 : rts) {
      stk.push_back({r0, 0});
      while (!stk.empty()) {
        auto& [v, ci] = stk.back();
        if (ci < nodes[v].kids.size()) {
          int32_t c = nodes[v].kids[ci++];
          stk.push_back({c, 0});
        } else {
          final_nodes.push_back(v);
          stk.pop_back();
        }
      }
    }
  }
  const int32_t ns = int32_t(final_nodes.size());
  std::vector<int32_t> fidx(nodes.size(), -1);
  for (int32_t K = 0; K < ns; ++K) fidx[final_nodes[K]] = K;

  // column numbering: each node's own supervariables, in post-order of nodes
  std::vector<int32_t> sv_col0(nsv, -1);  // by post-order sv position
  out.perm.resize(n);
  out.iperm.resize(n);
  out.first.assign(ns + 1, 0);
  int32_t col = 0;
  for (int32_t K = 0; K < ns; ++K) {
    out.first[K] = col;
    for (int32_t v : nodes[final_nodes[K]].svs) {
      sv_col0[v] = col;
      for (int32_t c0 : members[sv_at[v]]) {
        out.perm[col] = c0;
        out.iperm[c0] = col;
        ++col;
      }
    }
  }
  out.first[ns] = col;
  if (col != n) { err = "column numbering incomplete"; return PEXSI_ERR_INTERNAL; }

  out.nsuper = ns;
  out.parent.assign(ns, -1);
  out.rptr.assign(ns + 1, 0);
  std::vector<int32_t> col2sn(n);
  for (int32_t K = 0; K < ns; ++K) {
    const Node& nd = nodes[final_nodes[K]];
    out.parent[K] = nd.parent < 0 ? -1 : fidx[nd.parent];
    for (int32_t c = out.first[K]; c < out.first[K + 1]; ++c) col2sn[c] = K;
    std::vector<int32_t> rws;
    for (int32_t v : nd.strc) {
      int32_t c0 = sv_col0[v];
      for (int32_t t = 0; t < g.w[sv_at[v]]; ++t) rws.push_back(c0 + t);
    }
    std::sort(rws.begin(), rws.end());
    if (!rws.empty() && rws[0] < out.first[K + 1]) { err = "structure row inside its own supernode"; return PEXSI_ERR_INTERNAL; }
    out.rows.insert(out.rows.end(), rws.begin(), rws.end());
    out.rptr[K + 1] = int64_t(out.rows.size());
  }
  // parents must own the smallest structure row (Eq. parent)
  for (int32_t K = 0; K < ns; ++K) {
    if (out.r(K) == 0) {
      if (out.parent[K] != -1) { err = "root with a parent"; return PEXSI_ERR_INTERNAL; }
      continue;
    }
    if (col2sn[out.rows[out.rptr[K]]] != out.parent[K]) { err = "parent is not the owner of min structure row"; return PEXSI_ERR_INTERNAL; }
    if (out.parent[K] <= K) { err = "parent not after child"; return PEXSI_ERR_INTERNAL; }
  }
  // relative indices of each child's structure rows in its parent front
  out.rel.resize(out.rows.size());
  for (int32_t K = 0; K < ns; ++K) {
    int32_t P = out.parent[K];
    if (P < 0) continue;
    const int32_t* pr = out.rows.data() + out.rptr[P];
    const int32_t* pe = out.rows.data() + out.rptr[P + 1];
    for (int64_t t = out.rptr[K]; t < out.rptr[K + 1]; ++t) {
      int32_t i = out.rows[t];
      int32_t rl;
      if (i >= out.first[P] && i < out.first[P + 1]) rl = i - out.first[P];
      else {
        const int32_t* f = std::lower_bound(pr, pe, i);
        if (f == pe || *f != i) { err = "child structure not contained in parent front"; return PEXSI_ERR_INTERNAL; }
        rl = out.s(P) + int32_t(f - pr);
      }
      out.rel[t] = rl;
    }
  }
  // heights and levels
  out.height.assign(ns, 0);
  for (int32_t K = 0; K < ns; ++K)
    if (out.parent[K] >= 0) out.height[out.parent[K]] = std::max(out.height[out.parent[K]], out.height[K] + 1);
  out.nlevels = 0;
  for (int32_t K = 0; K < ns; ++K) out.nlevels = std::max(out.nlevels, out.height[K] + 1);
  out.level_fronts.assign(out.nlevels, {});
  for (int32_t K = 0; K < ns; ++K) out.level_fronts[out.height[K]].push_back(K);
  for (auto& lv : out.level_fronts)
    std::stable_sort(lv.begin(), lv.end(), [&](int32_t a, int32_t b) { return out.m(a) > out.m(b); });

  // front pool offsets and statistics
  out.front_off.assign(ns + 1, 0);
  for (int32_t K = 0; K < ns; ++K) {
    int64_t m = out.m(K), s = out.s(K), r = out.r(K);
    out.front_off[K + 1] = out.front_off[K] + m * m;
    out.nnz_L += s * (s + 1) / 2 + s * r;
    out.max_front = std::max(out.max_front, m);
    out.max_width = std::max(out.max_width, s);
  }
  out.front_elems = out.front_off[ns];

  // map CSC entries to front positions of their lower-triangle copy
  out.entry_pos.resize(out.nnz);
  out.entry_lower.resize(out.nnz);
  out.entry_pos_up.resize(out.nnz);
  for (int64_t j = 0; j < n; ++j) {
    int32_t b = out.iperm[j];
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      int32_t a = out.iperm[rowind[e]];
      int32_t row = std::max(a, b), cl = std::min(a, b);
      int32_t K = col2sn[cl];
      int32_t lc = cl - out.first[K];
      int32_t lr;
      if (row < out.first[K + 1]) lr = row - out.first[K];
      else {
        const int32_t* pr = out.rows.data() + out.rptr[K];
        const int32_t* pe = out.rows.data() + out.rptr[K + 1];
        const int32_t* f = std::lower_bound(pr, pe, row);
        if (f == pe || *f != row) { err = "pattern entry outside the symbolic factor"; return PEXSI_ERR_INTERNAL; }
        lr = out.s(K) + int32_t(f - pr);
      }
      out.entry_pos[e] = out.front_off[K] + int64_t(lc) * out.m(K) + lr;
      out.entry_pos_up[e] = out.front_off[K] + int64_t(lr) * out.m(K) + lc;
      out.entry_lower[e] = a >= b ? 1 : 0;
    }
  }
  return PEXSI_OK;
}

FlopCounts count_flops(const Symbolic& sym, int b) {
  FlopCounts f;
  for (int32_t K = 0; K < sym.nsuper; ++K) {
    int64_t s = sym.s(K), r = sym.r(K), m = s + r;
    for (int64_t p0 = 0; p0 < s; p0 += b) {
      double bb = double(std::min<int64_t>(b, s - p0));
      double mp = double(m - p0) - bb;
      f.diag += 8.0 * bb * bb * bb;
      f.factor_gemm += 8.0 * (mp * bb * bb + mp * (mp + 1) / 2 * bb);
      f.selinv_gemm += 8.0 * (mp * mp * bb + bb * bb * mp);
    }
    f.gather_bytes += 2.0 * 16.0 * double(r) * double(r);
  }
  return f;
}

}  // namespace pexsi
