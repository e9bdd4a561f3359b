// Chemical-potential search (Sec. II.C): inertia-count bracketing of
// N_beta(mu) = N_e with the two-root gap rule and progressive narrowing, then
// a safeguarded Newton iteration that takes N'(mu) = Tr[Gamma^d S] from the
// same P-pole evaluation as N(mu) = Tr[DM S] (Eq. Nmu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plan.hpp"

using pexsi::CudaError;
using pexsi::ck;

namespace {

// N_beta(mu): the linear interpolation of the counts N_inf(eps_q), constant
// outside [eps_0, eps_{Q-1}], smoothed with (beta/4) sech^2(beta (eps-mu)/2),
// i.e. -f'/2 for the spin-2 Fermi function (Eq. finiteelectronnumber).
double n_beta(const std::vector<double>& eps, const std::vector<double>& ninf, double beta, double mu) {
  const int G = 2001;
  const double half = 40.0 / beta;
  double acc = 0.0, wsum = 0.0;
  for (int g = 0; g < G; ++g) {
    double x = -half + 2.0 * half * g / (G - 1);
    double e = mu + x;
    double nl;
    if (e <= eps.front()) nl = ninf.front();
    else if (e >= eps.back()) nl = ninf.back();
    else {
      size_t q = size_t(std::upper_bound(eps.begin(), eps.end(), e) - eps.begin());
      double t = (e - eps[q - 1]) / (eps[q] - eps[q - 1]);
      nl = ninf[q - 1] + t * (ninf[q] - ninf[q - 1]);
    }
    double c = std::cosh(0.5 * beta * x);
    double k = 0.25 * beta / (c * c);
    double w = (g == 0 || g == G - 1) ? 0.5 : 1.0;
    acc += w * k * nl;
    wsum += w * k;
  }
  return acc / wsum;
}

// mu in [lo, hi] with n_beta(mu) = target (n_beta is non-decreasing).
double root(const std::vector<double>& eps, const std::vector<double>& ninf, double beta, double target, double lo,
            double hi) {
  for (int it = 0; it < 100; ++it) {
    double mid = 0.5 * (lo + hi);
    if (n_beta(eps, ninf, beta, mid) < target) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

extern "C" int pexsi_mu_opts_default(pexsi_mu_opts* o) {
  if (!o) return PEXSI_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->tol_ne = 1e-6;
  o->delta_n = 0.1;
  o->n_shifts = 16;
  o->max_inertia = 3;
  o->max_newton = 16;
  return PEXSI_OK;
}

extern "C" int pexsi_mu_solve(pexsi_plan* p, const double* H, const double* S, double beta, int32_t n_poles,
                              double delta_e, const pexsi_mu_opts* opts, double* dm, double* edm, double* fdm,
                              pexsi_mu_info* info) {
  if (!p || !H || !opts || p->opts.device < 0) return PEXSI_ERR_INVALID_ARG;
  if (!(opts->mu_hi > opts->mu_lo) || opts->n_shifts < 2 || opts->n_shifts > 64 || !(beta > 0))
    return PEXSI_ERR_INVALID_ARG;
  pexsi_mu_info loc;
  std::memset(&loc, 0, sizeof(loc));
  const double Ne = opts->n_electrons, dN = opts->delta_n > 0 ? opts->delta_n : 0.1;
  const double tol = opts->tol_ne > 0 ? opts->tol_ne : 1e-6;
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    int rc = pexsi::plan_workspace(p);
    if (rc) return rc;
    pexsi::Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    ck(cudaMemcpyAsync(ws.H, H, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(ws.S, S, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
    const double* dS = S ? ws.S : nullptr;
    std::string err;
    double lo = opts->mu_lo, hi = opts->mu_hi, mu = 0.5 * (lo + hi);
    const int Q = opts->n_shifts;
    int expansions = 0;
    // ---- inertia counting cycles
    for (int cyc = 0; cyc < opts->max_inertia;) {
      std::vector<double> eps(Q), ninf(Q);
      std::vector<int64_t> cnt(Q);
      // a shift that lands on an eigenvalue breaks the LDL^T down; move the
      // whole set by a small irrational fraction of the spacing and retry
      for (int attempt = 0;; ++attempt) {
        const double nudge = attempt * 0.0137 * (hi - lo) / (Q - 1);
        for (int q = 0; q < Q; ++q) eps[q] = lo + (hi - lo) * q / (Q - 1) + (q == 0 ? -nudge : q == Q - 1 ? nudge : nudge * 0.618);
        rc = pexsi::inertia_range(p, ws, &p->prof, ws.H, dS, eps.data(), Q, cnt.data(), &err);
        if (rc != PEXSI_ERR_BREAKDOWN || attempt == 3) break;
      }
      if (rc) { p->last_error = err; return rc; }
      lo = eps.front();
      hi = eps.back();
      for (int q = 0; q < Q; ++q) ninf[q] = 2.0 * double(cnt[q]);
      if (ninf.front() > Ne - dN || ninf.back() < Ne + dN) {
        if (++expansions > 8) { p->last_error = "cannot bracket the electron count"; return PEXSI_ERR_INVALID_ARG; }
        double w = hi - lo;
        if (ninf.front() > Ne - dN) lo -= w;
        if (ninf.back() < Ne + dN) hi += w;
        continue;
      }
      double el = root(eps, ninf, beta, Ne - dN, lo, hi);
      double eh = root(eps, ninf, beta, Ne + dN, lo, hi);
      mu = 0.5 * (el + eh);
      // narrow to the samples enclosing [eps_l, eps_h]
      int ql = 0, qh = Q - 1;
      for (int q = 0; q < Q; ++q)
        if (eps[q] <= el && ninf[q] <= Ne - dN) ql = q;
      for (int q = Q - 1; q >= 0; --q)
        if (eps[q] >= eh && ninf[q] >= Ne + dN) qh = q;
      // widen by the Fermi tail: an eigenvalue just above eps[ql] already
      // adds to N_beta(eps[ql]) at finite temperature, so the bracket keeps a
      // margin of 16 / beta (exp(-16) ~ 1e-7 per state) on each side
      lo = eps[ql] - 16.0 / beta;
      hi = eps[qh] + 16.0 / beta;
      ++cyc;
      loc.inertia_cycles = cyc;
      if (hi - lo < 50.0 / beta) break;
    }
    loc.mu_inertia = mu;
    // ---- Newton on N(mu) = N_e with N'(mu) = Tr[Gamma^d S]
    double *o_dm = ws.out, *o_edm = ws.out + nnz, *o_fdm = ws.out + 2 * nnz;
    pexsi_dm_info di;
    for (int it = 0; it < std::max(1, opts->max_newton); ++it) {
      rc = pexsi::dm_range(p, ws, &p->prof, ws.H, dS, mu, beta, n_poles, delta_e, 0, n_poles, 0, o_dm, o_edm, o_fdm,
                           &di, &err);
      if (rc) { p->last_error = err; return rc; }
      loc.newton_iters = it + 1;
      loc.mu = mu;
      loc.n_e = di.trace_dm_s;
      loc.dn_dmu = di.trace_ddm_s;
      double r = di.trace_dm_s - Ne;
      if (std::fabs(r) <= tol) { loc.converged = 1; break; }
      if (r < 0) lo = std::max(lo, mu);
      else hi = std::min(hi, mu);
      double next = mu - r / di.trace_ddm_s;
      if (!(di.trace_ddm_s > 0) || !(next > lo && next < hi)) next = 0.5 * (lo + hi);
      mu = next;
    }
    loc.bracket_lo = lo;
    loc.bracket_hi = hi;
    if (dm) ck(cudaMemcpyAsync(dm, o_dm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(dm)");
    if (edm) ck(cudaMemcpyAsync(edm, o_edm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(edm)");
    if (fdm) ck(cudaMemcpyAsync(fdm, o_fdm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(fdm)");
    ck(cudaStreamSynchronize(ws.stream), "sync");
  } catch (const CudaError& ce) {
    p->last_error = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
    return PEXSI_ERR_CUDA;
  }
  if (info) *info = loc;
  return PEXSI_OK;
}
