// Density of states and local density of states (Sec. II.D): the CDOS from
// inertia counts (Eq. cdos) and its numerical derivative; the LDOS matrix
// from one selected inversion at eps + i eta (Eq. LDOSGreen).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plan.hpp"

using pexsi::CudaError;
using pexsi::ck;

namespace {
constexpr double kPi = 3.14159265358979323846;

int stage(pexsi_plan* p, const double* H, const double* S, const double** dS) {
  ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
  int rc = pexsi::plan_workspace(p);
  if (rc) return rc;
  pexsi::Workspace& ws = p->ws;
  const size_t nnz = size_t(p->sym.nnz);
  ck(cudaMemcpyAsync(ws.H, H, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
  if (S) ck(cudaMemcpyAsync(ws.S, S, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
  *dS = S ? ws.S : nullptr;
  return PEXSI_OK;
}
}  // namespace

extern "C" int pexsi_dos(pexsi_plan* p, const double* H, const double* S, double e_lo, double e_hi,
                         int32_t n_points, double* eps, double* cdos, double* dos) {
  if (!p || !H || !eps || !cdos || !dos || n_points < 2 || !(e_hi > e_lo) || p->opts.device < 0)
    return PEXSI_ERR_INVALID_ARG;
  try {
    const double* dS = nullptr;
    int rc = stage(p, H, S, &dS);
    if (rc) return rc;
    std::vector<int64_t> cnt(n_points);
    for (int k = 0; k < n_points; ++k) eps[k] = e_lo + (e_hi - e_lo) * k / (n_points - 1);
    std::string err;
    rc = pexsi::inertia_range(p, p->ws, &p->prof, p->ws.H, dS, eps, n_points, cnt.data(), &err);
    if (rc) { p->last_error = err; return rc; }
    for (int k = 0; k < n_points; ++k) cdos[k] = 2.0 * double(cnt[k]);
    for (int k = 0; k < n_points; ++k) {
      int a = k > 0 ? k - 1 : 0, b = k + 1 < n_points ? k + 1 : n_points - 1;
      dos[k] = (cdos[b] - cdos[a]) / (eps[b] - eps[a]);
    }
  } catch (const CudaError& ce) {
    p->last_error = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
    return PEXSI_ERR_CUDA;
  }
  return PEXSI_OK;
}

extern "C" int pexsi_ldos(pexsi_plan* p, const double* H, const double* S, double eps, double eta, double* ldos) {
  if (!p || !H || !ldos || !(eta > 0) || p->opts.device < 0) return PEXSI_ERR_INVALID_ARG;
  try {
    const double* dS = nullptr;
    int rc = stage(p, H, S, &dS);
    if (rc) return rc;
    pexsi::Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    std::string err;
    // the selected inverse stays in ws.Y; only the scaled imaginary part is read out
    if (!ws.ainv) ck(cudaMalloc(&ws.ainv, sizeof(double2) * nnz), "cudaMalloc(ainv)");
    rc = pexsi::selinv_one(p, ws, ws.H, dS, eps, eta, ws.ainv, &err);
    if (rc) { p->last_error = err; return rc; }
    pexsi::launch_scaled_imag(ws.Y, p->d_entry_pos, p->sym.nnz, 2.0 / kPi, ws.out, ws.stream);
    ck(cudaGetLastError(), "ldos");
    ck(cudaMemcpyAsync(ldos, ws.out, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(ldos)");
    ck(cudaStreamSynchronize(ws.stream), "sync");
  } catch (const CudaError& ce) {
    p->last_error = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
    return PEXSI_ERR_CUDA;
  }
  return PEXSI_OK;
}
