// Internal definitions shared by the plan API (engine.cu) and the request
// server (server.cu): the device plan, per-computation workspaces and the
// batched numeric drivers.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/pexsi_gb300.h"
#include "kernels.cuh"
#include "symbolic.hpp"

namespace pexsi {

int pole_table(double beta, double delta_e, int P, double mu, std::vector<std::complex<double>>& z,
               std::vector<std::complex<double>>& w_rho, std::vector<std::complex<double>>& w_E,
               std::vector<std::complex<double>>& w_F, std::vector<std::complex<double>>* w_d = nullptr);

// An NVTX range over a host-side phase (visible in timeline profilers; a
// no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct CudaError {
  cudaError_t e;
  const char* what;
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaError{e, what};
}

// Host-side launch geometry of one level of the supernodal tree: fronts sorted
// by width descending, so the fronts still active at panel offset p0 (s > p0)
// are a prefix.
struct Level {
  int64_t front_off = 0;  // into the device list of level fronts
  std::vector<int32_t> fronts, s, m;
  std::vector<int64_t> ea_off;   // extend-add groups: rank k = k-th child of each parent
  std::vector<int32_t> ea_count, ea_tiles;
  std::vector<double> ea_elems;  // elements moved by each extend-add launch
  int64_t gather_tiles = 0;
  double gather_bytes = 0;
  // flat tile lists: prefix sums of the fronts' (or children's) 32x32 tiles in
  // the plan's d_tile_pref, so that a launch has exactly one block per tile
  int64_t gather_pref_off = 0, gather_total = 0;
  std::vector<int64_t> ea_pref_off, ea_total;
  // the same for the whole r x r update block of each child (LDU fronts)
  std::vector<int64_t> ea_pref_off_full, ea_total_full;
  std::vector<double> ea_elems_full;
  int32_t max_s = 0;
};

// CUDA-event bracketing of kernel launches, per launch class.
struct Profiler {
  bool on = false;
  struct Pending {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
    int kernels;
    double tensor;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[PEXSI_PROFILE_CLASSES] = {};
  double ms[PEXSI_PROFILE_CLASSES] = {}, flops[PEXSI_PROFILE_CLASSES] = {}, bytes[PEXSI_PROFILE_CLASSES] = {};
  double tensor[PEXSI_PROFILE_CLASSES] = {};
  cudaEvent_t begin(cudaStream_t st);
  void end(cudaEvent_t a, int cls, cudaStream_t st, double fl, double by, int kernels = 1, double tensor_fl = 0.0);
  void drain();
  void reset();
  void destroy();
};

enum ProfClass {
  P_ASSEMBLE, P_EXTEND, P_DIAG, P_PANEL, P_SCHUR, P_GATHER, P_OFFDIAG, P_DPART, P_DRED, P_POLESUM, P_TRACE, P_SLICE
};

// Device buffers of one in-flight computation: fronts for `batch` poles (or
// 2 x batch real shifts), split-K partials, status words, trace scratch, and
// staging for host-buffer calls; plus the stream the work runs on.
struct Workspace {
  int batch = 0;
  double2 *F = nullptr, *Y = nullptr, *part = nullptr;
  double2* kpart = nullptr;  // split-K partials of the FP64 Takahashi step
  void* dsave = nullptr;     // inertia shifts: panel blocks before inversion (counted afterwards)
  int* brk = nullptr;
  unsigned long long* minpiv = nullptr;
  int* neg = nullptr;
  double* partials = nullptr;
  double* trace3 = nullptr;
  double *H = nullptr, *S = nullptr, *out = nullptr;  // nnz, nnz, 4 nnz (DM, EDM, FDM, Gamma^d)
  double2* ainv = nullptr;
  uint8_t *ozA = nullptr, *ozB = nullptr;  // split-precision slice tiles
  int *exA = nullptr, *exB = nullptr, *ozfail = nullptr;
  uint32_t* ymax = nullptr;  // split path: row maxima of Y per pole
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // captured level schedules (factorisation + selected inversion of nb
  // complex poles at a Schur block width) and the stream they are captured on
  struct Graph {
    int nb, block;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t capture = nullptr;
  bool use_graphs = true;
  bool async = false;  // buffers from cudaMallocAsync on `stream`
  int64_t bytes = 0;
};

}  // namespace pexsi

struct pexsi_plan {
  pexsi::Symbolic sym;
  pexsi_opts opts{};
  std::string last_error;
  int b = 64;
  uint64_t wait_ns = 1000000000ull;  // bound of the device-side waits (opts.wait_ns, 0 = 1 s)
  int64_t* d_front_off = nullptr;
  int32_t *d_s = nullptr, *d_m = nullptr, *d_parent = nullptr, *d_rel = nullptr;
  int64_t* d_rptr = nullptr;
  int64_t *d_asm_src = nullptr, *d_asm_pos = nullptr;
  int64_t nlow = 0;
  int64_t* d_entry_pos = nullptr;
  int32_t* d_level_fronts = nullptr;
  int32_t* d_ea = nullptr;
  int32_t* d_tile_pref = nullptr;  // see Level::gather_pref_off / ea_pref_off
  int64_t* d_part_off = nullptr;
  int64_t part_stride = 0;  // partial-scratch elements per batch member
  double* d_ident = nullptr;
  // split-precision scratch layout (per front offsets within a level; strides
  // per batch member): slice tiles of A and B, exponents of A rows, B columns
  int oz_slices = 0;
  int oz_block = pexsi::kOzBlockPanels;  // panels per block of the split Schur update (1..kOzBlockPanels; tunable)
  int64_t *d_ozA_off = nullptr, *d_ozB_off = nullptr, *d_exA_off = nullptr, *d_exB_off = nullptr;
  int64_t* d_ymax_off = nullptr;  // first row of each front among all fronts' rows
  int64_t ymax_stride = 0;        // sum of m_K
  int64_t ozA_stride = 0, ozB_stride = 0, exA_stride = 0, exB_stride = 0;
  // the same for the real Schur update of the inertia factorisation (twice
  // as many batch members share the scratch; exponents use the offsets above)
  int64_t *d_ozA_off_r = nullptr, *d_ozB_off_r = nullptr;
  int64_t ozA_stride_r = 0, ozB_stride_r = 0;
  std::vector<pexsi::Level> levels;
  pexsi::FlopCounts flops;
  int trace_blocks = 256;
  pexsi::Profiler prof;
  pexsi::Workspace ws;  // the plan's own workspace (plan API calls)
  // complex Hermitian variant (LDU fronts), created on its first call: the
  // front position of each CSC entry and of its transpose, a complex
  // identity S, and the plan API's complex staging (H, S: nnz; outputs: 4 nnz)
  int64_t *d_pos_full = nullptr, *d_pos_t = nullptr;
  int32_t *d_col0 = nullptr, *d_bk_slots = nullptr;  // first column per front; (front, p0) of every panel
  int32_t n_bk_slots = 0;
  std::vector<int64_t> diag_entries;  // CSC entries on the diagonal
  // A plan that merges several systems (pexsi_group): the first CSC entry of
  // each system among the concatenated entries (nsys + 1), and each system's
  // range of the assembly list; {0, nnz} and {0, nlow} for a single system.
  std::vector<int64_t> sys_entry_off, sys_asm_off;
  double2 *d_ident_c = nullptr, *d_hH = nullptr, *d_hS = nullptr, *d_hout = nullptr;

  pexsi::DevFronts fronts() const {
    pexsi::DevFronts f;
    f.off = d_front_off;
    f.s = d_s;
    f.m = d_m;
    f.parent = d_parent;
    f.rptr = d_rptr;
    f.rel = d_rel;
    f.pool = sym.front_elems;
    return f;
  }
};

namespace pexsi {

// Bytes of workspace one pole adds (F and Y fronts + partials).
int64_t bytes_per_pole(const pexsi_plan* p);
// Fixed bytes of a workspace (staging + status + trace scratch).
int64_t bytes_fixed(const pexsi_plan* p);

// Allocates ws for `batch` poles on `stream` (cudaMallocAsync when async).
void workspace_alloc(const pexsi_plan* p, Workspace& ws, int batch, cudaStream_t stream, bool async);
void workspace_free(Workspace& ws);

// Poles [begin, end) of the P-pole table into d_dm/d_edm/d_fdm (device, any
// may be NULL), accumulating when `accumulate`; traces and status into info
// when info != NULL (synchronises ws.stream). Returns a PEXSI code; message
// in *err.
// Gamma^d (for N'(mu), Sec. II.C) accumulates into ws.out + 3 nnz with the
// same `accumulate` rule, and its trace goes to info->trace_ddm_s.
int dm_range(const pexsi_plan* p, Workspace& ws, Profiler* prof, const double* dH, const double* dS, double mu,
             double beta, int P, double delta_e, int begin, int end, int accumulate, double* d_dm, double* d_edm,
             double* d_fdm, pexsi_dm_info* info, std::string* err);

// Inertia counts of H - shifts[m] S (host shifts and counts); synchronises.
int inertia_range(const pexsi_plan* p, Workspace& ws, Profiler* prof, const double* dH, const double* dS,
                  const double* shifts, int n_shifts, int64_t* counts, std::string* err);

// The plan's own workspace (created on first use); PEXSI code.
int plan_workspace(pexsi_plan* p);

// Complex Hermitian H and S (interleaved complex, nnz each; dS NULL = I):
// poles [begin, end) into complex d_dm / d_edm / d_fdm (any may be NULL)
// through LDU fronts; Gamma^d into the plan's staging. Same status rules as
// dm_range. Needs the plan's Hermitian maps (hermitian_prepare).
int hermitian_prepare(pexsi_plan* p);
int inertia_range_herm(const pexsi_plan* p, Workspace& ws, const double2* dH, const double2* dS, const double* shifts,
                       int n_shifts, int64_t* counts, std::string* err);
int selinv_one_herm(const pexsi_plan* p, Workspace& ws, const double2* dH, const double2* dS, double z_re, double z_im,
                    double2* d_ainv, std::string* err);
int dm_range_herm(const pexsi_plan* p, Workspace& ws, Profiler* prof, const double2* dH, const double2* dS, double mu,
                  double beta, int P, double delta_e, int begin, int end, int accumulate, double2* d_dm,
                  double2* d_edm, double2* d_fdm, pexsi_dm_info* info, std::string* err);

// Groups of systems (one merged plan): the symbolic structures side by side,
// and the batched driver over all systems' poles.
Symbolic merge_symbolic(const std::vector<const Symbolic*>& parts);
int dm_range_group(const pexsi_plan* p, Workspace& ws, Profiler* prof, int wave, const double* const* dH,
                   const double* const* dS, const double* mu, const double* beta, int P, const double* delta_e,
                   int begin, int end, int accumulate, double* const* d_dm, double* const* d_edm, double* const* d_fdm,
                   pexsi_dm_info* info, const std::vector<int32_t>& f_off, std::string* err);

// Selected inverse of one complex shift into d_ainv (device, nnz complex);
// synchronises ws.stream.
int selinv_one(const pexsi_plan* p, Workspace& ws, const double* dH, const double* dS, double z_re, double z_im,
               double2* d_ainv, std::string* err);

}  // namespace pexsi
