// Device kernels of the multifrontal LDL^T + selected inversion (Sec. II.B,
// steps 3 and 4) and of the pole sum (Eq. gammapole, Eq. gammaF).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pexsi {

constexpr int kMaxBatch = 64;  // poles (or shifts) processed together
constexpr int kTile = 64;      // GEMM output tile edge
constexpr int kMaxKsplit = 8;  // K splits of the FP64 Takahashi step (kpart slots per 64-row tile)

// Shifts of one batch, passed by value: complex z_b (re, im) for poles, or
// real sigma_b (im = 0) for inertia shifts. Weights of the pole sum.
struct BatchShifts {
  int nb;
  double re[kMaxBatch], im[kMaxBatch];
  double wr_re[kMaxBatch], wr_im[kMaxBatch];  // w^rho
  double we_re[kMaxBatch], we_im[kMaxBatch];  // w^E
  double wf_re[kMaxBatch], wf_im[kMaxBatch];  // w^F
  double wd_re[kMaxBatch], wd_im[kMaxBatch];  // w^d (mu-derivative of the Fermi function)
};

// Front geometry on the device.
struct DevFronts {
  const int64_t* off;   // element offset of each front in one pole's pool
  const int32_t* s;     // width s_K
  const int32_t* m;     // m_K = s_K + r_K
  const int32_t* parent;
  const int64_t* rptr;  // offsets into rel
  const int32_t* rel;   // child structure rows -> parent front rows
  int64_t pool;         // elements per pole
};

// Error reporting shared by all kernels of one call.
struct DevStatus {
  int* breakdown_front;              // atomicMin of the first failing front (INT_MAX = none)
  unsigned long long* min_pivot;     // atomicMin of the bit pattern of min |pivot| / max |entry|
  int* neg_count;                    // per batch member: negative eigenvalues of D (inertia)
  // inertia: the panel blocks D saved before inversion, counted afterwards by
  // launch_bk_count_all off the factorisation's critical path; the block of
  // (front f, panel p0) of member b sits at dsave + b * dsave_stride + (col0[f] + p0) * b_panel
  void* dsave;
  const int32_t* col0;               // first column of each front
  int64_t dsave_stride;
};

// Scratch of the split-precision GEMM: bf16 slice tiles of A = Y[S,S] and
// B = L[S,P], their power-of-two exponents (per row / column), per front
// offsets within one batch member, strides between batch members, and a
// failure flag (a bounded wait ran out).
struct OzScratch {
  uint8_t* A;
  const int64_t* A_off;
  int64_t A_stride;
  uint8_t* B;
  const int64_t* B_off;
  int64_t B_stride;
  int* exA;
  const int64_t* exA_off;
  int64_t exA_stride;
  int* exB;
  const int64_t* exB_off;
  int64_t exB_stride;
  int* fail;
  // selected inversion: per front row r, the largest high word of |Re|, |Im|
  // over the part of row r of Y already computed (columns from the current
  // panel on), kept up to date by the kernels that write Y
  uint32_t* ymax;
  const int64_t* ymax_off;  // first row of each front
  int64_t ymax_stride;      // rows per pole
  uint64_t wait_ns;         // bound of every wait on another role (wall time)
  int stall;                // testing: CTA 0 of the short-K GEMM issues no copy
};

// ---- launchers (T = double for real inertia, double2 for complex poles) ----
template <typename T>
void launch_assemble(T* F, const double* H, const double* S, const int64_t* src, const int64_t* pos, int64_t nlow,
                     int64_t pool, const BatchShifts& sh, cudaStream_t st);

template <typename T>
void launch_extend_add(T* F, const DevFronts& fr, const int32_t* children, int nchild, const int32_t* pref,
                       int64_t total_tiles, const BatchShifts& sh, cudaStream_t st);

template <typename T>
void launch_diag_inv(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0, int b,
                     const BatchShifts& sh, DevStatus status, bool count_inertia, cudaStream_t st);

template <typename T>
void launch_panel_solve(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_row_tiles, int p0,
                        int b, const BatchShifts& sh, cudaStream_t st);

template <typename T>
void launch_trailing(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles, int p0, int b,
                     const BatchShifts& sh, cudaStream_t st);

void launch_gather(double2* Y, const DevFronts& fr, const int32_t* fronts, int nfronts, const int32_t* pref,
                   int64_t total_tiles, const BatchShifts& sh, cudaStream_t st);

// kpart (kstride elements per batch member, kMaxKsplit * kTile * b per tile
// slot of part_off) enables the split-K form; NULL runs one block per tile.
void launch_selinv_offdiag(double2* Y, const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts,
                           int max_row_tiles, int max_mp, int p0, int b, const BatchShifts& sh, double2* kpart,
                           const int64_t* part_off, int64_t kstride, cudaStream_t st);

void launch_selinv_diag_partial(const double2* Y, const double2* F, double2* part, const int64_t* part_off,
                                int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts,
                                int max_row_tiles, int p0, int b, const BatchShifts& sh, cudaStream_t st);

void launch_selinv_diag_reduce(double2* Y, const double2* F, const double2* part, const int64_t* part_off,
                               int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0,
                               int b, const BatchShifts& sh, cudaStream_t st);

void launch_pole_sum(const double2* Y, int64_t pool, const int64_t* entry_pos, int64_t nnz, const BatchShifts& sh,
                     int overwrite, double* dm, double* edm, double* fdm, double* ddm, cudaStream_t st);

void launch_extract(const double2* Y, const int64_t* entry_pos, int64_t nnz, double2* out, cudaStream_t st);

// out[e] = scale * Im Y[entry_pos[e]] (the LDOS matrix from one selected inverse).
void launch_scaled_imag(const double2* Y, const int64_t* entry_pos, int64_t nnz, double scale, double* out,
                        cudaStream_t st);

// Split-precision Takahashi step Y[S,P] = -Y[S,S] L[S,P] and its mirror, with
// A = Y[S,S] sliced on the fly inside the GEMM: prep = true computes the row
// exponents of A and slices B, prep = false runs the GEMM.
// Row maxima of Y for the rows of each front when its selected inversion
// starts (the update set from Y[U,U], the supernode rows 0); the Takahashi
// kernel and the Y[P,P] reduction keep them up to date, and they give the
// row exponents of A = Y[S,S] without reading Y[S,S] for every panel.
void launch_oz_rowmax_init(const double2* Y, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_m,
                           const OzScratch& oz, int nb, cudaStream_t st);
void launch_oz_takahashi(double2* Y, const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts,
                         int max_mp, int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, bool prep);
// Split-precision Y[P,P] = D^-1 - L[S,P]^T Y[S,P] (panel width 64): stage 0
// exponents of the Y[S,P] columns, stage 1 split-K GEMM into `part` (exact
// int64 sums per 256-deep K range), stage 2 reduction and symmetrisation.
void launch_oz_dpart(double2* Y, const double2* F, double2* part, const int64_t* part_off, int64_t part_stride,
                     const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp, int p0, int b, int S,
                     const OzScratch& oz, int nb, cudaStream_t st, int stage);
// Split-precision Schur update F[S,S] -= L[S,P] W[S,P]^T (lower triangle):
// slicing of L rows and W rows, then the tcgen05 GEMM with an FP64
// read-modify-write (max_tiles = max over fronts of oz_schur_tiles(m_p)).
// The panels are taken in blocks of kOzBlockPanels: with cb > 0 (the end
// column of the block) a panel updates only the columns before min(cb, s)
// (max_tiles = max of oz_block_tiles), and after the block one call with
// p0 = the block start, b = the block width and cb = 0 updates the rest with
// K = the block width (at most 256, one exact chunk of the FP32 accumulators).
constexpr int kOzBlockPanels = 4;
void launch_oz_slice_schur(const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp,
                           int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb);
void launch_oz_gemm_schur(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles, int p0,
                          int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb);
int oz_schur_tiles(int mp);
int oz_block_tiles(int mp, int cs, bool cplx);
size_t oz_smem_bytes(int S);
// Slice-tile scratch of one front per pole (both phases), for its largest m_p.
int64_t oz_front_bytes_A(int64_t mp, int b, int S);
int64_t oz_front_bytes_B(int64_t mp, int b, int S);
int64_t oz_front_bytes_A_real(int64_t mp, int b, int S);
int64_t oz_front_bytes_B_real(int64_t mp, int b, int S);
// Split-precision real Schur update of the inertia factorisation (LDL^T of
// H - sigma S): slicing of L rows and W rows, then the tcgen05 GEMM on
// 128 x 64 lower-triangle tiles (max_tiles = max of oz_schur_tiles_real).
int oz_schur_tiles_real(int mp);
// Split-precision panel solve L[S,P] = W[S,P] D^-1 (W^T kept in the upper
// triangle): gemm = false launches the slicing, gemm = true the tcgen05 GEMM.
void launch_oz_panel(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp, int p0, int b,
                     int S, const OzScratch& oz, int nb, cudaStream_t st, bool gemm);
void launch_oz_panel_real(double* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp, int p0,
                          int b, int S, const OzScratch& oz, int nb, cudaStream_t st, bool gemm);
void launch_oz_slice_schur_real(const double* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp,
                                int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb);
void launch_oz_gemm_schur_real(double* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles,
                               int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb);
cudaError_t oz_configure(int S);

// ---- LDU fronts (complex Hermitian H and S, Sec. IV's k-point / spin-orbit
// variant): A = H - z S is only structurally symmetric, so a front holds L
// below and U above its diagonal blocks, the Schur update covers the whole
// trailing square, and selected inversion computes Y[S,P] = -Y[S,S] L[S,P]
// and Y[P,S] = -U[P,S] Y[S,S] separately, with Y[P,P] = D^-1 - U[P,S] Y[S,P].
void launch_assemble_gen(double2* F, const double2* H, const double2* S, const int64_t* pos, int64_t nnz,
                         int64_t pool, const BatchShifts& sh, cudaStream_t st);
void launch_extend_add_full(double2* F, const DevFronts& fr, const int32_t* children, int nchild, const int32_t* pref,
                            int64_t total_tiles, const BatchShifts& sh, cudaStream_t st);
// count_inertia (real shifts of Hermitian H, S): Hermitian Bunch-Kaufman count of each D block
void launch_diag_inv_gen(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0, int b,
                         const BatchShifts& sh, DevStatus status, bool count_inertia, cudaStream_t st);
// upper = false: L[S,P] = A[S,P] D^-1 (A[P,S] stays); upper = true: U[P,S] = D^-1 A[P,S]
void launch_panel_solve_gen(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_row_tiles,
                            int p0, int b, const BatchShifts& sh, cudaStream_t st, bool upper);
void launch_trailing_full(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_row_tiles,
                          int p0, int b, const BatchShifts& sh, cudaStream_t st);
void launch_selinv_offdiag_gen(double2* Y, const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts,
                               int max_row_tiles, int p0, int b, const BatchShifts& sh, cudaStream_t st);
void launch_selinv_diag_partial_gen(const double2* Y, const double2* F, double2* part, const int64_t* part_off,
                                    int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts,
                                    int max_row_tiles, int p0, int b, const BatchShifts& sh, cudaStream_t st);
void launch_selinv_diag_reduce_gen(double2* Y, const double2* F, const double2* part, const int64_t* part_off,
                                   int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0,
                                   int b, const BatchShifts& sh, cudaStream_t st);
// (w G - conj(w) G^H) / 2i at each CSC entry: pos = its own position, pos_t = that of its transpose
void launch_pole_sum_herm(const double2* Y, int64_t pool, const int64_t* pos, const int64_t* pos_t, int64_t nnz,
                          const BatchShifts& sh, int overwrite, double2* dm, double2* edm, double2* fdm, double2* ddm,
                          cudaStream_t st);

// Inertia counts of all saved panel blocks (slots: (front, p0) pairs, nslots
// of them) for nb batch members: one CTA per block and member, a Bunch-Kaufman
// LDL^T (real, or Hermitian for T = double2) adding its negative eigenvalues
// to status.neg_count and flagging singular blocks.
template <typename T>
void launch_bk_count_all(const int32_t* slots, int nslots, const DevFronts& fr, int b, int nb, DevStatus status,
                         cudaStream_t st);

// Raises the dynamic shared-memory limits the kernels need for panel width b.
cudaError_t configure_kernels(int b);

// Deterministic Tr[X S] for up to four X (NULL entries give 0): partial sums
// of fixed ranges in `partials` (4 * nblocks doubles), then one ordered sum.
void launch_traces(const double* dm, const double* edm, const double* fdm, const double* ddm, const double* S,
                   int64_t nnz, double* partials, int nblocks, double* out4, cudaStream_t st);

}  // namespace pexsi
