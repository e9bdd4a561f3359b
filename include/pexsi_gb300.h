/*
 * pexsi_gb300.h -- C ABI of the GB300 (sm_103a) PEXSI hot path.
 *
 * The library computes, for a sparse symmetric pair (H, S) on a shared
 * pattern, the selected elements (those on the pattern of H) of
 *
 *   DM  = Im sum_l w^rho_l (H - (z_l + mu) S)^{-1}     (Sec. II.A, Eq. gammapole)
 *   EDM = Im sum_l w^E_l   (H - (z_l + mu) S)^{-1}     (Sec. II.A, Eq. gammaF)
 *   FDM = Im sum_l w^F_l   (H - (z_l + mu) S)^{-1}     (Sec. II.A, Eq. gammaF)
 *
 * through a supernodal LDL^T factorisation of each complex-symmetric shifted
 * matrix followed by selected inversion (Sec. II.B, steps 1-4), and the
 * inertia count of real shifted matrices H - sigma S (Sec. II.C, Sylvester's
 * law of inertia). Steps 1-2 (ordering, symbolic analysis) run on the host
 * once per pattern in pexsi_setup; steps 3-4 and the pole sum run in CUDA
 * kernels on one GPU.
 *
 * Conventions shared by every call:
 *  - Patterns are 0-based CSC: colptr[n+1] (int64), rowind[nnz] (int32), row
 *    indices strictly increasing within each column, every diagonal entry
 *    present, and the pattern structurally symmetric (the FULL symmetric
 *    pattern is stored, both triangles). It is the pattern of H; the pattern
 *    of S must be a subset (store explicit zeros).
 *  - Value arrays (H, S, DM, EDM, FDM) hold nnz float64 entries in that CSC
 *    order. Selected-inverse outputs hold nnz complex values as interleaved
 *    (re, im) float64 pairs.
 *  - Every call returns PEXSI_OK (0) or a negative PEXSI_ERR_* code; no C++
 *    exception crosses the ABI. pexsi_strerror() names a code and
 *    pexsi_last_error_detail() gives the plan's last message.
 *  - A plan is not thread-safe: callers serialise calls on one plan.
 *  - "Host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory on the plan's device; `stream` is a cudaStream_t passed as
 *    void* (NULL = the legacy default stream).
 */
#ifndef PEXSI_GB300_H
#define PEXSI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
enum {
  PEXSI_OK = 0,
  PEXSI_ERR_INVALID_ARG = -1,   /* bad size, NULL where required, bad CSC      */
  PEXSI_ERR_NOT_SYMMETRIC = -2, /* pattern not structurally symmetric          */
  PEXSI_ERR_NOMEM = -3,         /* host or device allocation failed            */
  PEXSI_ERR_CUDA = -4,          /* a CUDA runtime call or kernel launch failed */
  PEXSI_ERR_BREAKDOWN = -5,     /* zero / non-finite pivot in a diagonal block */
  PEXSI_ERR_INTERNAL = -6,      /* violated internal invariant (a bug)         */
  PEXSI_ERR_CANCELLED = -7,     /* server request cancelled before completion  */
  PEXSI_ERR_TIMEOUT = -8,       /* a bounded device-side wait ran out (split-
                                   precision kernels; pexsi_opts.wait_ns)      */
  PEXSI_PENDING = 1             /* server request not finished yet (poll)      */
};

typedef struct pexsi_plan pexsi_plan;

/* Options of pexsi_setup. Zero-initialised fields take the defaults that
 * pexsi_opts_default() writes. */
typedef struct pexsi_opts {
  int32_t device;          /* CUDA device ordinal (default 0); -1 builds a host-only
                              plan (ordering and symbolic analysis, no device memory)
                              on which the numeric calls return INVALID_ARG          */
  int32_t panel;           /* panel width b of the blocked front factorisation,
                              16..64 (default 64)                                    */
  int32_t leaf_cols;       /* nested-dissection leaf size in columns (default 96)    */
  int32_t amalgamate;      /* 1: relaxed supernode amalgamation (default), 0: off    */
  int32_t max_batch;       /* poles / shifts per device batch, 0 = automatic         */
  int32_t split_slices;    /* 0: FP64 GEMMs (default). 2..6: the supernode GEMMs
                              (panel solve L = W D^-1, Schur update F -= L W^T,
                              Takahashi step Y[S,P] = -Y[S,S] L[S,P] and Y[P,P] =
                              D^-1 - L[S,P]^T Y[S,P]; real ones of the inertia
                              LDL^T too) run on the tcgen05 tensor cores as exact
                              products of this many bf16 slices per operand (Ozaki
                              scheme; 6 slices ~ 42 bits), FP64 in and out; the
                              diagonal-block inverses and the pole sum stay FP64.
                              Requires panel = 64; other values are INVALID_ARG. */
  int64_t hbm_budget;      /* bytes of device workspace the batch may use, 0 = auto  */
  int64_t wait_ns;         /* bound, in ns of wall time, of every wait of one role of
                              a split-precision kernel on another (an mbarrier phase
                              of a copy, of the MMAs, of a TMEM drain); 0 = 1 s. A
                              wait that runs out stops the launch cleanly (every
                              role returns, TMEM is freed, later launches of the
                              call return at once) and the call returns
                              PEXSI_ERR_TIMEOUT. No other kernel waits.           */
  int32_t inject;          /* fault injection for tests of the error paths, 0 = off
                              (default). 1: CTA 0 of every short-K split GEMM launch
                              issues no operand copy, so that its MMA issuer's wait
                              runs out after wait_ns (PEXSI_ERR_TIMEOUT; split_slices
                              > 0 only). 2: a breakdown of front 0 is recorded from
                              the host after the first pole batch of every call with
                              accumulate = 0 (PEXSI_ERR_BREAKDOWN at the end of the
                              chain).                                             */
  int32_t split_block;     /* split-precision path: panels per block of the Schur
                              update, 1..4 (0 = 4). Each panel updates the rest of
                              its block, then one update of K = 64 x split_block
                              covers everything to the right; 1 is the unblocked
                              per-panel update (exponents over 64 columns of L).  */
} pexsi_opts;

/* Symbolic statistics of a plan. Flop counts are algorithmic real flops of
 * ONE pole (complex multiply-add = 8 flops) for the blocked front algorithm
 * the kernels run; the diagonal-block inversions are counted separately. */
typedef struct pexsi_plan_stats {
  int64_t n, nnz;
  int64_t nsuper;          /* supernodes (fronts) after amalgamation      */
  int64_t nlevels;         /* height of the supernodal elimination tree   */
  int64_t nnz_L;           /* entries of L below and on the diagonal      */
  int64_t front_elems;     /* sum over fronts of m_K^2 (one pole)         */
  int64_t max_front;       /* max m_K = s_K + r_K                         */
  int64_t max_width;       /* max s_K                                     */
  double factor_gemm_flops;/* panel solves + Schur (trailing) updates     */
  double selinv_gemm_flops;/* Y(S,P) = -Y(S,S) L(S,P) and Y(P,P) updates  */
  double diag_flops;       /* diagonal-block inversions                   */
  double gather_bytes;     /* bytes moved by the Ainv(C,C) gathers, 1 pole*/
  int64_t batch;           /* poles per device batch chosen for this plan */
  int64_t workspace_bytes; /* device workspace at that batch              */
} pexsi_plan_stats;

/* Per-call report of pexsi_dm / pexsi_dm_device. */
typedef struct pexsi_dm_info {
  double trace_dm_s;       /* Tr[DM S] = N_e (Eq. Nmu); computed on the device   */
  double trace_edm_s;      /* Tr[EDM S]                                          */
  double trace_fdm_s;      /* Tr[FDM S] (grand potential)                        */
  double min_pivot_ratio;  /* min over diagonal blocks of |pivot| / max |entry|, |z| = |Re z| + |Im z| */
  double ms_total;         /* wall time of the call (device events)             */
  double gemm_flops;       /* algorithmic GEMM flops executed by the call       */
  int32_t n_poles;         /* poles evaluated by the call                       */
  int32_t breakdown_front; /* front of the first breakdown, -1 if none          */
  double trace_ddm_s;      /* Tr[Gamma^d S] = N'(mu) (Sec. II.C): Gamma^d uses the
                              weights of d f / d mu with the same poles; it is
                              accumulated like the outputs (plan workspace)     */
} pexsi_dm_info;

/* Fill *opts with the defaults. */
int pexsi_opts_default(pexsi_opts* opts);

/* Steps 1-2 of Sec. II.B: fill-reducing ordering (nested dissection on the
 * supervariable graph, or the caller's permutation), elimination tree
 * (Sec. II.B, Eq. parent), supernodes, front structure and the maps that the
 * kernels use; then uploads the plan to the device.
 *   n, colptr, rowind : the pattern (see conventions); the library copies it.
 *   perm_or_null      : optional fill-reducing order, perm[new] = old; the
 *                       library still post-orders it. NULL = own ordering.
 *   opts              : NULL = defaults.
 *   out               : receives the plan; free it with pexsi_plan_destroy.
 * Errors: INVALID_ARG (bad CSC, missing diagonal, bad perm), NOT_SYMMETRIC,
 * NOMEM, CUDA. On error *out is NULL. */
int pexsi_setup(int64_t n, const int64_t* colptr, const int32_t* rowind,
                const int32_t* perm_or_null, const pexsi_opts* opts, pexsi_plan** out);

/* Release the plan and all of its host and device memory. NULL is a no-op. */
int pexsi_plan_destroy(pexsi_plan* plan);

int pexsi_plan_get_stats(const pexsi_plan* plan, pexsi_plan_stats* stats);

/* Write the final column order, perm[new] = old (n entries). */
int pexsi_plan_get_perm(const pexsi_plan* plan, int32_t* perm);

/* The pole expansion of Eq. polerho / Eq. gammaF (the construction the paper
 * cites: contour quadrature of the Fermi-Dirac function around the spectrum
 * through an elliptic-function map). For n_poles = P (even, >= 2) it writes
 * P complex shifts z_l + mu (Im > 0) and the weights w^rho, w^E, w^F as
 * interleaved (re, im) pairs, 2P doubles each. Any weight pointer may be
 * NULL. Such that for eps in [mu - delta_e, mu + delta_e]:
 *   2/(1+exp(beta (eps-mu)))          ~= Im sum_l w^rho_l / (eps - z_l)
 *   eps * 2/(1+exp(beta (eps-mu)))    ~= Im sum_l w^E_l   / (eps - z_l)
 *   -(2/beta) ln(1+exp(-beta(eps-mu)))~= Im sum_l w^F_l   / (eps - z_l)
 * Errors: INVALID_ARG (P odd or < 2, beta or delta_e not positive). */
int pexsi_pole_table(double beta, double delta_e, int32_t n_poles, double mu,
                     double* z, double* w_rho, double* w_E, double* w_F);

/* DM, EDM and FDM on the pattern for the P-pole expansion at (mu, beta,
 * delta_e) -- Eq. gammapole and Eq. gammaF. Host buffers of nnz doubles; any
 * output may be NULL. S == NULL means S = I (H's diagonal positions). The
 * call is synchronous. On error the outputs are undefined.
 * Errors: INVALID_ARG, NOMEM, CUDA, BREAKDOWN (info->breakdown_front),
 * TIMEOUT (split-precision path only: a bounded device-side wait ran out). */
int pexsi_dm(pexsi_plan* plan, const double* H, const double* S, double mu, double beta,
             int32_t n_poles, double delta_e, double* dm, double* edm, double* fdm,
             pexsi_dm_info* info);

/* Host-buffer form over the pole subrange [pole_begin, pole_end) of the
 * P-pole table (the end-to-end call: copies H and S to the device, computes,
 * copies the outputs back; synchronous). accumulate = 1 adds to the outputs.
 * Errors as pexsi_dm. */
int pexsi_dm_poles(pexsi_plan* plan, const double* H, const double* S, double mu, double beta,
                   int32_t n_poles, double delta_e, int32_t pole_begin, int32_t pole_end,
                   int32_t accumulate, double* dm, double* edm, double* fdm, pexsi_dm_info* info);

/* Device form of pexsi_dm over the pole subrange [pole_begin, pole_end) of
 * the same P-pole table: dH, dS, d_dm, d_edm, d_fdm are device buffers of nnz
 * doubles (dS may be NULL for S = I; outputs may be NULL). accumulate = 0
 * overwrites the outputs, 1 adds this subrange's contribution to them. The
 * work is enqueued on `stream`; the call returns after enqueueing unless
 * info != NULL, in which case it synchronises `stream` to fill info.
 * Status of a chain of calls: a call with accumulate = 0 clears the plan's
 * breakdown / timeout status, calls with accumulate = 1 keep it, and the
 * first call with info != NULL returns the status of every batch since the
 * chain began (BREAKDOWN, TIMEOUT). A chain that is never read with info
 * reports nothing; pass info on its last call. Inertia calls keep status
 * words of their own and do not disturb a chain. */
int pexsi_dm_device(pexsi_plan* plan, const double* dH, const double* dS, double mu,
                    double beta, int32_t n_poles, double delta_e, int32_t pole_begin,
                    int32_t pole_end, int32_t accumulate, double* d_dm, double* d_edm,
                    double* d_fdm, void* stream, pexsi_dm_info* info);

/* Selected elements of (H - z S)^{-1} on the pattern for one complex shift z
 * with Im z != 0 (one pole of Sec. II.A; also the LDOS kernel of Sec. II.D,
 * Eq. LDOSGreen, with z = eps + i eta). Host buffers; ainv receives nnz
 * interleaved complex values. Errors as pexsi_dm. */
int pexsi_selinv(pexsi_plan* plan, const double* H, const double* S, double z_re,
                 double z_im, double* ainv);

/* Inertia counts (Sec. II.C): counts[m] = number of generalised eigenvalues
 * of (H, S) below shifts[m] (per spin; N_infinity = 2 * counts), obtained as
 * the number of negative eigenvalues of D in the real block LDL^T of
 * H - shifts[m] S. Host buffers. A shift on (or numerically at) an
 * eigenvalue gives BREAKDOWN; perturb it and retry. */
int pexsi_inertia(pexsi_plan* plan, const double* H, const double* S, const double* shifts,
                  int32_t n_shifts, int64_t* counts);

/* Device form of pexsi_inertia: dH, dS device buffers; shifts and counts are
 * host arrays; synchronises `stream` before returning. */
int pexsi_inertia_device(pexsi_plan* plan, const double* dH, const double* dS,
                         const double* shifts, int32_t n_shifts, int64_t* counts, void* stream);

/* Supernodal structure of a plan (Sec. II.B, Eq. parent), new numbering:
 * first[nsuper+1] first column of each supernode, rptr[nsuper+1] offsets of
 * each off-diagonal row structure in rows[rptr[nsuper]] (ascending rows), and
 * parent[nsuper] (-1 for roots). Sizes come from pexsi_plan_get_stats (nsuper)
 * and this call with rows == NULL, which only writes first, rptr and parent. */
int pexsi_plan_get_supernodes(const pexsi_plan* plan, int32_t* first, int64_t* rptr, int32_t* rows,
                              int32_t* parent);

/* ------------------------------------------------------------ complex Hermitian H and S
 * The variant Sec. IV names for k-point sampling and spin-orbit coupling:
 * H and S complex Hermitian on the same structurally symmetric pattern. For
 * the folded shifts z_l (Im z_l > 0) of Eq. polerho, (H - conj(z) S)^{-1} =
 * ((H - z S)^{-1})^H, so the pole sum becomes
 *   Gamma = sum_l (w_l G_l - conj(w_l) G_l^H) / (2i),  G_l = (H - z_l S)^{-1},
 * a complex Hermitian matrix on the pattern (for real H and S it reduces to
 * Im sum_l w_l G_l of pexsi_dm). A = H - z S is only structurally symmetric,
 * so the fronts hold an unpivoted (across panels) L D U factorisation and
 * selected inversion runs the two-sided Takahashi recursion Y[S,P] =
 * -Y[S,S] L[S,P], Y[P,S] = -U[P,S] Y[S,S], Y[P,P] = D^-1 - U[P,S] Y[S,P]
 * (Sec. II.B steps 3-4 with U in place of L^T). These calls run the FP64
 * kernels whatever the plan's split_slices.
 * Layout: H, S, DM, EDM, FDM and ainv hold nnz complex values as interleaved
 * (re, im) doubles (2 nnz doubles) in the plan's CSC order; H[(r,c)] must be
 * conj(H[(c,r)]) (likewise S), S positive definite. S == NULL means S = I.
 * The traces in info are Tr[X S] = sum_e X_e conj(S_e) (real for Hermitian
 * X and S). Ownership, status chains and errors as pexsi_dm /
 * pexsi_dm_device; the first Hermitian call on a plan builds its maps and
 * staging (4 x 8 nnz + 6 x 16 nnz bytes of device memory, kept with the plan). */
int pexsi_dm_hermitian(pexsi_plan* plan, const double* H, const double* S, double mu, double beta,
                       int32_t n_poles, double delta_e, double* dm, double* edm, double* fdm,
                       pexsi_dm_info* info);
/* Device form over the pole subrange [pole_begin, pole_end) (device buffers of
 * 2 nnz doubles each, enqueued on `stream`; accumulate and info as
 * pexsi_dm_device). */
int pexsi_dm_hermitian_device(pexsi_plan* plan, const double* dH, const double* dS, double mu,
                              double beta, int32_t n_poles, double delta_e, int32_t pole_begin,
                              int32_t pole_end, int32_t accumulate, double* d_dm, double* d_edm,
                              double* d_fdm, void* stream, pexsi_dm_info* info);
/* Selected elements G[r, c] of (H - z S)^{-1} at every CSC entry (r, c), for
 * one complex shift z with Im z != 0 (host buffers, ainv: 2 nnz doubles). */
int pexsi_selinv_hermitian(pexsi_plan* plan, const double* H, const double* S, double z_re, double z_im,
                           double* ainv);
/* Inertia counts of the Hermitian pencil (Sec. II.C): counts[m] = number of
 * eigenvalues of (H, S) below shifts[m], from the Hermitian Bunch-Kaufman
 * count of each diagonal block D of the L D L^H fronts of H - shifts[m] S
 * (Sylvester's law with Haynsworth's inertia additivity). */
int pexsi_inertia_hermitian(pexsi_plan* plan, const double* H, const double* S, const double* shifts,
                            int32_t n_shifts, int64_t* counts);

/* ------------------------------------------------------------ groups of systems
 * Batching across systems (poles and systems are independent, Sec. II.B; the
 * elimination-tree concurrency of Eq. parent): the fronts of several
 * systems of different sizes are concatenated into one pool and their
 * elimination trees into one forest, so that each launch of the level
 * schedule -- block inverses, panel solves, Schur updates, Takahashi steps,
 * persistent split-precision GEMMs -- covers the fronts of every system at
 * that height of its tree, for all poles of a wave. Assembly and the pole
 * sum run per system (its own H, S, mu, beta, Delta E). A system's result is
 * the one its own plan gives with the same wave size and options.
 *
 * pexsi_group_create: plans[q] (n_plans of them) supply the symbolic
 * structure of system q (host-only plans, device = -1, suffice; the group
 * copies what it needs and the plans may be destroyed afterwards); all must
 * share opts->panel. opts: device, split_slices, max_batch (the most poles
 * per wave), hbm_budget, wait_ns of the group. Errors: INVALID_ARG (no
 * plans, NULL plan, panel mismatch, host-only device), NOMEM (one pole of
 * all systems does not fit the budget), CUDA. */
typedef struct pexsi_group pexsi_group;

/* Schedule of a group: poles per wave, and the panels per block of the
 * split-precision Schur update (one K = 64 * oz_block update per block). */
typedef struct pexsi_schedule {
  int32_t wave;        /* poles of every system per wave, 1..batch capacity   */
  int32_t oz_block;    /* 1, 2, 3 or 4 (split_slices > 0; ignored otherwise)  */
  double ms_per_pole;  /* the tuner's measurement (0 when set by hand)         */
  int32_t from_cache;  /* 1: the tuner took it from the cache file             */
  int32_t candidates;  /* schedules the tuner timed                           */
} pexsi_schedule;

int pexsi_group_create(const pexsi_plan* const* plans, int32_t n_plans, const pexsi_opts* opts,
                       pexsi_group** out);
int pexsi_group_destroy(pexsi_group* group);
/* Statistics of the merged plan (sums over the systems; batch = capacity). */
int pexsi_group_get_stats(const pexsi_group* group, pexsi_plan_stats* stats);
int pexsi_group_get_schedule(const pexsi_group* group, pexsi_schedule* out);
/* wave = 0 means the batch capacity. Errors: INVALID_ARG (out of range). */
int pexsi_group_set_schedule(pexsi_group* group, const pexsi_schedule* schedule);
/* DM / EDM / FDM of every system over the pole subrange [pole_begin,
 * pole_end) of its n_poles-pole table (the same P for all systems). dH[q],
 * dS[q] (NULL or dS == NULL: S = I), d_dm[q], d_edm[q], d_fdm[q] (any may be
 * NULL): device arrays of system q's nnz; mu, beta, delta_e: arrays of
 * n_plans. info: NULL (return after enqueueing on `stream`) or n_plans
 * reports (synchronises; traces per system; breakdown_front is the front
 * index within its system). Status chains and errors as pexsi_dm_device. */
int pexsi_group_dm_device(pexsi_group* group, const double* const* dH, const double* const* dS,
                          const double* mu, const double* beta, int32_t n_poles, const double* delta_e,
                          int32_t pole_begin, int32_t pole_end, int32_t accumulate, double* const* d_dm,
                          double* const* d_edm, double* const* d_fdm, void* stream, pexsi_dm_info* info);
/* Host-buffer form over all n_poles poles (synchronous; S may be NULL). */
int pexsi_group_dm(pexsi_group* group, const double* const* H, const double* const* S, const double* mu,
                   const double* beta, int32_t n_poles, const double* delta_e, double* const* dm,
                   double* const* edm, double* const* fdm, pexsi_dm_info* info);
/* The group's own schedule tuner: times each candidate schedule (wave = the
 * batch capacity, half, a quarter; oz_block = 4, 2, 1 on the split path) on
 * the device with CUDA events, on poles [0, wave) of the given device inputs
 * (as pexsi_group_dm_device), keeps the fastest per pole, and appends it to
 * the text file cache_path (NULL = no cache) under a fingerprint of the
 * device, the precision, the batch capacity and the systems' structure. When
 * the file already holds the fingerprint, that schedule is applied and
 * nothing is timed, unless force != 0. out (may be NULL) gets the schedule.
 * The group's output buffers are overwritten. Errors as
 * pexsi_group_dm_device. */
int pexsi_group_tune(pexsi_group* group, const double* const* dH, const double* const* dS, const double* mu,
                     const double* beta, int32_t n_poles, const double* delta_e, const char* cache_path,
                     int32_t force, pexsi_schedule* out);
const char* pexsi_group_last_error_detail(const pexsi_group* group);

/* ------------------------------------------------------------ chemical potential
 * Sec. II.C: find mu with N_beta(mu) = Tr[DM S] = N_e (Eq. Nmu).
 * 1. Inertia counting: N_inf(eps) = 2 x (# eigenvalues of (H,S) below eps) at
 *    n_shifts points across [mu_lo, mu_hi]; N_beta is the linear interpolation
 *    of those counts smoothed by -f'(eps - mu) (Eq. finiteelectronnumber). Two
 *    roots N_beta(eps_l) = N_e - delta_n and N_beta(eps_h) = N_e + delta_n give
 *    mu = (eps_l + eps_h)/2 (the gap rule) and a narrower bracket (the samples
 *    enclosing the two roots, widened by 16/beta for the Fermi tail); this
 *    repeats up to max_inertia times. A bracket that does not contain the
 *    target count is widened by its own width (at most 8 times).
 * 2. Newton: N(mu) = Tr[DM S] and N'(mu) = Tr[Gamma^d S] from one P-pole
 *    evaluation each (Gamma^d shares the poles), mu <- mu - (N - N_e)/N',
 *    bisection inside the bracket when the step leaves it, until
 *    |N - N_e| <= tol_ne or max_newton evaluations.
 * delta_e must cover the spectrum around every mu the search visits. dm,
 * edm, fdm (host, nnz each, may be NULL) receive the matrices of the last
 * evaluation. Errors as pexsi_dm; PEXSI_ERR_INVALID_ARG also when the target
 * count cannot be bracketed. */
typedef struct pexsi_mu_opts {
  double mu_lo, mu_hi;   /* initial bracket                                     */
  double n_electrons;    /* target N_e (both spins)                             */
  double tol_ne;         /* |Tr[DM S] - N_e| tolerance (default 1e-6)            */
  double delta_n;        /* gap-rule offset delta N (default 0.1)               */
  int32_t n_shifts;      /* inertia shifts per counting cycle (default 16)      */
  int32_t max_inertia;   /* counting cycles (default 3; 0 = Newton only)        */
  int32_t max_newton;    /* P-pole evaluations (default 16)                     */
  int32_t reserved0;
} pexsi_mu_opts;

typedef struct pexsi_mu_info {
  double mu;             /* final chemical potential                           */
  double n_e;            /* Tr[DM S] at mu                                      */
  double dn_dmu;         /* Tr[Gamma^d S] at mu                                 */
  double mu_inertia;     /* estimate after the inertia-counting cycles          */
  double bracket_lo, bracket_hi;
  int32_t inertia_cycles, newton_iters, converged, reserved0;
} pexsi_mu_info;

int pexsi_mu_opts_default(pexsi_mu_opts* opts);
int pexsi_mu_solve(pexsi_plan* plan, const double* H, const double* S, double beta, int32_t n_poles,
                   double delta_e, const pexsi_mu_opts* opts, double* dm, double* edm, double* fdm,
                   pexsi_mu_info* info);

/* ------------------------------------------------------------ DOS and LDOS
 * Sec. II.D. pexsi_dos samples the cumulative density of states
 * C(eps_k) = N_inf(eps_k) = 2 x #{eigenvalues of (H,S) < eps_k} (Eq. cdos; the
 * factor 2 is spin, Eq. DOS) at n_points energies evenly spaced on
 * [e_lo, e_hi] by inertia counting, and the DOS g(eps_k) as the derivative of
 * the linear interpolation of C (central differences inside, one-sided at
 * the ends). eps, cdos, dos: host arrays of n_points (n_points >= 2).
 * pexsi_ldos writes the selected elements of the LDOS matrix
 * (2/pi) Im [H - (eps + i eta) S]^{-1} on the pattern (Eq. LDOSGreen; its
 * contraction with the basis functions, g(x, eps), is left to the caller).
 * ldos: host array of nnz. eta > 0. Errors as pexsi_inertia / pexsi_selinv. */
int pexsi_dos(pexsi_plan* plan, const double* H, const double* S, double e_lo, double e_hi, int32_t n_points,
              double* eps, double* cdos, double* dos);
int pexsi_ldos(pexsi_plan* plan, const double* H, const double* S, double eps, double eta, double* ldos);

/* ------------------------------------------------------------ request server
 * A continuous-batching request loop for DM and inertia solves of systems of
 * different sizes (the serving pattern around Sec. II.C's inertia counting and
 * Sec. II.A's pole expansion). The server owns `slots` worker threads, each
 * with its own CUDA stream. Requests queue in arrival order; when a slot is
 * free, the first one whose device footprint (fronts of `batch` poles of its
 * plan plus staging) fits the HBM budget still unused is admitted (a request
 * passed over 8 times by later, smaller ones holds back everything behind it
 * until it fits, so none starves); its
 * workspace is taken from the stream-ordered allocator, and its kernels run
 * concurrently with those of the other admitted requests. Plans (symbolic
 * structure and device maps) stay resident across requests; several requests
 * may share one plan. Per request: the inertia counts at its shifts first,
 * then the P-pole DM/EDM/FDM, copied into the caller's buffers. Results are
 * the same as the plan calls give alone (the kernels are deterministic). */
typedef struct pexsi_server pexsi_server;

typedef struct pexsi_server_opts {
  int32_t device;      /* CUDA device (default 0)                                 */
  int32_t slots;       /* concurrently admitted requests (default 4)              */
  int32_t batch;       /* poles per device batch of one request (default 8)       */
  int32_t reserved0;
  int64_t hbm_budget;  /* bytes all admitted workspaces may use, 0 = 60% of free  */
} pexsi_server_opts;

/* One request. H, S and shifts are copied at submit; the plan and the output
 * buffers must stay valid until the request completes or is cancelled. */
typedef struct pexsi_request {
  const pexsi_plan* plan;   /* built by pexsi_setup on the server's device        */
  const double* H;          /* nnz values (host)                                  */
  const double* S;          /* nnz values (host), NULL = identity                 */
  double mu, beta, delta_e; /* pole expansion parameters (Eq. polerho)            */
  int32_t n_poles;          /* P (even); 0 = inertia only                         */
  int32_t n_shifts;         /* number of inertia shifts, may be 0                 */
  const double* shifts;     /* n_shifts real shifts (host)                        */
  double* dm;               /* outputs, nnz each (host), any may be NULL          */
  double* edm;
  double* fdm;
  int64_t* counts;          /* n_shifts inertia counts (host)                     */
} pexsi_request;

typedef struct pexsi_result {
  int32_t status;           /* PEXSI_OK or a PEXSI_ERR_* code                     */
  int32_t breakdown_front;  /* -1 if none                                         */
  double trace_dm_s, trace_edm_s, trace_fdm_s;
  double queue_ms;          /* submit -> admission                                */
  double run_ms;            /* admission -> outputs in the caller's buffers       */
  double latency_ms;        /* submit -> outputs ready                            */
  int64_t footprint_bytes;  /* device bytes the request was admitted with         */
  int32_t batch;            /* poles per device batch used                        */
  int32_t max_concurrent;   /* requests running on the device at its admission    */
} pexsi_result;

typedef struct pexsi_server_stats {
  int64_t submitted, completed, cancelled, failed;
  int64_t queued, running;
  int64_t bytes_in_use, peak_bytes, budget;
  int32_t peak_concurrent, reserved0;
} pexsi_server_stats;

int pexsi_server_opts_default(pexsi_server_opts* opts);
/* Errors: INVALID_ARG, CUDA, NOMEM. */
int pexsi_server_create(const pexsi_server_opts* opts, pexsi_server** out);
/* Queues a request; *ticket identifies it. Errors: INVALID_ARG (bad request,
 * plan on another device or host-only), NOMEM (a single pole of this plan can
 * never fit the budget). */
int pexsi_server_submit(pexsi_server* server, const pexsi_request* req, int64_t* ticket);
/* PEXSI_OK and *result when finished (also for failed or cancelled requests,
 * see result->status), PEXSI_PENDING otherwise, INVALID_ARG for an unknown
 * ticket. A finished ticket stays readable until pexsi_server_release. */
int pexsi_server_poll(pexsi_server* server, int64_t ticket, pexsi_result* result);
/* Blocks until the request finishes; returns as pexsi_server_poll. */
int pexsi_server_wait(pexsi_server* server, int64_t ticket, pexsi_result* result);
/* A queued request is removed at once; a running one stops after its current
 * device batch. Its status becomes PEXSI_ERR_CANCELLED. */
int pexsi_server_cancel(pexsi_server* server, int64_t ticket);
/* Forget a finished ticket. */
int pexsi_server_release(pexsi_server* server, int64_t ticket);
int pexsi_server_get_stats(pexsi_server* server, pexsi_server_stats* stats);
/* Cancels queued requests, waits for running ones, joins the workers. */
int pexsi_server_destroy(pexsi_server* server);

/* Allocation-free Tr[X S] for device-resident DM / EDM / FDM (no counterpart
 * in the paper; the traces themselves are Eq. Nmu and its energy analogues).
 * For callers that cannot allocate device memory when they need the traces --
 * for example while capturing a stream into a CUDA graph, inside a runtime
 * that owns a fixed memory arena, or in a serving loop that must not touch
 * the allocator -- this call allocates nothing: its scratch (the block
 * partial sums) is a file-scope device array of 3 x 1024 doubles (24 KiB)
 * that every GPU which loads the library holds until the process exits.
 *   d_dm, d_edm, d_fdm : device arrays of nnz doubles, any may be NULL (its
 *                        trace is then written as 0)
 *   d_S                : device array of nnz doubles (the overlap on the same
 *                        pattern; an identity S gives the plain trace)
 *   nnz                : 0 <= nnz <= 2^30 (1024 blocks x 2^20 entries);
 *                        larger sizes return PEXSI_ERR_INVALID_ARG
 *   d_out3             : device array of 3 doubles, receives
 *                        (Tr[DM S], Tr[EDM S], Tr[FDM S])
 *   stream             : cudaStream_t (void*), NULL = legacy default stream
 * Runs on the current device and returns after enqueueing. The first call on
 * a device looks up the scratch array's device address (with that device
 * current) and caches it; make that first call before any stream capture.
 * Every call shares the one scratch array per device and overwrites it, so
 * calls that overlap on the GPU (concurrent streams) race; serialise them.
 * Errors: INVALID_ARG (NULL d_S / d_out3, nnz out of range), CUDA. */
int pexsi_trace_noalloc(const double* d_dm, const double* d_edm, const double* d_fdm,
                        const double* d_S, int64_t nnz, double* d_out3, void* stream);

/* Per-kernel-class timing (instrumentation, not part of the method). When
 * enabled, every kernel launch of the plan is bracketed by CUDA events on the
 * stream it runs on; pexsi_profile_read accumulates the elapsed times after
 * the work has completed. Classes (index: name):
 *   0 assemble, 1 extend_add, 2 diag_inv, 3 panel_solve, 4 schur_update,
 *   5 gather, 6 selinv_offdiag, 7 selinv_diag_partial, 8 selinv_diag_reduce,
 *   9 pole_sum, 10 trace, 11 split_slice (the bf16 slicing kernels of the
 *   split-precision path; its GEMMs stay in classes 4 and 6)
 * flops / bytes are the algorithmic counts of the launches (complex
 * multiply-add = 8 flops, real = 2; bytes = one read of each input element and
 * one write of each output element). tensor_flops: the bf16 tensor-core flops
 * the split-precision GEMMs execute (2 per multiply-add of every slice
 * product), 0 elsewhere. */
typedef struct pexsi_kernel_profile {
  char name[24];
  int64_t launches;
  double ms;
  double flops;
  double bytes;
  double tensor_flops;
} pexsi_kernel_profile;

#define PEXSI_PROFILE_CLASSES 12

int pexsi_profile_enable(pexsi_plan* plan, int32_t on);
/* Synchronises the plan's pending work, then writes PEXSI_PROFILE_CLASSES
 * entries (totals since the last reset) into out. */
int pexsi_profile_read(pexsi_plan* plan, pexsi_kernel_profile* out);
int pexsi_profile_reset(pexsi_plan* plan);

const char* pexsi_strerror(int code);
const char* pexsi_last_error_detail(const pexsi_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* PEXSI_GB300_H */
