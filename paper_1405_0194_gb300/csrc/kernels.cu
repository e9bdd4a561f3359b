// CUDA kernels of the multifrontal LDL^T factorisation and selected inversion
// (Sec. II.B, steps 3-4) and of the pole sum (Eq. gammapole, Eq. gammaF).
//
// Storage: every front K of every batch member is an m_K x m_K column-major
// block in a pool (one pool per batch member, `pool` elements apart).
//   factor pool F: lower triangle = the front; after the panel loop its first
//     s_K columns hold L (unit lower, diagonal blocks overwritten by D^{-1} of
//     each panel) and its trailing r_K x r_K block the Schur complement that
//     the parent assembles. The upper triangle holds W^T = (L D)^T of the
//     current panel (the unscaled panel the Schur update needs).
//   inverse pool Y: the full (both triangles) selected inverse restricted to
//     the front's rows and columns, Ainv(K u C_K, K u C_K).
//
// Panel algorithm for front K (panel of width bb at p0, rows below q0 = p0+bb):
//   D = F[P,P];  F[P,P] <- D^{-1}                      (in-block pivoting)
//   W = F[S,P];  F[P,S] <- W^T;  F[S,P] <- L = W D^{-1}
//   F[S,S] -= L W^T                                   (lower triangle)
// Selected inversion for K, panels from last to first (Takahashi recursion,
// derived from A^{-1} = L^{-T} D^{-1} L^{-1}):
//   Y[C,C]  <- gathered from the parent's Y through the relative indices
//   Y[S,P]  = -Y[S,S] L[S,P];   Y[P,S] = Y[S,P]^T
//   Y[P,P]  = D^{-1} - L[S,P]^T Y[S,P]
#include <cfloat>
#include <climits>

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace pexsi {
namespace {

// ------------------------------------------------------------ arithmetic
__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double one_of(double) { return 1.0; }
__device__ __forceinline__ double2 one_of(double2) { return make_double2(1.0, 0.0); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double2 fmac(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double mulv(double a, double b) { return a * b; }
__device__ __forceinline__ double2 mulv(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double subv(double a, double b) { return a - b; }
// c - a b as fused multiply-adds: 1 for real, 4 for complex (instead of 6
// separate multiplies and adds); FP64 issue bounds the block inversion.
__device__ __forceinline__ double fmsv(double c, double a, double b) { return fma(-a, b, c); }
__device__ __forceinline__ double2 fmsv(double2 c, double2 a, double2 b) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 subv(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double addv(double a, double b) { return a + b; }
__device__ __forceinline__ double2 addv(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double negv(double a) { return -a; }
__device__ __forceinline__ double2 negv(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ double scalev(double a, double s) { return a * s; }
__device__ __forceinline__ double2 scalev(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ double absv(double2 a) { return hypot(a.x, a.y); }
// Magnitudes for partial pivoting in the block inverses: |Re| + |Im| (the
// norm of LAPACK's complex i?amax). The search compares FP32 copies (the
// FP64 pipe of an SM does 2 operations per clock, and a search is on the
// critical path of every pivot step); the chosen pivot's magnitude for the
// pivot ratio is taken in FP64. Entries below the FP32 range (1e-45) compare
// as zero: in a column whose entries all lie below it the search keeps the
// diagonal entry, unpivoted (far outside the scale of H - zS here; a zero or
// relatively tiny pivot still reports a breakdown through the pivot ratio).
__device__ __forceinline__ float pivmag(double a) { return fabsf(__double2float_rn(a)); }
__device__ __forceinline__ float pivmag(double2 a) {
  return fabsf(__double2float_rn(a.x)) + fabsf(__double2float_rn(a.y));
}
__device__ __forceinline__ double mag1(double a) { return fabs(a); }
__device__ __forceinline__ double mag1(double2 a) { return fabs(a.x) + fabs(a.y); }
// Reciprocal of a pivot: 1 / a by the correctly rounded reciprocal; for
// complex a = x + iy, (x - iy) / (x^2 + y^2) with x and y first scaled by a
// power of two (exact) that puts max(|x|, |y|) in [1, 2), so that the sum of
// squares neither overflows nor underflows; one reciprocal instead of the
// three divisions of Smith's method.
__device__ __forceinline__ double recip_piv(double a) { return __drcp_rn(a); }
__device__ __forceinline__ double2 recip_piv(double2 a) {
  const double m = fmax(fabs(a.x), fabs(a.y));
  const int e = min(((__double2hiint(m) >> 20) & 0x7FF) - 1023, 1022);  // exponent of m (subnormal: -1023)
  const double sc = __hiloint2double((1023 - e) << 20, 0);             // 2^-e
  const double x = a.x * sc, y = a.y * sc;
  const double r = __drcp_rn(fma(x, x, y * y));
  return make_double2(x * r * sc, -(y * r) * sc);
}
__device__ __forceinline__ bool finitev(double a) { return isfinite(a); }
__device__ __forceinline__ bool finitev(double2 a) { return isfinite(a.x) && isfinite(a.y); }

template <typename T> __device__ __forceinline__ T make_shift(double h, double s, const BatchShifts& sh, int b);
template <> __device__ __forceinline__ double make_shift<double>(double h, double s, const BatchShifts& sh, int b) {
  return fma(-sh.re[b], s, h);
}
template <> __device__ __forceinline__ double2 make_shift<double2>(double h, double s, const BatchShifts& sh, int b) {
  return make_double2(fma(-sh.re[b], s, h), -sh.im[b] * s);
}

// lower-triangle tile index t -> (I, J), I >= J
// Owner of tile t in a flat tile list: the largest item f with pref[f] <= t
// (pref[0] = 0, pref[n] = the total; items without tiles repeat a value).
__device__ __forceinline__ int tile_owner(const int32_t* __restrict__ pref, int n, int t) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pref[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void tri_tile(int t, int& I, int& J) {
  int i = int((sqrt(8.0 * double(t) + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// K splits of the FP64 Takahashi step of a front with m_p trailing rows:
// at least 384 of K per split, at most kMaxKsplit splits.
__host__ __device__ __forceinline__ int ksplit_of(int mp) {
  const int k = mp / 384;
  return k < 1 ? 1 : (k > kMaxKsplit ? kMaxKsplit : k);
}

// ------------------------------------------------------------ GEMM tile
// acc[i][j] += sum_k A(r, k) B(k, c) for the 64 x 64 output tile, r = tx + 16 i,
// c = ty + 16 j (tx = tid & 15, ty = tid >> 4, 256 threads).
// A(r, k) is A[r + lda k] (AT = false) or A[k + lda r] (AT = true);
// B(k, c) is B[k + ldb c]. Rows >= Mv, columns >= Nv and k >= K read as 0.
constexpr int kKc = 16;      // k-chunk staged per step
constexpr int kLd = 65;      // padded smem row stride (elements)

template <typename T, bool AT>
__device__ __forceinline__ void gemm_tile(T (&acc)[4][4], const T* __restrict__ A, int64_t lda,
                                          const T* __restrict__ B, int64_t ldb, int Mv, int Nv, int K, T* As,
                                          T* Bs) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const T z = zero_of(T());
  for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, r, k;
      if (!AT) { r = idx & 63; k = idx >> 6; }
      else { k = idx & 15; r = idx >> 4; }
      T v = z;
      if (r < Mv && k0 + k < K) v = AT ? A[(k0 + k) + lda * r] : A[r + lda * (k0 + k)];
      As[k * kLd + r] = v;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, k = idx & 15, c = idx >> 4;
      T v = z;
      if (c < Nv && k0 + k < K) v = B[(k0 + k) + ldb * c];
      Bs[k * kLd + c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kKc; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k * kLd + tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k * kLd + ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmac(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// Complex tile by the 3-multiplication (Gauss) form: with T1 = sum ar br,
// T2 = sum ai bi, T3 = sum (ar + ai)(br + bi), the product is T1 - T2 +
// i (T3 - T1 - T2). Three real multiply-adds per complex multiply-add instead
// of four; the operand sums are formed once per staged element. Shared memory
// (dynamic, kSmem3m bytes): six 16 x 65 double planes.
constexpr int kPlane = kKc * kLd;
constexpr size_t kSmem3m = 6 * kPlane * sizeof(double);

template <bool AT>
__device__ __forceinline__ void gemm_tile_3m(double2 (&acc)[4][4], const double2* __restrict__ A, int64_t lda,
                                             const double2* __restrict__ B, int64_t ldb, int Mv, int Nv, int K,
                                             double* sm) {
  double* Ar = sm;
  double* Ai = sm + kPlane;
  double* As = sm + 2 * kPlane;
  double* Br = sm + 3 * kPlane;
  double* Bi = sm + 4 * kPlane;
  double* Bs = sm + 5 * kPlane;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;
  // The global loads of the next 16-deep chunk are issued into registers
  // before the current chunk's multiply-adds, so that their latency hides
  // behind them (one CTA per SM leaves no other CTA to cover it).
  double2 va[4], vb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, r, k;
      if (!AT) { r = idx & 63; k = idx >> 6; }
      else { k = idx & 15; r = idx >> 4; }
      va[q] = make_double2(0.0, 0.0);
      if (r < Mv && k0 + k < K) va[q] = AT ? A[(k0 + k) + lda * r] : A[r + lda * (k0 + k)];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, k = idx & 15, c = idx >> 4;
      vb[q] = make_double2(0.0, 0.0);
      if (c < Nv && k0 + k < K) vb[q] = B[(k0 + k) + ldb * c];
    }
  };
  if (K > 0) load(0);
  for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, r, k;
      if (!AT) { r = idx & 63; k = idx >> 6; }
      else { k = idx & 15; r = idx >> 4; }
      Ar[k * kLd + r] = va[q].x;
      Ai[k * kLd + r] = va[q].y;
      As[k * kLd + r] = va[q].x + va[q].y;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q, k = idx & 15, c = idx >> 4;
      Br[k * kLd + c] = vb[q].x;
      Bi[k * kLd + c] = vb[q].y;
      Bs[k * kLd + c] = vb[q].x + vb[q].y;
    }
    __syncthreads();
    if (k0 + kKc < K) load(k0 + kKc);
#pragma unroll 2
    for (int k = 0; k < kKc; ++k) {
      double ar[4], ai[4], as[4], br[4], bi[4], bs[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = Ar[k * kLd + tx + 16 * i];
        ai[i] = Ai[k * kLd + tx + 16 * i];
        as[i] = As[k * kLd + tx + 16 * i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        br[j] = Br[k * kLd + ty + 16 * j];
        bi[j] = Bi[k * kLd + ty + 16 * j];
        bs[j] = Bs[k * kLd + ty + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          t1[i][j] = fma(ar[i], br[j], t1[i][j]);
          t2[i][j] = fma(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fma(as[i], bs[j], t3[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      acc[i][j] = make_double2(t1[i][j] - t2[i][j], (t3[i][j] - t1[i][j]) - t2[i][j]);
}

// Dispatch: complex tiles take the 3M form, real tiles the plain one.
template <typename T, bool AT>
__device__ __forceinline__ void gemm_any(T (&acc)[4][4], const T* A, int64_t lda, const T* B, int64_t ldb, int Mv,
                                         int Nv, int K, double* sm);
template <>
__device__ __forceinline__ void gemm_any<double, false>(double (&acc)[4][4], const double* A, int64_t lda,
                                                        const double* B, int64_t ldb, int Mv, int Nv, int K,
                                                        double* sm) {
  gemm_tile<double, false>(acc, A, lda, B, ldb, Mv, Nv, K, sm, sm + kPlane);
}
template <>
__device__ __forceinline__ void gemm_any<double2, false>(double2 (&acc)[4][4], const double2* A, int64_t lda,
                                                         const double2* B, int64_t ldb, int Mv, int Nv, int K,
                                                         double* sm) {
  gemm_tile_3m<false>(acc, A, lda, B, ldb, Mv, Nv, K, sm);
}
template <>
__device__ __forceinline__ void gemm_any<double2, true>(double2 (&acc)[4][4], const double2* A, int64_t lda,
                                                        const double2* B, int64_t ldb, int Mv, int Nv, int K,
                                                        double* sm) {
  gemm_tile_3m<true>(acc, A, lda, B, ldb, Mv, Nv, K, sm);
}

template <typename T>
__device__ __forceinline__ void zero_acc(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero_of(T());
}

// ------------------------------------------------------------ assembly
template <typename T>
__global__ void k_assemble(T* __restrict__ F, const double* __restrict__ H, const double* __restrict__ S,
                           const int64_t* __restrict__ src, const int64_t* __restrict__ pos, int64_t nlow,
                           int64_t pool, BatchShifts sh) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < nlow; t += int64_t(gridDim.x) * blockDim.x) {
    int64_t e = src[t], p = pos[t];
    double h = H[e], s = S[e];
    for (int b = 0; b < sh.nb; ++b) F[b * pool + p] = make_shift<T>(h, s, sh, b);
  }
}

// U_c (trailing r x r block of child c: its lower triangle, or with FULL the
// whole square of an LDU front) added into the parent front.
template <typename T, bool FULL = false>
__global__ void k_extend_add(T* __restrict__ F, DevFronts fr, const int32_t* __restrict__ children, int nchild,
                             const int32_t* __restrict__ pref) {
  // one block per 32x32 tile (lower-triangle tiles unless FULL) of some child's update block
  const int ci = tile_owner(pref, nchild, int(blockIdx.x));
  const int c = children[ci];
  const int64_t base = int64_t(blockIdx.z) * fr.pool;
  const int s = fr.s[c], m = fr.m[c], r = m - s;
  const int P = fr.parent[c];
  const int mP = fr.m[P];
  int I, J;
  if (FULL) {
    const int Tn = (r + 31) / 32, t = int(blockIdx.x) - pref[ci];
    I = t % Tn;
    J = t / Tn;
  } else {
    tri_tile(int(blockIdx.x) - pref[ci], I, J);
  }
  const T* Fc = F + base + fr.off[c];
  T* Fp = F + base + fr.off[P];
  const int32_t* rel = fr.rel + fr.rptr[c];
  const int i = I * 32 + threadIdx.x;
  if (i >= r) return;
  const int64_t ri = rel[i];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int j = J * 32 + threadIdx.y + 8 * q;
    if (j < r && (FULL || j <= i)) {
      T u = Fc[(s + i) + int64_t(m) * (s + j)];
      T* d = Fp + ri + int64_t(mP) * rel[j];
      *d = addv(*d, u);
    }
  }
}

// ------------------------------------------------------------ diagonal blocks
// Inverse of the (complex-)symmetric panel block D by Gauss-Jordan with
// partial (row) pivoting, written back as the full block; for real symmetric
// D (inertia) also the number of negative eigenvalues, from a Bunch-Kaufman
// symmetric-pivoted LDL^T of D (Sylvester's law, Sec. II.C).
template <typename T>
__device__ void bk_count(T* Bm, int n, int ld, int* out_neg, bool* singular);

__device__ __forceinline__ double2 conjv(double2 a) { return make_double2(a.x, -a.y); }

// Complex Hermitian D (a real shift of Hermitian H and S): the same
// Bunch-Kaufman pivoting on moduli, D = L E L^H with Hermitian 1x1 / 2x2
// blocks E; a 1x1 pivot d (real) is negative when d < 0, a 2x2 pivot
// [a conj(b); b c] (a, c real) holds one negative eigenvalue when its
// determinant a c - |b|^2 < 0 and two when it is positive with a + c < 0.
template <>
__device__ void bk_count<double2>(double2* Bm, int n, int ld, int* out_neg, bool* singular) {
  __shared__ int s_piv[3];
  __shared__ int s_neg;
  __shared__ double s_div;
  __shared__ double2 s_u[64], s_w[64];
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  if (threadIdx.x == 0) s_neg = 0;
  __syncthreads();
  int k = 0;
  while (k < n) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double lam = 0.0;
      int r = k;
      for (int i = k + 1 + lane; i < n; i += 32) {
        const double a = absv(Bm[i * ld + k]);
        if (a > lam) { lam = a; r = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ol = __shfl_xor_sync(0xffffffffu, lam, o);
        const int orr = __shfl_xor_sync(0xffffffffu, r, o);
        if (ol > lam || (ol == lam && orr < r)) { lam = ol; r = orr; }
      }
      const double akk = fabs(Bm[k * ld + k].x);
      int kind = 1, swapr = k;
      bool sing = false;
      if (lam == 0.0 && akk == 0.0) { sing = true; kind = 1; }
      else if (akk >= alpha * lam) { kind = 1; }
      else {
        double sig = 0.0;
        for (int j = k + lane; j < n; j += 32)
          if (j != r) sig = fmax(sig, absv(Bm[r * ld + j]));
        for (int o = 16; o > 0; o >>= 1) sig = fmax(sig, __shfl_xor_sync(0xffffffffu, sig, o));
        if (akk * sig >= alpha * lam * lam) kind = 1;
        else if (fabs(Bm[r * ld + r].x) >= alpha * sig) { kind = 1; swapr = r; }
        else { kind = 2; swapr = r; }
      }
      if (lane == 0) {
        s_piv[0] = kind;
        s_piv[1] = swapr;
        if (sing) *singular = true;
      }
    }
    __syncthreads();
    const int kind = s_piv[0], sr = s_piv[1];
    const int tgt = (kind == 1) ? k : k + 1;
    if (sr != tgt) {  // symmetric swap of rows/columns tgt and sr (keeps D Hermitian)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double2 t = Bm[tgt * ld + j]; Bm[tgt * ld + j] = Bm[sr * ld + j]; Bm[sr * ld + j] = t;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double2 t = Bm[i * ld + tgt]; Bm[i * ld + tgt] = Bm[i * ld + sr]; Bm[i * ld + sr] = t;
      }
      __syncthreads();
    }
    if (kind == 1) {
      const double d = Bm[k * ld + k].x;
      if (threadIdx.x == 0) {
        if (d < 0) ++s_neg;
        if (d == 0.0) *singular = true;
      }
      if (threadIdx.x == 0) s_div = d != 0.0 ? 1.0 / d : 0.0;  // one division per pivot
      __syncthreads();
      const double inv = s_div;
      // u_j = D(k, j) / d = conj(D(j, k)) / d
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) s_u[j] = scalev(conjv(Bm[j * ld + k]), inv);
      __syncthreads();
      for (int idx = threadIdx.x; idx < (n - k - 1) * (n - k - 1); idx += blockDim.x) {
        int i = k + 1 + idx % (n - k - 1), j = k + 1 + idx / (n - k - 1);
        Bm[i * ld + j] = fmsv(Bm[i * ld + j], Bm[i * ld + k], s_u[j]);
      }
      __syncthreads();
      k += 1;
    } else {
      const double a = Bm[k * ld + k].x, c = Bm[(k + 1) * ld + (k + 1)].x;
      const double2 bq = Bm[(k + 1) * ld + k];  // E = [a conj(b); b c]
      const double det = a * c - (bq.x * bq.x + bq.y * bq.y);
      if (threadIdx.x == 0) {
        if (det < 0) s_neg += 1;
        else if (det > 0 && a + c < 0) s_neg += 2;
        if (det == 0.0) *singular = true;
      }
      if (threadIdx.x == 0) s_div = det != 0.0 ? 1.0 / det : 0.0;
      __syncthreads();
      const double id = s_div;
      const int nn = n - k - 2;
      // E^{-1} = [c -conj(b); -b a] / det applied to (x0, x1) = (D(k, j), D(k+1, j))
      for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) {
        const double2 x0 = conjv(Bm[j * ld + k]), x1 = conjv(Bm[j * ld + k + 1]);
        s_u[j] = scalev(subv(scalev(x0, c), mulv(conjv(bq), x1)), id);
        s_w[j] = scalev(subv(scalev(x1, a), mulv(bq, x0)), id);
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nn * nn; idx += blockDim.x) {
        int i = k + 2 + idx % nn, j = k + 2 + idx / nn;
        Bm[i * ld + j] = fmsv(fmsv(Bm[i * ld + j], Bm[i * ld + k], s_u[j]), Bm[i * ld + k + 1], s_w[j]);
      }
      __syncthreads();
      k += 2;
    }
  }
  if (threadIdx.x == 0) *out_neg = s_neg;
  __syncthreads();
}

template <>
__device__ void bk_count<double>(double* Bm, int n, int ld, int* out_neg, bool* singular) {
  __shared__ int s_piv[3];  // kind (1 or 2), row r, flag
  __shared__ int s_neg;
  __shared__ double s_div;
  __shared__ double s_u[64], s_w[64];  // the pivot columns times the pivot's inverse, per row j
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  if (threadIdx.x == 0) s_neg = 0;
  __syncthreads();
  int k = 0;
  while (k < n) {
    if (threadIdx.x < 32) {  // pivot choice by warp 0: same decisions as a serial scan (first maximum)
      const int lane = threadIdx.x;
      double lam = 0.0;
      int r = k;
      for (int i = k + 1 + lane; i < n; i += 32) {
        const double a = fabs(Bm[i * ld + k]);
        if (a > lam) { lam = a; r = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ol = __shfl_xor_sync(0xffffffffu, lam, o);
        const int orr = __shfl_xor_sync(0xffffffffu, r, o);
        if (ol > lam || (ol == lam && orr < r)) { lam = ol; r = orr; }
      }
      const double akk = fabs(Bm[k * ld + k]);
      int kind = 1, swapr = k;
      bool sing = false;
      if (lam == 0.0 && akk == 0.0) { sing = true; kind = 1; }
      else if (akk >= alpha * lam) { kind = 1; }
      else {
        double sig = 0.0;
        for (int j = k + lane; j < n; j += 32)
          if (j != r) sig = fmax(sig, fabs(Bm[r * ld + j]));
        for (int o = 16; o > 0; o >>= 1) sig = fmax(sig, __shfl_xor_sync(0xffffffffu, sig, o));
        if (akk * sig >= alpha * lam * lam) kind = 1;
        else if (fabs(Bm[r * ld + r]) >= alpha * sig) { kind = 1; swapr = r; }
        else { kind = 2; swapr = r; }
      }
      if (lane == 0) {
        s_piv[0] = kind;
        s_piv[1] = swapr;
        if (sing) *singular = true;
      }
    }
    __syncthreads();
    const int kind = s_piv[0], sr = s_piv[1];
    const int tgt = (kind == 1) ? k : k + 1;
    if (sr != tgt) {  // symmetric swap of rows/columns tgt and sr
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double t = Bm[tgt * ld + j]; Bm[tgt * ld + j] = Bm[sr * ld + j]; Bm[sr * ld + j] = t;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double t = Bm[i * ld + tgt]; Bm[i * ld + tgt] = Bm[i * ld + sr]; Bm[i * ld + sr] = t;
      }
      __syncthreads();
    }
    if (kind == 1) {
      double d = Bm[k * ld + k];
      if (threadIdx.x == 0) {
        if (d < 0) ++s_neg;
        if (d == 0.0) *singular = true;
      }
      if (threadIdx.x == 0) s_div = d != 0.0 ? 1.0 / d : 0.0;  // one division per pivot
      __syncthreads();
      const double inv = s_div;
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) s_u[j] = Bm[j * ld + k] * inv;
      __syncthreads();
      for (int idx = threadIdx.x; idx < (n - k - 1) * (n - k - 1); idx += blockDim.x) {
        int i = k + 1 + idx % (n - k - 1), j = k + 1 + idx / (n - k - 1);
        Bm[i * ld + j] = fma(-Bm[i * ld + k], s_u[j], Bm[i * ld + j]);
      }
      __syncthreads();
      k += 1;
    } else {
      double a = Bm[k * ld + k], b = Bm[(k + 1) * ld + k], c = Bm[(k + 1) * ld + (k + 1)];
      double det = a * c - b * b;
      if (threadIdx.x == 0) {
        if (det < 0) s_neg += 1;
        else if (det > 0 && a + c < 0) s_neg += 2;
        if (det == 0.0) *singular = true;
      }
      if (threadIdx.x == 0) s_div = det != 0.0 ? 1.0 / det : 0.0;
      __syncthreads();
      const double id = s_div;
      int nn = n - k - 2;
      // [xi0 xi1] E^{-1} [xj0; xj1], E^{-1} = [c -b; -b a] / det: the
      // factor E^{-1} [xj0; xj1] = (u_j, w_j) once per row j
      for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) {
        const double xj0 = Bm[j * ld + k], xj1 = Bm[j * ld + k + 1];
        s_u[j] = (c * xj0 - b * xj1) * id;
        s_w[j] = (-b * xj0 + a * xj1) * id;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nn * nn; idx += blockDim.x) {
        int i = k + 2 + idx % nn, j = k + 2 + idx / nn;
        Bm[i * ld + j] = fma(-Bm[i * ld + k], s_u[j], fma(-Bm[i * ld + k + 1], s_w[j], Bm[i * ld + j]));
      }
      __syncthreads();
      k += 2;
    }
  }
  if (threadIdx.x == 0) *out_neg = s_neg;
  __syncthreads();
}

// Threads of a block inversion (8 warps; 16 measured slower: the FP64 pipe
// of each SM is the bound, not the latency of its multiply-adds).
constexpr int kDiagThreads = 256;

template <typename T, bool GEN = false>
__global__ void __launch_bounds__(kDiagThreads) k_diag_inv(T* __restrict__ F, DevFronts fr, const int32_t* __restrict__ fronts, int p0, int b,
                           DevStatus st, int count_inertia) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Aug = reinterpret_cast<T*>(smem_raw);  // bb x bb, row-major, stride b+1, inverted in place
  const int f = fronts[blockIdx.x];
  const int pb = blockIdx.y;
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0);
  const int ld = b + 1;
  T* Fd = F + int64_t(pb) * fr.pool + fr.off[f] + p0 + int64_t(m) * p0;
  __shared__ double s_max;
  __shared__ int s_piv;
  __shared__ double s_pmin;
  __shared__ bool s_bad;
  __shared__ T s_fac[64];
  __shared__ T s_inv;
  __shared__ int s_perm[64];
  if (threadIdx.x == 0) { s_max = 0.0; s_pmin = DBL_MAX; s_bad = false; }
  __syncthreads();
  double lmax = 0.0;
  for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
    int i = idx % bb, j = idx / bb;
    // symmetric fronts hold the lower triangle; LDU fronts (GEN) both
    T v = (GEN || i >= j) ? Fd[i + int64_t(m) * j] : Fd[j + int64_t(m) * i];
    Aug[i * ld + j] = v;
    lmax = fmax(lmax, mag1(v));
  }
  // block max |entry| for the pivot ratio
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(&s_max), __double_as_longlong(lmax));
  __syncthreads();

  if (count_inertia && st.dsave) {
    // the block as it is before inversion, counted later (launch_bk_count_all)
    T* save = reinterpret_cast<T*>(st.dsave) + int64_t(pb) * st.dsave_stride + int64_t(st.col0[f] + p0) * b;
    for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
      const int i = idx / bb, j = idx % bb;
      save[i * b + j] = Aug[i * ld + j];
    }
  } else if (count_inertia) {
    // Bunch-Kaufman count on a copy placed after the augmented matrix
    // (real symmetric blocks, or Hermitian ones of an LDU front with a real shift)
    if constexpr (sizeof(T) == sizeof(double) || GEN) {
      T* Bm = Aug + bb * ld;
      for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
        int i = idx % bb, j = idx / bb;
        Bm[i * b + j] = Aug[i * ld + j];
      }
      __syncthreads();
      __shared__ int s_neg;
      __shared__ bool s_sing;
      if (threadIdx.x == 0) s_sing = false;
      __syncthreads();
      bk_count<T>(Bm, bb, b, &s_neg, &s_sing);
      if (threadIdx.x == 0) {
        atomicAdd(&st.neg_count[pb], s_neg);
        if (s_sing) atomicMin(st.breakdown_front, f);
      }
    }
  }

  for (int k = 0; k < bb; ++k) {
    if (threadIdx.x < 32) {
      float bestf = -1.0f;
      int bi = k;
      for (int i = k + threadIdx.x; i < bb; i += 32) {
        const float a = pivmag(Aug[i * ld + k]);
        if (a > bestf) { bestf = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, bestf, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > bestf || (ob == bestf && oi < bi)) { bestf = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        const double best = mag1(Aug[bi * ld + k]);
        s_piv = bi;
        s_pmin = fmin(s_pmin, best);
        if (!(best > 0.0) || !isfinite(best)) s_bad = true;
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (threadIdx.x == 0) s_perm[k] = pr;
    if (pr != k)
      for (int j = threadIdx.x; j < bb; j += blockDim.x) {
        T t = Aug[k * ld + j]; Aug[k * ld + j] = Aug[pr * ld + j]; Aug[pr * ld + j] = t;
      }
    __syncthreads();
    // in-place Gauss-Jordan step: column k keeps the multipliers' negatives
    // over the pivot, row k is scaled by the pivot's reciprocal (one thread
    // takes the reciprocal: the FP64 pipe of an SM does 2 multiply-adds per clock)
    if (threadIdx.x == 0) s_inv = s_bad ? zero_of(T()) : recip_piv(Aug[k * ld + k]);
    for (int i = threadIdx.x; i < bb; i += blockDim.x) s_fac[i] = Aug[i * ld + k];
    __syncthreads();
    const T inv = s_inv;
    for (int j = threadIdx.x; j < bb; j += blockDim.x) Aug[k * ld + j] = (j == k) ? inv : mulv(Aug[k * ld + j], inv);
    __syncthreads();
    for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
      const int i = idx / bb, j = idx % bb;
      if (i == k) continue;
      Aug[i * ld + j] = (j == k) ? fmsv(zero_of(T()), s_fac[i], inv) : fmsv(Aug[i * ld + j], s_fac[i], Aug[k * ld + j]);
    }
    __syncthreads();
  }
  // the row interchanges become column interchanges of the inverse, undone in reverse order
  for (int k = bb - 1; k >= 0; --k) {
    const int pr = s_perm[k];
    if (pr != k)
      for (int i = threadIdx.x; i < bb; i += blockDim.x) {
        T t = Aug[i * ld + k]; Aug[i * ld + k] = Aug[i * ld + pr]; Aug[i * ld + pr] = t;
      }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
    int i = idx % bb, j = idx / bb;
    Fd[i + int64_t(m) * j] = Aug[i * ld + j];
  }
  if (threadIdx.x == 0) {
    double ratio = s_max > 0 ? s_pmin / s_max : 0.0;
    atomicMin(st.min_pivot, (unsigned long long)__double_as_longlong(ratio));
    if (s_bad || ratio < 1e-13) atomicMin(st.breakdown_front, f);
  }
}

// The same inversion of a complex panel block, split over a cluster of
// kDiagCluster (2, 4 or 8) CTAs (one SM each): CTA r owns columns [r W, (r+1) W) of the
// bb x bb block (W = ceil(bb / kDiagCluster)) in its shared memory. At pivot
// step k the owner of column k searches it for the pivot, swaps rows k and
// pr in its columns and writes the pivot row index, the reciprocal of the
// pivot and the (swapped) column k into every CTA's shared memory
// (distributed shared memory, double-buffered by step parity); after one
// cluster barrier every CTA swaps, scales row k and updates its own columns.
// The buffer written at step k + 2 is no longer read then: every CTA has
// passed the barrier of step k + 1, after its update of step k. The final
// column interchanges are applied when the columns are written back. One
// inversion thus runs on kDiagCluster SMs' FP64 pipes instead of one.
template <typename T, bool GEN, int kDiagCluster>
__global__ void __launch_bounds__(kDiagThreads) k_diag_inv_cluster(T* __restrict__ F, DevFronts fr,
                                                                   const int32_t* __restrict__ fronts, int p0, int b,
                                                                   DevStatus st) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ T A[64][64 / kDiagCluster + 1];  // this CTA's columns (row-major in i)
  __shared__ T pub_fac[2][64];
  __shared__ T pub_inv[2];
  __shared__ T s_inv;
  __shared__ int pub_piv[2];
  __shared__ double pub_best[2];
  __shared__ double s_maxes[kDiagCluster];
  __shared__ int s_perm[64];
  __shared__ double s_lmax;
  const int f = fronts[blockIdx.x / kDiagCluster];
  const int r = int(cluster.block_rank());
  const int pb = blockIdx.y;
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;  // the same for every CTA of the cluster
  const int bb = min(b, s - p0);
  const int W = (bb + kDiagCluster - 1) / kDiagCluster;
  const int c0 = r * W, nc = max(0, min(bb, c0 + W) - c0);
  T* Fd = F + int64_t(pb) * fr.pool + fr.off[f] + p0 + int64_t(m) * p0;
  if (threadIdx.x == 0) s_lmax = 0.0;
  __syncthreads();
  double lmax = 0.0;
  for (int idx = threadIdx.x; idx < bb * nc; idx += blockDim.x) {
    const int i = idx % bb, jl = idx / bb, j = c0 + jl;
    const T v = (GEN || i >= j) ? Fd[i + int64_t(m) * j] : Fd[j + int64_t(m) * i];
    A[i][jl] = v;
    lmax = fmax(lmax, mag1(v));
  }
  if (st.dsave) {  // inertia shifts: this CTA's columns of the block before inversion, counted later
    T* save = reinterpret_cast<T*>(st.dsave) + int64_t(pb) * st.dsave_stride + int64_t(st.col0[f] + p0) * b;
    for (int idx = threadIdx.x; idx < bb * nc; idx += blockDim.x) {
      const int i = idx % bb, jl = idx / bb;
      save[i * b + c0 + jl] = A[i][jl];
    }
  }
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(&s_lmax), __double_as_longlong(lmax));
  __syncthreads();
  cluster.sync();  // every CTA of the cluster runs before any distributed shared memory access
  if (threadIdx.x == 0) *cluster.map_shared_rank(&s_maxes[r], 0) = s_lmax;  // block max, gathered in CTA 0
  bool bad = false;
  double pmin = DBL_MAX;
  for (int k = 0; k < bb; ++k) {
    const int par = k & 1, owner = k / W;
    if (r == owner) {
      const int lk = k - c0;
      if (threadIdx.x < 32) {
        float bestf = -1.0f;
        int bi = k;
        for (int i = k + threadIdx.x; i < bb; i += 32) {
          const float a = pivmag(A[i][lk]);
          if (a > bestf) { bestf = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, bestf, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > bestf || (ob == bestf && oi < bi)) { bestf = ob; bi = oi; }
        }
        if (threadIdx.x == 0) {
          pub_piv[par] = bi;
          pub_best[par] = mag1(A[bi][lk]);
        }
      }
      __syncthreads();
      const int pr = pub_piv[par];
      if (pr != k)
        for (int jl = threadIdx.x; jl < nc; jl += blockDim.x) {
          const T t = A[k][jl]; A[k][jl] = A[pr][jl]; A[pr][jl] = t;
        }
      __syncthreads();
      const double best = pub_best[par];
      const bool now_bad = bad || !(best > 0.0) || !isfinite(best);
      // one thread takes the reciprocal (the FP64 pipe of an SM does 2 multiply-adds per clock)
      if (threadIdx.x == 0) s_inv = now_bad ? zero_of(T()) : recip_piv(A[k][lk]);
      __syncthreads();
      const T inv = s_inv;
      // publish into every CTA of the cluster, all (CTA, row) pairs at once
      for (int idx = threadIdx.x; idx < kDiagCluster * bb; idx += blockDim.x) {
        const int q = idx / bb, i = idx - q * bb;
        *cluster.map_shared_rank(&pub_fac[par][i], q) = A[i][lk];
      }
      if (threadIdx.x < kDiagCluster) {
        const int q = threadIdx.x;
        *cluster.map_shared_rank(&pub_inv[par], q) = inv;
        *cluster.map_shared_rank(&pub_piv[par], q) = pr;
        *cluster.map_shared_rank(&pub_best[par], q) = best;
      }
    }
    cluster.sync();
    const int pr = pub_piv[par];
    const double best = pub_best[par];
    const T inv = pub_inv[par];
    bad = bad || !(best > 0.0) || !isfinite(best);
    pmin = fmin(pmin, best);
    if (threadIdx.x == 0) s_perm[k] = pr;
    if (r != owner && pr != k)
      for (int jl = threadIdx.x; jl < nc; jl += blockDim.x) {
        const T t = A[k][jl]; A[k][jl] = A[pr][jl]; A[pr][jl] = t;
      }
    __syncthreads();
    // row k scaled by the pivot's reciprocal; column k keeps the multipliers' negatives over the pivot
    for (int jl = threadIdx.x; jl < nc; jl += blockDim.x) A[k][jl] = (c0 + jl == k) ? inv : mulv(A[k][jl], inv);
    __syncthreads();
    const T* fac = pub_fac[par];
    for (int idx = threadIdx.x; idx < bb * nc; idx += blockDim.x) {
      const int i = idx / nc, jl = idx % nc;
      if (i == k) continue;
      A[i][jl] = (c0 + jl == k) ? fmsv(zero_of(T()), fac[i], inv) : fmsv(A[i][jl], fac[i], A[k][jl]);
    }
    __syncthreads();
  }
  // write back: the row interchanges are column interchanges of the inverse,
  // undone in reverse order, applied to each column's destination index
  for (int jl = 0; jl < nc; ++jl) {
    int pos = c0 + jl;
    for (int k = bb - 1; k >= 0; --k) {
      const int q = s_perm[k];
      if (pos == k) pos = q;
      else if (pos == q) pos = k;
    }
    for (int i = threadIdx.x; i < bb; i += blockDim.x) Fd[i + int64_t(m) * pos] = A[i][jl];
  }
  cluster.sync();  // every remote write of the cluster is done before any CTA leaves
  if (r == 0 && threadIdx.x == 0) {
    double mx = 0.0;
    for (int q = 0; q < kDiagCluster; ++q) mx = fmax(mx, s_maxes[q]);
    const double ratio = mx > 0 ? pmin / mx : 0.0;
    atomicMin(st.min_pivot, (unsigned long long)__double_as_longlong(ratio));
    if (bad || ratio < 1e-13) atomicMin(st.breakdown_front, f);
  }
}

// Deferred inertia count: one CTA per (saved panel block, batch member).
template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_bk_count_all(const int32_t* __restrict__ slots, DevFronts fr, int b,
                                                               DevStatus st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Bm = reinterpret_cast<T*>(smem_raw);  // bb x bb, row stride b
  const int f = slots[2 * blockIdx.x], p0 = slots[2 * blockIdx.x + 1];
  const int pb = blockIdx.y;
  const int bb = min(b, fr.s[f] - p0);
  const T* save = reinterpret_cast<const T*>(st.dsave) + int64_t(pb) * st.dsave_stride + int64_t(st.col0[f] + p0) * b;
  for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
    const int i = idx / bb, j = idx % bb;
    Bm[i * b + j] = save[i * b + j];
  }
  __syncthreads();
  __shared__ int s_neg;
  __shared__ bool s_sing;
  if (threadIdx.x == 0) s_sing = false;
  __syncthreads();
  bk_count<T>(Bm, bb, b, &s_neg, &s_sing);
  if (threadIdx.x == 0) {
    if (s_neg) atomicAdd(&st.neg_count[pb], s_neg);
    if (s_sing) atomicMin(st.breakdown_front, f);
  }
}

// ------------------------------------------------------------ panel solve
template <typename T, bool GEN = false>
__global__ void __launch_bounds__(256) k_panel_solve(T* __restrict__ F, DevFronts fr, const int32_t* __restrict__ fronts,
                                                     int p0, int b) {
  extern __shared__ __align__(16) double gsm[];
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int I0 = blockIdx.x * kTile;
  if (I0 >= mp) return;
  T* Fb = F + int64_t(blockIdx.z) * fr.pool + fr.off[f];
  const int Mv = min(kTile, mp - I0);
  T acc[4][4];
  zero_acc(acc);
  gemm_any<T, false>(acc, Fb + q0 + I0 + int64_t(m) * p0, m, Fb + p0 + int64_t(m) * p0, m, Mv, bb, bb, gsm);
  // W^T into the upper triangle (rows p0.., columns q0+I0..); an LDU front
  // (GEN) already holds its own row panel A[P,S] there
  if (!GEN)
    for (int idx = threadIdx.x; idx < Mv * bb; idx += blockDim.x) {
      int k = idx % bb, r = idx / bb;
      Fb[(p0 + k) + int64_t(m) * (q0 + I0 + r)] = Fb[(q0 + I0 + r) + int64_t(m) * (p0 + k)];
    }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = tx + 16 * i, c = ty + 16 * j;
      if (r < Mv && c < bb) Fb[(q0 + I0 + r) + int64_t(m) * (p0 + c)] = acc[i][j];
    }
}

// Row panel of an LDU front: U[P,S] = D^{-1} A[P,S] over 64-column tiles of
// S, in place (each CTA reads and writes its own columns only), after the
// Schur update has used A[P,S].
__global__ void __launch_bounds__(256) k_panel_upper(double2* __restrict__ F, DevFronts fr,
                                                     const int32_t* __restrict__ fronts, int p0, int b) {
  extern __shared__ __align__(16) double gsm[];
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int I0 = blockIdx.x * kTile;
  if (I0 >= mp) return;
  double2* Fb = F + int64_t(blockIdx.z) * fr.pool + fr.off[f];
  const int Nv = min(kTile, mp - I0);
  double2 acc[4][4];
  zero_acc(acc);
  gemm_any<double2, false>(acc, Fb + p0 + int64_t(m) * p0, m, Fb + p0 + int64_t(m) * (q0 + I0), m, bb, Nv, bb, gsm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = tx + 16 * i, c = ty + 16 * j;
      if (r < bb && c < Nv) Fb[(p0 + r) + int64_t(m) * (q0 + I0 + c)] = acc[i][j];
    }
}

// ------------------------------------------------------------ Schur update
// F[S,S] -= L[S,P] B[P,S] with B the stored W^T (symmetric fronts: lower
// triangle tiles) or the row panel A[P,S] of an LDU front (FULL: all tiles).
template <typename T, bool FULL = false>
__global__ void __launch_bounds__(256) k_trailing(T* __restrict__ F, DevFronts fr, const int32_t* __restrict__ fronts,
                                                  int p0, int b) {
  extern __shared__ __align__(16) double gsm[];
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int Tn = (mp + kTile - 1) / kTile;
  if (int(blockIdx.x) >= (FULL ? Tn * Tn : Tn * (Tn + 1) / 2)) return;
  int I, J;
  if (FULL) {
    I = int(blockIdx.x) % Tn;
    J = int(blockIdx.x) / Tn;
  } else {
    tri_tile(blockIdx.x, I, J);
  }
  T* Fb = F + int64_t(blockIdx.z) * fr.pool + fr.off[f];
  const int r0 = q0 + I * kTile, c0 = q0 + J * kTile;
  const int Mv = min(kTile, m - r0), Nv = min(kTile, m - c0);
  T acc[4][4];
  zero_acc(acc);
  gemm_any<T, false>(acc, Fb + r0 + int64_t(m) * p0, m, Fb + p0 + int64_t(m) * c0, m, Mv, Nv, bb, gsm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = tx + 16 * i, c = ty + 16 * j;
      if (r < Mv && c < Nv && (FULL || I != J || r >= c)) {
        T* d = Fb + (r0 + r) + int64_t(m) * (c0 + c);
        *d = subv(*d, acc[i][j]);
      }
    }
}

// ------------------------------------------------------------ selected inversion
__global__ void k_gather(double2* __restrict__ Y, DevFronts fr, const int32_t* __restrict__ fronts, int nfronts,
                         const int32_t* __restrict__ pref) {
  // one block per 32x32 tile of some front's Y[C,C] (fronts without a parent have none)
  const int fi = tile_owner(pref, nfronts, int(blockIdx.x));
  const int f = fronts[fi];
  const int P = fr.parent[f];
  const int s = fr.s[f], m = fr.m[f], r = m - s, mP = fr.m[P];
  const int Tn = (r + 31) / 32;
  const int t = int(blockIdx.x) - pref[fi];
  const int I = t % Tn, J = t / Tn;
  const int64_t base = int64_t(blockIdx.z) * fr.pool;
  double2* Yf = Y + base + fr.off[f];
  const double2* Yp = Y + base + fr.off[P];
  const int32_t* rel = fr.rel + fr.rptr[f];
  const int i = I * 32 + threadIdx.x;
  if (i >= r) return;
  const int64_t ri = rel[i];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int j = J * 32 + threadIdx.y + 8 * q;
    if (j < r) Yf[(s + i) + int64_t(m) * (s + j)] = Yp[ri + int64_t(mP) * rel[j]];
  }
}

// Y[S,P] = -Y[S,S] L[S,P] over 64-row tiles of S, and its mirror Y[P,S] =
// Y[S,P]^T. LDU fronts (GEN) have no mirror: blocks blockIdx.x >= gridDim.x
// / 2 compute Y[P,S] = -U[P,S] Y[S,S] over 64-column tiles of S instead.
//
// Split-K (complex-symmetric fronts, kpart != NULL): a front's ks = ksplit_of(m_p)
// blocks per tile (block x = tile * ks + split) take ks contiguous K ranges
// (multiples of 16) and write their 64 x bb partial products to kpart;
// k_offdiag_reduce adds the partials in split order and writes Y[S,P] and
// its mirror. The CTAs of a long-K launch are equal in size, so their last
// wave can leave most SMs idle (the FP64 pipe of each SM is the bound);
// ks times as many, ks times shorter CTAs fill the waves. ks depends on the
// front alone, so results do not depend on the batch or on the launch's
// other fronts.
template <bool GEN = false>
__global__ void __launch_bounds__(256) k_selinv_offdiag(double2* __restrict__ Y, const double2* __restrict__ F, DevFronts fr,
                                                        const int32_t* __restrict__ fronts, int p0, int b,
                                                        double2* __restrict__ kpart, const int64_t* __restrict__ part_off,
                                                        int64_t kstride) {
  extern __shared__ __align__(16) double gsm[];
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int half = GEN ? int(gridDim.x) / 2 : int(gridDim.x);
  const bool upper = GEN && int(blockIdx.x) >= half;
  const int ks = (GEN || kpart == nullptr) ? 1 : ksplit_of(mp);
  const int tile = GEN ? (upper ? int(blockIdx.x) - half : int(blockIdx.x)) : int(blockIdx.x) / ks;
  const int split = GEN ? 0 : int(blockIdx.x) % ks;
  const int I0 = tile * kTile;
  if (I0 >= mp) return;
  const int64_t base = int64_t(blockIdx.z) * fr.pool + fr.off[f];
  double2* Yb = Y + base;
  const double2* Fb = F + base;
  const int Mv = min(kTile, mp - I0);
  // this block's K range (the whole of it unless split)
  const int kc = ks > 1 ? ((mp + ks - 1) / ks + 15) / 16 * 16 : mp;
  const int k0 = min(mp, split * kc), k1 = min(mp, k0 + kc);
  double2 acc[4][4];
  zero_acc(acc);
  if (upper)  // U[P,S] (bb x mp) times the columns I0.. of Y[S,S]
    gemm_any<double2, false>(acc, Fb + p0 + int64_t(m) * q0, m, Yb + q0 + int64_t(m) * (q0 + I0), m, bb, Mv, mp, gsm);
  else
    gemm_any<double2, false>(acc, Yb + q0 + I0 + int64_t(m) * (q0 + k0), m, Fb + q0 + k0 + int64_t(m) * p0, m, Mv, bb,
                             k1 - k0, gsm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (!GEN && ks > 1) {
    const int64_t slot = part_off[f] / (int64_t(b) * b) + tile;
    double2* out = kpart + int64_t(blockIdx.z) * kstride + (slot * kMaxKsplit + split) * (int64_t(kTile) * b);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int r = tx + 16 * i, c = ty + 16 * j;
        if (r < Mv && c < bb) out[r + kTile * c] = acc[i][j];
      }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = tx + 16 * i, c = ty + 16 * j;
      if (upper) {
        if (r < bb && c < Mv) Yb[(p0 + r) + int64_t(m) * (q0 + I0 + c)] = negv(acc[i][j]);
      } else if (r < Mv && c < bb) {
        double2 v = negv(acc[i][j]);
        Yb[(q0 + I0 + r) + int64_t(m) * (p0 + c)] = v;
        if (!GEN) Yb[(p0 + c) + int64_t(m) * (q0 + I0 + r)] = v;
      }
    }
}

__global__ void __launch_bounds__(256) k_offdiag_reduce(double2* __restrict__ Y, DevFronts fr,
                                                        const int32_t* __restrict__ fronts, int p0, int b,
                                                        const double2* __restrict__ kpart,
                                                        const int64_t* __restrict__ part_off, int64_t kstride) {
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int ks = ksplit_of(mp);
  const int I0 = blockIdx.x * kTile;
  if (ks == 1 || I0 >= mp) return;
  const int Mv = min(kTile, mp - I0);
  double2* Yb = Y + int64_t(blockIdx.z) * fr.pool + fr.off[f];
  const int64_t slot = part_off[f] / (int64_t(b) * b) + blockIdx.x;
  const double2* in = kpart + int64_t(blockIdx.z) * kstride + slot * kMaxKsplit * (int64_t(kTile) * b);
  for (int idx = threadIdx.x; idx < Mv * bb; idx += blockDim.x) {
    const int r = idx % Mv, c = idx / Mv;
    double2 v = in[r + kTile * c];
    for (int j = 1; j < ks; ++j) v = addv(v, in[j * (int64_t(kTile) * b) + r + kTile * c]);
    v = negv(v);
    Yb[(q0 + I0 + r) + int64_t(m) * (p0 + c)] = v;
    Yb[(p0 + c) + int64_t(m) * (q0 + I0 + r)] = v;
  }
}

template <bool GEN = false>
__global__ void __launch_bounds__(256) k_selinv_diag_partial(const double2* __restrict__ Y, const double2* __restrict__ F,
                                                             double2* __restrict__ part, const int64_t* __restrict__ part_off,
                                                             int64_t part_stride, DevFronts fr,
                                                             const int32_t* __restrict__ fronts, int p0, int b) {
  extern __shared__ __align__(16) double gsm[];
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int I0 = blockIdx.x * kTile;
  if (I0 >= mp) return;
  const int64_t base = int64_t(blockIdx.z) * fr.pool + fr.off[f];
  const double2* Yb = Y + base;
  const double2* Fb = F + base;
  const int Kv = min(kTile, mp - I0);
  double2 acc[4][4];
  zero_acc(acc);
  // partial(c1, c2) = sum_{i in tile} L[i, p0+c1] Y[i, p0+c2], or for an LDU
  // front sum_{i in tile} U[p0+c1, i] Y[i, p0+c2]
  if (GEN)
    gemm_any<double2, false>(acc, Fb + p0 + int64_t(m) * (q0 + I0), m, Yb + q0 + I0 + int64_t(m) * p0, m, bb, bb, Kv,
                             gsm);
  else
    gemm_any<double2, true>(acc, Fb + q0 + I0 + int64_t(m) * p0, m, Yb + q0 + I0 + int64_t(m) * p0, m, bb, bb, Kv, gsm);
  double2* out = part + int64_t(blockIdx.z) * part_stride + part_off[f] + int64_t(blockIdx.x) * b * b;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = tx + 16 * i, c = ty + 16 * j;
      if (r < bb && c < bb) out[r + b * c] = acc[i][j];
    }
}

template <bool GEN = false>
__global__ void k_selinv_diag_reduce(double2* __restrict__ Y, const double2* __restrict__ F,
                                     const double2* __restrict__ part, const int64_t* __restrict__ part_off,
                                     int64_t part_stride, DevFronts fr, const int32_t* __restrict__ fronts, int p0, int b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tmp = reinterpret_cast<double2*>(smem_raw);  // bb x bb
  const int f = fronts[blockIdx.x];
  const int s = fr.s[f], m = fr.m[f];
  if (p0 >= s) return;
  const int bb = min(b, s - p0), q0 = p0 + bb, mp = m - q0;
  const int nt = (mp + kTile - 1) / kTile;
  const int64_t base = int64_t(blockIdx.y) * fr.pool + fr.off[f];
  double2* Yb = Y + base;
  const double2* Fb = F + base;
  const double2* pp = part + int64_t(blockIdx.y) * part_stride + part_off[f];
  for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
    int r = idx % bb, c = idx / bb;
    double2 v = Fb[(p0 + r) + int64_t(m) * (p0 + c)];
    for (int t = 0; t < nt; ++t) v = subv(v, pp[int64_t(t) * b * b + r + b * c]);
    tmp[r + bb * c] = v;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < bb * bb; idx += blockDim.x) {
    int r = idx % bb, c = idx / bb;
    double2 a = tmp[r + bb * c], t = tmp[c + bb * r];
    // Y[P,P] of a complex-symmetric front is symmetrised; an LDU front's is not symmetric
    Yb[(p0 + r) + int64_t(m) * (p0 + c)] = GEN ? a : make_double2(0.5 * (a.x + t.x), 0.5 * (a.y + t.y));
  }
}

// ------------------------------------------------------------ pole sum
__global__ void k_pole_sum(const double2* __restrict__ Y, int64_t pool, const int64_t* __restrict__ entry_pos,
                           int64_t nnz, BatchShifts sh, int overwrite, double* __restrict__ dm,
                           double* __restrict__ edm, double* __restrict__ fdm, double* __restrict__ ddm) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = entry_pos[e];
    double a = 0.0, ae = 0.0, af = 0.0, ad = 0.0;
    for (int b = 0; b < sh.nb; ++b) {
      double2 v = Y[b * pool + p];
      // Im(w v) = w.re v.im + w.im v.re
      a = fma(sh.wr_re[b], v.y, fma(sh.wr_im[b], v.x, a));
      ae = fma(sh.we_re[b], v.y, fma(sh.we_im[b], v.x, ae));
      af = fma(sh.wf_re[b], v.y, fma(sh.wf_im[b], v.x, af));
      ad = fma(sh.wd_re[b], v.y, fma(sh.wd_im[b], v.x, ad));
    }
    if (dm) dm[e] = overwrite ? a : dm[e] + a;
    if (edm) edm[e] = overwrite ? ae : edm[e] + ae;
    if (fdm) fdm[e] = overwrite ? af : fdm[e] + af;
    if (ddm) ddm[e] = overwrite ? ad : ddm[e] + ad;
  }
}

// Assembly of an LDU front from complex H and S (interleaved, nnz each):
// every CSC entry at its own position (both triangles), A = H - z S.
__global__ void k_assemble_gen(double2* __restrict__ F, const double2* __restrict__ H, const double2* __restrict__ S,
                               const int64_t* __restrict__ pos, int64_t nnz, int64_t pool, BatchShifts sh) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = pos[e];
    const double2 h = H[e], v = S[e];
    for (int b = 0; b < sh.nb; ++b)  // (hr + i hi) - (zr + i zi)(sr + i si)
      F[b * pool + p] = make_double2(h.x - fma(sh.re[b], v.x, -sh.im[b] * v.y), h.y - fma(sh.re[b], v.y, sh.im[b] * v.x));
  }
}

// Pole sum of the Hermitian variant: with G = (H - z S)^{-1} and (H - conj(z)
// S)^{-1} = G^H, the folded pole pair contributes (w G - conj(w) G^H) / 2i;
// at entry (r, c), with a = w G[r,c] and t = w G[c,r], that is
// ((a.im + t.im) + i (t.re - a.re)) / 2. Complex outputs (interleaved).
__global__ void k_pole_sum_herm(const double2* __restrict__ Y, int64_t pool, const int64_t* __restrict__ pos,
                                const int64_t* __restrict__ pos_t, int64_t nnz, BatchShifts sh, int overwrite,
                                double2* __restrict__ dm, double2* __restrict__ edm, double2* __restrict__ fdm,
                                double2* __restrict__ ddm) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = pos[e], q = pos_t[e];
    double2 o[4] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int b = 0; b < sh.nb; ++b) {
      const double2 g = Y[b * pool + p], gt = Y[b * pool + q];
      const double wr[4] = {sh.wr_re[b], sh.we_re[b], sh.wf_re[b], sh.wd_re[b]};
      const double wi[4] = {sh.wr_im[b], sh.we_im[b], sh.wf_im[b], sh.wd_im[b]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double2 w = make_double2(wr[k], wi[k]);
        const double2 a = mulv(w, g), t = mulv(w, gt);
        o[k].x += 0.5 * (a.y + t.y);
        o[k].y += 0.5 * (t.x - a.x);
      }
    }
    double2* outs[4] = {dm, edm, fdm, ddm};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (outs[k]) outs[k][e] = overwrite ? o[k] : addv(outs[k][e], o[k]);
  }
}

__global__ void k_extract(const double2* __restrict__ Y, const int64_t* __restrict__ entry_pos, int64_t nnz,
                          double2* __restrict__ out) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x)
    out[e] = Y[entry_pos[e]];
}

__global__ void k_scaled_imag(const double2* __restrict__ Y, const int64_t* __restrict__ entry_pos, int64_t nnz,
                              double scale, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x)
    out[e] = scale * Y[entry_pos[e]].y;
}

__global__ void k_trace_partial(const double* dm, const double* edm, const double* fdm, const double* ddm,
                                const double* __restrict__ S, int64_t nnz, double* partials) {
  __shared__ double red[4][256];
  const int64_t chunk = (nnz + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(nnz, lo + chunk);
  double a = 0, b = 0, c = 0, d = 0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    double sv = S[e];
    if (dm) a = fma(dm[e], sv, a);
    if (edm) b = fma(edm[e], sv, b);
    if (fdm) c = fma(fdm[e], sv, c);
    if (ddm) d = fma(ddm[e], sv, d);
  }
  red[0][threadIdx.x] = a; red[1][threadIdx.x] = b; red[2][threadIdx.x] = c; red[3][threadIdx.x] = d;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) partials[4 * blockIdx.x + q] = red[q][0];
}

__global__ void k_trace_final(const double* partials, int nblocks, double* out4) {
  if (threadIdx.x < 4) {
    double s = 0;
    for (int t = 0; t < nblocks; ++t) s += partials[4 * t + threadIdx.x];
    out4[threadIdx.x] = s;
  }
}

inline int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return int(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

// ------------------------------------------------------------ launchers
template <typename T>
void launch_assemble(T* F, const double* H, const double* S, const int64_t* src, const int64_t* pos, int64_t nlow,
                     int64_t pool, const BatchShifts& sh, cudaStream_t st) {
  k_assemble<T><<<grid_for(nlow, 256), 256, 0, st>>>(F, H, S, src, pos, nlow, pool, sh);
}

template <typename T>
void launch_extend_add(T* F, const DevFronts& fr, const int32_t* children, int nchild, const int32_t* pref,
                       int64_t total_tiles, const BatchShifts& sh, cudaStream_t st) {
  if (nchild <= 0 || total_tiles <= 0) return;
  dim3 grid(unsigned(total_tiles), 1, sh.nb), block(32, 8);
  k_extend_add<T><<<grid, block, 0, st>>>(F, fr, children, nchild, pref);
}

// One cluster of C CTAs per block inverse (complex poles, which need no
// inertia count).
template <typename T, bool GEN, int C>
void launch_diag_inv_cluster_c(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0, int b,
                               const BatchShifts& sh, DevStatus status, cudaStream_t st) {
  constexpr int kDiagCluster = C;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(nfronts * kDiagCluster), unsigned(sh.nb), 1);
  cfg.blockDim = dim3(kDiagThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kDiagCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_diag_inv_cluster<T, GEN, C>, F, fr, fronts, p0, b, status);
}

// The cluster size: wide enough to spread the launch's inversions over the
// SMs, 1 (the single-CTA kernel) once they already fill them.
int diag_cluster_size(int inversions) {
  return inversions >= 152 ? 1 : inversions >= 76 ? 2 : inversions >= 38 ? 4 : 8;
}

template <typename T, bool GEN>
bool launch_diag_inv_cluster(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0, int b,
                             const BatchShifts& sh, DevStatus status, cudaStream_t st) {
  switch (diag_cluster_size(nfronts * sh.nb)) {
    case 8: launch_diag_inv_cluster_c<T, GEN, 8>(F, fr, fronts, nfronts, p0, b, sh, status, st); return true;
    case 4: launch_diag_inv_cluster_c<T, GEN, 4>(F, fr, fronts, nfronts, p0, b, sh, status, st); return true;
    case 2: launch_diag_inv_cluster_c<T, GEN, 2>(F, fr, fronts, nfronts, p0, b, sh, status, st); return true;
    default: return false;
  }
}

template <typename T>
void launch_diag_inv(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0, int b,
                     const BatchShifts& sh, DevStatus status, bool count_inertia, cudaStream_t st) {
  if (nfronts <= 0) return;
  // the cluster kernel: complex poles, and inertia shifts whose blocks are
  // saved for the deferred count
  if ((!count_inertia || status.dsave) && b <= 64 &&
      launch_diag_inv_cluster<T, false>(F, fr, fronts, nfronts, p0, b, sh, status, st))
    return;
  size_t smem = sizeof(T) * size_t(b) * (b + 1) + (count_inertia ? sizeof(double) * b * b : 0);
  dim3 grid(nfronts, sh.nb);
  k_diag_inv<T><<<grid, kDiagThreads, smem, st>>>(F, fr, fronts, p0, b, status, count_inertia ? 1 : 0);
}

template <typename T>
void launch_panel_solve(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_row_tiles, int p0,
                        int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  dim3 grid(max_row_tiles, nfronts, sh.nb);
  k_panel_solve<T><<<grid, 256, kSmem3m, st>>>(F, fr, fronts, p0, b);
}

template <typename T>
void launch_trailing(T* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles, int p0, int b,
                     const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || max_tiles <= 0) return;
  dim3 grid(max_tiles, nfronts, sh.nb);
  k_trailing<T><<<grid, 256, kSmem3m, st>>>(F, fr, fronts, p0, b);
}

void launch_gather(double2* Y, const DevFronts& fr, const int32_t* fronts, int nfronts, const int32_t* pref,
                   int64_t total_tiles, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || total_tiles <= 0) return;
  dim3 grid(unsigned(total_tiles), 1, sh.nb), block(32, 8);
  k_gather<<<grid, block, 0, st>>>(Y, fr, fronts, nfronts, pref);
}

void launch_selinv_offdiag(double2* Y, const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts,
                           int max_row_tiles, int max_mp, int p0, int b, const BatchShifts& sh, double2* kpart,
                           const int64_t* part_off, int64_t kstride, cudaStream_t st) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  // every front's ks tiles fit: ksplit_of is non-decreasing in m_p
  const int ks = kpart ? ksplit_of(max_mp) : 1;
  dim3 grid(max_row_tiles * ks, nfronts, sh.nb);
  k_selinv_offdiag<false><<<grid, 256, kSmem3m, st>>>(Y, F, fr, fronts, p0, b, kpart, part_off, kstride);
  if (ks > 1)
    k_offdiag_reduce<<<dim3(max_row_tiles, nfronts, sh.nb), 256, 0, st>>>(Y, fr, fronts, p0, b, kpart, part_off,
                                                                            kstride);
}

void launch_selinv_diag_partial(const double2* Y, const double2* F, double2* part, const int64_t* part_off,
                                int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts,
                                int max_row_tiles, int p0, int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  dim3 grid(max_row_tiles, nfronts, sh.nb);
  k_selinv_diag_partial<<<grid, 256, kSmem3m, st>>>(Y, F, part, part_off, part_stride, fr, fronts, p0, b);
}

void launch_selinv_diag_reduce(double2* Y, const double2* F, const double2* part, const int64_t* part_off,
                               int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0,
                               int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0) return;
  dim3 grid(nfronts, sh.nb);
  k_selinv_diag_reduce<<<grid, 256, sizeof(double2) * b * b, st>>>(Y, F, part, part_off, part_stride, fr, fronts, p0, b);
}

void launch_pole_sum(const double2* Y, int64_t pool, const int64_t* entry_pos, int64_t nnz, const BatchShifts& sh,
                     int overwrite, double* dm, double* edm, double* fdm, double* ddm, cudaStream_t st) {
  k_pole_sum<<<grid_for(nnz, 256), 256, 0, st>>>(Y, pool, entry_pos, nnz, sh, overwrite, dm, edm, fdm, ddm);
}

void launch_extract(const double2* Y, const int64_t* entry_pos, int64_t nnz, double2* out, cudaStream_t st) {
  k_extract<<<grid_for(nnz, 256), 256, 0, st>>>(Y, entry_pos, nnz, out);
}

void launch_scaled_imag(const double2* Y, const int64_t* entry_pos, int64_t nnz, double scale, double* out,
                        cudaStream_t st) {
  k_scaled_imag<<<grid_for(nnz, 256), 256, 0, st>>>(Y, entry_pos, nnz, scale, out);
}

void launch_traces(const double* dm, const double* edm, const double* fdm, const double* ddm, const double* S,
                   int64_t nnz, double* partials, int nblocks, double* out4, cudaStream_t st) {
  k_trace_partial<<<nblocks, 256, 0, st>>>(dm, edm, fdm, ddm, S, nnz, partials);
  k_trace_final<<<1, 32, 0, st>>>(partials, nblocks, out4);
}

cudaError_t configure_kernels(int b) {
  size_t need_c = sizeof(double2) * size_t(b) * (b + 1);
  size_t need_r = sizeof(double) * size_t(b) * (b + 1) + sizeof(double) * b * b;
  cudaError_t e = cudaFuncSetAttribute(k_diag_inv<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(need_c));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_diag_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(need_r));
  if (e != cudaSuccess) return e;
  // LDU fronts: the Hermitian inertia count keeps a complex copy of the block
  e = cudaFuncSetAttribute(k_bk_count_all<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(sizeof(double2) * b * b));
  if (e != cudaSuccess) return e;
  const size_t need_g = sizeof(double2) * size_t(b) * (b + 1) + sizeof(double2) * b * b;
  e = cudaFuncSetAttribute(k_diag_inv<double2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(need_g));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_selinv_diag_reduce<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(sizeof(double2) * b * b));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_selinv_diag_reduce<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(sizeof(double2) * b * b));
  if (e != cudaSuccess) return e;
  const void* gemms[] = {(const void*)k_panel_solve<double>, (const void*)k_panel_solve<double2>,
                         (const void*)k_panel_solve<double2, true>, (const void*)k_panel_upper,
                         (const void*)k_trailing<double>, (const void*)k_trailing<double2>,
                         (const void*)k_trailing<double2, true>, (const void*)k_selinv_offdiag<false>,
                         (const void*)k_selinv_offdiag<true>, (const void*)k_selinv_diag_partial<false>,
                         (const void*)k_selinv_diag_partial<true>};
  for (const void* fn : gemms) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmem3m));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---- LDU fronts of complex Hermitian H and S (general complex shifted matrices)
void launch_assemble_gen(double2* F, const double2* H, const double2* S, const int64_t* pos, int64_t nnz,
                         int64_t pool, const BatchShifts& sh, cudaStream_t st) {
  k_assemble_gen<<<grid_for(nnz, 256), 256, 0, st>>>(F, H, S, pos, nnz, pool, sh);
}

void launch_extend_add_full(double2* F, const DevFronts& fr, const int32_t* children, int nchild, const int32_t* pref,
                            int64_t total_tiles, const BatchShifts& sh, cudaStream_t st) {
  if (nchild <= 0 || total_tiles <= 0) return;
  dim3 grid(unsigned(total_tiles), 1, sh.nb), block(32, 8);
  k_extend_add<double2, true><<<grid, block, 0, st>>>(F, fr, children, nchild, pref);
}

void launch_diag_inv_gen(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0, int b,
                         const BatchShifts& sh, DevStatus status, bool count_inertia, cudaStream_t st) {
  if (nfronts <= 0) return;
  if ((!count_inertia || status.dsave) && b <= 64 &&
      launch_diag_inv_cluster<double2, true>(F, fr, fronts, nfronts, p0, b, sh, status, st))
    return;
  size_t smem = sizeof(double2) * size_t(b) * (b + 1) + (count_inertia ? sizeof(double2) * b * b : 0);
  dim3 grid(nfronts, sh.nb);
  k_diag_inv<double2, true><<<grid, kDiagThreads, smem, st>>>(F, fr, fronts, p0, b, status, count_inertia ? 1 : 0);
}

void launch_panel_solve_gen(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_row_tiles,
                            int p0, int b, const BatchShifts& sh, cudaStream_t st, bool upper) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  dim3 grid(max_row_tiles, nfronts, sh.nb);
  if (upper) k_panel_upper<<<grid, 256, kSmem3m, st>>>(F, fr, fronts, p0, b);
  else k_panel_solve<double2, true><<<grid, 256, kSmem3m, st>>>(F, fr, fronts, p0, b);
}

void launch_trailing_full(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_row_tiles,
                          int p0, int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  dim3 grid(max_row_tiles * max_row_tiles, nfronts, sh.nb);
  k_trailing<double2, true><<<grid, 256, kSmem3m, st>>>(F, fr, fronts, p0, b);
}

void launch_selinv_offdiag_gen(double2* Y, const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts,
                               int max_row_tiles, int p0, int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  dim3 grid(2 * max_row_tiles, nfronts, sh.nb);
  k_selinv_offdiag<true><<<grid, 256, kSmem3m, st>>>(Y, F, fr, fronts, p0, b, nullptr, nullptr, 0);
}

void launch_selinv_diag_partial_gen(const double2* Y, const double2* F, double2* part, const int64_t* part_off,
                                    int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts,
                                    int max_row_tiles, int p0, int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0 || max_row_tiles <= 0) return;
  dim3 grid(max_row_tiles, nfronts, sh.nb);
  k_selinv_diag_partial<true><<<grid, 256, kSmem3m, st>>>(Y, F, part, part_off, part_stride, fr, fronts, p0, b);
}

void launch_selinv_diag_reduce_gen(double2* Y, const double2* F, const double2* part, const int64_t* part_off,
                                   int64_t part_stride, const DevFronts& fr, const int32_t* fronts, int nfronts, int p0,
                                   int b, const BatchShifts& sh, cudaStream_t st) {
  if (nfronts <= 0) return;
  dim3 grid(nfronts, sh.nb);
  k_selinv_diag_reduce<true><<<grid, 256, sizeof(double2) * b * b, st>>>(Y, F, part, part_off, part_stride, fr, fronts,
                                                                          p0, b);
}

void launch_pole_sum_herm(const double2* Y, int64_t pool, const int64_t* pos, const int64_t* pos_t, int64_t nnz,
                          const BatchShifts& sh, int overwrite, double2* dm, double2* edm, double2* fdm, double2* ddm,
                          cudaStream_t st) {
  k_pole_sum_herm<<<grid_for(nnz, 256), 256, 0, st>>>(Y, pool, pos, pos_t, nnz, sh, overwrite, dm, edm, fdm, ddm);
}

template <typename T>
void launch_bk_count_all(const int32_t* slots, int nslots, const DevFronts& fr, int b, int nb, DevStatus status,
                         cudaStream_t st) {
  if (nslots <= 0 || nb <= 0) return;
  k_bk_count_all<T><<<dim3(nslots, nb), kDiagThreads, sizeof(T) * b * b, st>>>(slots, fr, b, status);
}
template void launch_bk_count_all<double>(const int32_t*, int, const DevFronts&, int, int, DevStatus, cudaStream_t);
template void launch_bk_count_all<double2>(const int32_t*, int, const DevFronts&, int, int, DevStatus, cudaStream_t);

#define PEXSI_INSTANTIATE(T)                                                                                        \
  template void launch_assemble<T>(T*, const double*, const double*, const int64_t*, const int64_t*, int64_t,    \
                                   int64_t, const BatchShifts&, cudaStream_t);                                   \
  template void launch_extend_add<T>(T*, const DevFronts&, const int32_t*, int, const int32_t*, int64_t,        \
                                     const BatchShifts&, cudaStream_t);                                           \
  template void launch_diag_inv<T>(T*, const DevFronts&, const int32_t*, int, int, int, const BatchShifts&,      \
                                   DevStatus, bool, cudaStream_t);                                                \
  template void launch_panel_solve<T>(T*, const DevFronts&, const int32_t*, int, int, int, int,                  \
                                      const BatchShifts&, cudaStream_t);                                          \
  template void launch_trailing<T>(T*, const DevFronts&, const int32_t*, int, int, int, int, const BatchShifts&, \
                                   cudaStream_t);
PEXSI_INSTANTIATE(double)
PEXSI_INSTANTIATE(double2)

}  // namespace pexsi
