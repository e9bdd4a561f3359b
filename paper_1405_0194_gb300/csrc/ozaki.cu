// Split-precision (Ozaki-scheme) complex and real GEMMs on the tcgen05 tensor
// cores: the Schur update F[S,S] -= L[S,P] W[S,P]^T and the panel solve
// L[S,P] = W[S,P] D^-1 of the factorisation (short K = bb, persistent
// kernel k_oz_gemm), and the Takahashi step Y[S,P] = -Y[S,S] L[S,P] of
// selected inversion (long K = m_p, k_oz_tak_fused, which slices A itself).
//
// Error-free splitting (Ozaki, Ogita, Oishi and Rump 2012): each row i of A
// and each row j of B (both stored K-major) is scaled by a power of two
// 2^e > max |entry| and cut into S slices of small integers,
//   x = A_ik / 2^e_i = sum_s a_s 2^(-7 s) + r,  |a_1| <= 128, |a_s| <= 64 (s > 1),
// |r| <= 2^(-7 S - 1), each slice exact in bfloat16. The cut rounds to a
// 7S-bit fixed-point integer (half of the entries by one FP64 fused
// multiply-add, half from the bit pattern with integer operations, which
// balances the two pipes) and takes its balanced base-128 digits without a
// carry chain (one mask and one float add per digit).
//
// Complex products as real MMAs: a tile of 64 complex rows of A becomes the
// 128 x K real operand [Ar; Ai] (P1) and, one slice block further on,
// [Ai; -Ar] (P2); with B = Br + i Bi (64 complex columns as 64 real rows),
//   P1 Br^T + P2 (-Bi)^T = [Ar Br - Ai Bi; Ai Br + Ar Bi] = [Re; Im],
// the -Bi coming from the MMA's negate-B bit. So each slice pair (s, t) is
// two M = 128, N = 64 products per 16-deep K step into ONE accumulator, and
// the slice tile of A stores the three 64-row blocks Ar, Ai, -Ar back to
// back. The B slices of a K tile are stored Br of slices 1..S, then Bi of
// slices 1..S, so the products of slice s of A with up to four consecutive
// B slices are one MMA of N = 64 g.
//
// A product of two slices is exact in FP32; the tensor core adds them in FP32
// accumulators in TMEM, one accumulator (64 columns) per "diagonal"
// D = s + t (products of equal scale 2^(-7 D)). With S <= 6 and K chunks of
// 256 every accumulator holds an integer of magnitude at most 2^24 (for
// S = 6 the last diagonal holds 6 pairs: 2 (2 * 2^13 + 4 * 2^12) per k), so
// the accumulation is exact. After each chunk the epilogue warps convert the
// accumulators to integers and combine them exactly in 64-bit integers,
// sum_D acc_D 2^(7 (S + 1 - D)) (magnitude below 2^58.1 per chunk, so eight
// chunks stay below 2^61.1, inside int64); the final scaling by 2^(e_i + f_j - 7 (S + 1)) is
// folded into an integer-only int64 -> double conversion. Pairs with
// s + t > S + 1 are dropped (their contribution is below 2^(-7 (S + 2)) of
// |A_i| |B_j|).
//
// Operands are pre-tiled by the slicing kernel into the no-swizzle K-major
// core-matrix layout the MMA descriptors read: a block of R rows x 32 k of
// one slice stores element (r, k) at byte (r/8)*512 + (k/8)*128 + (r%8)*16 +
// (k%8)*2 (LBO 128 B, SBO 512 B). One (row tile, K tile) holds the S slices
// one after another: 12 KiB each for A (Ar, Ai, -Ar); for B the S blocks of
// Br, then the S blocks of Bi (4 KiB each); so one bulk async copy stages a
// slice of A or all slices of B.
//
// The GEMM CTAs are warp-specialised: a producer streams slices (bulk async
// copies with mbarrier transaction counts, or slices cut in shared memory by
// worker warps); one thread issues tcgen05.mma and releases each slot with
// tcgen05.commit; epilogue warps drain TMEM while the next slices load. Every wait is bounded (1 s of wall time); a wait that runs
// out records where in a status word, lets the other roles stop, waits
// (bounded) for its own copies and MMAs in flight, frees TMEM and returns,
// and CTAs that start after a failure return at once.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace pexsi {
namespace {

constexpr int kOzRows = 64;   // complex rows of A (and of B) per tile
constexpr int kOzK = 32;      // K per staged tile
constexpr int kOzFlush = 8;   // chunks per 64-bit integer partial sum
constexpr int kBlk = kOzRows * kOzK * 2;  // bytes of one 64-row block of one slice (4 KiB)
constexpr int kSliceA = 3 * kBlk;         // Ar, Ai, -Ar (12 KiB)
constexpr int kSliceB = 2 * kBlk;         // Br, Bi (8 KiB)
constexpr int kSlotsA = 8;    // A ring: one slice of one K tile per slot
constexpr int kSlotsB = 2;    // B ring: all S slices of one K tile per slot
constexpr int kEpiWarps = 8;  // two per TMEM lane quarter, 32 columns each
constexpr int kGemmThreads = (kEpiWarps + 2) * 32;  // + producer warp + MMA warp
constexpr int kNanExp = 0x7FFF;                     // exponent marker of a row holding Inf or NaN
constexpr uint64_t kWaitNs = 1000000000ull;         // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle, K-major: LBO = 128 B between
// core matrices along K, SBO = 512 B between 8-row groups, version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFF) >> 4) | (uint64_t(128 >> 4) << 16) | (uint64_t(512 >> 4) << 32) |
         (uint64_t(1) << 46);
}

// The same for 16-deep K tiles: SBO = 256 B.
__device__ __forceinline__ uint64_t sdesc16(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFF) >> 4) | (uint64_t(128 >> 4) << 16) | (uint64_t(256 >> 4) << 32) |
         (uint64_t(1) << 46);
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major,
// M = 128, N = 64 g; optionally B negated.
__host__ __device__ constexpr uint32_t idesc(int g, bool negate_b) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (negate_b ? (1u << 14) : 0u) | (uint32_t(64 * g >> 3) << 17) |
         (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (budget_ns of wall time, the plan's wait bound) for the
// completion of the barrier phase of the given parity; gives up early once
// another role has recorded a failure.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, const volatile int* fail, uint64_t budget_ns) {
  if (bar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (bar_try(bar, parity)) return true;
    if (*fail) return false;
    if ((it & 255u) == 0 && global_ns() - t0 > budget_ns) return false;
  }
}

// Bounded wait that ignores failures (draining own copies / MMAs in flight):
// always the full second, whatever the plan's wait bound, since what it
// waits for was issued and completes on its own.
__device__ __forceinline__ bool bar_wait_all(uint32_t bar, uint32_t parity) {
  if (bar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (bar_try(bar, parity)) return true;
    if ((it & 255u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void bar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate));
}

// Arrives on `bar` once every tcgen05.mma this thread issued so far is done.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Descriptor d moved by off 16-byte units: the start address field is the
// low 14 bits and shared-memory addresses stay below 2^18, so the low word
// takes the add without a carry.
__device__ __forceinline__ uint64_t desc_off(uint64_t d, uint32_t off) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(uint32_t(d) + off), "r"(uint32_t(d >> 32)));
  return r;
}

// Products of one slice of A with the B slices T0 + 1 .. T0 + G of a K tile
// (KSTEPS steps of 16): the G slices of Br (and of Bi) are consecutive 64-row
// blocks of BLK bytes, and the accumulators of their diagonals consecutive
// 64-column blocks of TMEM, so one MMA with N = 64 G covers all G diagonals.
// a1, a2, br, bi: descriptors of [Ar; Ai], [Ai; -Ar], Br slice 1, Bi slice 1
// (real operands: a1 and br only); acc: the TMEM column of diagonal s + 1.
template <bool CPLX, int KSTEPS, int BLK, int T0, int G>
__device__ __forceinline__ void mma_group(uint32_t acc, uint64_t a1, uint64_t a2, uint64_t br, uint64_t bi,
                                          uint32_t first) {
#pragma unroll
  for (int ks = 0; ks < KSTEPS; ++ks) {
    const uint32_t ko = uint32_t(ks * 16);  // two core matrices along K (256 B, in 16-byte units)
    const uint32_t bo = uint32_t(T0 * BLK / 16) + ko;
    mma(acc + uint32_t(T0 * 64), desc_off(a1, ko), desc_off(br, bo), idesc(G, false), ks == 0 ? first : 1u);
    if (CPLX) mma(acc + uint32_t(T0 * 64), desc_off(a2, ko), desc_off(bi, bo), idesc(G, true), 1u);
  }
}

// All products of slice s of A with the B slices t = 1 .. c (c = S + 1 - s,
// the pairs s + t <= S + 1), c diagonals in groups of at most four. The MMA
// of N = 64 is bound by its operand fetch from shared memory (6 KiB in 48
// cycles, against 32 cycles of math), N >= 128 runs at the tensor rate; and
// one straight-line issue per slice keeps the issuing thread ahead of the
// tensor pipe.
template <bool CPLX, int KSTEPS, int BLK>
__device__ __forceinline__ void mma_slice(int c, uint32_t acc, uint64_t a1, uint64_t a2, uint64_t br, uint64_t bi,
                                          uint32_t first) {
  switch (c) {
    case 6:
      mma_group<CPLX, KSTEPS, BLK, 0, 4>(acc, a1, a2, br, bi, first);
      mma_group<CPLX, KSTEPS, BLK, 4, 2>(acc, a1, a2, br, bi, first);
      break;
    case 5:
      mma_group<CPLX, KSTEPS, BLK, 0, 3>(acc, a1, a2, br, bi, first);
      mma_group<CPLX, KSTEPS, BLK, 3, 2>(acc, a1, a2, br, bi, first);
      break;
    case 4:
      mma_group<CPLX, KSTEPS, BLK, 0, 4>(acc, a1, a2, br, bi, first);
      break;
    case 3:
      mma_group<CPLX, KSTEPS, BLK, 0, 3>(acc, a1, a2, br, bi, first);
      break;
    case 2:
      mma_group<CPLX, KSTEPS, BLK, 0, 2>(acc, a1, a2, br, bi, first);
      break;
    default:
      mma_group<CPLX, KSTEPS, BLK, 0, 1>(acc, a1, a2, br, bi, first);
      break;
  }
}

// 32 lanes x 8 consecutive TMEM columns, without the wait: tcgen05.wait::ld
// before any register is read.
__device__ __forceinline__ void tmem_ld8_nw(uint32_t addr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(addr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 consecutive TMEM columns, without the wait.
__device__ __forceinline__ void tmem_ld16_nw(uint32_t addr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
}

__device__ __forceinline__ void tmem_st16(uint32_t addr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          addr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// w_c += v_c 2^sh on the 64-bit integers w_c = (w[2c + 1], w[2c]), c < 8,
// for FP32 accumulators v_c holding exact integers (|v_c| <= 2^24). When
// every |v_c| of the warp is below 2^22, 1.5 2^23 + v_c is exact with v_c in
// its low mantissa bits (one add, one integer subtract); otherwise the
// conversion instruction takes them.
__device__ __forceinline__ void acc_add8(uint32_t (&w)[16], const uint32_t (&v)[8], int sh) {
  float mx = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) mx = fmaxf(mx, fabsf(__uint_as_float(v[c])));
  int iv[8];
  if (__all_sync(0xFFFFFFFFu, mx < 4194304.0f)) {
#pragma unroll
    for (int c = 0; c < 8; ++c) iv[c] = __float_as_int(__uint_as_float(v[c]) + 12582912.0f) - 0x4B400000;
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) iv[c] = __float2int_rn(__uint_as_float(v[c]));
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    unsigned long long a64 = (static_cast<unsigned long long>(w[2 * c + 1]) << 32) | w[2 * c];
    a64 += static_cast<unsigned long long>(static_cast<long long>(iv[c])) << sh;
    w[2 * c] = uint32_t(a64);
    w[2 * c + 1] = uint32_t(a64 >> 32);
  }
}

// w_c += sum over the diagonals D = 2 .. S + 1 of v[D - 2]_c 2^(7 (S + 1 - D)),
// c < 8, for the FP32 accumulators of all S diagonals at once. When every
// |v| of the warp is below 2^22, each converts by the add-and-subtract and
// adjacent diagonals pair in 32 bits: the biased words h = 0x4B400000 + a
// and l = 0x4B400000 + b give a 2^7 + b = 128 h + l - 129 0x4B400000 modulo
// 2^32, exact since |a 2^7 + b| < 2^30; one multiply-add per pair and one
// 64-bit multiply-add by 2^shift. Otherwise each diagonal takes the
// conversion instruction.
template <int S>
__device__ __forceinline__ void acc_add_diags8(uint32_t (&w)[16], const uint32_t (&v)[S][8]) {
  float mx = 0.0f;
#pragma unroll
  for (int t = 0; t < S; ++t)
#pragma unroll
    for (int c = 0; c < 8; ++c) mx = fmaxf(mx, fabsf(__uint_as_float(v[t][c])));
  if (!__all_sync(0xFFFFFFFFu, mx < 4194304.0f)) {
#pragma unroll
    for (int D = 2; D <= S + 1; ++D) acc_add8(w, v[D - 2], 7 * (S + 1 - D));
    return;
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    unsigned long long a64 = (static_cast<unsigned long long>(w[2 * c + 1]) << 32) | w[2 * c];
#pragma unroll
    for (int D = 2; D <= S + 1; D += 2) {
      const uint32_t h = __float_as_uint(__uint_as_float(v[D - 2][c]) + 12582912.0f);
      if (D + 1 <= S + 1) {
        const uint32_t l = __float_as_uint(__uint_as_float(v[D - 1][c]) + 12582912.0f);
        const int pr = int(h * 128u + l - 0x4B400000u * 129u);
        a64 += static_cast<unsigned long long>(static_cast<long long>(pr) * (1LL << (7 * (S - D))));
      } else {
        const int a = int(h - 0x4B400000u);
        a64 += static_cast<unsigned long long>(static_cast<long long>(a) * (1LL << (7 * (S + 1 - D))));
      }
    }
    w[2 * c] = uint32_t(a64);
    w[2 * c + 1] = uint32_t(a64 >> 32);
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// The integer X nearest to x 2^(7 S - e) (|x| < 2^e, so |X| <= 2^(7 S)),
// from the bit pattern: the mantissa shifted right by n >= 10 with rounding,
// no floating-point arithmetic.
__device__ __forceinline__ long long fixed_point(double x, int e, int S) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = int((bits >> 52) & 0x7FF);
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  int Ee = 1;  // subnormals: exponent of the smallest normal, no hidden bit
  if (E != 0) {
    mant |= 1ull << 52;
    Ee = E;
  }
  const int n = 1075 - Ee - 7 * S + e;
  long long X = 0;
  if (n > 0 && n < 54) X = static_cast<long long>((mant + (1ull << (n - 1))) >> n);
  return (bits >> 63) ? -X : X;
}

// The same rounded to nearest even by one FP64 fused multiply-add, for rows
// whose scale 2^(7 S - e) is a normal double (fma_scale): x 2^(7 S - e) is
// exact, and adding 1.5 2^52 leaves the integer (|X| <= 2^42) in the low
// mantissa bits. One FP64 instruction instead of some 17 integer ones on the
// busier integer pipe.
__device__ __forceinline__ long long fixed_point_fma(double x, double scale) {
  return __double_as_longlong(fma(x, scale, 6755399441055744.0)) - 0x4338000000000000LL;
}

// 2^(7 S - e) when it is a normal double and the row is finite, else 0.
__device__ __forceinline__ double fma_scale(int e, int S) {
  const int be = 1023 + 7 * S - e;
  return (e != kNanExp && be >= 1 && be <= 2046) ? __longlong_as_double(static_cast<long long>(be) << 52) : 0.0;
}

// The fixed-point integer of x for a row of exponent e: by the FP64
// multiply-add when the scale is a normal double (every row but those of
// extreme range or holding Inf / NaN), else by the bit pattern. Both round to
// nearest (ties to even, resp. away from zero). The cutting kernels send
// half of the entries (real parts; even k of real operands) this way and
// half by the bit pattern, which keeps the FP64 and integer pipes balanced.
__device__ __forceinline__ long long fixed_of(double x, double scale, int e, int S) {
  return scale != 0.0 ? fixed_point_fma(x, scale) : fixed_point(x, e, S);
}

// High word of |x|: ordered like |x| for finite x, >= 0x7FF00000 for Inf / NaN.
__device__ __forceinline__ uint32_t abs_hi(double x) { return uint32_t(__double2hiint(x)) & 0x7FFFFFFFu; }

// Row exponent e (2^e > every |entry|) from the largest high word of the row.
__device__ __forceinline__ int exp_of_hi(uint32_t mx) {
  return mx >= 0x7FF00000u ? kNanExp : mx != 0 ? int(mx >> 20) - 1022 : 0;
}

// Balanced base-128 digits of X: X = d_0 128^(S-1) + ... + d_(S-1), the
// lower digits in [-64, 63] and |d_0| <= 128. Without a carry chain: the
// digits of Y = X + C, C = 64 (1 + 128 + ... + 128^(S-2)), below the top one
// are d_s + 64 in [0, 127] (the representation is unique), so each is a
// shift and a mask, and the top digit d_0 is Y >> 7 (S - 1) itself.
__host__ __device__ constexpr long long digit_bias(int S) {
  long long c = 0;
  for (int k = 1; k < S; ++k) c = 128 * c + 64;
  return c;
}

// Slice sl (0 = the most significant) of Y = X + digit_bias(S) as a float
// holding the digit exactly. A lower digit u sits at bit p <= 14 of the low
// word (digits 0-2 from the low end) or of Y >> 21 (digits 3-4); under the
// exponent field of 2^(23 - p) those bits make the float 2^(23 - p) + u, and
// subtracting 2^(23 - p) + 64 leaves u - 64: one mask and one add, no shift.
// The top digit is 1.5 2^23 + d_0 - 1.5 2^23.
template <int S>
__device__ __forceinline__ float slice_digit(long long Y, int sl) {
  if (sl == 0) return __int_as_float(0x4B400000 + int(Y >> (7 * (S - 1)))) - 12582912.0f;
  const int k = S - 1 - sl;  // digit index from the low end, 0 .. 4
  const int p = k <= 2 ? 7 * k : 7 * k - 21;
  const uint32_t w = k <= 2 ? uint32_t(Y) : uint32_t(Y >> 21);
  return __uint_as_float((uint32_t(150 - p) << 23) | (w & (127u << p))) - (float(1 << (23 - p)) + 64.0f);
}

// 32-bit word of two bfloat16 values (a in the low half, b in the high half)
// from floats holding integers of at most 8 significant bits (exact in bf16).
__device__ __forceinline__ uint32_t bf16x2_of(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// The S slice words of 8 complex entries along K (Y[2u], Y[2u + 1]: real and
// imaginary part of entry u as X + digit_bias(S)): slice sl of the real parts
// goes to re + sl * step, of the imaginary parts to im + sl * step, and when
// neg is given, of the negated real parts to neg + sl * step (sign bits
// flipped: -0 for a zero digit, an exact zero).
template <int S>
__device__ __forceinline__ void store_slices_c(const long long (&Y)[16], uint8_t* re, uint8_t* im, uint8_t* neg,
                                               int step) {
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    float f[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) f[t] = slice_digit<S>(Y[t], sl);
    const uint4 wre = make_uint4(bf16x2_of(f[0], f[2]), bf16x2_of(f[4], f[6]), bf16x2_of(f[8], f[10]),
                                 bf16x2_of(f[12], f[14]));
    const uint4 wim = make_uint4(bf16x2_of(f[1], f[3]), bf16x2_of(f[5], f[7]), bf16x2_of(f[9], f[11]),
                                 bf16x2_of(f[13], f[15]));
    *reinterpret_cast<uint4*>(re + sl * step) = wre;
    *reinterpret_cast<uint4*>(im + sl * step) = wim;
    if (neg != nullptr)
      *reinterpret_cast<uint4*>(neg + sl * step) =
          make_uint4(wre.x ^ 0x80008000u, wre.y ^ 0x80008000u, wre.z ^ 0x80008000u, wre.w ^ 0x80008000u);
  }
}

// The same for 8 real entries: slice sl to dst + sl * step.
template <int S>
__device__ __forceinline__ void store_slices_r(const long long (&Y)[8], uint8_t* dst, int step) {
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    float f[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) f[t] = slice_digit<S>(Y[t], sl);
    *reinterpret_cast<uint4*>(dst + sl * step) =
        make_uint4(bf16x2_of(f[0], f[1]), bf16x2_of(f[2], f[3]), bf16x2_of(f[4], f[5]), bf16x2_of(f[6], f[7]));
  }
}

// Calls f(std::integral_constant<int, S>) for the slice count S in 2..6.
template <typename Fn>
__device__ __forceinline__ void with_slices(int S, Fn&& f) {
  switch (S) {
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    default: f(std::integral_constant<int, 6>{}); break;
  }
}

// v 2^sc rounded to the nearest double (ties to even) with integer
// operations only; results outside the normal range go through ldexp.
__device__ __forceinline__ double i64_scaled(long long v, int sc) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = v < 0 ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
  const int lz = __clzll(static_cast<long long>(u));
  u <<= lz;                            // leading one at bit 63
  unsigned long long mant = u >> 11;   // 53 significant bits
  const unsigned long long rest = u & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
  int E = 63 - lz + sc + 1023;
  if (mant >> 53) {
    mant >>= 1;
    ++E;
  }
  if (E <= 0 || E >= 2047) return ldexp(static_cast<double>(v), sc);
  return __longlong_as_double(
      static_cast<long long>(sign | (static_cast<unsigned long long>(E) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// Per-(front, pole) geometry of the active panel.
struct PanelDims {
  int f, s, m, bb, q0, mp;
};

__device__ __forceinline__ bool panel_dims(const DevFronts& fr, const int32_t* fronts, int fi, int p0, int b,
                                           PanelDims& d) {
  d.f = fronts[fi];
  d.s = fr.s[d.f];
  d.m = fr.m[d.f];
  if (p0 >= d.s) return false;
  d.bb = min(b, d.s - p0);
  d.q0 = p0 + d.bb;
  d.mp = d.m - d.q0;
  return d.mp > 0;
}

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- slicing
// PHASE 1 (Schur): A = L[S,P] (row i = front row q0 + i, K = the panel's bb
//   columns), B = W[S,P] (row j = column q0 + j of the stored W^T).
// PHASE 2 (panel solve L = W D^-1): A = W[S,P] by rows (where L will be
//   written; each entry is also copied to W^T in the upper triangle), B =
//   the columns of the symmetric D^-1.
// One block of 256 threads per group of 8 operand rows; grid (groups of A,
// then groups of B; fronts; poles). Pass 1: warp w finds the exponent of row
// 8g + w. Pass 2: thread (r, o) cuts the 8 entries of row 8g + r at K octet
// o into 16-byte words, per slice: Ar, Ai and -Ar for A, Br and Bi for B,
// at the place the MMA descriptors read them. Rows past the operand (inside
// the last group) and K past its end are written as zeros.
template <int PHASE>
__global__ void __launch_bounds__(256) k_oz_slice(const double2* __restrict__ /*Y*/, double2* __restrict__ F,
                                                  DevFronts fr, const int32_t* __restrict__ fronts, int p0, int b,
                                                  int S, int groupsA, OzScratch oz, int cb) {
  PanelDims d;
  if (!panel_dims(fr, fronts, blockIdx.y, p0, b, d)) return;
  const int pole = blockIdx.z;
  const bool isA = int(blockIdx.x) < groupsA;
  const int g = isA ? int(blockIdx.x) : int(blockIdx.x) - groupsA;
  const int64_t fo = int64_t(pole) * fr.pool + fr.off[d.f];
  const int K = d.bb;
  const int rows = (PHASE == 2 && !isA) ? d.bb : (isA || cb <= 0) ? d.mp : min(d.mp, min(cb, d.s) - d.q0);
  const double2* src = isA ? F + fo + d.q0 + int64_t(d.m) * p0 : F + fo + p0 + int64_t(d.m) * (PHASE == 2 ? p0 : d.q0);
  const int64_t si = isA ? 1 : d.m, sk = isA ? d.m : 1;
  const int nkt = ceil_div(K, kOzK);
  const int slice = isA ? kSliceA : kSliceB;
  uint8_t* dst = isA ? oz.A + int64_t(pole) * oz.A_stride + oz.A_off[d.f]
                     : oz.B + int64_t(pole) * oz.B_stride + oz.B_off[d.f];
  int* ex = isA ? oz.exA + int64_t(pole) * oz.exA_stride + oz.exA_off[d.f]
                : oz.exB + int64_t(pole) * oz.exB_stride + oz.exB_off[d.f];
  if (g * 8 >= rows) return;

  __shared__ int s_e[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const int i = g * 8 + warp;
    uint32_t mx = 0;  // largest high word of |re|, |im|: carries the largest exponent
    if (i < rows)
      for (int k = lane; k < K; k += 32) {
        const double2 v = src[int64_t(i) * si + int64_t(k) * sk];
        mx = max(mx, max(uint32_t(__double2hiint(v.x)) & 0x7FFFFFFFu, uint32_t(__double2hiint(v.y)) & 0x7FFFFFFFu));
      }
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    int e = 0;  // 2^e > max |entry|
    if (mx >= 0x7FF00000u)
      e = kNanExp;
    else if (mx != 0)
      e = int(mx >> 20) - 1022;
    if (lane == 0) {
      s_e[warp] = e;
      if (i < rows) ex[i] = e;
    }
  }
  __syncthreads();

  const int r = threadIdx.x & 7;
  const int i = g * 8 + r;
  const int e = s_e[r];
  // row tile i / 64; inside it, the 8-row group of i and row i % 8
  uint8_t* rowbase = dst + int64_t(i / kOzRows) * nkt * S * slice + ((i % kOzRows) >> 3) * 512 + r * 16;
  const double2* row = src + int64_t(i) * si;
  const long long bias = digit_bias(S);
  const double scale = fma_scale(e, S);
  for (int o = threadIdx.x >> 3; o < nkt * (kOzK / 8); o += 32) {
    long long Y[16];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = o * 8 + u;
      double2 v = make_double2(0.0, 0.0);
      if (i < rows && k < K) {
        v = row[int64_t(k) * sk];
        if (PHASE == 2 && isA) F[fo + p0 + int64_t(d.m) * (d.q0 + i) + k] = v;  // W^T (rows p0.., column q0 + i)
      }
      Y[2 * u] = fixed_of(v.x, scale, e, S) + bias;
      Y[2 * u + 1] = fixed_point(v.y, e, S) + bias;
    }
    uint8_t* p = rowbase + int64_t(o >> 2) * S * slice + (o & 3) * 128;
    with_slices(S, [&](auto SC) {
      if (isA)  // slice s: Ar, Ai, -Ar
        store_slices_c<decltype(SC)::value>(Y, p, p + kBlk, p + 2 * kBlk, slice);
      else  // Br of slices 1..S, then Bi of slices 1..S
        store_slices_c<decltype(SC)::value>(Y, p, p + S * kBlk, nullptr, kBlk);
    });
  }
}

// Real operands (LDL^T of H - sigma S for inertia counts), PHASE 1 (Schur):
// A = L[S,P] rows (tiles of 128 rows), B = W[S,P] rows (tiles of 64 rows);
// PHASE 2 (panel solve): A = W[S,P] rows (copied to W^T on the way), B = the
// columns of D^-1; K = the panel's bb columns; one 16-byte word per slice and
// row octet, in the same core-matrix layout (a slice of A is two 64-row
// blocks, one of B is one block). Grid and passes as k_oz_slice.
template <int PHASE>
__global__ void __launch_bounds__(256) k_oz_slice_real(double* __restrict__ F, DevFronts fr,
                                                       const int32_t* __restrict__ fronts, int p0, int b, int S,
                                                       int groupsA, OzScratch oz, int cb) {
  PanelDims d;
  if (!panel_dims(fr, fronts, blockIdx.y, p0, b, d)) return;
  const int pole = blockIdx.z;
  const bool isA = int(blockIdx.x) < groupsA;
  const int g = isA ? int(blockIdx.x) : int(blockIdx.x) - groupsA;
  const int64_t fo = int64_t(pole) * fr.pool + fr.off[d.f];
  const int rows = (PHASE == 2 && !isA) ? d.bb : (isA || cb <= 0) ? d.mp : min(d.mp, min(cb, d.s) - d.q0);
  const int K = d.bb, nkt = ceil_div(K, kOzK);
  const double* src = isA ? F + fo + d.q0 + int64_t(d.m) * p0 : F + fo + p0 + int64_t(d.m) * (PHASE == 2 ? p0 : d.q0);
  const int64_t si = isA ? 1 : d.m, sk = isA ? d.m : 1;
  const int R = isA ? 2 * kOzRows : kOzRows;
  const int slice = isA ? 2 * kBlk : kBlk;
  uint8_t* dst = isA ? oz.A + int64_t(pole) * oz.A_stride + oz.A_off[d.f]
                     : oz.B + int64_t(pole) * oz.B_stride + oz.B_off[d.f];
  int* ex = isA ? oz.exA + int64_t(pole) * oz.exA_stride + oz.exA_off[d.f]
                : oz.exB + int64_t(pole) * oz.exB_stride + oz.exB_off[d.f];
  if (g * 8 >= rows) return;

  __shared__ int s_e[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const int i = g * 8 + warp;
    uint32_t mx = 0;
    if (i < rows)
      for (int k = lane; k < K; k += 32)
        mx = max(mx, uint32_t(__double2hiint(src[int64_t(i) * si + int64_t(k) * sk])) & 0x7FFFFFFFu);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    int e = 0;
    if (mx >= 0x7FF00000u)
      e = kNanExp;
    else if (mx != 0)
      e = int(mx >> 20) - 1022;
    if (lane == 0) {
      s_e[warp] = e;
      if (i < rows) ex[i] = e;
    }
  }
  __syncthreads();

  const int r = threadIdx.x & 7;
  const int i = g * 8 + r;
  const int e = s_e[r];
  uint8_t* rowbase = dst + int64_t(i / R) * nkt * S * slice + ((i % R) >> 3) * 512 + r * 16;
  const double* row = src + int64_t(i) * si;
  const long long bias = digit_bias(S);
  const double scale = fma_scale(e, S);
  for (int o = threadIdx.x >> 3; o < nkt * (kOzK / 8); o += 32) {
    long long Y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = o * 8 + u;
      double v = 0.0;
      if (i < rows && k < K) {
        v = row[int64_t(k) * sk];
        if (PHASE == 2 && isA) F[fo + p0 + int64_t(d.m) * (d.q0 + i) + k] = v;  // W^T into the upper triangle
      }
      Y[u] = ((u & 1) ? fixed_point(v, e, S) : fixed_of(v, scale, e, S)) + bias;
    }
    uint8_t* p = rowbase + int64_t(o >> 2) * S * slice + (o & 3) * 128;
    with_slices(S, [&](auto SC) { store_slices_r<decltype(SC)::value>(Y, p, slice); });
  }
}

// Where a wait ran out: site (1..8) + 16 * (K tile mod 16), below 256; the
// launch reports 1 + (mode << 28) + (this << 20) + CTA index, mode 1-3 for the
// short-K GEMM (its MODE), 0 for the Takahashi / Y[P,P] kernel.
__device__ __forceinline__ void record_fail(int* s_fail, int site, int kt) {
  atomicCAS(s_fail, 0, site + 16 * (kt & 15));
}

// ---------------------------------------------------------------- GEMM (short K)
// Output tiles of one front at the active panel (m_p rows below it); MODE 3
// only the first cs columns (the rest of the panel block).
template <int MODE, bool CPLX>
__host__ __device__ inline int front_tiles(int mp, int cs) {
  if (mp <= 0) return 0;
  if (MODE == 2) return ceil_div(mp, CPLX ? kOzRows : 2 * kOzRows);
  if (MODE == 3) {  // column tiles nt < nc, row tiles on and below the diagonal
    const int nnt = ceil_div(mp, kOzRows), nc = cs <= 0 ? 0 : min(nnt, ceil_div(cs, kOzRows));
    if (CPLX) return nc * nnt - nc * (nc - 1) / 2;
    const int nmt = ceil_div(mp, 2 * kOzRows);
    int t = 0;
    for (int nt = 0; nt < nc; ++nt) t += nmt - nt / 2;
    return t;
  }
  if (CPLX) {
    const int n = ceil_div(mp, kOzRows);
    return n * (n + 1) / 2;  // 64 x 64 tiles on and below the diagonal
  }
  const int nmt = ceil_div(mp, 2 * kOzRows), nnt = ceil_div(mp, kOzRows);
  return nmt * (nmt + 1) - (2 * nmt - nnt);  // 128 x 64 tiles: 2r + 2 in row r, fewer in the last
}

// Row tile mt and column tile nt of tile t of a front.
template <int MODE, bool CPLX>
__device__ __forceinline__ void tile_coords(int t, int mp, int& mt, int& nt) {
  if (MODE == 2) {
    mt = t;
    nt = 0;
  } else if (MODE == 3) {  // column by column: column nt holds the row tiles from the diagonal down
    const int first_of = CPLX ? 0 : 1;  // real tiles: 128 rows, so row tile nt / 2 holds the diagonal
    const int nrows = CPLX ? ceil_div(mp, kOzRows) : ceil_div(mp, 2 * kOzRows);
    nt = 0;
    while (t >= nrows - (first_of ? nt / 2 : nt)) {
      t -= nrows - (first_of ? nt / 2 : nt);
      ++nt;
    }
    mt = (first_of ? nt / 2 : nt) + t;
  } else if (CPLX) {  // t = mt (mt + 1) / 2 + nt, nt <= mt
    mt = int((sqrtf(8.0f * float(t) + 1.0f) - 1.0f) * 0.5f);
    while (mt * (mt + 1) / 2 > t) --mt;
    while ((mt + 1) * (mt + 2) / 2 <= t) ++mt;
    nt = t - mt * (mt + 1) / 2;
  } else {  // t = mt (mt + 1) + nt, nt <= 2 mt + 1
    mt = int((sqrtf(4.0f * float(t) + 1.0f) - 1.0f) * 0.5f);
    while (mt * (mt + 1) > t) --mt;
    while ((mt + 1) * (mt + 2) <= t) ++mt;
    nt = t - mt * (mt + 1);
  }
}

// MODE 1, Schur update F[S,S] -= A B^T on the lower triangle, A = L[S,P],
//   B = W[S,P] (K = bb <= 64); complex 64 x 64 tiles or real 128 x 64 tiles.
// MODE 2, panel solve L[S,P] = A B^T with A = W[S,P] and B = D^-1, written
//   where W was; one tile per row tile of S.
// MODE 3, MODE 1 restricted to the columns before min(cb, s): the update of
//   the rest of a block of panels, whose update of the columns after the
//   block waits for one MODE 1 launch over the whole block (K up to 256).
// Persistent: each CTA walks the (pole, front, tile) items of the launch with
// stride gridDim.x. The slot rings run on across items, so the next tile's
// slices load during this tile's MMAs; the epilogue warps drain TMEM into
// registers and release it at once, so the next tile's MMAs overlap this
// tile's global read-modify-write. Warps 0-7 epilogue, warp 8 producer, warp
// 9 MMA issuer (and TMEM owner).
template <int MODE, bool CPLX>
__global__ void __launch_bounds__(kGemmThreads, 1) k_oz_gemm(void* __restrict__ Yv, DevFronts fr,
                                                             const int32_t* __restrict__ fronts, int nfronts, int p0,
                                                             int b, int S, int nb, OzScratch oz, int cb) {
  extern __shared__ __align__(128) uint8_t osm[];
  __shared__ __align__(8) uint64_t full_a[kSlotsA], empty_a[kSlotsA], full_b[kSlotsB], empty_b[kSlotsB];
  __shared__ __align__(8) uint64_t acc_full, acc_empty, mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  constexpr int TR = CPLX ? kOzRows : 2 * kOzRows;  // output rows per tile
  constexpr int SA = CPLX ? kSliceA : 2 * kBlk;     // bytes of one slice of A (one K tile)
  constexpr int SB = CPLX ? kSliceB : kBlk;         // bytes of one slice of B (one K tile: Br, Bi; or Br)
  constexpr bool SCHUR = MODE != 2;                  // read-modify-write of the trailing block
  // An earlier CTA gave up (the result is void anyway): the whole CTA leaves
  // together, on one read of the flag, before any barrier or TMEM is set up.
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = *static_cast<volatile int*>(oz.fail);
  __syncthreads();
  if (s_skip) return;
  uint8_t* sA = osm;                                 // kSlotsA x one slice of A (Ar, Ai, -Ar; or Ar)
  uint8_t* sB = osm + kSlotsA * kSliceA;             // kSlotsB x S slices of B (Br, Bi; or Br)
  int* s_pref = reinterpret_cast<int*>(sB + kSlotsB * 6 * kSliceB);  // tiles before front f
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* fail = &s_fail;

  if (warp == 0) {  // prefix sums of the fronts' tile counts
    int carry = 0;
    if (lane == 0) s_pref[0] = 0;
    for (int f0 = 0; f0 < nfronts; f0 += 32) {
      int v = 0;
      if (f0 + lane < nfronts) {
        PanelDims d;
        v = panel_dims(fr, fronts, f0 + lane, p0, b, d) ? front_tiles<MODE, CPLX>(d.mp, min(cb, d.s) - d.q0) : 0;
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += u;
      }
      if (f0 + lane < nfronts) s_pref[f0 + lane + 1] = carry + v;
      carry += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int j = 0; j < kSlotsA; ++j) {
      bar_init(smem_u32(&full_a[j]), 1);
      bar_init(smem_u32(&empty_a[j]), 1);
    }
    for (int j = 0; j < kSlotsB; ++j) {
      bar_init(smem_u32(&full_b[j]), 1);
      bar_init(smem_u32(&empty_b[j]), 1);
    }
    bar_init(smem_u32(&acc_full), 1);
    bar_init(smem_u32(&acc_empty), kEpiWarps);
    bar_init(smem_u32(&mma_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == kEpiWarps + 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const int T = s_pref[nfronts];
  const int items = T * nb;

  // item -> (pole, front, tile): binary search of the prefix sums
  auto decode = [&](int it, int& pole, PanelDims& d, int& mt, int& nt) -> bool {
    pole = it / T;
    const int t = it - pole * T;
    int lo = 0, hi = nfronts;  // largest f with s_pref[f] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_pref[mid] <= t) lo = mid;
      else hi = mid;
    }
    if (!panel_dims(fr, fronts, lo, p0, b, d)) return false;
    tile_coords<MODE, CPLX>(t - s_pref[lo], d.mp, mt, nt);
    return true;
  };

  if (warp == kEpiWarps) {
    if (lane == 0) {  // ---- producer
      int na = 0, nbf = 0;
      // fault injection (testing the timeout path): CTA 0 issues no copy, so
      // the MMA issuer's first wait runs out and the launch reports it
      bool ok = !(oz.stall && blockIdx.x == 0);
      for (int it = blockIdx.x; it < items && ok && !*fail; it += gridDim.x) {
        int pole, mt, nt;
        PanelDims d;
        if (!decode(it, pole, d, mt, nt)) continue;
        const int nkt = ceil_div(d.bb, kOzK);
        const uint8_t* gA = oz.A + int64_t(pole) * oz.A_stride + oz.A_off[d.f] + int64_t(mt) * nkt * S * SA;
        const uint8_t* gB = oz.B + int64_t(pole) * oz.B_stride + oz.B_off[d.f] + int64_t(nt) * nkt * S * SB;
        for (int kt = 0; kt < nkt && ok; ++kt) {
          const int sb = nbf % kSlotsB, ub = nbf / kSlotsB;
          if (ub > 0 && !bar_wait(smem_u32(&empty_b[sb]), (ub - 1) & 1, fail, oz.wait_ns)) {
            record_fail(&s_fail, 1, kt);
            ok = false;
            break;
          }
          bar_expect(smem_u32(&full_b[sb]), uint32_t(S * SB));
          bulk_load(smem_u32(sB + sb * 6 * kSliceB), gB + int64_t(kt) * S * SB, uint32_t(S * SB),
                    smem_u32(&full_b[sb]));
          ++nbf;
          for (int s = 0; s < S; ++s) {
            const int sa = na % kSlotsA, ua = na / kSlotsA;
            if (ua > 0 && !bar_wait(smem_u32(&empty_a[sa]), (ua - 1) & 1, fail, oz.wait_ns)) {
              record_fail(&s_fail, 2, kt);
              ok = false;
              break;
            }
            bar_expect(smem_u32(&full_a[sa]), uint32_t(SA));
            bulk_load(smem_u32(sA + sa * kSliceA), gA + (int64_t(kt) * S + s) * SA, uint32_t(SA),
                      smem_u32(&full_a[sa]));
            ++na;
          }
        }
      }
      // every copy issued has landed before the CTA leaves (bounded)
      for (int j = 0; j < kSlotsA; ++j)
        if (na > j && !bar_wait_all(smem_u32(&full_a[j]), ((na - 1 - j) / kSlotsA) & 1)) record_fail(&s_fail, 3, 0);
      for (int j = 0; j < kSlotsB; ++j)
        if (nbf > j && !bar_wait_all(smem_u32(&full_b[j]), ((nbf - 1 - j) / kSlotsB) & 1)) record_fail(&s_fail, 3, 1);
    }
  } else if (warp == kEpiWarps + 1) {
    if (lane == 0) {  // ---- MMA issuer
      int na = 0, nbf = 0, ti = 0;
      bool ok = true;
      // one instance per slice count: the slices of a K tile are issued as
      // straight-line code with constant descriptor offsets
      with_slices(S, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
          int pole, mt, nt;
          PanelDims d;
          if (!decode(it, pole, d, mt, nt)) continue;
          const int nkt = ceil_div(d.bb, kOzK);
          if (ti > 0 && !bar_wait(smem_u32(&acc_empty), (ti - 1) & 1, fail, oz.wait_ns)) {  // previous tile drained
            record_fail(&s_fail, 4, 0);
            ok = false;
            break;
          }
          for (int kt = 0; kt < nkt && ok; ++kt) {
            const int sb = nbf % kSlotsB;
            if (!bar_wait(smem_u32(&full_b[sb]), (nbf / kSlotsB) & 1, fail, oz.wait_ns)) {
              record_fail(&s_fail, 5, kt);
              ok = false;
              break;
            }
            // Br slices 1..S, then Bi slices 1..S
            const uint64_t br = sdesc(smem_u32(sB + sb * 6 * kSliceB)), bi = desc_off(br, SS * kBlk / 16);
#pragma unroll
            for (int s = 1; s <= SS; ++s) {
              const int sa = na % kSlotsA;
              if (!bar_wait(smem_u32(&full_a[sa]), (na / kSlotsA) & 1, fail, oz.wait_ns)) {
                record_fail(&s_fail, 6, kt);
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
              const uint64_t a1 = sdesc(smem_u32(sA + sa * kSliceA));  // [Ar; Ai], then [Ai; -Ar] (or 128 real rows)
              // the first product into each accumulator of a tile overwrites
              // it: for diagonal D that is the pair (1, D - 1) at the first K step
              mma_slice<CPLX, kOzK / 16, kBlk>(SS + 1 - s, tmem + uint32_t((s - 1) * 64), a1, desc_off(a1, kBlk / 16), br,
                                               bi, (kt == 0 && s == 1) ? 0u : 1u);
              mma_commit(smem_u32(&empty_a[sa]));
              ++na;
            }
            if (!ok) break;
            mma_commit(smem_u32(&empty_b[sb]));
            ++nbf;
          }
          if (!ok) break;
          mma_commit(smem_u32(&acc_full));
          ++ti;
        }
      });
      // every MMA issued has completed before TMEM is read for the last time or freed
      mma_commit(smem_u32(&mma_done));
      if (!bar_wait_all(smem_u32(&mma_done), 0)) record_fail(&s_fail, 7, 0);
    }
  } else {  // ---- epilogue: exact FP32 integers -> 64-bit integers -> FP64 outputs
    const int q = warp & 3, h = (warp >> 2) & 1;
    // complex: lanes 0-63 hold real parts, 64-127 imaginary parts of the
    // tile's 64 complex rows; real: lane = row of the 128-row tile
    const int ri = CPLX ? (q & 1) * 32 + lane : q * 32 + lane;
    const int part = CPLX ? q >> 1 : 0;
    constexpr int ES = CPLX ? 2 : 1;  // doubles per element
    int ti = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      int pole, mt, nt;
      PanelDims d;
      if (!decode(it, pole, d, mt, nt)) continue;
      const int i = mt * TR + ri;  // row of the trailing block
      const bool row_in = i < d.mp;
      double* Yb = static_cast<double*>(Yv) + ES * (int64_t(pole) * fr.pool + fr.off[d.f]) + part;
      // the exponents are requested before the accumulators are ready; the
      // exponent of column h*32 + lane is broadcast by shuffles below (every
      // lane takes part; the row test only guards memory accesses)
      const int jl = nt * kOzRows + h * 32 + lane;
      // Schur columns: j <= i below the panel, MODE 3 only before the block end
      const int jmax = MODE == 2 ? d.bb : MODE == 3 ? min(d.mp, min(cb, d.s) - d.q0) : d.mp;
      const int eb_lane = jl < jmax ? oz.exB[int64_t(pole) * oz.exB_stride + oz.exB_off[d.f] + jl] : 0;
      const int ea = row_in ? oz.exA[int64_t(pole) * oz.exA_stride + oz.exA_off[d.f] + i] : 0;
      bool ok = true;
      if (lane == 0) ok = bar_wait(smem_u32(&acc_full), ti & 1, fail, oz.wait_ns);
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) record_fail(&s_fail, 8, ti);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned long long acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = 0ull;
      for (int D = 2; D <= S + 1; ++D) {  // one TMEM round trip per diagonal
        const int sh = 7 * (S + 1 - D);
        uint32_t v[32];
        tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t((D - 2) * 64 + h * 32), v);
#pragma unroll
        for (int c = 0; c < 32; ++c)
          acc[c] += static_cast<unsigned long long>(static_cast<long long>(__float2int_rn(__uint_as_float(v[c])))) << sh;
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) bar_arrive(smem_u32(&acc_empty));  // TMEM free for the next tile
      ++ti;
      // Schur: the old values of 16 columns are loaded before any of them is
      // stored, so that their loads are in flight together
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        double old[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = nt * kOzRows + h * 32 + c0 + c;
          const bool in = row_in && j < jmax && (!SCHUR || j <= i);
          old[c] = (SCHUR && in) ? Yb[ES * ((d.q0 + i) + int64_t(d.m) * (d.q0 + j))] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = nt * kOzRows + h * 32 + c0 + c;
          const bool in = row_in && j < jmax && (!SCHUR || j <= i);
          const int ebc = __shfl_sync(0xFFFFFFFFu, eb_lane, c0 + c);
          if (in) {
            double v = i64_scaled(static_cast<long long>(acc[c0 + c]), ea + ebc - 7 * (S + 1));
            if (ea == kNanExp || ebc == kNanExp) v = __longlong_as_double(0x7FF8000000000000LL);
            if (SCHUR)
              Yb[ES * ((d.q0 + i) + int64_t(d.m) * (d.q0 + j))] = old[c] - v;
            else
              Yb[ES * ((d.q0 + i) + int64_t(d.m) * (p0 + j))] = v;
          }
        }
      }
    }
  }

  __syncthreads();
  if (s_fail && threadIdx.x == 0)  // where the wait gave up: mode, site + 16 * K tile, CTA
    atomicMax(oz.fail, 1 + (MODE << 28) + (min(s_fail, 255) << 20) + min(int(blockIdx.x), (1 << 20) - 1));
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == kEpiWarps + 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------- fused Takahashi step
// Y[S,P] = -Y[S,S] L[S,P] with A = Y[S,S] sliced on the fly: the worker warps
// read the FP64 trailing block straight from the front and write its slices
// into shared memory, so A never makes a round trip through HBM as slices
// (16 B per complex entry read once, instead of 16 B read, 36 B written and
// 36 B read again). Row exponents of A and the slices of B = L[S,P] come from
// k_oz_tak_prep. K tiles of 16; a ring of three slots, each holding all S
// slices of A (6 KiB each: Ar, Ai, -Ar) and of B (Br of slices 1..S, then
// Bi of slices 1..S, 2 KiB each).
constexpr int kFK = 16;                     // K per tile
constexpr int kFBlk = kOzRows * kFK * 2;    // one 64-row block of one slice (2 KiB)
constexpr int kFSliceA = 3 * kFBlk;
constexpr int kFSliceB = 2 * kFBlk;
constexpr int kFSlots = 3;
constexpr int kFSlotA = 6 * kFSliceA;       // A part of a slot (S <= 6)
constexpr int kFSlot = kFSlotA + 6 * kFSliceB;
constexpr int kFChunk = 256 / kFK;          // K tiles per exact chunk
constexpr int kFWorkers = 8;
constexpr int kFThreads = (kFWorkers + 1) * 32;
constexpr int kFSmem = kFSlots * kFSlot;

// Row exponents of A = Y[S,S] from the row maxima of Y (A groups, 256 rows
// each) and the slices of B = L[S,P] in the 16-deep tile layout (B groups, 8
// rows each); grid (groups of A, then of B; fronts; poles).
__global__ void __launch_bounds__(256) k_oz_tak_prep(const double2* __restrict__ /*Y*/, const double2* __restrict__ F,
                                                     DevFronts fr, const int32_t* __restrict__ fronts, int p0, int b,
                                                     int S, int groupsA, OzScratch oz) {
  PanelDims d;
  if (!panel_dims(fr, fronts, blockIdx.y, p0, b, d)) return;
  const int pole = blockIdx.z;
  const bool isA = int(blockIdx.x) < groupsA;
  const int g = isA ? int(blockIdx.x) : int(blockIdx.x) - groupsA;
  const int64_t fo = int64_t(pole) * fr.pool + fr.off[d.f];
  if (isA) {  // rows of Y[S,S]: from the row maxima kept up to date as Y is written
    const int i = g * 256 + int(threadIdx.x);
    if (i < d.mp)
      oz.exA[int64_t(pole) * oz.exA_stride + oz.exA_off[d.f] + i] =
          exp_of_hi(oz.ymax[int64_t(pole) * oz.ymax_stride + oz.ymax_off[d.f] + d.q0 + i]);
    return;
  }
  const double2* src = F + fo + int64_t(p0) * d.m + d.q0;
  const int rows = d.bb, K = d.mp;
  int* ex = oz.exB + int64_t(pole) * oz.exB_stride + oz.exB_off[d.f];
  if (g * 8 >= rows) return;
  __shared__ int s_e[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const int i = g * 8 + warp;
    uint32_t mx = 0;
    if (i < rows)
      for (int k = lane; k < K; k += 32) {
        const double2 v = src[int64_t(i) * d.m + k];
        mx = max(mx, max(uint32_t(__double2hiint(v.x)) & 0x7FFFFFFFu, uint32_t(__double2hiint(v.y)) & 0x7FFFFFFFu));
      }
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    int e = 0;
    if (mx >= 0x7FF00000u)
      e = kNanExp;
    else if (mx != 0)
      e = int(mx >> 20) - 1022;
    if (lane == 0) {
      s_e[warp] = e;
      if (i < rows) ex[i] = e;
    }
  }
  __syncthreads();
  const int r = threadIdx.x & 7;
  const int j = g * 8 + r;
  const int e = s_e[r];
  const int nkt = ceil_div(K, kFK);
  uint8_t* rowbase = oz.B + int64_t(pole) * oz.B_stride + oz.B_off[d.f] + (j >> 3) * 256 + r * 16;
  const double2* row = src + int64_t(j) * d.m;
  const long long bias = digit_bias(S);
  const double scale = fma_scale(e, S);
  for (int o = threadIdx.x >> 3; o < nkt * (kFK / 8); o += 32) {
    long long Y[16];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = o * 8 + u;
      const double2 v = (j < rows && k < K) ? row[k] : make_double2(0.0, 0.0);
      Y[2 * u] = fixed_of(v.x, scale, e, S) + bias;
      Y[2 * u + 1] = fixed_point(v.y, e, S) + bias;
    }
    uint8_t* p = rowbase + int64_t(o >> 1) * S * kFSliceB + (o & 1) * 128;  // Br slices 1..S, then Bi
    with_slices(S, [&](auto SC) { store_slices_c<decltype(SC)::value>(Y, p, p + S * kFBlk, nullptr, kFBlk); });
  }
}

// Row maxima of Y when a front's selected inversion starts: rows of the update
// set U = [s, m) over the columns of U (Y[U,U] as gathered from the parent; Y
// is symmetric, so row r is read as column r), 0 for the rows of the
// supernode, whose columns are computed later. One warp per row; grid (rows /
// 8, fronts, poles).
__global__ void __launch_bounds__(256) k_oz_rowmax_init(const double2* __restrict__ Y, DevFronts fr,
                                                        const int32_t* __restrict__ fronts, OzScratch oz) {
  const int f = fronts[blockIdx.y];
  const int s = fr.s[f], m = fr.m[f];
  const int r = int(blockIdx.x) * 8 + int(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= m) return;  // whole warps
  const int pole = blockIdx.z;
  uint32_t mx = 0;
  if (r >= s) {
    const double2* col = Y + int64_t(pole) * fr.pool + fr.off[f] + int64_t(m) * r;
    for (int c = s + lane; c < m; c += 32) {
      const double2 v = col[c];
      mx = max(mx, max(abs_hi(v.x), abs_hi(v.y)));
    }
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  }
  if (lane == 0) oz.ymax[int64_t(pole) * oz.ymax_stride + oz.ymax_off[f] + r] = mx;
}

// KIND 0, Takahashi step: one CTA per 64-row tile of S (front, pole); A =
//   Y[S,S] rows cut on the fly, B = L[S,P] slices staged by k_oz_tak_prep;
//   its epilogue writes Y[S,P] and Y[P,S] and raises the row maxima of Y
//   (rows S, and by a warp reduction over its rows, rows P).
// KIND 1, the product L[S,P]^T Y[S,P] of Y[P,P] = D^-1 - L[S,P]^T Y[S,P]:
//   one CTA per 256-deep K range (front, pole); A = L[S,P] columns and B =
//   Y[S,P] columns both cut on the fly; the exact int64 sums of the range go
//   to `part` and k_oz_dpart_reduce adds the ranges.
// Warps 0-7: workers (warps 0-3 produce the even K tiles, 4-7 the odd ones:
// thread (row r, octet o) cuts 8 entries of row r into S x 3 words of A (and
// for KIND 1, S x 2 words of B); every warp also drains its part of TMEM
// after each chunk); warp 8: TMEM owner and MMA issuer.
template <int KIND>
__global__ void __launch_bounds__(kFThreads, 1) k_oz_tak_fused(double2* __restrict__ Y, DevFronts fr,
                                                              const int32_t* __restrict__ fronts, int p0, int b,
                                                              int S, OzScratch oz, const double2* __restrict__ F,
                                                              long long* __restrict__ part,
                                                              const int64_t* __restrict__ part_off, int64_t part_stride) {
  constexpr bool DP = KIND == 1;
  extern __shared__ __align__(128) uint8_t osm[];
  __shared__ __align__(8) uint64_t full_a[kFSlots], full_b[kFSlots], empty[kFSlots];
  __shared__ __align__(8) uint64_t acc_full, acc_empty, mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ int s_last_b[kFSlots];
  __shared__ int s_ea[kOzRows], s_eb[kOzRows];
  PanelDims d;
  if (!panel_dims(fr, fronts, blockIdx.y, p0, b, d)) return;
  // an earlier CTA gave up: leave together, on one read of the flag
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = *static_cast<volatile int*>(oz.fail);
  __syncthreads();
  if (s_skip) return;
  const int mt = DP ? 0 : int(blockIdx.x);
  if (DP ? int(blockIdx.x) * kFChunk >= ceil_div(d.mp, kFK) : mt >= ceil_div(d.mp, kOzRows)) return;
  const int pole = blockIdx.z;
  // K tiles kt0 .. kt0 + nkt - 1 (KIND 1: one 256-deep range per CTA)
  const int kt0 = DP ? int(blockIdx.x) * kFChunk : 0;
  const int nkt = DP ? min(kFChunk, ceil_div(d.mp, kFK) - kt0) : ceil_div(d.mp, kFK);
  const int nchunks = ceil_div(nkt, kFChunk);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* fail = &s_fail;
  const uint8_t* gB = oz.B + int64_t(pole) * oz.B_stride + oz.B_off[d.f];

  if (threadIdx.x < 2 * kOzRows) {
    const int* exa = oz.exA + int64_t(pole) * oz.exA_stride + oz.exA_off[d.f];
    const int* exb = oz.exB + int64_t(pole) * oz.exB_stride + oz.exB_off[d.f];
    if (threadIdx.x < kOzRows) {  // rows of A: Y[S,S] rows, or L[S,P] columns
      const int i = mt * kOzRows + threadIdx.x;
      s_ea[threadIdx.x] = DP ? (i < d.bb ? exb[i] : 0) : (i < d.mp ? exa[i] : 0);
    } else {  // rows of B: L[S,P] columns, or Y[S,P] columns
      const int j = threadIdx.x - kOzRows;
      s_eb[j] = j < d.bb ? (DP ? exa[j] : exb[j]) : 0;
    }
  }
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int j = 0; j < kFSlots; ++j) {
      bar_init(smem_u32(&full_a[j]), 4 * 32);  // the producing half: 128 threads
      bar_init(smem_u32(&full_b[j]), 1);
      bar_init(smem_u32(&empty[j]), 1);
      s_last_b[j] = -1;
    }
    bar_init(smem_u32(&acc_full), 1);
    bar_init(smem_u32(&acc_empty), kFWorkers);
    bar_init(smem_u32(&mma_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == kFWorkers) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const bool multi = !DP && nchunks > kOzFlush;

  const int q = warp & 3, h = (warp >> 2) & 1;
  // this warp's exact int64 partial sums live in TMEM columns 384 + 64 h ..
  // (lo, hi words of column c at 2c, 2c + 1), next to the six accumulators
  const uint32_t tsum = tmem + (uint32_t(q * 32) << 16) + uint32_t(6 * 64 + h * 64);
  // output row of this thread's TMEM lane (real part in lanes 0-63, imaginary in 64-127)
  const int orow = mt * kOzRows + (q & 1) * 32 + lane;
  double* Yout = reinterpret_cast<double*>(Y + int64_t(pole) * fr.pool + fr.off[d.f]) + (q >> 1);

  if (warp == kFWorkers) {
    if (lane == 0) {  // ---- MMA issuer
      // one instance per slice count: every descriptor offset is a constant
      with_slices(S, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        for (int kt = 0; kt < nkt; ++kt) {
          const int c = kt / kFChunk, in_chunk = kt % kFChunk;
          if (in_chunk == 0 && c > 0 && !bar_wait(smem_u32(&acc_empty), (c - 1) & 1, fail, oz.wait_ns)) {
            record_fail(&s_fail, 4, kt);
            break;
          }
          const int slot = kt % kFSlots;
          const uint32_t par = (kt / kFSlots) & 1;
          if (!bar_wait(smem_u32(&full_a[slot]), par, fail, oz.wait_ns) || (!DP && !bar_wait(smem_u32(&full_b[slot]), par, fail, oz.wait_ns))) {
            record_fail(&s_fail, 6, kt);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t da = sdesc16(smem_u32(osm + slot * kFSlot)), db = desc_off(da, kFSlotA / 16);
#pragma unroll
          for (int s = 1; s <= SS; ++s) {  // [Ar; Ai], then [Ai; -Ar] of slice s; Br 1..S, then Bi 1..S
            const uint64_t a1 = desc_off(da, (s - 1) * kFSliceA / 16);
            mma_slice<true, 1, kFBlk>(SS + 1 - s, tmem + uint32_t((s - 1) * 64), a1, desc_off(a1, kFBlk / 16), db,
                                      desc_off(db, SS * kFBlk / 16), (in_chunk == 0 && s == 1) ? 0u : 1u);
          }
          mma_commit(smem_u32(&empty[slot]));
          if (in_chunk == kFChunk - 1 || kt == nkt - 1) mma_commit(smem_u32(&acc_full));
        }
      });
      mma_commit(smem_u32(&mma_done));
      if (!bar_wait_all(smem_u32(&mma_done), 0)) record_fail(&s_fail, 7, 0);
    }
  } else {  // ---- workers: produce A slices, drain TMEM after each chunk
    const int half = warp >> 2;
    const int item = q * 32 + lane;        // 0..127
    const int r = item & (kOzRows - 1), oct = item >> 6;
    const int i = mt * kOzRows + r;
    const bool rowok = DP ? r < d.bb : i < d.mp;
    const int e = s_ea[r], eB = s_eb[r];
    const int64_t fo = int64_t(pole) * fr.pool + fr.off[d.f];
    // A row: KIND 0 column q0 + i of Y (rows q0..), KIND 1 panel column p0 + r of L
    const double2* col = DP ? F + fo + int64_t(p0 + (rowok ? r : 0)) * d.m + d.q0
                            : Y + fo + int64_t(d.q0 + (rowok ? i : 0)) * d.m + d.q0;
    // B row (KIND 1): panel column p0 + r of Y, rows q0..
    const double2* colB = Y + fo + int64_t(p0 + (rowok ? r : 0)) * d.m + d.q0;
    const uint32_t wbase = uint32_t((r >> 3) * 256 + oct * 128 + (r & 7) * 16);
    const long long bias = digit_bias(S);
    const double scale = fma_scale(e, S);
    int drained = 0, pending = 0;
    bool ok = true;
    auto drain = [&](int ch) -> bool {
      bool got = true;
      if (lane == 0) got = bar_wait(smem_u32(&acc_full), ch & 1, fail, oz.wait_ns);
      got = __shfl_sync(0xFFFFFFFFu, got, 0);
      if (!got) {
        if (lane == 0) record_fail(&s_fail, 8, ch * kFChunk);
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool flush = multi && pending + 1 == kOzFlush && ch != nchunks - 1;
#pragma unroll 1
      for (int hh = 0; hh < 4; ++hh) {  // 8 output columns at a time
        uint32_t w[16];
        // the partial sum and every diagonal's 8 columns in one TMEM round trip
        with_slices(S, [&](auto SC) {
          constexpr int SS = decltype(SC)::value;
          uint32_t v[SS][8];
          if (pending > 0) tmem_ld16_nw(tsum + hh * 16, w);
          const uint32_t ta = tmem + (uint32_t(q * 32) << 16) + uint32_t(h * 32 + hh * 8);
#pragma unroll
          for (int t = 0; t < SS; ++t) tmem_ld8_nw(ta + uint32_t(t * 64), v[t]);
          tmem_wait_ld();
          if (pending == 0) {
#pragma unroll
            for (int c = 0; c < 16; ++c) w[c] = 0u;
          }
          acc_add_diags8<SS>(w, v);  // diagonal D at columns 64 (D - 2)
        });
        if (flush) {
          // K > 2048: move the exact partial sum into this thread's own
          // Y[S,P] entries (rounded once), which no operand of the launch reads
          if (orow < d.mp) {
            const int ea = s_ea[orow - mt * kOzRows];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const int j = h * 32 + hh * 8 + c;
              if (j < d.bb) {
                double* o = Yout + 2 * ((d.q0 + orow) + int64_t(d.m) * (p0 + j));
                const long long a64 = static_cast<long long>((static_cast<unsigned long long>(w[2 * c + 1]) << 32) | w[2 * c]);
                const double v = i64_scaled(a64, ea + s_eb[j] - 7 * (S + 1));
                *o = (ch + 1 == kOzFlush ? 0.0 : *o) + v;
              }
            }
          }
        } else {
          tmem_st16(tsum + hh * 16, w);
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) bar_arrive(smem_u32(&acc_empty));
      pending = (multi && pending + 1 == kOzFlush && ch != nchunks - 1) ? 0 : pending + 1;
      return true;
    };
    // the FP64 entries of A for this half's next tile are loaded into
    // registers one tile ahead, so that their latency hides behind the
    // cutting of the current one (no shared-memory staging: the MMAs' operand
    // fetch already takes most of the shared-memory bandwidth)
    double2 an[8];
    auto load_a = [&](int kt) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = (kt0 + kt) * kFK + oct * 8 + u;
        an[u] = (kt < nkt && rowok && k < d.mp) ? col[k] : make_double2(0.0, 0.0);
      }
    };
    load_a(half);
    for (int kt = half; kt < nkt && ok; kt += 2) {
      // the slot of tile kt is freed only by MMAs of the next chunk, which
      // wait for the drain of the previous one: drain it first; and drain as
      // soon as the chunk's MMAs are done once this half is past the chunk,
      // so that the tensor pipe idles for the drain alone
      if (drained < nchunks && kt >= kFChunk * (drained + 1)) {
        bool now = kt >= kFChunk * (drained + 1) + kFSlots;
        if (!now && lane == 0) now = bar_try(smem_u32(&acc_full), drained & 1);
        if (__shfl_sync(0xFFFFFFFFu, now, 0)) ok = drain(drained++);
      }
      if (!ok) break;
      const int slot = kt % kFSlots, use = kt / kFSlots;
      bool free_slot = true;
      if (use > 0) {
        if (lane == 0) free_slot = bar_wait(smem_u32(&empty[slot]), (use - 1) & 1, fail, oz.wait_ns);
        free_slot = __shfl_sync(0xFFFFFFFFu, free_slot, 0);
      }
      if (!free_slot) {
        if (lane == 0) record_fail(&s_fail, 2, kt);
        ok = false;
        break;
      }
      uint8_t* sbase = osm + slot * kFSlot;
      if (!DP && item == 0) {  // B: all S slices of this K tile, one bulk copy
        bar_expect(smem_u32(&full_b[slot]), uint32_t(S * kFSliceB));
        bulk_load(smem_u32(sbase + kFSlotA), gB + int64_t(kt) * S * kFSliceB, uint32_t(S * kFSliceB),
                  smem_u32(&full_b[slot]));
        atomicMax(&s_last_b[slot], kt);
      }
      if (DP) {  // B: 8 entries of Y[S,P] column r, cut into Br, Bi words
        long long YB[16];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = (kt0 + kt) * kFK + oct * 8 + u;
          const double2 v = (rowok && k < d.mp) ? colB[k] : make_double2(0.0, 0.0);
          YB[2 * u] = fixed_point(v.x, eB, S) + bias;  // A already loads the FP64 pipe here
          YB[2 * u + 1] = fixed_point(v.y, eB, S) + bias;
        }
        uint8_t* pb = sbase + kFSlotA + wbase;  // Br slices 1..S, then Bi slices 1..S
        with_slices(S, [&](auto SC) { store_slices_c<decltype(SC)::value>(YB, pb, pb + S * kFBlk, nullptr, kFBlk); });
      }
      // A: 8 entries of row r at k = 16 kt + 8 oct .. + 7, cut into Ar, Ai, -Ar words
      long long Y[16];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        Y[2 * u] = fixed_of(an[u].x, scale, e, S) + bias;
        Y[2 * u + 1] = fixed_point(an[u].y, e, S) + bias;
      }
      load_a(kt + 2);
      uint8_t* ps = sbase + wbase;
      with_slices(S, [&](auto SC) { store_slices_c<decltype(SC)::value>(Y, ps, ps + kFBlk, ps + 2 * kFBlk, kFSliceA); });
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(smem_u32(&full_a[slot]));
    }
    while (ok && drained < nchunks) ok = drain(drained++);
  }

  __syncthreads();
  if (threadIdx.x == 0)  // bulk copies still in flight after a failure land before the CTA leaves
    for (int j = 0; j < kFSlots; ++j)
      if (s_last_b[j] >= 0 && !bar_wait_all(smem_u32(&full_b[j]), (s_last_b[j] / kFSlots) & 1))
        record_fail(&s_fail, 3, j);
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0)
      atomicMax(oz.fail, 1 + (0 << 28) + (min(s_fail, 255) << 20) + min(int(blockIdx.x), (1 << 20) - 1));
  } else if (DP && warp < kFWorkers) {
    // the range's exact sums: lane row (0-63 real, 64-127 imaginary parts of
    // row p of the product), 64 columns q, as int64 in `part`
    asm volatile("tcgen05.fence::after_thread_sync;");
    long long* pp = part + (int64_t(pole) * part_stride + part_off[d.f]) * 2 +
                    int64_t(blockIdx.x) * (2 * kOzRows * kOzRows) + int64_t(q * 32 + lane) * kOzRows + h * 32;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint32_t w[32];
      tmem_ld32(tsum + hh * 32, w);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        pp[hh * 16 + c] = static_cast<long long>((static_cast<unsigned long long>(w[2 * c + 1]) << 32) | w[2 * c]);
    }
  } else if (!DP && warp < kFWorkers) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int ea = orow < d.mp ? s_ea[orow - mt * kOzRows] : 0;
    // the largest high words of what is written, per row (this thread) and
    // per column (a warp reduction; lane c keeps column h*32 + c), go into
    // the row maxima: Y[S,P] extends rows S, and its columns are the rows P
    uint32_t rmax = 0, cmax = 0;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint32_t w[32];
      tmem_ld32(tsum + hh * 32, w);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int j = h * 32 + hh * 16 + c;
        uint32_t hv = 0;
        if (orow < d.mp && j < d.bb) {
          const int eb = s_eb[j];
          double* o = Yout + 2 * ((d.q0 + orow) + int64_t(d.m) * (p0 + j));
          const long long a64 =
              static_cast<long long>((static_cast<unsigned long long>(w[2 * c + 1]) << 32) | w[2 * c]);
          double v = i64_scaled(a64, ea + eb - 7 * (S + 1));
          if (multi) v += *o;  // the partial sums moved out every eight chunks
          if (ea == kNanExp || eb == kNanExp) v = __longlong_as_double(0x7FF8000000000000LL);
          *o = -v;
          Yout[2 * ((p0 + j) + int64_t(d.m) * (d.q0 + orow))] = -v;
          hv = abs_hi(v);
        }
        rmax = max(rmax, hv);
        const uint32_t cm = __reduce_max_sync(0xFFFFFFFFu, hv);
        if (lane == hh * 16 + c) cmax = cm;
      }
    }
    uint32_t* ym = oz.ymax + int64_t(pole) * oz.ymax_stride + oz.ymax_off[d.f];
    if (orow < d.mp) atomicMax(ym + d.q0 + orow, rmax);
    if (h * 32 + lane < d.bb) atomicMax(ym + p0 + h * 32 + lane, cmax);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == kFWorkers) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Exponents of the panel columns of Y[S,P] (rows q0..m-1) into exA[0..bb):
// one warp per column; grid (ceil(b / 8), fronts, poles).
__global__ void __launch_bounds__(256) k_oz_col_exp(const double2* __restrict__ Y, DevFronts fr,
                                                    const int32_t* __restrict__ fronts, int p0, int b, OzScratch oz) {
  PanelDims d;
  if (!panel_dims(fr, fronts, blockIdx.y, p0, b, d)) return;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= d.bb) return;
  const int pole = blockIdx.z;
  const double2* col = Y + int64_t(pole) * fr.pool + fr.off[d.f] + int64_t(p0 + j) * d.m + d.q0;
  uint32_t mx = 0;
  for (int k = lane; k < d.mp; k += 32) {
    const double2 v = col[k];
    mx = max(mx, max(uint32_t(__double2hiint(v.x)) & 0x7FFFFFFFu, uint32_t(__double2hiint(v.y)) & 0x7FFFFFFFu));
  }
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  if (lane == 0)
    oz.exA[int64_t(pole) * oz.exA_stride + oz.exA_off[d.f] + j] =
        mx >= 0x7FF00000u ? kNanExp : (mx != 0 ? int(mx >> 20) - 1022 : 0);
}

// (double) of an exact 128-bit sum: high and low parts, each rounded once.
__device__ __forceinline__ double i128_scaled(__int128 v, int sc) {
  const long long hi = static_cast<long long>(v >> 62);
  const long long lo = static_cast<long long>(v - (static_cast<__int128>(hi) << 62));
  return i64_scaled(hi, sc + 62) + i64_scaled(lo, sc);
}

// Y[P,P] = D^-1 - L[S,P]^T Y[S,P]: the K ranges' exact int64 sums added in
// 128-bit integers (order-free, hence deterministic), scaled by the row and
// column exponents, subtracted from D^-1 (in the diagonal block of F) and
// symmetrised; one CTA per (front, pole).
__global__ void __launch_bounds__(256) k_oz_dpart_reduce(double2* __restrict__ Y, const double2* __restrict__ F,
                                                         const long long* __restrict__ part,
                                                         const int64_t* __restrict__ part_off, int64_t part_stride,
                                                         DevFronts fr, const int32_t* __restrict__ fronts, int p0,
                                                         int b, int S, OzScratch oz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tmp = reinterpret_cast<double2*>(smem_raw);  // bb x bb
  PanelDims d;
  panel_dims(fr, fronts, blockIdx.x, p0, b, d);  // m_p = 0 still needs Y[P,P] = D^-1
  if (p0 >= d.s) return;
  const int pole = blockIdx.y;
  const int nsplit = d.mp > 0 ? ceil_div(ceil_div(d.mp, kFK), kFChunk) : 0;
  const int64_t base = int64_t(pole) * fr.pool + fr.off[d.f];
  const long long* pp = part + (int64_t(pole) * part_stride + part_off[d.f]) * 2;
  const int* exa = oz.exA + int64_t(pole) * oz.exA_stride + oz.exA_off[d.f];  // Y[S,P] columns
  const int* exb = oz.exB + int64_t(pole) * oz.exB_stride + oz.exB_off[d.f];  // L[S,P] columns
  __shared__ uint32_t s_rmax[kOzRows];  // row maxima of Y[P,P] (high words)
  if (threadIdx.x < kOzRows) s_rmax[threadIdx.x] = 0;
  for (int idx = threadIdx.x; idx < d.bb * d.bb; idx += blockDim.x) {
    const int r = idx % d.bb, c = idx / d.bb;
    __int128 re = 0, im = 0;
    for (int t = 0; t < nsplit; ++t) {
      re += pp[int64_t(t) * 2 * kOzRows * kOzRows + int64_t(r) * kOzRows + c];
      im += pp[int64_t(t) * 2 * kOzRows * kOzRows + int64_t(kOzRows + r) * kOzRows + c];
    }
    const int ea = exb[r], eb = exa[c];
    double2 v = F[base + (p0 + r) + int64_t(d.m) * (p0 + c)];
    if (ea == kNanExp || eb == kNanExp) {
      v = make_double2(__longlong_as_double(0x7FF8000000000000LL), __longlong_as_double(0x7FF8000000000000LL));
    } else {
      const int sc = ea + eb - 7 * (S + 1);
      v.x -= i128_scaled(re, sc);
      v.y -= i128_scaled(im, sc);
    }
    tmp[r + d.bb * c] = v;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < d.bb * d.bb; idx += blockDim.x) {
    const int r = idx % d.bb, c = idx / d.bb;
    const double2 a = tmp[r + d.bb * c], t = tmp[c + d.bb * r];
    const double2 v = make_double2(0.5 * (a.x + t.x), 0.5 * (a.y + t.y));
    Y[base + (p0 + r) + int64_t(d.m) * (p0 + c)] = v;
    atomicMax(&s_rmax[r], max(abs_hi(v.x), abs_hi(v.y)));
  }
  __syncthreads();
  if (threadIdx.x < d.bb)  // the rows P of Y now extend over the columns P
    atomicMax(oz.ymax + int64_t(pole) * oz.ymax_stride + oz.ymax_off[d.f] + p0 + threadIdx.x, s_rmax[threadIdx.x]);
}

}  // namespace

constexpr int kMaxPersistFronts = 4096;  // fronts per launch of the persistent GEMM (prefix sums in smem)

size_t oz_smem_bytes(int /*S*/) {
  return size_t(kSlotsA) * kSliceA + size_t(kSlotsB) * 6 * kSliceB + sizeof(int) * (kMaxPersistFronts + 1);
}

// Scratch bytes of one front (per pole) whose first panel leaves mp rows
// below it, for the phases that stage slices in HBM: Schur A = L[S,P]
// (mp x bb) and B = W[S,P] (mp x bb); panel solve A = W[S,P], B = D^-1;
// the fused Takahashi step stages only B = L[S,P] (bb x mp, 16-deep tiles).
int64_t oz_front_bytes_A(int64_t mp, int b, int S) {
  const int64_t rt = (mp + kOzRows - 1) / kOzRows;
  return rt * ((b + kOzK - 1) / kOzK) * S * kSliceA;
}

int64_t oz_front_bytes_B(int64_t mp, int b, int S) {
  const int64_t tak = ((mp + kFK - 1) / kFK) * S * kFSliceB;
  const int64_t sch = ((mp + kOzRows - 1) / kOzRows) * ((b + kOzK - 1) / kOzK) * S * kSliceB;
  return std::max(tak, sch);
}

cudaError_t oz_configure(int S) {
  const int smem = int(oz_smem_bytes(S));
  cudaError_t e = cudaFuncSetAttribute(k_oz_gemm<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_oz_gemm<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_oz_gemm<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_oz_gemm<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_oz_gemm<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_oz_gemm<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_oz_tak_fused<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kFSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_oz_tak_fused<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kFSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_oz_dpart_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(sizeof(double2) * kOzRows * kOzRows));
  return e;
}

int64_t oz_front_bytes_A_real(int64_t mp, int b, int S) {
  return ((mp + 2 * kOzRows - 1) / (2 * kOzRows)) * ((b + kOzK - 1) / kOzK) * S * (2 * kBlk);
}

int64_t oz_front_bytes_B_real(int64_t mp, int b, int S) {
  return ((mp + kOzRows - 1) / kOzRows) * ((b + kOzK - 1) / kOzK) * S * kBlk;
}

namespace {

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 148;
  }
  return cached[dev];
}

// One persistent launch per group of at most kMaxPersistFronts fronts; the
// grid is one CTA per SM (fewer when the launch holds fewer tiles).
template <int MODE, bool CPLX>
void launch_persistent(void* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles, int p0, int b,
                       int S, const OzScratch& oz, int nb, cudaStream_t st, int cb = 0) {
  if (nfronts <= 0 || max_tiles <= 0) return;
  for (int f0 = 0; f0 < nfronts; f0 += kMaxPersistFronts) {
    const int nf = std::min(kMaxPersistFronts, nfronts - f0);
    const int64_t bound = int64_t(max_tiles) * nf * nb;
    const int grid = int(std::min<int64_t>(sm_count(), bound));
    k_oz_gemm<MODE, CPLX><<<grid, kGemmThreads, oz_smem_bytes(S), st>>>(F, fr, fronts + f0, nf, p0, b, S, nb, oz, cb);
  }
}

}  // namespace

int oz_schur_tiles_real(int mp) {
  const int nmt = ceil_div(mp, 2 * kOzRows), nnt = ceil_div(mp, kOzRows);
  return mp > 0 ? nmt * (nmt + 1) - (2 * nmt - nnt) : 0;
}

int oz_schur_tiles(int mp) {
  const int nmt = ceil_div(mp, kOzRows);
  return nmt * (nmt + 1) / 2;
}

void launch_oz_slice_schur_real(const double* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp,
                                int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb) {
  if (nfronts <= 0 || max_mp <= 0) return;
  const int groups = (max_mp + 7) / 8;
  dim3 g(2 * groups, nfronts, nb);
  k_oz_slice_real<1><<<g, 256, 0, st>>>(const_cast<double*>(F), fr, fronts, p0, b, S, groups, oz, cb);
}

void launch_oz_gemm_schur_real(double* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles,
                               int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb) {
  if (cb > 0)
    launch_persistent<3, false>(F, fr, fronts, nfronts, max_tiles, p0, b, S, oz, nb, st, cb);
  else
    launch_persistent<1, false>(F, fr, fronts, nfronts, max_tiles, p0, b, S, oz, nb, st);
}

void launch_oz_slice_schur(const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp,
                           int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb) {
  if (nfronts <= 0 || max_mp <= 0) return;
  const int groups = (max_mp + 7) / 8;
  dim3 g(2 * groups, nfronts, nb);
  k_oz_slice<1><<<g, 256, 0, st>>>(F, const_cast<double2*>(F), fr, fronts, p0, b, S, groups, oz, cb);
}

void launch_oz_gemm_schur(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_tiles, int p0,
                          int b, int S, const OzScratch& oz, int nb, cudaStream_t st, int cb) {
  if (cb > 0)
    launch_persistent<3, true>(F, fr, fronts, nfronts, max_tiles, p0, b, S, oz, nb, st, cb);
  else
    launch_persistent<1, true>(F, fr, fronts, nfronts, max_tiles, p0, b, S, oz, nb, st);
}

int oz_block_tiles(int mp, int cs, bool cplx) {
  return cplx ? front_tiles<3, true>(mp, cs) : front_tiles<3, false>(mp, cs);
}

// Split-precision panel solve L[S,P] = W[S,P] D^-1 (complex poles and real
// inertia shifts): slicing of W rows (W^T saved on the way) and of D^-1, then
// the GEMM writing L over W.
void launch_oz_panel(double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp, int p0, int b,
                     int S, const OzScratch& oz, int nb, cudaStream_t st, bool gemm) {
  if (nfronts <= 0 || max_mp <= 0) return;
  if (!gemm) {
    const int groupsA = (max_mp + 7) / 8, groupsB = (b + 7) / 8;
    dim3 g(groupsA + groupsB, nfronts, nb);
    k_oz_slice<2><<<g, 256, 0, st>>>(nullptr, F, fr, fronts, p0, b, S, groupsA, oz, 0);
  } else {
    launch_persistent<2, true>(F, fr, fronts, nfronts, ceil_div(max_mp, kOzRows), p0, b, S, oz, nb, st);
  }
}

void launch_oz_panel_real(double* F, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp, int p0,
                          int b, int S, const OzScratch& oz, int nb, cudaStream_t st, bool gemm) {
  if (nfronts <= 0 || max_mp <= 0) return;
  if (!gemm) {
    const int groupsA = (max_mp + 7) / 8, groupsB = (b + 7) / 8;
    dim3 g(groupsA + groupsB, nfronts, nb);
    k_oz_slice_real<2><<<g, 256, 0, st>>>(F, fr, fronts, p0, b, S, groupsA, oz, 0);
  } else {
    launch_persistent<2, false>(F, fr, fronts, nfronts, ceil_div(max_mp, 2 * kOzRows), p0, b, S, oz, nb, st);
  }
}

// Fused Takahashi step: exponents of A and slices of B (prep = true), then
// the GEMM that slices A on the fly (prep = false).
void launch_oz_rowmax_init(const double2* Y, const DevFronts& fr, const int32_t* fronts, int nfronts, int max_m,
                           const OzScratch& oz, int nb, cudaStream_t st) {
  if (nfronts <= 0 || max_m <= 0) return;
  dim3 g(ceil_div(max_m, 8), nfronts, nb);
  k_oz_rowmax_init<<<g, 256, 0, st>>>(Y, fr, fronts, oz);
}

void launch_oz_takahashi(double2* Y, const double2* F, const DevFronts& fr, const int32_t* fronts, int nfronts,
                         int max_mp, int p0, int b, int S, const OzScratch& oz, int nb, cudaStream_t st, bool prep) {
  if (nfronts <= 0 || max_mp <= 0) return;
  if (prep) {
    const int groupsA = (max_mp + 255) / 256, groupsB = (b + 7) / 8;
    dim3 g(groupsA + groupsB, nfronts, nb);
    k_oz_tak_prep<<<g, 256, 0, st>>>(Y, F, fr, fronts, p0, b, S, groupsA, oz);
  } else {
    dim3 gg(ceil_div(max_mp, kOzRows), nfronts, nb);
    k_oz_tak_fused<0><<<gg, kFThreads, size_t(kFSmem), st>>>(Y, fr, fronts, p0, b, S, oz, nullptr,
                                                                      nullptr, nullptr, 0);
  }
}

// Split-precision Y[P,P] = D^-1 - L[S,P]^T Y[S,P]: stage 0 finds the
// exponents of the Y[S,P] columns, stage 1 runs the split-K GEMM into
// `part` (int64 sums per 256-deep range), stage 2 reduces and symmetrises.
void launch_oz_dpart(double2* Y, const double2* F, double2* part, const int64_t* part_off, int64_t part_stride,
                     const DevFronts& fr, const int32_t* fronts, int nfronts, int max_mp, int p0, int b, int S,
                     const OzScratch& oz, int nb, cudaStream_t st, int stage) {
  if (nfronts <= 0 || (stage < 2 && max_mp <= 0)) return;
  if (stage == 0) {
    dim3 g(ceil_div(b, 8), nfronts, nb);
    k_oz_col_exp<<<g, 256, 0, st>>>(Y, fr, fronts, p0, b, oz);
  } else if (stage == 1) {
    dim3 g(ceil_div(ceil_div(max_mp, kFK), kFChunk), nfronts, nb);
    k_oz_tak_fused<1><<<g, kFThreads, size_t(kFSmem), st>>>(
        Y, fr, fronts, p0, b, S, oz, F, reinterpret_cast<long long*>(part), part_off, part_stride);
  } else {
    dim3 g(nfronts, nb);
    k_oz_dpart_reduce<<<g, 256, sizeof(double2) * kOzRows * kOzRows, st>>>(
        Y, F, reinterpret_cast<const long long*>(part), part_off, part_stride, fr, fronts, p0, b, S, oz);
  }
}

}  // namespace pexsi
