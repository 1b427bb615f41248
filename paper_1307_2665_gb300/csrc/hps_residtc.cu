// FP64 residual (and leaf fluxes) of the refinement with the derivative
// products on the tensor cores, for leaves of order p = 16 whose operator has
// no first-order or mixed term (c11, c22 and c only: Laplace- and
// Helmholtz-type problems).
//
// Per leaf and grid w (16 x 16 FP64 values at the tensor Chebyshev nodes) the
// residual needs the second derivatives along x and y, X = w D2^T (row a of w
// against row b of D^2) and Y = D2 w, then r = -(A w) = k11 X + k22 Y + k0 w at
// the 196 interior nodes (Section 3.1); the leaf fluxes need rows 0 and 15 of D
// along x and y, then the side interpolant at the Gauss points (Section 3.2,
// Steps 3-4).  As FP64 FMAs these contractions bound the refinement on the FP64
// pipe (2 FMAs per clock per SM on this part).  Here they run as exact integer
// products on the BF16 tensor cores (Ozaki's splitting):
//   * the interior rows of D^2 are only needed at interior nodes, so one table
//     B = [D_0 ; D^2_1 .. D^2_14 ; D_15] (16 x 16) gives both the second
//     derivatives and the side derivatives;
//   * every grid is scaled by 2^-e_g, e_g the exponent of its largest |w|, and
//     rounded to a signed 56-bit fixed-point value written as 7 balanced
//     base-256 digits (the top one in [-256, 256], the others in [-128, 127]);
//     every row n of B likewise relative to its own exponent f_n, to 62 bits in
//     8 digits.  Every digit is exact in BF16;
//   * eight grids form one M = 128 operand: rows (grid, a) with K = b for the x
//     products, rows (grid, b) with K = a for the y products.  For every digit
//     pair (s, t) with s + t <= 9 one tcgen05.mma (M = 128, N = 16, K = 16) adds
//     the exact integer products into the FP32 tensor-memory accumulator of its
//     diagonal d = s + t; a diagonal holds at most 7 pairs of 16 products, so
//     every sum is an integer below 2^21 and exact in FP32;
//   * the drain reads the eight diagonal sums of an output, forms the exact
//     integer U = sum_d P_d 256^(9-d) (up to 79 bits) and rounds it to a double
//     with integer instructions only: X = U 2^(e_g + f_n + 2 - 72).
// The dropped pairs (s + t >= 10) and the two roundings to fixed point weigh
// below 2^-56 of max|w| max|B_n.|, under the rounding of an FP64 product, so
// the result is the FP64 residual to rounding.  The FP64 pipe keeps the
// combination k11 X + k22 Y + k0 w and the fluxes' Gauss interpolation.  The
// tables D and D^2 are the ones every other kernel applies.
//
// kFromY: the grids are the columns of [L1 ; Y] of each leaf (the residual of
// the leaf systems in the build), no fluxes.  kFlux: the fluxes L4 L3 w are
// stored to hp (FP64), as the FP64-pipe kernel does.
//
// A grid holding an infinity or NaN gives NaN at every output.  A grid whose
// largest |w| is below 2^-900 is taken as zero.  Waits on the tensor cores are
// bounded; a CTA whose wait gives up sets *status to -1 (a device error),
// waits (bounded again) for its products still in flight and frees its
// tensor memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"
#include "hps_tc.cuh"

namespace hps {

namespace {

struct CoefPtrs {
  const double* c[6];  // c11, c12, c22, c1, c2, c (null = absent)
};

constexpr int kRP = 16;                // order p of the leaves this kernel takes
constexpr int kRPP = kRP * kRP;
constexpr int kRNi = (kRP - 2) * (kRP - 2);
constexpr int kRG = 8;                 // grids per block: M = 8 x 16 = 128 rows
constexpr int kRThreads = 256;
constexpr int kRSA = 7;                // digits of a grid value (56 bits)
constexpr int kRSB = 8;                // digits of a table entry (62 bits)
constexpr int kRDiag = 8;              // diagonals d = 2 .. 9
constexpr int kRCols = 2 * kRDiag * kRP;  // TMEM columns: x and y accumulators
constexpr int kRWp = kRP + 1;          // padded row pitch of the FP64 tiles (doubles)
constexpr int kRGs = kRP * kRWp;       // one grid
constexpr int kRFlB = 4;               // blocks per interpolation of the side derivatives
constexpr int kRFl = kRFlB * kRG * 4;  // lines per interpolation: 128 = M
constexpr int kASliceB = 128 * kRP * 2;  // bytes of one A digit slice (4 KB)
constexpr int kBSliceB = kRP * kRP * 2;  // bytes of one B digit slice (512 B)
constexpr long kRSpin = 1L << 20;      // bound of every wait (iterations)
constexpr int kRExpMin = -900;         // grids below 2^-900 are taken as zero
constexpr int kRExpNaN = 4096;         // marks a grid holding an infinity or NaN
// worst diagonal: the top digits (256 x 128, 128 x 64) and five pairs of 128 x 128
static_assert((256 * 128 + 128 * 64 + 5 * 128 * 128) * kRP < (1 << 22),
              "diagonal sums exact in FP32");

// Offset (elements) of operand element (row r, k) in the K-major, no-swizzle
// layout of a 16-wide K: core matrices of 8 rows x 8 k (128 bytes), the two K
// cores of a row group adjacent (LBO 128 B), row groups 256 B apart (SBO).
__device__ __forceinline__ int op_off(int r, int k) {
  return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// e with |x| < 2^e for every x of a set, from the largest high word of |x|
// (exponent field and top mantissa bits): kRExpMin for zero and tiny sets,
// kRExpNaN when an infinity or NaN is present.
__device__ __forceinline__ int exp_bound(uint32_t hmax) {
  const int ex = (int)(hmax >> 20);
  if (ex == 0x7ff) return kRExpNaN;
  return max(ex - 1022, kRExpMin);
}

// round(x 2^(kBits - e)) (|x| < 2^e; ties away from zero) as a two's-complement
// integer plus 128 at every digit but the top one: byte j of the result is then
// digit (n - j) + 128 for the n - 1 lower digits, and the arithmetic shift by
// 8 (n - 1) is the signed top digit (|F| < 2^kBits, so nothing overflows).
template <int kBits, int kDigits>
__device__ __forceinline__ unsigned long long fixed_point(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & 0xfffffffffffffULL;
  if (ex != 0) m |= 1ULL << 52;
  const int sh = (ex == 0 ? -1074 : ex - 1075) + kBits - e;  // |x| = m 2^(sh - kBits + e)
  unsigned long long F = 0;
  if (e < kRExpNaN) {
    if (sh >= 0)
      F = m << sh;
    else if (sh > -54)
      F = (m + (1ULL << (-sh - 1))) >> (-sh);
  }
  if (bits >> 63) F = 0ULL - F;
  constexpr unsigned long long kOff =
      kDigits == 7 ? 0x808080808080ULL : 0x80808080808080ULL;  // 128 at digits 2..n
  return F + kOff;
}

// A lower digit as a float: PRMT places byte j of the word under the exponent
// bits of 1.5 2^23, and the subtraction removes the bias and the 128.
__device__ __forceinline__ float digit_lo(uint32_t word, int j) {
  return __uint_as_float(__byte_perm(word, 0x4B400000u, 0x7650u | (uint32_t)j)) - 12583040.0f;
}
// The signed top digit as a float (|t| <= 256).
__device__ __forceinline__ float digit_top(int t) {
  return __int_as_float(0x4B400000 + t) - 12582912.0f;
}
// Two floats holding BF16-exact values as one packed BF16 pair (lo, hi).
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
// Digit s (1-based, s = 1 the top) of a fixed_point value with n digits.
template <int kDigits>
__device__ __forceinline__ float digit(unsigned long long G, int s) {
  if (s == 1) return digit_top((int)((long long)G >> (8 * (kDigits - 1))));
  const int j = kDigits - s;  // byte index
  return digit_lo(j < 4 ? (uint32_t)G : (uint32_t)(G >> 32), j & 3);
}
// Slice s of 8 fixed_point values as 8 packed BF16 (16 bytes) at a shared address.
template <int kDigits>
__device__ __forceinline__ void store_slice(uint32_t saddr, const unsigned long long* G, int s) {
  const uint32_t w0 = pack_bf16(digit<kDigits>(G[0], s), digit<kDigits>(G[1], s));
  const uint32_t w1 = pack_bf16(digit<kDigits>(G[2], s), digit<kDigits>(G[3], s));
  const uint32_t w2 = pack_bf16(digit<kDigits>(G[4], s), digit<kDigits>(G[5], s));
  const uint32_t w3 = pack_bf16(digit<kDigits>(G[6], s), digit<kDigits>(G[7], s));
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(saddr), "r"(w0), "r"(w1), "r"(w2),
               "r"(w3)
               : "memory");
}

// The integer held exactly by an FP32 accumulator (|v| < 2^22), plus the bias
// 0x4B400000 (the bits of v + 1.5 2^23); pair_acc removes the bias.
__device__ __forceinline__ uint32_t acc_bits(uint32_t v) {
  return __float_as_uint(__uint_as_float(v) + 12582912.0f);
}
// P_e 256 + P_o from the biased bits of two consecutive diagonals (modulo 2^32,
// where the true value, below 2^30 in magnitude, is exact).
__device__ __forceinline__ int pair_acc(uint32_t be, uint32_t bo) {
  return (int)(be * 256u + bo - 257u * 0x4B400000u);
}

// U 2^scale rounded to the nearest double (ties to even), for the exact integer
// U = A1 2^48 + A2 2^32 + A3 2^16 + A4 (|A| < 2^30), by integer instructions.
__device__ __forceinline__ double u_to_double(int A1, int A2, int A3, int A4, int scale) {
  const long long hi = (long long)A1 * 65536 + A2;
  const long long lo = (long long)A3 * 65536 + A4;
  long long uh = hi + (lo >> 32);  // U = uh 2^32 + ul, 0 <= ul < 2^32
  uint32_t ul = (uint32_t)lo;
  const bool neg = uh < 0;
  if (neg) {
    uh = -uh - (ul != 0u ? 1 : 0);
    ul = 0u - ul;
  }
  unsigned long long m;
  int E;
  if (uh < (1LL << 21)) {  // U < 2^53: exact
    const unsigned long long N = ((unsigned long long)uh << 32) | ul;
    if (N == 0) return 0.0;
    const int t = 63 - __clzll((long long)N);
    m = N << (52 - t);
    E = t + scale;
  } else {
    const int t = 63 - __clzll(uh);
    const int k = t - 20;  // 1 .. 27 bits drop out of ul
    m = ((unsigned long long)uh << (32 - k)) | (ul >> k);
    const uint32_t rem = ul & ((1u << k) - 1u), half = 1u << (k - 1);
    m += (rem > half || (rem == half && (m & 1ULL))) ? 1ULL : 0ULL;
    E = t + 32 + scale;
  }
  unsigned long long b;
  if (E > 1023)
    b = 0x7ff0000000000000ULL;  // beyond the double range: infinity
  else
    b = ((unsigned long long)(E + 1022) << 52) + m;  // m carries the hidden bit
  if (neg) b |= 1ULL << 63;
  return __longlong_as_double((long long)b);
}

// A float as a double by integer instructions (normal numbers and zeros; the
// conversion instruction for the rest).
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) {
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
    return (double)f;
  }
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(ex + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// A double rounded to the nearest float by integer instructions (the
// conversion instruction for zeros below the float range, infinities, NaN).
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ff) - 1023;
  if ((b << 1) == 0ULL) return __uint_as_float(sign);
  if (E < -126 || E == 1024) return (float)x;
  if (E > 127) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long mant = b & 0xfffffffffffffULL;
  uint32_t m = (uint32_t)(mant >> 29);
  const uint32_t rem = (uint32_t)mant & 0x1fffffffu;
  m += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | (((uint32_t)(E + 127) << 23) + m));  // a carry raises E
}
template <typename R>
__device__ __forceinline__ R to_r(double x) {
  if constexpr (sizeof(R) == 4)
    return d2f(x);
  else
    return x;
}

// Eight outputs of one TMEM lane: columns c0 .. c0 + 7 of the eight diagonal
// accumulators starting at column tb, as doubles scaled by 2^(e + f_n + 2 - 72).
__device__ __forceinline__ void drain8(uint32_t tb, int c0, int e, const int* fn, double* out) {
  int A[4][8];
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // diagonals 4 h + 2 .. 4 h + 5, one wait
    uint32_t v[4][8];
#pragma unroll
    for (int t = 0; t < 4; ++t) tc::ld8(tb + (uint32_t)((4 * h + t) * kRP + c0), v[t]);
    tc::wait_ld();
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      A[2 * h][n] = pair_acc(acc_bits(v[0][n]), acc_bits(v[1][n]));
      A[2 * h + 1][n] = pair_acc(acc_bits(v[2][n]), acc_bits(v[3][n]));
    }
  }
#pragma unroll
  for (int n = 0; n < 8; ++n)
    out[n] = e == kRExpNaN ? __longlong_as_double(0x7ff8000000000000LL)
                           : u_to_double(A[0][n], A[1][n], A[2][n], A[3][n],
                                         e + fn[c0 + n] + 2 - 72);
}

// ------------------------------------------------------------------ kernel
// One CTA per leaf (two per SM), blocks of 8 grids (right-hand sides).  Per
// block:
//   1. warp g moves grid g (loaded one block ahead) into shared memory and
//      finds e_g;
//   2. each thread writes the digits of 8 values of one row of the x and of
//      the y operand;
//   3. thread 0 issues the 70 products and commits them to an mbarrier;
//   4. every warp drains 8 columns of its TMEM lane quadrant, first of the y
//      accumulators (Y and the side derivatives d/dy to shared memory), then
//      of the x accumulators, forming r = k11 X + k22 Y + k0 w at once;
//   5. the coalesced store of r.
// kFlux: the side derivatives of 4 blocks (32 grids x 4 sides = 128 lines of
// 16 values) are interpolated to the Gauss points as one more digit product
// (M = 128 lines, N = 16 rows of Pc2g, K = 16), which every warp drains.
// After the products are complete the operand buffer holds Y and r, then the
// digits of the lines.
template <typename R, bool kFromY, bool kFlux>
__global__ void __launch_bounds__(kRThreads, 2) k_leaf_resid_tc(
    CoefPtrs cp, int l0, int q, const double2* __restrict__ hsc, const double* __restrict__ gD,
    const double* __restrict__ gPm, double* const* __restrict__ wptr,
    const int64_t* __restrict__ wrs, int nrhs, R* __restrict__ rbuf, const R* __restrict__ Ysrc,
    int64_t ys, const int64_t* __restrict__ leaf_off, int64_t ext_total, double* __restrict__ hp,
    int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* As = smraw;                     // x, y: 7 digit slices each
  unsigned char* Bs = As + 2 * kRSA * kASliceB;  // 8 digit slices of the table
  unsigned char* Bp = Bs + kRSB * kBSliceB;      // kFlux: 8 digit slices of Pc2g
  double* W = reinterpret_cast<double*>(Bp + (kFlux ? kRSB * kBSliceB : 0));  // 8 grids, 16 x 17
  double* Kc = W + kRG * kRGs;                   // k11, k22, k0: 16 x 17 each
  double* Fq = Kc + 3 * kRGs;                    // kFlux: 128 lines of pitch 17
  double* Pm = Fq + (kFlux ? kRFl * kRWp : 0);   // kFromY: Pg2c (16 x q)
  // aliases of the operand buffer, live from the end of the products to the
  // next digits written there
  double* Ys = reinterpret_cast<double*>(As);    // 8 grids of 16 x 17
  R* Rs = reinterpret_cast<R*>(Ys + kRG * kRGs);  // 8 grids x 196
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int eg[kRG];
  __shared__ int fn[kRP];
  __shared__ int fq[kRP];   // kFlux: exponents of the rows of Pc2g
  __shared__ int el[kRFl];  // kFlux: exponents of the 128 lines
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int jl = blockIdx.x, l = l0 + jl;  // group-local and global leaf
  const double sx = hsc[l].x, sy = hsc[l].y;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_base)),
                 "r"(kRCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // row n of the table: D_0, D^2_1 .. D^2_14, D_15
  auto brow = [&](int n, int k) -> double {
    if (n == 0 || n == kRP - 1) return gD[n * kRP + k];
    return gD[kRPP + n * kRP + k];  // D^2 follows D
  };
  // kFlux: row n of Pc2g (q x 16), zero rows after it
  auto prow = [&](int n, int k) -> double { return n < q ? gPm[n * kRP + k] : 0.0; };
  auto row_exp = [&](int n, bool pc) {
    uint32_t hm = 0;
    for (int k = 0; k < kRP; ++k)
      hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(pc ? prow(n, k)
                                                                         : brow(n, k)) >>
                              32) &
                       0x7fffffffu);
    return exp_bound(hm);
  };
  for (int e = tid; e < kRPP; e += kRThreads) {
    const size_t g = (size_t)jl * kRPP + e;
    const int t = (e >> 4) * kRWp + (e & 15);
    Kc[t] = cp.c[0] ? cp.c[0][g] * sx * sx : 0.0;
    Kc[kRGs + t] = cp.c[2] ? cp.c[2][g] * sy * sy : 0.0;
    Kc[2 * kRGs + t] = cp.c[5] ? -cp.c[5][g] : 0.0;
  }
  if constexpr (kFromY)
    for (int e = tid; e < kRP * q; e += kRThreads) Pm[e] = gPm[e];
  if (tid < kRP) fn[tid] = row_exp(tid, false);
  if constexpr (kFlux)
    if (tid >= 32 && tid < 32 + kRP) fq[tid - 32] = row_exp(tid - 32, true);
  __syncthreads();
  // digits of the tables: thread (n, half) writes 8 entries of row n per slice
  if (tid < 2 * kRP || (kFlux && tid >= 64 && tid < 64 + 2 * kRP)) {
    const bool pc = tid >= 64;
    const int n = (tid & 63) >> 1, half = tid & 1;
    unsigned long long G[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = half * 8 + j;
      G[j] = fixed_point<62, kRSB>(pc ? prow(n, k) : brow(n, k), pc ? fq[n] : fn[n]);
    }
    const uint32_t base = tc::smem_u32((pc ? Bp : Bs) + op_off(n, half * 8) * 2);
#pragma unroll
    for (int t = 1; t <= kRSB; ++t) store_slice<kRSB>(base + (t - 1) * kBSliceB, G, t);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int64_t off = kFlux ? leaf_off[l] : 0;
  const double* wl = kFromY ? nullptr : wptr[l];
  const int64_t wstride = kFromY ? 0 : wrs[l];
  const int row = 32 * (warp & 3) + lane;  // TMEM lane = operand row (grid, i)
  const int rg = row >> 4, ri = row & 15;
  const int c0 = 8 * (warp >> 2);          // the 8 columns this warp drains
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  // the values of grid `warp` of a block held by this lane (nodes lane + 32 j),
  // loaded one block ahead so that the loads run during the previous block
  using PreT = typename std::conditional<kFromY, R, double>::type;
  PreT pre[kRPP / 32];
  auto fetch = [&](int rb0) {
    const int g = rb0 + warp;
#pragma unroll
    for (int j = 0; j < kRPP / 32; ++j) {
      const int node = lane + 32 * j, a = node >> 4, b = node & 15;
      PreT v = PreT(0);
      if (g < nrhs) {
        if constexpr (kFromY) {
          if (a > 0 && a < kRP - 1 && b > 0 && b < kRP - 1)
            v = Ysrc[(size_t)jl * ys + (a - 1) * (kRP - 2) + (b - 1) + (size_t)g * kRNi];
        } else {
          v = wl[(size_t)g * wstride + node];
        }
      }
      pre[j] = v;
    }
  };
  // one commit per product batch; waits take the parity of the next phase
  uint32_t phase = 0;
  auto products_done = [&]() -> bool {
    const bool ok = tc::mbar_wait(&bar, phase, kRSpin);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
  };
  fetch(0);
  bool fail = false;
  int blk = 0;
  for (int r0 = 0; r0 < nrhs; r0 += kRG, ++blk) {
    const int nb = min(kRG, nrhs - r0);
    // ---- 1. grid `warp` into shared memory, its exponent
    {
      const int gi = warp, g = r0 + gi;
      uint32_t hm = 0;
#pragma unroll
      for (int j = 0; j < kRPP / 32; ++j) {
        const int node = lane + 32 * j, a = node >> 4, b = node & 15;
        double v;
        if constexpr (kFromY) {
          if (a > 0 && a < kRP - 1 && b > 0 && b < kRP - 1) {
            v = sizeof(R) == 4 ? f2d((float)pre[j]) : (double)pre[j];
          } else {  // column g is Gauss node k of side s: L1's entry at this node
            v = 0.0;
            const int s = g / q, k = g % q;
            int jj = -1;
            if (s == 0 && a == 0) jj = b;
            if (s == 2 && a == kRP - 1) jj = b;
            if (s == 1 && b == kRP - 1) jj = a;
            if (s == 3 && b == 0) jj = a;
            if (jj >= 0 && gi < nb) v = ((jj == 0 || jj == kRP - 1) ? 0.5 : 1.0) * Pm[jj * q + k];
          }
        } else {
          v = pre[j];
        }
        W[gi * kRGs + a * kRWp + b] = v;
        hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu);
      }
      hm = __reduce_max_sync(0xffffffffu, hm);
      if (lane == 0) eg[gi] = exp_bound(hm);
    }
    fetch(r0 + kRG);  // the next block's values, in flight during this block
    __syncthreads();
    // ---- 2. digits of the x operand (row (g, a), K = b) and of the y operand
    // (row (g, b), K = a): thread (row, half) writes 8 values per slice
    {
      const int r = tid >> 1, half = tid & 1;
      const int g = r >> 4, i = r & 15;
      const int e = eg[g];
      const double* Wg = W + g * kRGs;
#pragma unroll
      for (int dw = 0; dw < 2; ++dw) {
        unsigned long long G[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          G[j] = fixed_point<56, kRSA>(
              dw == 0 ? Wg[i * kRWp + half * 8 + j] : Wg[(half * 8 + j) * kRWp + i], e);
        const uint32_t base = tc::smem_u32(As + dw * kRSA * kASliceB + op_off(r, half * 8) * 2);
#pragma unroll
        for (int s = 1; s <= kRSA; ++s) store_slice<kRSA>(base + (s - 1) * kASliceB, G, s);
      }
      // the tensor cores read shared memory through the async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // ---- 3. the products: diagonal d of direction dw (0 = x, 1 = y)
    // accumulates in columns (dw * 8 + d - 2) * 16 .. + 15
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
      constexpr uint32_t idesc = tc::idesc_bf16(128, kRP);
      for (int dw = 0; dw < 2; ++dw)
        for (int d = 2; d <= kRDiag + 1; ++d) {
          uint32_t acc = 0;
          for (int s = max(1, d - kRSB); s <= min(kRSA, d - 1); ++s) {
            const uint64_t da =
                tc::desc_kmajor(a0 + (uint32_t)((dw * kRSA + s - 1) * kASliceB), 128, 256);
            const uint64_t db = tc::desc_kmajor(b0 + (uint32_t)((d - s - 1) * kBSliceB), 128, 256);
            tc::mma_bf16(tmem + (uint32_t)((dw * kRDiag + d - 2) * kRP), da, db, idesc, acc);
            acc = 1;
          }
        }
      tc::commit(&bar);
    }
    if (!products_done()) {
      fail = true;
      break;
    }
    const int slot = blk & (kRFlB - 1);  // kFlux: this block's lines in Fq
    // ---- 4a. y: this lane is column b = ri of grid rg; outputs n = c0 .. c0 + 7
    // are Y(n, b) (n = 1 .. 14), d/dy at row 0 (n = 0) and at row 15 (n = 15)
    {
      double out[8];
      drain8(tmem + tlane + (uint32_t)(kRDiag * kRP), c0, eg[rg], fn, out);
      if (ri >= 1 && ri <= kRP - 2) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = c0 + j;
          if (n >= 1 && n <= kRP - 2) Ys[rg * kRGs + n * kRWp + ri] = out[j];
        }
      }
      if constexpr (kFlux) {  // lines S (0) and N (2) of grid rg
        double* F = Fq + (slot * kRG * 4 + rg * 4) * kRWp + ri;
        if (c0 == 0) F[0] = out[0];
        else F[2 * kRWp] = out[7];
      }
    }
    __syncthreads();
    // ---- 4b. x: this lane is row a = ri of grid rg; outputs n = c0 .. c0 + 7
    // are X(a, n), d/dx at column 0 (n = 0) and at column 15 (n = 15); r at
    // the interior nodes (a, n)
    {
      double out[8];
      drain8(tmem + tlane, c0, eg[rg], fn, out);
      if (ri >= 1 && ri <= kRP - 2 && rg < nb) {
        const double* Wr = W + rg * kRGs + ri * kRWp;
        const double* Yr = Ys + rg * kRGs + ri * kRWp;
        const double* Kr = Kc + ri * kRWp;
        R* rr = Rs + rg * kRNi + (ri - 1) * (kRP - 2) - 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = c0 + j;
          if (n >= 1 && n <= kRP - 2) {
            double r = Kr[2 * kRGs + n] * Wr[n];
            r = fma(Kr[kRGs + n], Yr[n], r);
            r = fma(Kr[n], out[j], r);
            rr[n] = to_r<R>(r);
          }
        }
      }
      if constexpr (kFlux) {  // lines E (1) and W (3) of grid rg
        double* F = Fq + (slot * kRG * 4 + rg * 4) * kRWp + ri;
        if (c0 == 0) F[3 * kRWp] = out[0];
        else F[kRWp] = out[7];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- 5. r of the block, coalesced (grids r0 .. r0 + nb - 1 are contiguous)
    {
      R* rdst = rbuf + (size_t)jl * kRNi * nrhs + (size_t)r0 * kRNi;
      for (int e = tid; e < nb * kRNi; e += kRThreads) rdst[e] = Rs[e];
    }
    // ---- kFlux, every 4 blocks and after the last: the lines at the Gauss
    // points, (L4 L3 w)(s, k) = scale_s sum_j Pc2g[k][j] line_s[j]
    if constexpr (kFlux) {
      if (slot == kRFlB - 1 || r0 + kRG >= nrhs) {
        __syncthreads();  // r has left the operand buffer
        {
          const int line = tid >> 1, half = tid & 1;
          const double* src = Fq + line * kRWp + half * 8;
          double v[8];
          uint32_t hm = 0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            v[j] = src[j];
            hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(v[j]) >> 32) &
                             0x7fffffffu);
          }
          hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, 1));
          const int e = exp_bound(hm);
          if (half == 0) el[line] = e;
          unsigned long long G[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) G[j] = fixed_point<56, kRSA>(v[j], e);
          const uint32_t base = tc::smem_u32(As + op_off(line, half * 8) * 2);
#pragma unroll
          for (int s = 1; s <= kRSA; ++s) store_slice<kRSA>(base + (s - 1) * kASliceB, G, s);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bp);
          constexpr uint32_t idesc = tc::idesc_bf16(128, kRP);
          for (int d = 2; d <= kRDiag + 1; ++d) {
            uint32_t acc = 0;
            for (int s = max(1, d - kRSB); s <= min(kRSA, d - 1); ++s) {
              const uint64_t da = tc::desc_kmajor(a0 + (uint32_t)((s - 1) * kASliceB), 128, 256);
              const uint64_t db =
                  tc::desc_kmajor(b0 + (uint32_t)((d - s - 1) * kBSliceB), 128, 256);
              tc::mma_bf16(tmem + (uint32_t)((d - 2) * kRP), da, db, idesc, acc);
              acc = 1;
            }
          }
          tc::commit(&bar);
        }
        if (!products_done()) {
          fail = true;
          break;
        }
        {
          // lane = line (block slot, grid, side); outputs: Gauss points c0 .. c0 + 7
          double out[8];
          drain8(tmem + tlane, c0, el[row], fq, out);
          const int sl = row >> 5, g = (row >> 2) & 7, s = row & 3;
          const int grid = r0 - slot * kRG + sl * kRG + g;
          if (grid < nrhs) {
            const double sc = (s & 1) ? sx : sy;
            double* dst = hp + (size_t)grid * ext_total + off + s * q;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (c0 + j < q) dst[c0 + j] = sc * out[j];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
    }
  }
  if (fail && tid == 0) {
    // the products that gave up may still be in flight: let them finish
    // (bounded) before the tensor memory is released
    tc::mbar_wait(&bar, phase, kRSpin);
    if (status) atomicCAS(status, 0, -1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRCols));
}

// ---------------------------------------------- leaf boundary rows, L1 u_e
// The boundary rows of a mixed solve's leaf values (Section 3.2, Step 1: each
// side's q Gauss values interpolated to its p Chebyshev points), which must
// be FP64 values in the range of L1 and identical in both leaves of a side:
// each (right-hand side, leaf, side) line is rounded to a 56-bit fixed point
// relative to its own largest exponent (so its result depends on the line
// alone) and interpolated as one exact digit product, 128 lines per tcgen05
// product against the digits of Pg2c (p x q, zero past q), drained by every
// warp into correctly rounded doubles.  Line id = (r nl + l) 4 + side;
// out[id p + j] = (Pg2c u_e(line))_j.  A persistent grid: CTA c takes rounds
// c, c + gridDim.x, ...
constexpr int kICols = kRDiag * kRP;  // TMEM columns: 8 diagonals x 16 points

__global__ void __launch_bounds__(kRThreads, 3) k_bnd_interp_tc(
    const double* __restrict__ uext, const int64_t* __restrict__ leaf_off, int l0, int nl,
    int64_t ext_total, int q, int nrhs, const double* __restrict__ gPg2c,
    double* __restrict__ out, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* As = smraw;                 // 7 digit slices: 128 lines
  unsigned char* Bp = As + kRSA * kASliceB;  // 8 digit slices of Pg2c
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int fq[kRP];  // exponents of the rows of Pg2c
  __shared__ int el[128];  // exponents of the lines
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nlines = (int64_t)nrhs * nl * 4;
  const int64_t rounds = (nlines + 127) / 128;
  if ((int64_t)blockIdx.x >= rounds) return;  // uniform: before any allocation
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_base)),
                 "r"(kICols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // row j of Pg2c (p x q), zero past q
  auto prow = [&](int j, int k) -> double { return k < q ? gPg2c[j * q + k] : 0.0; };
  if (tid < kRP) {
    uint32_t hm = 0;
    for (int k = 0; k < kRP; ++k)
      hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(prow(tid, k)) >> 32) &
                       0x7fffffffu);
    fq[tid] = exp_bound(hm);
  }
  __syncthreads();
  if (tid < 2 * kRP) {  // digits of Pg2c: thread (j, half), 8 entries of row j per slice
    const int j = tid >> 1, half = tid & 1;
    unsigned long long G[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) G[i] = fixed_point<62, kRSB>(prow(j, half * 8 + i), fq[j]);
    const uint32_t base = tc::smem_u32(Bp + op_off(j, half * 8) * 2);
#pragma unroll
    for (int t = 1; t <= kRSB; ++t) store_slice<kRSB>(base + (t - 1) * kBSliceB, G, t);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int row = 32 * (warp & 3) + lane;  // TMEM lane = line of the round
  const int c0 = 8 * (warp >> 2);          // the Chebyshev points this warp drains
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  bool fail = false;
  uint32_t phase = 0;
  // Gauss values half*8 .. +7 of line tid/2 of round rd (zero past q and
  // past the last line), loaded one round ahead
  double v[8];
  auto fetch = [&](int64_t rd) {
    const int half = tid & 1;
    const int64_t id = rd * 128 + (tid >> 1);
    const double* src = nullptr;
    if (rd < rounds && id < nlines) {
      const int side = (int)(id & 3);
      const int64_t rl = id >> 2;
      const int l = (int)(rl % nl), r = (int)(rl / nl);
      src = uext + (size_t)r * ext_total + leaf_off[l0 + l] + side * q;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = half * 8 + i;
      v[i] = (src && k < q) ? src[k] : 0.0;
    }
  };
  fetch(blockIdx.x);
  for (int64_t rd = blockIdx.x; rd < rounds; rd += gridDim.x) {
    __syncthreads();  // the previous round's products read As: complete (waited)
    // ---- thread (line, half) holds Gauss values half*8 .. +7 of its line
    {
      const int line = tid >> 1, half = tid & 1;
      uint32_t hm = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(v[i]) >> 32) &
                         0x7fffffffu);
      hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, 1));
      const int e = exp_bound(hm);
      if (half == 0) el[line] = e;
      unsigned long long G[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) G[i] = fixed_point<56, kRSA>(v[i], e);
      const uint32_t base = tc::smem_u32(As + op_off(line, half * 8) * 2);
#pragma unroll
      for (int s = 1; s <= kRSA; ++s) store_slice<kRSA>(base + (s - 1) * kASliceB, G, s);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bp);
      constexpr uint32_t idesc = tc::idesc_bf16(128, kRP);
      for (int d = 2; d <= kRDiag + 1; ++d) {
        uint32_t acc = 0;
        for (int s = max(1, d - kRSB); s <= min(kRSA, d - 1); ++s) {
          const uint64_t da = tc::desc_kmajor(a0 + (uint32_t)((s - 1) * kASliceB), 128, 256);
          const uint64_t db = tc::desc_kmajor(b0 + (uint32_t)((d - s - 1) * kBSliceB), 128, 256);
          tc::mma_bf16(tmem + (uint32_t)((d - 2) * kRP), da, db, idesc, acc);
          acc = 1;
        }
      }
      tc::commit(&bar);
    }
    fetch(rd + gridDim.x);  // in flight while the products run and drain
    {
      const bool ok = tc::mbar_wait(&bar, phase, kRSpin);
      if (__syncthreads_or(!ok)) {
        fail = true;
        break;
      }
      phase ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
      double o[8];
      drain8(tmem + tlane, c0, el[row], fq, o);
      const int64_t id = rd * 128 + row;
      if (id < nlines) {
        double2* dst = reinterpret_cast<double2*>(out + id * kRP + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_double2(o[2 * i], o[2 * i + 1]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (fail && tid == 0) {
    tc::mbar_wait(&bar, phase, kRSpin);  // the products that gave up finish first
    if (status) atomicCAS(status, 0, -1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kICols));
}

// ------------------------------------------------------------------ host
template <typename R, bool kFlux>
size_t resid_tc_smem(int q) {
  return (size_t)2 * kRSA * kASliceB + (size_t)(kFlux ? 2 : 1) * kRSB * kBSliceB +
         sizeof(double) * ((size_t)kRG * kRGs + 3 * kRGs +
                           (kFlux ? (size_t)kRFl * kRWp : (size_t)kRP * q));
}

// The operator and leaf shape the kernel takes: p = 16, q <= 16, no mixed or
// first-order term.
bool resid_tc_fits(const double* const* coef, int p, int q) {
  return p == kRP && q >= 1 && q <= kRP && !coef[1] && !coef[3] && !coef[4];
}

template <typename R, bool kFromY, bool kFlux>
void launch_resid_tc(const double* const* coef, int l0, int nl, int q, const double2* hsc,
                     const double* d_D, const double* d_Pm, double* const* wptr,
                     const int64_t* wrs, int nrhs, R* rbuf, const R* Y, int64_t ys,
                     const int64_t* leaf_off, int64_t ext_total, double* hp, int* status,
                     const char* name, cudaStream_t st) {
  static_assert((size_t)kRG * kRGs * 8 + kRG * kRNi * sizeof(R) <= (size_t)2 * kRSA * kASliceB,
                "Y and r fit in the operand buffer");
  if (nl <= 0 || nrhs <= 0) return;
  CoefPtrs cp;
  for (int k = 0; k < 6; ++k) cp.c[k] = coef[k];
  const size_t smem = resid_tc_smem<R, kFlux>(q);
  const void* kern = reinterpret_cast<const void*>(&k_leaf_resid_tc<R, kFromY, kFlux>);
  // the ceiling covers q <= 16 (a launch asking for more fails its launch check)
  if (!opt_in_smem(kern, (int)resid_tc_smem<R, kFlux>(kRP))) return;
  // the operation's FP64 flops per grid (what the FP64 pipe would execute):
  // X and Y at the interior nodes (16-term sums), the combination (3 per
  // node), the side derivatives (4 x 16 sums of 16 terms) and their Gauss
  // interpolation (4 q sums of 16 terms); bytes: the grid, r, the fluxes, and
  // the leaf's coefficients
  const double per = 2.0 * (2.0 * kRNi * kRP + 3.0 * kRNi +
                            (kFlux ? 4.0 * kRP * kRP + 4.0 * q * kRP : 0.0));
  const double in_bytes = kFromY ? (double)kRNi * sizeof(R) : (double)kRPP * 8.0;
  prof::Scope sc(name, st, (double)nl * nrhs * per,
                 (double)nl * (nrhs * (in_bytes + kRNi * sizeof(R) + (kFlux ? 32.0 * q : 0.0)) +
                               3.0 * kRPP * 8.0));
  k_leaf_resid_tc<R, kFromY, kFlux><<<nl, kRThreads, smem, st>>>(
      cp, l0, q, hsc, d_D, d_Pm, wptr, wrs, nrhs, rbuf, Y, ys, leaf_off, ext_total, hp, status);
}

}  // namespace

bool leaf_bnd_interp_tc(const double* uext, const int64_t* leaf_ext_off, int l0, int nleaves,
                        int64_t ext_total, int p, int q, int nrhs, const double* d_Pg2c,
                        double* out, int* status, cudaStream_t st) {
  if (p != kRP || q < 1 || q > kRP || !status) return false;
  if (nleaves <= 0 || nrhs <= 0) return true;
  const int64_t lines = (int64_t)nrhs * nleaves * 4, rounds = (lines + 127) / 128;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(rounds, (int64_t)std::max(nsm, 1) * 3);
  const size_t smem = (size_t)kRSA * kASliceB + (size_t)kRSB * kBSliceB;
  prof::Scope sc("leaf_bnd_tc<f64>", st, (double)lines * kRP * q * 2.0,
                 (double)lines * (q + kRP) * 8.0);
  k_bnd_interp_tc<<<grid, kRThreads, smem, st>>>(uext, leaf_ext_off, l0, nleaves, ext_total, q,
                                                  nrhs, d_Pg2c, out, status);
  return true;
}

template <typename R>
bool leaf_resflux_tc(const double* const* coef, int l0, int nl, int p, int q, const double2* hsc,
                     const double* d_D, const double* d_Pc2g, double* const* wptr,
                     const int64_t* wrs, int nrhs, R* rbuf, const int64_t* leaf_off,
                     int64_t ext_total, double* hp, int* status, cudaStream_t st) {
  if (!resid_tc_fits(coef, p, q)) return false;
  launch_resid_tc<R, false, true>(coef, l0, nl, q, hsc, d_D, d_Pc2g, wptr, wrs, nrhs, rbuf,
                                  nullptr, 0, leaf_off, ext_total, hp, status,
                                  "leaf_resflux_tc<f64>", st);
  return true;
}

template <typename R>
bool leaf_y_residual_tc(const double* const* coef, int l0, int nl, int p, int q,
                        const double2* hsc, const double* d_D, const double* d_Pg2c, const R* Y,
                        int64_t ys, R* rbuf, int* status, cudaStream_t st) {
  if (!resid_tc_fits(coef, p, q)) return false;
  launch_resid_tc<R, true, false>(coef, l0, nl, q, hsc, d_D, d_Pg2c, nullptr, nullptr, 4 * q,
                                  rbuf, Y, ys, nullptr, 0, nullptr, status,
                                  "leaf_yresid_tc<f64>", st);
  return true;
}

#define HPS_RESID_TC_INST(R)                                                                   \
  template bool leaf_resflux_tc<R>(const double* const*, int, int, int, int, const double2*,  \
                                   const double*, const double*, double* const*,               \
                                   const int64_t*, int, R*, const int64_t*, int64_t, double*,  \
                                   int*, cudaStream_t);                                        \
  template bool leaf_y_residual_tc<R>(const double* const*, int, int, int, int,                \
                                      const double2*, const double*, const double*, const R*,  \
                                      int64_t, R*, int*, cudaStream_t);
HPS_RESID_TC_INST(float)
HPS_RESID_TC_INST(double)
#undef HPS_RESID_TC_INST

}  // namespace hps
