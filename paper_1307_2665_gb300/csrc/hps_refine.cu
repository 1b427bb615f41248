// Accelerated iterative refinement: the vector work of one Anderson step.
//
// Refinement (mixed precision) produces, at iterate w_j of one right-hand side
// ("column"), the low-precision correction F_j (the elimination of Algorithms
// 1-2 applied to the FP64 residual of the global collocation system).  Plain
// refinement sets w_{j+1} = w_j + F_j.  Anderson acceleration of depth m keeps
// the last m differences dF_i = F_{i+1} - F_i and dW_i = w_{i+1} - w_i and sets
//   gamma   = argmin || F_j - sum_i gamma_i dF_i ||_2,
//   w_{j+1} = w_j + F_j - sum_i gamma_i (dW_i + dF_i),
// which on a linear fixed-point map is the GMRES iterate of the same Krylov
// space (Walker & Ni, SIAM J. Numer. Anal. 49, 2011).  The error of the FP32
// factors is dominated by a few slowly decaying modes; acceleration removes
// them in a few steps where plain refinement contracts by a fixed ratio.
//
// Layout ("F space"): column c = (problem k, right-hand side r) is one
// contiguous range [off_c, off_c + len_c) of every work vector, matching the
// element order of u (leaf-major, p*p nodes per leaf).  Everything that enters
// the new iterate is FP64: F, the previous F, the last update dW and the ring
// slots G = dW + dF.  A history rounded to FP32 would add, at every step, noise
// of 2^-24 times the early (large) differences, partly in smooth modes whose
// residual lies below the rounding level of the FP64 residual, where no later
// correction can see it.  Only the copies of dF that set the least-squares
// weights are FP32, and the dot products run in FP32 (weights need few digits;
// the FP64 pipe is the scarce one).
//
// The number of live history slots is a template parameter of both kernels:
// FP64 instructions of lanes predicated off still occupy the FP64 pipe (2 per
// clock per SM), so a loop unrolled to the maximum depth with a runtime guard
// cost the update 8 FP64 FMAs per element for 3 live slots.
//
// Reductions are deterministic: every column is cut into fixed chunks of
// kChunk elements (independent of the other columns), each chunk reduces in a
// fixed order into its own partial, and the partials of a column are summed
// in chunk order.  A column's results therefore do not depend on which other
// columns or problems share the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"

namespace hps {

namespace {

constexpr int kThreads = 256;
static_assert(kAaMaxDepth == 8, "the launch switches below cover depths 0..8");

// max of two non-negative doubles (or NaN patterns with the sign bit clear,
// which compare above every finite value and +inf) on their bit patterns
__device__ __forceinline__ double bitmax(double a, double b) {
  return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ long long absbits(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

// One CTA per chunk.  Partials, per chunk: [0] max|F|, [1] max|w|,
// [2 + s] <dF_s, F>, [2 + kAaMaxDepth + s] <dF_s, dF_new> for s < nslots (NS).
template <int NS>
__global__ void __launch_bounds__(kThreads) k_aa_reduce(const AaCol* __restrict__ cols,
                                                        const int* __restrict__ col_of,
                                                        const double* __restrict__ F,
                                                        double* Fprev,
                                                        const double* __restrict__ dWlast,
                                                        float* __restrict__ dF,
                                                        double* __restrict__ G, int64_t nu, int j,
                                                        int slot_new,
                                                        double* __restrict__ part) {
  constexpr int nslots = NS;
  const int64_t b = blockIdx.x;
  const AaCol c = cols[col_of[b]];
  const int64_t e0 = (b - c.ch0) * kAaChunk;
  const int64_t e1 = min(e0 + (int64_t)kAaChunk, c.len);
  long long mf = 0, mw = 0;  // |F|, |w| maxima as bit patterns (exact, NaN-preserving)
  float accF[NS > 0 ? NS : 1], accD[NS > 0 ? NS : 1];
#pragma unroll
  for (int s = 0; s < NS; ++s) accF[s] = accD[s] = 0.0f;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
    const int64_t i = c.off + e;
    const double fv = F[i];
    const float f32 = (float)fv;
    mf = max(mf, absbits(fv));
    mw = max(mw, absbits(c.w[e]));
    float dfn = 0.0f;
    if (j >= 1) {
      const double d = fv - Fprev[i];
      dfn = (float)d;
      dF[(int64_t)slot_new * nu + i] = dfn;
      G[(int64_t)slot_new * nu + i] = dWlast[i] + d;
    }
    if (Fprev) Fprev[i] = fv;  // null for plain refinement (no history)
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float d = (s == slot_new) ? dfn : dF[(int64_t)s * nu + i];
      accF[s] = fmaf(d, f32, accF[s]);
      accD[s] = fmaf(d, dfn, accD[s]);
    }
  }
  // fixed-order block reduction
  constexpr int Q = kAaQ;
  __shared__ double red[kThreads / 32][Q];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  auto warp_sum = [&](float v) {
    double x = v;  // per-thread sums in FP32, the rest of the tree in FP64
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  auto warp_max = [&](long long v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return __longlong_as_double(v);
  };
  const double mfd = warp_max(mf), mwd = warp_max(mw);
  if (lane == 0) {
    red[wid][0] = mfd;
    red[wid][1] = mwd;
  }
#pragma unroll
  for (int s = 0; s < kAaMaxDepth; ++s) {
    const double a = s < NS ? warp_sum(accF[s < NS ? s : 0]) : 0.0;
    const double d = s < NS ? warp_sum(accD[s < NS ? s : 0]) : 0.0;
    if (lane == 0) {
      red[wid][2 + s] = a;
      red[wid][2 + kAaMaxDepth + s] = d;
    }
  }
  __syncthreads();
  if (threadIdx.x < Q) {
    const int q = threadIdx.x;
    double v = red[0][q];
    for (int w = 1; w < kThreads / 32; ++w) v = (q < 2) ? bitmax(v, red[w][q]) : v + red[w][q];
    part[b * Q + q] = v;
  }
}

// One CTA per column: sums (or maxima) of its chunks' partials in chunk order.
__global__ void k_aa_colsum(const AaCol* __restrict__ cols, const double* __restrict__ part,
                            double* __restrict__ colsum) {
  const AaCol c = cols[blockIdx.x];
  const int64_t nch = (c.len + kAaChunk - 1) / kAaChunk;
  const int q = threadIdx.x;
  if (q >= kAaQ) return;
  double v = 0.0;
  for (int64_t k = 0; k < nch; ++k) {
    const double x = part[(c.ch0 + k) * kAaQ + q];
    v = (q < 2) ? bitmax(v, x) : v + x;
  }
  colsum[(int64_t)blockIdx.x * kAaQ + q] = v;
}

// coef[c*(kAaMaxDepth+1)]: 0 frozen, 1 accelerated update, 2 plain update
// (w += F); then gamma_s for the NS live slots.
template <int NS>
__global__ void __launch_bounds__(kThreads) k_aa_update(const AaCol* __restrict__ cols,
                                                        const int* __restrict__ col_of,
                                                        const double* __restrict__ F,
                                                        double* __restrict__ dWlast,
                                                        const double* __restrict__ G, int64_t nu,
                                                        const double* __restrict__ coef) {
  const int64_t b = blockIdx.x;
  const int ci = col_of[b];
  const AaCol c = cols[ci];
  const double* cf = coef + (int64_t)ci * (kAaMaxDepth + 1);
  const int mode = (int)cf[0];
  if (mode == 0) return;
  double g[NS > 0 ? NS : 1];
#pragma unroll
  for (int s = 0; s < NS; ++s) g[s] = mode == 1 ? cf[1 + s] : 0.0;
  const int64_t e0 = (b - c.ch0) * kAaChunk;
  const int64_t e1 = min(e0 + (int64_t)kAaChunk, c.len);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
    const int64_t i = c.off + e;
    double d = F[i];
    if (mode == 1) {
#pragma unroll
      for (int s = 0; s < NS; ++s) d = fma(-g[s], G[(int64_t)s * nu + i], d);
      dWlast[i] = d;
    }
    c.w[e] += d;
  }
}

}  // namespace

void aa_reduce(const AaCol* cols, const int* col_of, int ncol, int64_t nchunks, const double* F,
               double* Fprev,
               const double* dWlast, float* dF, double* G, int64_t nu, int j, int slot_new,
               int nslots, double* part, double* colsum, cudaStream_t st) {
  if (ncol <= 0 || nchunks <= 0) return;
  // bytes: F, w, Fprev read and written; with history dW, dF_new, G_new and
  // the older dF slots
  prof::Scope sc("refine_reduce", st, 4.0 * nslots * (double)nu,
                 (double)nu * (8.0 + 8.0 + 16.0 + (j >= 1 ? 8.0 + 4.0 + 8.0 : 0.0) +
                               4.0 * std::max(nslots - 1, 0)));
  switch (nslots) {
#define HPS_AA_REDUCE(NS)                                                                        \
  case NS:                                                                                       \
    k_aa_reduce<NS><<<(unsigned)nchunks, kThreads, 0, st>>>(cols, col_of, F, Fprev, dWlast, dF, G, \
                                                          nu, j, slot_new, part);              \
    break;
    HPS_AA_REDUCE(0) HPS_AA_REDUCE(1) HPS_AA_REDUCE(2) HPS_AA_REDUCE(3) HPS_AA_REDUCE(4)
    HPS_AA_REDUCE(5) HPS_AA_REDUCE(6) HPS_AA_REDUCE(7) HPS_AA_REDUCE(8)
#undef HPS_AA_REDUCE
    default: return;  // beyond kAaMaxDepth: rejected by the caller
  }
  k_aa_colsum<<<(unsigned)ncol, 32, 0, st>>>(cols, part, colsum);
}

void aa_update(const AaCol* cols, const int* col_of, int ncol, int64_t nchunks, const double* F,
               double* dWlast,
               const double* G, int64_t nu, int nslots, const double* coef, cudaStream_t st) {
  if (ncol <= 0 || nchunks <= 0) return;
  prof::Scope sc("refine_update", st, 2.0 * nslots * (double)nu,
                 (double)nu * (8.0 + 16.0 + 8.0 + 8.0 * nslots));
  switch (nslots) {
#define HPS_AA_UPDATE(NS)                                                                     \
  case NS:                                                                                    \
    k_aa_update<NS><<<(unsigned)nchunks, kThreads, 0, st>>>(cols, col_of, F, dWlast, G, nu, \
                                                          coef);                            \
    break;
    HPS_AA_UPDATE(0) HPS_AA_UPDATE(1) HPS_AA_UPDATE(2) HPS_AA_UPDATE(3) HPS_AA_UPDATE(4)
    HPS_AA_UPDATE(5) HPS_AA_UPDATE(6) HPS_AA_UPDATE(7) HPS_AA_UPDATE(8)
#undef HPS_AA_UPDATE
    default: return;
  }
}

}  // namespace hps
