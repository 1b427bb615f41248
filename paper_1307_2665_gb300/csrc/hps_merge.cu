// Merge gather and downward-pass scatter kernels (Section 4, Algorithms 1-2).
//
// A merge of children alpha, beta into tau needs, in the parent's exterior
// ordering (J1, J2 interleaved as the parent's sides require):
//   Aw = T33^a - T33^b                       (m x m)
//   S  = [-T31^a | T32^b]                    (m x ne)   -> Aw^{-1} S by the LU
//   Cw = [T13^a ; T23^b]                     (ne x m)
//   Tp = diag(T11^a, T22^b)                  (ne x ne)  -> Tp + Cw S by a GEMM
// J3 is a contiguous run of each child's exterior (alpha's east or north side,
// beta's west or south side); src[k] names the child entry of parent position k.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"

namespace hps {

__device__ __forceinline__ double tload(const void* p, int f64, int64_t i) {
  return f64 ? static_cast<const double*>(p)[i] : (double)static_cast<const float*>(p)[i];
}

// I: the index type, 32-bit whenever every merge of the launch has fewer than
// 2^31 entries to write (integer division and modulo by m and ne per entry
// cost several times as much in 64 bits).
template <typename R, typename I>
__global__ void __launch_bounds__(256) k_merge_gather(const MergeDesc<R>* __restrict__ d,
                                                      int chunks, int64_t per_chunk) {
  const MergeDesc<R> g = d[blockIdx.x / chunks];
  const int chunk = blockIdx.x % chunks;
  const I m = g.m, ne = g.ne;
  const I nA = m * m, nS = m * ne, nC = ne * m, nT = g.Tp ? ne * ne : 0;
  const I nW = g.W ? m * m : 0;
  const I total = nA + nS + nC + nT + nW;
  const I beg = (I)(chunk * per_chunk);
  const I end = min(total, (I)(beg + per_chunk));
  const int64_t na = g.na, nb = g.nb;
  for (I e = beg + (I)threadIdx.x; e < end; e += (I)blockDim.x) {
    if (e < nA) {
      I i = e % m, j = e / m;
      g.Aw[e] = (R)(tload(g.Ta, g.ta64, (g.j3a + i) + (g.j3a + j) * na) -
                    tload(g.Tb, g.tb64, (g.j3b + i) + (g.j3b + j) * nb));
    } else if (e < nA + nS) {
      I x = e - nA, i = x % m, k = x / m;
      int s = g.src[k];
      g.S[x] = s >= 0 ? (R)(-tload(g.Ta, g.ta64, (g.j3a + i) + (int64_t)s * na))
                      : (R)tload(g.Tb, g.tb64, (g.j3b + i) + (int64_t)(-s - 1) * nb);
    } else if (e < nA + nS + nC) {
      I x = e - nA - nS, k = x % ne, i = x / ne;
      int s = g.src[k];
      g.Cw[x] = s >= 0 ? (R)tload(g.Ta, g.ta64, s + (g.j3a + i) * na)
                       : (R)tload(g.Tb, g.tb64, (int64_t)(-s - 1) + (g.j3b + i) * nb);
    } else if (e >= nA + nS + nC + nT) {
      I x = e - nA - nS - nC - nT;
      g.W[x] = (x % m == x / m) ? R(1) : R(0);
    } else {
      I x = e - nA - nS - nC, k = x % ne, k2 = x / ne;
      int s = g.src[k], s2 = g.src[k2];
      R v = R(0);
      if (s >= 0 && s2 >= 0)
        v = (R)tload(g.Ta, g.ta64, s + (int64_t)s2 * na);
      else if (s < 0 && s2 < 0)
        v = (R)tload(g.Tb, g.tb64, (int64_t)(-s - 1) + (int64_t)(-s2 - 1) * nb);
      g.Tp[x] = v;
    }
  }
}

template <typename R>
void merge_gather(const MergeDesc<R>* d_desc, int ndesc, int64_t max_work, cudaStream_t st,
                  double bytes) {
  if (ndesc <= 0 || max_work <= 0) return;
  const int64_t per_chunk = 256 * 16;
  int chunks = (int)((max_work + per_chunk - 1) / per_chunk);
  prof::Scope sc(sizeof(R) == 8 ? "merge_gather<f64>" : "merge_gather<f32>", st, 0.0, bytes);
  if (max_work < ((int64_t)1 << 31) - per_chunk)
    k_merge_gather<R, int><<<(unsigned)((int64_t)ndesc * chunks), 256, 0, st>>>(d_desc, chunks,
                                                                               per_chunk);
  else
    k_merge_gather<R, int64_t><<<(unsigned)((int64_t)ndesc * chunks), 256, 0, st>>>(
        d_desc, chunks, per_chunk);
}

// ------------------------------------------------------ body-load upward pass
// The body-load kernels below give a thread one entry of a merge and loop over
// the right-hand sides, eight loads before eight stores (the pools' source and
// destination parts are disjoint, which the compiler cannot know: one memory
// round trip per value otherwise); blocks of up to 256 threads per merge.
constexpr int kBodyBatch = 8;
static void body_grid(int nd, int max_n, int* threads, int* bpd) {
  *threads = max_n >= 256 ? 256 : std::max(32, ((max_n + 31) / 32) * 32);
  *bpd = (max_n + *threads - 1) / *threads;
  (void)nd;
}

// Right-hand side of a merge's interface equation for the correction:
// (T33^a - T33^b) z = h3^b - h3^a, the flux offsets of the two children at J3.
template <typename R>
__global__ void k_merge_rhs(const BodyDesc* __restrict__ d, int bpd,
                            const double* __restrict__ hp, int64_t ext_total, int nrhs,
                            R* __restrict__ zlev) {
  const BodyDesc g = d[blockIdx.x / bpd];
  const int i = (blockIdx.x % bpd) * blockDim.x + threadIdx.x;
  if (i >= g.m) return;
  const double* hb = hp + g.b_off + g.j3b + i;
  const double* ha = hp + g.a_off + g.j3a + i;
  R* z = zlev + g.z_off * nrhs + i;
  int r0 = 0;
  for (; r0 + kBodyBatch <= nrhs; r0 += kBodyBatch) {
    R v[kBodyBatch];
#pragma unroll
    for (int j = 0; j < kBodyBatch; ++j) {
      const size_t o = (size_t)(r0 + j) * ext_total;
      v[j] = (R)(hb[o] - ha[o]);
    }
#pragma unroll
    for (int j = 0; j < kBodyBatch; ++j) z[(size_t)(r0 + j) * g.m] = v[j];
  }
  for (; r0 < nrhs; ++r0) {
    const size_t o = (size_t)r0 * ext_total;
    z[(size_t)r0 * g.m] = (R)(hb[o] - ha[o]);
  }
}

// The parent's flux offsets before the Schur term: h^tau(k) = h^a(src) or h^b(src).
__global__ void k_merge_hpar(const BodyDesc* __restrict__ d, int bpd, double* __restrict__ hp,
                             int64_t ext_total, int nrhs) {
  const BodyDesc g = d[blockIdx.x / bpd];
  const int k = (blockIdx.x % bpd) * blockDim.x + threadIdx.x;
  if (k >= g.ne) return;
  const int s = g.src[k];
  const double* src = hp + (s >= 0 ? g.a_off + s : g.b_off + (-s - 1));
  double* dst = hp + g.par_off + k;
  int r0 = 0;
  for (; r0 + kBodyBatch <= nrhs; r0 += kBodyBatch) {
    double v[kBodyBatch];
#pragma unroll
    for (int j = 0; j < kBodyBatch; ++j) v[j] = src[(size_t)(r0 + j) * ext_total];
#pragma unroll
    for (int j = 0; j < kBodyBatch; ++j) dst[(size_t)(r0 + j) * ext_total] = v[j];
  }
  for (; r0 < nrhs; ++r0) dst[(size_t)r0 * ext_total] = src[(size_t)r0 * ext_total];
}

// u3 := z (the particular part of the interface values), before u3 += S u_parent.
template <typename R>
__global__ void k_z_to_u3(const BodyDesc* __restrict__ d, int bpd, const R* __restrict__ zlev,
                          double* __restrict__ u3, int64_t u3_total, int nrhs) {
  const BodyDesc g = d[blockIdx.x / bpd];
  const int i = (blockIdx.x % bpd) * blockDim.x + threadIdx.x;
  if (i >= g.m) return;
  const R* z = zlev + g.z_off * nrhs + i;
  double* u = u3 + g.u3_off + i;
  int r0 = 0;
  for (; r0 + kBodyBatch <= nrhs; r0 += kBodyBatch) {
    double v[kBodyBatch];
#pragma unroll
    for (int j = 0; j < kBodyBatch; ++j) v[j] = (double)z[(size_t)(r0 + j) * g.m];
#pragma unroll
    for (int j = 0; j < kBodyBatch; ++j) u[(size_t)(r0 + j) * u3_total] = v[j];
  }
  for (; r0 < nrhs; ++r0) u[(size_t)r0 * u3_total] = (double)z[(size_t)r0 * g.m];
}

template <typename R>
void merge_rhs(const BodyDesc* d, int nd, int max_m, const double* hp, int64_t ext_total,
               int nrhs, R* zlev, cudaStream_t st) {
  if (nd <= 0 || max_m <= 0) return;
  int threads, bpd;
  body_grid(nd, max_m, &threads, &bpd);
  prof::Scope sc("merge_rhs", st, 0.0, (double)nd * max_m * nrhs * (16.0 + sizeof(R)));
  k_merge_rhs<R><<<(unsigned)((int64_t)nd * bpd), threads, 0, st>>>(d, bpd, hp, ext_total, nrhs,
                                                                    zlev);
}

void merge_hpar(const BodyDesc* d, int nd, int max_ne, double* hp, int64_t ext_total, int nrhs,
                cudaStream_t st) {
  if (nd <= 0 || max_ne <= 0) return;
  int threads, bpd;
  body_grid(nd, max_ne, &threads, &bpd);
  prof::Scope sc("merge_hpar", st, 0.0, (double)nd * max_ne * nrhs * 16.0);
  k_merge_hpar<<<(unsigned)((int64_t)nd * bpd), threads, 0, st>>>(d, bpd, hp, ext_total, nrhs);
}

template <typename R>
void z_to_u3(const BodyDesc* d, int nd, int max_m, const R* zlev, double* u3, int64_t u3_total,
             int nrhs, cudaStream_t st) {
  if (nd <= 0 || max_m <= 0) return;
  int threads, bpd;
  body_grid(nd, max_m, &threads, &bpd);
  prof::Scope sc("z_to_u3", st, 0.0, (double)nd * max_m * nrhs * (8.0 + sizeof(R)));
  k_z_to_u3<R><<<(unsigned)((int64_t)nd * bpd), threads, 0, st>>>(d, bpd, zlev, u3, u3_total,
                                                                  nrhs);
}

// ----------------------------------------------------------- downward pass
// Exterior-value pool: uext[r*ext_total + box.ext_off + i] for right-hand side r.
__global__ void k_root_scatter(const RootDesc* __restrict__ d, int chunks, int nrhs,
                               double* __restrict__ uext, int64_t ext_total) {
  const RootDesc g = d[blockIdx.x / chunks];
  const int64_t n = (int64_t)g.nbnd * nrhs;
  for (int64_t e = (int64_t)(blockIdx.x % chunks) * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)chunks * blockDim.x) {
    const int k = (int)(e % g.nbnd);
    const int64_t r = e / g.nbnd;
    uext[r * ext_total + g.root_off + k] = g.f ? g.f[r * g.nbnd + g.rff[k]] : 0.0;
  }
}

void solve_root_scatter(const RootDesc* d, int nprob, int max_nbnd, int nrhs, double* uext,
                        int64_t ext_total, cudaStream_t st) {
  if (nprob <= 0) return;
  int chunks = (int)std::min<int64_t>(((int64_t)max_nbnd * nrhs + 255) / 256, 64);
  if (chunks < 1) return;
  prof::Scope sc("root_scatter", st, 0.0, 16.0 * nprob * (double)max_nbnd * nrhs);
  k_root_scatter<<<(unsigned)((int64_t)nprob * chunks), 256, 0, st>>>(d, chunks, nrhs, uext,
                                                                      ext_total);
}

// children's exterior values from the parent's and u3 = S u_parent.  A thread
// owns one exterior entry of a child (its source read once from the map) and
// copies it for every right-hand side, eight loads before eight stores (the
// source and destination are disjoint parts of the pools, which the compiler
// cannot know: one memory round trip per value otherwise).
__global__ void k_child_scatter(const SolveScatterDesc* __restrict__ d, int bpd,
                                const double* __restrict__ u3, int64_t u3_total,
                                double* __restrict__ uext, int64_t ext_total, int nrhs) {
  const SolveScatterDesc g = d[blockIdx.x / bpd];
  const int i = (blockIdx.x % bpd) * blockDim.x + threadIdx.x;
  if (i >= g.na + g.nb) return;
  const bool in_a = i < g.na;
  const int c = in_a ? g.cmap_a[i] : g.cmap_b[i - g.na];
  const int64_t dst = in_a ? g.a_off + i : g.b_off + (i - g.na);
  const double* src = c >= 0 ? uext + g.par_off + c : u3 + g.u3_off + (-c - 1);
  const int64_t ss = c >= 0 ? ext_total : u3_total;
  double* out = uext + dst;
  constexpr int kB = 8;
  int r0 = 0;
  for (; r0 + kB <= nrhs; r0 += kB) {
    double v[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) v[j] = src[(size_t)(r0 + j) * ss];
#pragma unroll
    for (int j = 0; j < kB; ++j) out[(size_t)(r0 + j) * ext_total] = v[j];
  }
  for (; r0 < nrhs; ++r0) out[(size_t)r0 * ext_total] = src[(size_t)r0 * ss];
}

void solve_child_scatter(const SolveScatterDesc* d_desc, int ndesc, int max_n, const double* u3,
                         int64_t u3_total, double* uext, int64_t ext_total, int nrhs,
                         cudaStream_t st) {
  if (ndesc <= 0 || max_n <= 0) return;
  const int threads = max_n >= 256 ? 256 : ((max_n + 31) / 32) * 32;
  const int bpd = (max_n + threads - 1) / threads;
  prof::Scope sc("child_scatter", st, 0.0, 2.0 * (double)ndesc * max_n * nrhs * 8.0);
  k_child_scatter<<<(unsigned)((int64_t)ndesc * bpd), threads, 0, st>>>(
      d_desc, bpd, u3, u3_total, uext, ext_total, nrhs);
}

template void merge_gather<double>(const MergeDesc<double>*, int, int64_t, cudaStream_t, double);
template void merge_gather<float>(const MergeDesc<float>*, int, int64_t, cudaStream_t, double);
template void merge_rhs<double>(const BodyDesc*, int, int, const double*, int64_t, int, double*,
                                cudaStream_t);
template void merge_rhs<float>(const BodyDesc*, int, int, const double*, int64_t, int, float*,
                               cudaStream_t);
template void z_to_u3<double>(const BodyDesc*, int, int, const double*, double*, int64_t, int,
                              cudaStream_t);
template void z_to_u3<float>(const BodyDesc*, int, int, const float*, double*, int64_t, int,
                             cudaStream_t);

}  // namespace hps
