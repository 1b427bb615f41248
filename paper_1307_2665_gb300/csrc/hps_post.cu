// Post-processing kernels: the root DtN map applied to Dirichlet data
// (Section 9.1 times it as T_apply, Table 1), and the solution evaluated at
// arbitrary points (Section 5.3).
//
// T^1 apply.  The root DtN T of a problem maps the Dirichlet values at the
// root's exterior Gauss nodes to the boundary fluxes v there (Section 2: d/dx
// on vertical sides, d/dy on horizontal sides, in the global direction); it is
// kept column-major in the root's exterior order, and rff[k] names the Gamma
// index of exterior position k.  g = T f is therefore a gather of f into the
// exterior order, a dense product, and a scatter back.  One right-hand side
// is HBM-bound (T read once, one FMA per element); from two on the FP64 FMAs
// bound the product, so 16 or more right-hand sides take the tensor-core FP64
// GEMM.  Fewer run as matvec passes of NR = 8, 4, 2, 1 right-hand sides
// (NR a template parameter: predicated-off FMAs would still occupy the FP64
// pipe): one thread per row, the columns split into fixed chunks of kDtnChunk
// whose partial sums are added in chunk order, so the result of a right-hand
// side does not depend on the others.
//
// Point evaluation.  Inside a leaf the solution is the tensor-product
// polynomial interpolant of its p x p Chebyshev values; it is evaluated with
// the barycentric formula for Chebyshev points of the second kind (Berrut &
// Trefethen, SIAM Review 46, 2004: weights (-1)^j, halved at the two ends).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"

namespace hps {

namespace {

constexpr int kDtnChunk = 128;  // columns per partial sum
constexpr int kDtnRows = 256;   // rows (threads) per CTA
constexpr int kDtnTcMin = 16;   // right-hand sides from which the tensor cores take the product

bool dtn_use_tc(int n, int nrhs) { return n >= 128 && nrhs >= kDtnTcMin; }

__global__ void k_dtn_gather(const double* __restrict__ f, const int* __restrict__ rff, int n,
                             int nrhs, double* __restrict__ fr) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int k = (int)(e % n);
  const int64_t r = e / n;
  fr[e] = f[r * n + rff[k]];
}

// part[(kc * nrhs + r) * n + i] = sum over the chunk's columns l of T[i, l] fr[r, l],
// for the right-hand sides r0 .. r0 + NR - 1 of this pass.  Eight column loads
// of a thread are issued before their FMAs.
template <int NR>
__global__ void __launch_bounds__(kDtnRows) k_dtn_matvec(const double* __restrict__ T, int n,
                                                         const double* __restrict__ fr, int nrhs,
                                                         int r0, double* __restrict__ part) {
  __shared__ double xs[NR][kDtnChunk];
  const int kc = blockIdx.y;
  const int c0 = kc * kDtnChunk, c1 = min(n, c0 + kDtnChunk);
  for (int e = threadIdx.x; e < NR * kDtnChunk; e += blockDim.x) {
    const int r = e / kDtnChunk, l = e % kDtnChunk;
    xs[r][l] = (c0 + l < c1) ? fr[(int64_t)(r0 + r) * n + c0 + l] : 0.0;
  }
  __syncthreads();
  const int i = blockIdx.x * kDtnRows + threadIdx.x;
  if (i >= n) return;
  double acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = 0.0;
  const double* col = T + i + (size_t)c0 * n;
  const int len = c1 - c0;
  int l = 0;
  for (; l + 8 <= len; l += 8) {
    double t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = col[(size_t)(l + u) * n];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] = fma(t[u], xs[r][l + u], acc[r]);
  }
  for (; l < len; ++l) {
    const double t = col[(size_t)l * n];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = fma(t, xs[r][l], acc[r]);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) part[((int64_t)kc * nrhs + r0 + r) * n + i] = acc[r];
}

// g[r * n + rff[i]] = sum over chunks kc (in order) of part[(kc * nrhs + r) * n + i]
__global__ void k_dtn_reduce(const double* __restrict__ part, int n, int nrhs, int nchunks,
                             const int* __restrict__ rff, double* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int i = (int)(e % n);
  const int64_t r = e / n;
  double s = 0.0;
  for (int kc = 0; kc < nchunks; ++kc) s += part[((int64_t)kc * nrhs + r) * n + i];
  g[r * n + rff[i]] = s;
}

__global__ void k_dtn_scatter(const double* __restrict__ gr, const int* __restrict__ rff, int n,
                              int nrhs, double* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int i = (int)(e % n);
  const int64_t r = e / n;
  g[r * n + rff[i]] = gr[e];
}

__global__ void k_f2d(const float* __restrict__ s, double* __restrict__ d, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) d[e] = (double)s[e];
}

__global__ void k_d2f(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) d[e] = (float)s[e];
}

// Barycentric Lagrange basis of the p Chebyshev points of the second kind
// ts (increasing), at t; exactly 1 / 0 when t is a node.
__device__ void cheb_basis(double t, int p, const double* ts, double* ell) {
  double den = 0.0;
  int hit = -1;
  for (int j = 0; j < p; ++j) {
    const double d = t - ts[j];
    if (d == 0.0) hit = j;
    double wj = (j & 1) ? -1.0 : 1.0;
    if (j == 0 || j == p - 1) wj *= 0.5;
    ell[j] = wj / d;
    den += ell[j];
  }
  if (hit >= 0) {
    for (int j = 0; j < p; ++j) ell[j] = (j == hit) ? 1.0 : 0.0;
    return;
  }
  const double inv = 1.0 / den;
  for (int j = 0; j < p; ++j) ell[j] *= inv;
}

// One thread per point (all right-hand sides); the nodes are computed once per
// CTA.  out[r * npts + i] = u_r(x_i, y_i).
__global__ void __launch_bounds__(128) k_interp(const double* __restrict__ u, int nrhs,
                                                int64_t per_rhs, InterpGrid s,
                                                const double* __restrict__ xy, int64_t npts,
                                                double* __restrict__ out,
                                                int* __restrict__ status) {
  __shared__ double ts[64];
  const int p = s.p;
  if (threadIdx.x < p) ts[threadIdx.x] = -cospi((double)threadIdx.x / (double)(p - 1));
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double x = xy[2 * i], y = xy[2 * i + 1];
  if (!(x >= s.x0 && x <= s.x1 && y >= s.y0 && y <= s.y1)) {
    for (int r = 0; r < nrhs; ++r) out[r * npts + i] = __longlong_as_double(0x7ff8000000000000LL);
    if (status) atomicCAS(status, 0, 1);
    return;
  }
  // leaf: the one to the east (north) of a shared edge, the last one on the
  // domain's east (north) side
  const double sx = (x - s.x0) / (s.x1 - s.x0) * s.nx;
  const double sy = (y - s.y0) / (s.y1 - s.y0) * s.ny;
  const int ix = min((int)floor(sx), s.nx - 1), iy = min((int)floor(sy), s.ny - 1);
  double lx[64], ly[64];
  cheb_basis(2.0 * (sx - ix) - 1.0, p, ts, lx);
  cheb_basis(2.0 * (sy - iy) - 1.0, p, ts, ly);
  const int64_t leaf = ((int64_t)iy * s.nx + ix) * p * p;
  for (int r = 0; r < nrhs; ++r) {
    const double* w = u + r * per_rhs + leaf;
    double acc = 0.0;
    for (int a = 0; a < p; ++a) {
      double row = 0.0;
      for (int b = 0; b < p; ++b) row = fma(lx[b], w[a * p + b], row);
      acc = fma(ly[a], row, acc);
    }
    out[r * npts + i] = acc;
  }
}

}  // namespace

size_t dtn_apply_ws_bytes(int n, int nrhs) {
  const size_t fr = (size_t)n * nrhs * sizeof(double);
  const int nchunks = (n + kDtnChunk - 1) / kDtnChunk;
  if (dtn_use_tc(n, nrhs)) {
    std::vector<OzDesc> h(1);
    h[0].M = n;
    h[0].N = nrhs;
    h[0].K = n;
    const size_t oz = (oz_plan(h) + 255) & ~size_t(255);
    return 2 * ((fr + 255) & ~size_t(255)) + oz + 256;
  }
  return ((fr + 255) & ~size_t(255)) + (size_t)nchunks * n * nrhs * sizeof(double);
}

cudaError_t dtn_apply(const double* T, int n, const int* rff, const double* f, int nrhs,
                      double* g, void* ws, size_t ws_bytes, int* status, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (ws_bytes < dtn_apply_ws_bytes(n, nrhs)) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(ws);
  double* fr = reinterpret_cast<double*>(w);
  w += ((size_t)n * nrhs * sizeof(double) + 255) & ~size_t(255);
  const int64_t tot = (int64_t)n * nrhs;
  const unsigned eb = (unsigned)((tot + 255) / 256);
  {
    prof::Scope sc("dtn_gather", st, 0.0, 16.0 * tot);
    k_dtn_gather<<<eb, 256, 0, st>>>(f, rff, n, nrhs, fr);
  }
  if (dtn_use_tc(n, nrhs)) {
    double* gr = reinterpret_cast<double*>(w);
    w += ((size_t)n * nrhs * sizeof(double) + 255) & ~size_t(255);
    std::vector<OzDesc> h(1);
    h[0].A = T;
    h[0].B = fr;
    h[0].C = gr;
    h[0].M = n;
    h[0].N = nrhs;
    h[0].K = n;
    h[0].lda = n;
    h[0].ldb = n;
    h[0].ldc = n;
    const size_t ob = oz_plan(h);
    OzDesc* dd = reinterpret_cast<OzDesc*>(w);
    void* ow = w + 256;
    cudaError_t e = cudaMemcpyAsync(dd, h.data(), sizeof(OzDesc), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = oz_gemm(dd, h, ow, ob, 1.0, 0.0, status, st, "dtn_apply_tc<f64>");
    if (e != cudaSuccess) return e;
    prof::Scope sc("dtn_scatter", st, 0.0, 16.0 * tot);
    k_dtn_scatter<<<eb, 256, 0, st>>>(gr, rff, n, nrhs, g);
    return cudaGetLastError();
  }
  double* part = reinterpret_cast<double*>(w);
  const int nchunks = (n + kDtnChunk - 1) / kDtnChunk;
  const dim3 grid((unsigned)((n + kDtnRows - 1) / kDtnRows), (unsigned)nchunks);
  for (int r0 = 0; r0 < nrhs;) {
    const int nr = nrhs - r0 >= 8 ? 8 : nrhs - r0 >= 4 ? 4 : nrhs - r0 >= 2 ? 2 : 1;
    // bytes: T once per pass, the data and the partial sums
    prof::Scope sc("dtn_matvec", st, 2.0 * n * (double)n * nr,
                   8.0 * ((double)n * n + (double)n * nr * (1 + nchunks)));
    switch (nr) {
      case 8: k_dtn_matvec<8><<<grid, kDtnRows, 0, st>>>(T, n, fr, nrhs, r0, part); break;
      case 4: k_dtn_matvec<4><<<grid, kDtnRows, 0, st>>>(T, n, fr, nrhs, r0, part); break;
      case 2: k_dtn_matvec<2><<<grid, kDtnRows, 0, st>>>(T, n, fr, nrhs, r0, part); break;
      default: k_dtn_matvec<1><<<grid, kDtnRows, 0, st>>>(T, n, fr, nrhs, r0, part); break;
    }
    r0 += nr;
  }
  prof::Scope sc("dtn_reduce", st, (double)tot * nchunks, 8.0 * tot * (nchunks + 1));
  k_dtn_reduce<<<eb, 256, 0, st>>>(part, n, nrhs, nchunks, rff, g);
  return cudaGetLastError();
}

void f32_to_f64(const float* s, double* d, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  prof::Scope sc("f32_to_f64", st, 0.0, 12.0 * n);
  k_f2d<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, d, n);
}

void f64_to_f32(const double* s, float* d, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  prof::Scope sc("f64_to_f32", st, 0.0, 12.0 * n);
  k_d2f<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, d, n);
}

void interp_points(const double* u, int nrhs, const InterpGrid& s, const double* xy,
                   int64_t npts, double* out, int* status, cudaStream_t st) {
  if (npts <= 0 || nrhs <= 0) return;
  const int64_t tot = npts * nrhs;
  const int64_t pp = (int64_t)s.p * s.p;
  prof::Scope sc("interp_points", st, (double)tot * (2.0 * pp + 8.0 * s.p),
                 (double)tot * (8.0 * pp + 8.0) + 16.0 * npts);
  k_interp<<<(unsigned)((npts + 127) / 128), 128, 0, st>>>(u, nrhs, (int64_t)s.nx * s.ny * pp, s,
                                                          xy, npts, out, status);
}

}  // namespace hps
