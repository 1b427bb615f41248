// Leaf kernels (Section 3 and Section 5.3).
//
// On the p x p Chebyshev grid of a leaf the operator of eq. defA is the
// collocation matrix of Section 3.1,
//   A = -C11 Dx^2 - 2 C12 Dx Dy - C22 Dy^2 + C1 Dx + C2 Dy + C,
// with Dx = (2/hx) I (x) D acting along x and Dy = (2/hy) D (x) I along y.  The
// entries are generated on the fly from D, D^2 and the coefficient samples; no
// p^2 x p^2 matrix is ever stored.
//
//   leaf_assemble : A_ii (interior rows and columns) and B = -A_ie L1, where L1
//                   (Step 1) extrapolates each side's degree q-1 Gauss
//                   interpolant to the side's p Chebyshev points and averages
//                   the two values at a corner.  The batched LU then turns B
//                   into Y = -A_ii^{-1} A_ie L1 (eq. leaf_solve).
//   leaf_dtn      : T = L4 L3 W with W = [L1 ; Y] the full-grid potential per
//                   unit Gauss datum (Steps 3-4: d/dy on horizontal sides, d/dx
//                   on vertical sides, then evaluation of the side interpolant
//                   at the q Gauss points).
//   leaf_post     : w_full = W u_e for the solve (Section 5.3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"

namespace hps {

namespace {

struct CoefPtrs {
  const double* c[6];  // c11, c12, c22, c1, c2, c (null = absent)
};

template <typename R>
const char* tname(const char* f64, const char* f32) {
  return sizeof(R) == 8 ? f64 : f32;
}

// Side visited at slot t of a derivative pass: S, N (d/dy), E, W (d/dx).
__device__ __forceinline__ int side_order(int t) { return t == 1 ? 2 : (t == 2 ? 1 : t); }

}  // namespace

// One CTA per leaf.
template <typename R>
__global__ void __launch_bounds__(256) k_leaf_assemble(CoefPtrs cp, int l0, int p, int q,
                                                       const double2* __restrict__ hsc,
                                                       const double* __restrict__ gD,
                                                       const double* __restrict__ gPg2c,
                                                       R* __restrict__ Aii, R* __restrict__ Y,
                                                       int64_t ys, int with_identity) {
  extern __shared__ __align__(16) double sm[];
  const int pp = p * p, pi = p - 2, ni = pi * pi, nq = 4 * q;
  double* D = sm;             // p x p
  double* D2 = D + pp;        // p x p  (D*D)
  double* Pg = D2 + pp;       // p x q
  double* G = Pg + p * q;     // p x q : G[b][k] = sum_d D[b][d] w(d) Pg[d][k]
  double* cf = G + p * q;     // 6 x pp coefficient samples
  const int j = blockIdx.x, l = l0 + j;  // group-local and global leaf
  const double sx = hsc[l].x, sy = hsc[l].y;
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D[e] = gD[e];
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) Pg[e] = gPg2c[e];
  for (int k = 0; k < 6; ++k)
    for (int e = threadIdx.x; e < pp; e += blockDim.x)
      cf[k * pp + e] = cp.c[k] ? cp.c[k][(size_t)j * pp + e] : 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D2[e] = gD[pp + e];  // D^2 follows D
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
    int b = e / q, k = e % q;
    double s = 0.0;
    for (int d = 0; d < p; ++d) {
      double w = (d == 0 || d == p - 1) ? 0.5 : 1.0;
      s = fma(D[b * p + d] * w, Pg[d * q + k], s);
    }
    G[e] = s;
  }
  __syncthreads();
  // per interior row r = (a, b): the coefficient products every entry of the
  // row uses, once (FP64; the FP64 pipe is scarce)
  const bool has12 = cp.c[1] != nullptr;
  double* rf = cf + 6 * pp;  // 5 x ni: -c11 sx^2, c1 sx, -c22 sy^2, c2 sy, -2 c12 sx sy
  for (int ri = threadIdx.x; ri < ni; ri += blockDim.x) {
    const int r = (ri / pi + 1) * p + ri % pi + 1;
    rf[ri] = -cf[r] * sx * sx;
    rf[ni + ri] = cf[3 * pp + r] * sx;
    rf[2 * ni + ri] = -cf[2 * pp + r] * sy * sy;
    rf[3 * ni + ri] = cf[4 * pp + r] * sy;
    rf[4 * ni + ri] = has12 ? -2.0 * cf[pp + r] * sx * sy : 0.0;
  }
  __syncthreads();
  const double* c0 = cf + 5 * pp;
  R* Al = Aii + (size_t)j * ni * ni;
  R* Yl = Y + (size_t)j * ys;
  // A_ii(ri, ci), ri = (a-1)*(p-2) + (b-1), ci = (c-1)*(p-2) + (d-1): thread
  // rows, columns uniform per iteration (no index divisions per entry)
  for (int ri0 = 0; ri0 < ni; ri0 += blockDim.x) {
    const int ri = ri0 + threadIdx.x;
    if (ri >= ni) break;
    const int a = ri / pi + 1, b = ri % pi + 1, r = a * p + b;
    const double fxx = rf[ri], fx = rf[ni + ri], fyy = rf[2 * ni + ri], fy = rf[3 * ni + ri],
                 fxy = rf[4 * ni + ri];
    if (!has12) {
      // a row reaches only the nodes of its own grid row (c == a) and column
      // (d == b): zeros first, then those entries.  No branch on a node's
      // position, whose FP64 work would run for every lane of a warp.
      for (int ci = 0; ci < ni; ++ci) {
        Al[ri + (size_t)ci * ni] = R(0);
        if (with_identity)  // columns nq .. nq+ni-1: the identity, so the solve also returns A_ii^{-1}
          Yl[(size_t)ni * nq + ri + (size_t)ci * ni] = (ri == ci) ? R(1) : R(0);
      }
      for (int d = 1; d < p - 1; ++d) {  // c == a
        double v = fxx * D2[b * p + d] + fx * D[b * p + d];
        if (d == b) {
          v += fyy * D2[a * p + a] + fy * D[a * p + a];
          v += c0[r];
        }
        Al[ri + (size_t)((a - 1) * pi + d - 1) * ni] = (R)v;
      }
      for (int c = 1; c < p - 1; ++c) {  // d == b, c != a
        if (c == a) continue;
        const double v = fyy * D2[a * p + c] + fy * D[a * p + c];
        Al[ri + (size_t)((c - 1) * pi + b - 1) * ni] = (R)v;
      }
      continue;
    }
    int c = 1, d = 1;
    for (int ci = 0; ci < ni; ++ci) {  // the mixed term reaches every node
      double v = 0.0;
      if (a == c) v += fxx * D2[b * p + d] + fx * D[b * p + d];
      if (b == d) v += fyy * D2[a * p + c] + fy * D[a * p + c];
      v += fxy * D[a * p + c] * D[b * p + d];
      if (a == c && b == d) v += c0[r];
      Al[ri + (size_t)ci * ni] = (R)v;
      if (with_identity)
        Yl[(size_t)ni * nq + ri + (size_t)ci * ni] = (ri == ci) ? R(1) : R(0);
      if (++d == p - 1) {
        d = 1;
        ++c;
      }
    }
  }
  // B = -A_ie L1 (ni x 4q).  For an interior row (a, b) only the boundary nodes
  // of row a / column b are reached by the pure x / pure y terms; the mixed term
  // reaches every node of a side, collapsed through G.
  for (int ri0 = 0; ri0 < ni; ri0 += blockDim.x) {
    const int ri = ri0 + threadIdx.x;
    if (ri >= ni) break;
    const int a = ri / pi + 1, b = ri % pi + 1;
    const double fxx = rf[ri], fx = rf[ni + ri], fyy = rf[2 * ni + ri], fy = rf[3 * ni + ri],
                 fxy = rf[4 * ni + ri];
    // the four sides' row factors, then the q Gauss columns of each side
    const double hS = -(fyy * D2[a * p] + fy * D[a * p]);
    const double hN = -(fyy * D2[a * p + p - 1] + fy * D[a * p + p - 1]);
    const double hE = -(fxx * D2[b * p + p - 1] + fx * D[b * p + p - 1]);
    const double hW = -(fxx * D2[b * p] + fx * D[b * p]);
    for (int k = 0; k < q; ++k) {
      double vS = hS * Pg[b * q + k], vN = hN * Pg[b * q + k];
      double vE = hE * Pg[a * q + k], vW = hW * Pg[a * q + k];
      if (has12) {
        vS -= fxy * D[a * p] * G[b * q + k];
        vN -= fxy * D[a * p + p - 1] * G[b * q + k];
        vE -= fxy * D[b * p + p - 1] * G[a * q + k];
        vW -= fxy * D[b * p] * G[a * q + k];
      }
      Yl[ri + (size_t)(0 * q + k) * ni] = (R)vS;
      Yl[ri + (size_t)(1 * q + k) * ni] = (R)vE;
      Yl[ri + (size_t)(2 * q + k) * ni] = (R)vN;
      Yl[ri + (size_t)(3 * q + k) * ni] = (R)vW;
    }
  }
}

template <typename R>
void leaf_assemble(const double* const* coef, int l0, int nleaves, int p, int q,
                   const double2* hsc, const double* d_D, const double* d_Pg2c, R* Aii, R* Y,
                   int64_t ys, int with_identity, cudaStream_t st) {
  if (nleaves <= 0) return;
  CoefPtrs cp;
  for (int k = 0; k < 6; ++k) cp.c[k] = coef[k];
  size_t smem = (size_t)(2 * p * p + 2 * p * q + 6 * p * p + 5 * (p - 2) * (p - 2)) *
                sizeof(double);
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_leaf_assemble<R>), 200 * 1024))
    return;  // reported by the caller's launch check
  const double ni = (double)(p - 2) * (p - 2);
  int ncoef = 0;
  for (int k = 0; k < 6; ++k) ncoef += coef[k] != nullptr;
  prof::Scope sc(tname<R>("leaf_assemble<f64>", "leaf_assemble<f32>"), st,
                 (double)nleaves * (ni * ni * 8.0 + ni * 4.0 * q * 6.0),
                 (double)nleaves * ((ni * ni + ni * 4.0 * q) * sizeof(R) + ncoef * p * p * 8.0));
  k_leaf_assemble<R><<<nleaves, 256, smem, st>>>(cp, l0, p, q, hsc, d_D, d_Pg2c, Aii, Y, ys,
                                                 with_identity);
}

// ------------------------------------------------------------------ leaf DtN
// One CTA per leaf; the 4q columns of W are processed in chunks of CH.
// With dY (a correction of Y from one refinement step against the FP64
// residual, leaf stride dys), the interior rows are Y + dY summed in FP64, so T
// is formed from the corrected operator before any rounding to R; the rounded
// sum is written back to Y for the solve.
template <typename R>
__global__ void __launch_bounds__(256) k_leaf_dtn(R* Y, int64_t ys, int l0, int p, int q,
                                                  const double2* __restrict__ hsc,
                                                  const double* __restrict__ gD,
                                                  const double* __restrict__ gPg2c,
                                                  const double* __restrict__ gPc2g,
                                                  R* __restrict__ T, const R* __restrict__ dY,
                                                  int64_t dys) {
  constexpr int CH = 8;
  extern __shared__ __align__(16) double sm[];
  const int pp = p * p, pi = p - 2, ni = pi * pi, nq = 4 * q;
  double* D = sm;               // p x p
  double* Pg = D + pp;          // p x q
  double* Pc = Pg + p * q;      // q x p
  double* W = Pc + q * p;       // pp x CH
  double* F = W + pp * CH;      // 4p x CH side fluxes at Chebyshev points
  const int l = blockIdx.x;      // group-local leaf
  const double sx = hsc[l0 + l].x, sy = hsc[l0 + l].y;
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D[e] = gD[e];
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
    Pg[e] = gPg2c[e];
    Pc[e] = gPc2g[e];
  }
  R* Yl = Y + (size_t)l * ys;
  const R* dYl = dY ? dY + (size_t)l * dys : nullptr;
  R* Tl = T + (size_t)l * nq * nq;
  for (int g0 = 0; g0 < nq; g0 += CH) {
    const int nc = min(CH, nq - g0);
    __syncthreads();
    // W[:, g] for g in chunk: boundary rows from L1, interior rows from Y
    for (int e = threadIdx.x; e < pp * nc; e += blockDim.x) {
      const int node = e % pp, cc = e / pp, g = g0 + cc;
      const int a = node / p, b = node % p;
      double v = 0.0;
      if (a > 0 && a < p - 1 && b > 0 && b < p - 1) {
        const size_t idx = (a - 1) * pi + (b - 1) + (size_t)g * ni;
        v = (double)Yl[idx];
        if (dYl) {
          v += (double)dYl[idx];
          Yl[idx] = (R)v;
        }
      } else {
        const int s = g / q, k = g % q;
        // the node lies on side s at position j?
        int j = -1;
        if (s == 0 && a == 0) j = b;
        if (s == 2 && a == p - 1) j = b;
        if (s == 1 && b == p - 1) j = a;
        if (s == 3 && b == 0) j = a;
        if (j >= 0) v = ((j == 0 || j == p - 1) ? 0.5 : 1.0) * Pg[j * q + k];
      }
      W[node + cc * pp] = v;
    }
    __syncthreads();
    // Step 3: fluxes at the Chebyshev points of each side
    for (int e = threadIdx.x; e < 4 * p * nc; e += blockDim.x) {
      // sides in the order S, N, E, W: a warp's lanes take one branch
      const int sj = e % (4 * p), cc = e / (4 * p);
      const int s = side_order(sj / p), j = sj % p;
      double acc = 0.0;
      const double* Wc = W + cc * pp;
      if (s == 0 || s == 2) {  // d/dy at node (0 or p-1, j)
        const int row = (s == 0) ? 0 : p - 1;
        for (int a = 0; a < p; ++a) acc = fma(D[row * p + a], Wc[a * p + j], acc);
        acc *= sy;
      } else {  // d/dx at node (j, p-1 or 0)
        const int col = (s == 1) ? p - 1 : 0;
        for (int b = 0; b < p; ++b) acc = fma(D[col * p + b], Wc[j * p + b], acc);
        acc *= sx;
      }
      F[s * p + j + cc * 4 * p] = acc;
    }
    __syncthreads();
    // Step 4: Gauss values of each side's flux interpolant
    for (int e = threadIdx.x; e < nq * nc; e += blockDim.x) {
      const int row = e % nq, cc = e / nq;
      const int s = row / q, k = row % q;
      double acc = 0.0;
      for (int j = 0; j < p; ++j) acc = fma(Pc[k * p + j], F[s * p + j + cc * 4 * p], acc);
      Tl[row + (size_t)(g0 + cc) * nq] = (R)acc;
    }
  }
}

template <typename R>
void leaf_dtn(R* Y, int64_t ys, int l0, int nleaves, int p, int q, const double2* hsc,
              const double* d_D, const double* d_Pg2c, const double* d_Pc2g, R* T,
              cudaStream_t st, const R* dY, int64_t dys) {
  if (nleaves <= 0) return;
  size_t smem = (size_t)(p * p + 2 * p * q + p * p * 8 + 4 * p * 8) * sizeof(double);
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_leaf_dtn<R>), 200 * 1024))
    return;  // reported by the caller's launch check
  const double ni = (double)(p - 2) * (p - 2), nq = 4.0 * q;
  prof::Scope sc(tname<R>("leaf_dtn<f64>", "leaf_dtn<f32>"), st,
                 (double)nleaves * nq * (8.0 * p * p + 2.0 * nq * p),
                 (double)nleaves * (ni * nq + nq * nq) * sizeof(R));
  k_leaf_dtn<R><<<nleaves, 256, smem, st>>>(Y, ys, l0, p, q, hsc, d_D, d_Pg2c, d_Pc2g, T, dY,
                                             dys);
}

// ------------------------------------------------------------ post-process
// w_full = W u_e + [0 ; z] with W = [L1 ; Y] (Section 5.3), right-hand sides in
// chunks of RC.  The interior rows Y u_e (+ z) run in the element type R of Y.
// The boundary rows L1 u_e run in FP64: they are the values that neighbouring
// leaves share and must stay consistent between them.  They are formed first,
// side by side for all threads (4 p values per right-hand side, each a q-term
// dot product), then read back per node: a corner is the mean of its two
// sides' values (Section 3.2, Step 1).
// u[(r*nl + l)*pp + node] receives w_full (accumulate = 0) or has it added in
// FP64 (accumulate = 1).  z (optional) holds per leaf ni x nrhs interior values
// (ld ni).  bndv (optional) holds the side values already formed, per
// right-hand side, leaf and side the p values L1 u_e ((r*nl + l)*4 + side)*p;
// the kernel then reads them instead of forming them.
template <typename R, int RC>
__global__ void __launch_bounds__(256) k_leaf_post(const R* __restrict__ Y, int64_t ys, int l0,
                                                   const double* __restrict__ uext,
                                                   const int64_t* __restrict__ leaf_off,
                                                   int64_t ext_total, int p, int q, int nrhs,
                                                   const double* __restrict__ gPg2c,
                                                   const R* __restrict__ z, int accumulate,
                                                   double* const* __restrict__ wptr,
                                                   const int64_t* __restrict__ wrs,
                                                   const double* __restrict__ bndv) {
  extern __shared__ __align__(16) double smd[];
  const int pp = p * p, pi = p - 2, ni = pi * pi, nq = 4 * q;
  double* Pg = smd;                               // p x q
  double* ued = Pg + p * q;                       // nq x RC, FP64 (boundary rows)
  double* bnd = ued + nq * RC;                    // 4 sides x p points x RC: L1 u_e per side
  R* uer = reinterpret_cast<R*>(bnd + 4 * p * RC);  // nq x RC, element type of Y (interior rows)
  const int l = blockIdx.x;  // group-local leaf
  const int64_t off = leaf_off[l0 + l];
  double* const wl = wptr[l0 + l];
  const int64_t wstride = wrs[l0 + l];
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) Pg[e] = gPg2c[e];
  const R* Yl = Y + (size_t)l * ys;
  const R* zl = z ? z + (size_t)l * ni * nrhs : nullptr;
  for (int r0 = 0; r0 < nrhs; r0 += RC) {
    const int nr = min(RC, nrhs - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nq * RC; e += blockDim.x) {
      const int g = e % nq, rr = e / nq;
      const double v = rr < nr ? uext[(size_t)(r0 + rr) * ext_total + off + g] : 0.0;
      ued[g * RC + rr] = v;
      uer[g * RC + rr] = (R)v;
    }
    __syncthreads();
    // side values: bnd[(sd*p + j)*RC + rr] = sum_k Pg[j][k] u_e[sd*q + k]
    if (bndv) {
      for (int e = threadIdx.x; e < 4 * p * RC; e += blockDim.x) {
        const int rr = e / (4 * p), s = e % (4 * p);
        if (rr < nr) bnd[s * RC + rr] = bndv[((size_t)(r0 + rr) * gridDim.x + l) * 4 * p + s];
      }
    } else {
      for (int e = threadIdx.x; e < 4 * p * RC; e += blockDim.x) {
        const int rr = e % RC, j = (e / RC) % p, sd = e / (RC * p);
        double v = 0.0;
        for (int k = 0; k < q; ++k) v = fma(Pg[j * q + k], ued[(sd * q + k) * RC + rr], v);
        bnd[e] = v;
      }
    }
    __syncthreads();
    // interior nodes: Y u_e (+ z) in the precision of Y.  Interior and
    // boundary nodes run in separate loops, so no warp issues the other
    // kind's FP64 work for lanes that do not need it.
    for (int ri = threadIdx.x; ri < ni; ri += blockDim.x) {
      const int node = (ri / pi + 1) * p + ri % pi + 1;
      R acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = R(0);
      for (int g = 0; g < nq; ++g) {
        const R y = Yl[ri + (size_t)g * ni];
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr] = fma(y, uer[g * RC + rr], acc[rr]);
      }
      if (zl)
        for (int rr = 0; rr < nr; ++rr) acc[rr] += zl[ri + (size_t)(r0 + rr) * ni];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) {
        if (rr < nr) {
          double* up = wl + (size_t)(r0 + rr) * wstride + node;
          double v = (double)acc[rr];
          if (accumulate) v += *up;
          *up = v;
        }
      }
    }
    // boundary nodes: the side value (S row a = 0 and N row a = p-1 indexed by
    // b, E column b = p-1 and W column b = 0 indexed by a), a corner the mean
    // of its two sides
    for (int t = threadIdx.x; t < 4 * (p - 1); t += blockDim.x) {
      int a, b;
      if (t < p) {
        a = 0;
        b = t;
      } else if (t < 2 * p) {
        a = p - 1;
        b = t - p;
      } else if (t < 3 * p - 2) {
        a = t - 2 * p + 1;
        b = 0;
      } else {
        a = t - 3 * p + 3;
        b = p - 1;
      }
      const int node = a * p + b;
      const int sides[4][2] = {{0, b}, {2, b}, {1, a}, {3, a}};
      const bool on[4] = {a == 0, a == p - 1, b == p - 1, b == 0};
      int s1 = -1, s2 = -1;
      for (int u = 0; u < 4; ++u)
        if (on[u]) {
          const int idx = sides[u][0] * p + sides[u][1];
          if (s1 < 0)
            s1 = idx;
          else
            s2 = idx;
        }
      for (int rr = 0; rr < nr; ++rr) {
        double* up = wl + (size_t)(r0 + rr) * wstride + node;
        double v = s2 < 0 ? bnd[s1 * RC + rr] : 0.5 * (bnd[s1 * RC + rr] + bnd[s2 * RC + rr]);
        if (accumulate) v += *up;
        *up = v;
      }
    }
  }
}

// Exact FP32 -> FP64 by integer instructions (the FP64 pipe, which also
// converts, is the GPU's slowest); zeros, subnormals, infinities and NaNs
// take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f), e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)f;
  }
  return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)),
                          (int)(b << 29));
}

// The post-process of a mixed solve at p = 16 (196 interior nodes = 28 x 7)
// with the boundary rows already formed (bndv, layout as for k_leaf_post):
// one leaf per block of 256 threads, its right-hand sides in chunks of 64.
// Y and the chunk's z (FP32) come into shared memory by asynchronous copies
// while the block stages u_e and writes the boundary nodes; then warp w forms
// the right-hand sides 8w .. 8w + 7 of the chunk, lane i < 28 the interior rows
// i, i + 28, ..., i + 168, each the same sequential FP32 FMA chain over the 4q
// exterior values as k_leaf_post (so the same bits), plus z.
constexpr int kPostP = 16, kPostNi = 196, kPostRows = 7, kPostLanes = 28;
constexpr int kPostRc = 64, kPostUs = kPostRc + 4;  // chunk width, row stride of Us
constexpr int kPostThreads = 256;
constexpr int kPostUe = kPostRc * 64 / kPostThreads;                      // u_e per thread
constexpr int kPostBn = (kPostRc * 4 * (kPostP - 1) + kPostThreads - 1) / kPostThreads;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Boundary node t (0 .. 4(p-1)-1) of a leaf: its node index and the side
// values (side * p + point) it takes, s2 >= 0 at a corner (the mean).
__device__ __forceinline__ void post_bnd_node(int t, int& node, int& s1, int& s2) {
  constexpr int p = kPostP;
  int a, b;
  s2 = -1;
  if (t < p) {
    a = 0, b = t, s1 = b;                       // S
  } else if (t < 2 * p) {
    a = p - 1, b = t - p, s1 = 2 * p + b;       // N
  } else if (t < 3 * p - 2) {
    a = t - 2 * p + 1, b = 0, s1 = 3 * p + a;   // W
  } else {
    a = t - 3 * p + 3, b = p - 1, s1 = p + a;   // E
  }
  if (a == 0 && b == 0) s2 = 3 * p;              // S and W
  if (a == 0 && b == p - 1) s2 = p;              // S and E
  if (a == p - 1 && b == 0) s2 = 3 * p + p - 1;  // N and W
  if (a == p - 1 && b == p - 1) s2 = p + p - 1;  // N and E
  node = a * p + b;
}

__global__ void __launch_bounds__(kPostThreads, 2) k_leaf_post_tiled(
    const float* __restrict__ Y, int64_t ys, int l0, const double* __restrict__ uext,
    const int64_t* __restrict__ leaf_off, int64_t ext_total, int nq, int nrhs,
    const float* __restrict__ z, double* const* __restrict__ wptr,
    const int64_t* __restrict__ wrs, const double* __restrict__ bndv) {
  extern __shared__ __align__(16) float smf[];
  constexpr int p = kPostP, ni = kPostNi, nb = 4 * (p - 1);
  float* Ys = smf;                 // ni x nq, column g at g*ni
  float* Us = Ys + ni * nq;        // nq x kPostUs: the chunk's u_e in FP32
  float* Zs = Us + nq * kPostUs;   // ni x kPostRc: the chunk's z
  const int l = blockIdx.x, nl = gridDim.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t off = leaf_off[l0 + l];
  double* const wl = wptr[l0 + l];
  const int64_t wstride = wrs[l0 + l];
  {
    const float* src = Y + (size_t)l * ys;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Ys);
    for (int e = tid; e < ni * nq / 4; e += kPostThreads) cp_async16(dst + 16u * e, src + 4 * e);
  }
  const float* zl = z ? z + (size_t)l * ni * nrhs : nullptr;
  for (int r0 = 0; r0 < nrhs; r0 += kPostRc) {
    const int nr = min(kPostRc, nrhs - r0);
    if (r0) __syncthreads();  // the previous chunk's reads of Us and Zs are done
    if (zl) {
      const float* src = zl + (size_t)r0 * ni;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Zs);
      for (int e = tid; e < nr * ni / 4; e += kPostThreads) cp_async16(dst + 16u * e, src + 4 * e);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    {  // u_e of the chunk: every load in flight before the first store
      double v[kPostUe];
#pragma unroll
      for (int i = 0; i < kPostUe; ++i) {
        const int e = tid + kPostThreads * i, g = e % nq, rr = e / nq;
        v[i] = (rr < nr) ? uext[(size_t)(r0 + rr) * ext_total + off + g] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kPostUe; ++i) {
        const int e = tid + kPostThreads * i, g = e % nq, rr = e / nq;
        if (rr < kPostRc) Us[g * kPostUs + rr] = (float)v[i];
      }
    }
    // boundary nodes, in batches of 8: loads first, then the means and stores
#pragma unroll
    for (int i0 = 0; i0 < kPostBn; i0 += 8) {
      double v1[8], v2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int e = tid + kPostThreads * (i0 + i), rr = e / nb;
        int node, s1, s2;
        post_bnd_node(e % nb, node, s1, s2);
        v1[i] = v2[i] = 0.0;
        if (i0 + i < kPostBn && rr < nr) {
          const double* bv = bndv + ((size_t)(r0 + rr) * nl + l) * 4 * p;
          v1[i] = bv[s1];
          if (s2 >= 0) v2[i] = bv[s2];
        }
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int e = tid + kPostThreads * (i0 + i), rr = e / nb;
        int node, s1, s2;
        post_bnd_node(e % nb, node, s1, s2);
        if (i0 + i < kPostBn && rr < nr)
          wl[(size_t)(r0 + rr) * wstride + node] = s2 < 0 ? v1[i] : 0.5 * (v1[i] + v2[i]);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (lane < kPostLanes && 8 * warp < nr) {
      float acc[kPostRows][8];
#pragma unroll
      for (int j = 0; j < kPostRows; ++j)
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) acc[j][rr] = 0.0f;
#pragma unroll 2
      for (int g = 0; g < nq; ++g) {
        const float4 ua = *reinterpret_cast<const float4*>(Us + g * kPostUs + 8 * warp);
        const float4 ub = *reinterpret_cast<const float4*>(Us + g * kPostUs + 8 * warp + 4);
        const float u[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
        for (int j = 0; j < kPostRows; ++j) {
          const float y = Ys[g * ni + lane + kPostLanes * j];
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) acc[j][rr] = fmaf(y, u[rr], acc[j][rr]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int rc = 8 * warp + rr;
        if (rc < nr) {
          double* up = wl + (size_t)(r0 + rc) * wstride;
#pragma unroll
          for (int j = 0; j < kPostRows; ++j) {
            const int ri = lane + kPostLanes * j;
            float v = acc[j][rr];
            if (zl) v += Zs[ri + rc * ni];
            up[(ri / (p - 2) + 1) * p + ri % (p - 2) + 1] = f2d_exact(v);
          }
        }
      }
    }
  }
}

template <typename R>
void leaf_post(const R* Y, int64_t ys, int l0, const double* uext, const int64_t* leaf_ext_off,
               int64_t ext_total, int nleaves, int p, int q, int nrhs, const double* d_Pg2c,
               double* const* wptr, const int64_t* wrs, cudaStream_t st, const R* z,
               int accumulate, const double* bndv) {
  if (nleaves <= 0 || nrhs <= 0) return;
  if constexpr (std::is_same<R, float>::value) {
    if (bndv && !accumulate && p == kPostP && 4 * q <= 64 && ys % 4 == 0 &&
        reinterpret_cast<uintptr_t>(Y) % 16 == 0 && reinterpret_cast<uintptr_t>(z) % 16 == 0) {
      const int nq = 4 * q;
      const size_t smem = ((size_t)nq * (kPostNi + kPostUs) + (size_t)kPostNi * kPostRc) *
                          sizeof(float);
      if (!opt_in_smem(reinterpret_cast<const void*>(&k_leaf_post_tiled), 200 * 1024))
        return;  // reported by the caller's launch check
      const double ni = kPostNi;
      prof::Scope sc("leaf_post<f32>", st, (double)nleaves * nrhs * 2.0 * ni * nq,
                     (double)nleaves * (ni * nq * sizeof(R) +
                                        nrhs * (nq + 4.0 * p + (double)p * p) * 8.0 +
                                        (z ? nrhs * ni * sizeof(R) : 0.0)));
      k_leaf_post_tiled<<<nleaves, kPostThreads, smem, st>>>(Y, ys, l0, uext, leaf_ext_off, ext_total, nq,
                                                     nrhs, z, wptr, wrs, bndv);
      return;
    }
  }
  // right-hand sides per block: the smallest power of two covering nrhs, at most
  // 16 (padded columns would still run their FMAs; per column the arithmetic
  // does not depend on the block width)
  const int rc = nrhs >= 16 ? 16 : nrhs > 4 ? (nrhs > 8 ? 16 : 8) : nrhs > 2 ? 4 : nrhs;
  const size_t smem = (size_t)(p * q + 4 * q * rc + 4 * p * rc) * sizeof(double) +
                      (size_t)4 * q * rc * sizeof(R);
  auto opt = [](const void* k) { return opt_in_smem(k, 200 * 1024); };
  if (!opt(reinterpret_cast<const void*>(&k_leaf_post<R, 1>)) ||
      !opt(reinterpret_cast<const void*>(&k_leaf_post<R, 2>)) ||
      !opt(reinterpret_cast<const void*>(&k_leaf_post<R, 4>)) ||
      !opt(reinterpret_cast<const void*>(&k_leaf_post<R, 8>)) ||
      !opt(reinterpret_cast<const void*>(&k_leaf_post<R, 16>)))
    return;  // reported by the caller's launch check
  const double ni = (double)(p - 2) * (p - 2), nq = 4.0 * q;
  prof::Scope sc(tname<R>("leaf_post<f64>", "leaf_post<f32>"), st,
                 (double)nleaves * nrhs * (2.0 * ni * nq + (bndv ? 0.0 : 2.0 * (4.0 * p) * q)),
                 (double)nleaves * (ni * nq * sizeof(R) +
                                    nrhs * (nq + (bndv ? 4.0 * p : 0.0) +
                                            (double)p * p * (accumulate ? 2 : 1)) * 8.0));
#define HPS_LEAF_POST(RC)                                                                     \
  k_leaf_post<R, RC><<<nleaves, 256, smem, st>>>(Y, ys, l0, uext, leaf_ext_off, ext_total, p, q, \
                                                 nrhs, d_Pg2c, z, accumulate, wptr, wrs, bndv)
  switch (rc) {
    case 1: HPS_LEAF_POST(1); break;
    case 2: HPS_LEAF_POST(2); break;
    case 4: HPS_LEAF_POST(4); break;
    case 8: HPS_LEAF_POST(8); break;
    default: HPS_LEAF_POST(16); break;
  }
#undef HPS_LEAF_POST
}

// ------------------------------------------------------------ FP64 residual
// r = -(A w_full) at the interior Chebyshev nodes of each leaf, in FP64, from
// the coefficient samples and D (O(p^3) per leaf and right-hand side):
//   A w = -c11 Dxx w - 2 c12 Dy (Dx w) - c22 Dyy w + c1 Dx w + c2 Dy w + c w.
// The leaf's scalings (2/h) and the signs are folded once per leaf into per-node
// coefficients (the FP64 pipe, 2 per clock per SM, bounds this kernel).  With
// kMerged, the second- and first-order terms of a direction, which act on the
// same grid line, are merged once per leaf into one row per interior node:
// Mx(node, k) = k11 D2(b, k) + k1 D(b, k), My(node, k) = k22 D2(a, k) + k2 D(a, k);
// each right-hand side then costs p FMAs per direction and node instead of 2p
// (the rows take 2 p (p-2)^2 doubles of shared memory, so the host merges only
// when both orders are present and the rows fit).  The mixed term goes
// through Dx w at every node.
// Output rbuf[l*ni*nrhs + i + r*ni] in the element type of the correction solve.
//
// kFromY: the grids are the columns of W = [L1 ; Y] of a leaf (Section 3.2,
// Step 1 and eq. leaf_solve), nrhs = 4q of them: boundary rows from L1 (the
// side's Gauss interpolant, corners averaged), interior rows from the leaf's
// low-precision Y (ld ni, leaf stride ys).  Then -(A W)_i = -A_ie L1 - A_ii Y is
// the FP64 residual of the leaf system A_ii Y = -A_ie L1 that the LU solved.
template <typename R, bool kMerged, bool kFromY>
__global__ void __launch_bounds__(256) k_leaf_residual(CoefPtrs cp, int l0, int p, int rb,
                                                       const double2* __restrict__ hsc,
                                                       const double* __restrict__ gD,
                                                       double* const* __restrict__ wptr,
                                                       const int64_t* __restrict__ wrs, int nrhs,
                                                       R* __restrict__ rbuf,
                                                       const R* __restrict__ Ysrc, int64_t ys,
                                                       int q, const double* __restrict__ gPg2c) {
  extern __shared__ __align__(16) double sm[];
  const int pp = p * p, pi = p - 2, ni = pi * pi;
  const int lp = p + 1;      // padded row pitch of D and D^2: rows walked across threads
  double* D = sm;
  double* D2 = D + p * lp;
  double* Pg = D2 + p * lp;  // kFromY: p x q side interpolation (Step 1)
  double* W = Pg + (kFromY ? p * q : 0);  // rb x pp: w of this block of right-hand sides
  double* Wx = W + rb * pp;  // rb x pp: Dx w, unscaled (only with the mixed term)
  double* K = Wx + rb * pp;  // merged: 2 x ni (k12, k0 per interior node), then Mx, My
                             // (p x ni each, k-major); else 6 x pp per-node coefficients
  const int jl = blockIdx.x, l = l0 + jl;  // group-local and global leaf
  const double sx = hsc[l].x, sy = hsc[l].y;
  const double* wl = kFromY ? nullptr : wptr[l];
  const int64_t wstride = kFromY ? 0 : wrs[l];
  if constexpr (kFromY)
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) Pg[e] = gPg2c[e];
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D[(e / p) * lp + e % p] = gD[e];
  __syncthreads();
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D2[(e / p) * lp + e % p] = gD[pp + e];
  R* rl = rbuf + (size_t)jl * ni * nrhs;
  const bool has11 = cp.c[0] != nullptr, has12 = cp.c[1] != nullptr,
             has22 = cp.c[2] != nullptr, has1 = cp.c[3] != nullptr, has2 = cp.c[4] != nullptr,
             has0 = cp.c[5] != nullptr;
  const bool hasx = has11 || has1, hasy = has22 || has2;
  double* Mx = K + 2 * ni;
  double* My = Mx + p * ni;
  if constexpr (kMerged) {
    // r = Mx w + My w + k12 Dy Dx w + k0 w, D unscaled
    __syncthreads();  // D2 complete
    for (int e = threadIdx.x; e < ni * p; e += blockDim.x) {
      const int ri = e % ni, k = e / ni;
      const int a = ri / pi + 1, b = ri % pi + 1;
      const size_t g = (size_t)jl * pp + a * p + b;
      if (hasx) {
        const double k11 = has11 ? cp.c[0][g] * sx * sx : 0.0;
        const double k1 = has1 ? -cp.c[3][g] * sx : 0.0;
        Mx[e] = fma(k1, D[b * lp + k], k11 * D2[b * lp + k]);
      }
      if (hasy) {
        const double k22 = has22 ? cp.c[2][g] * sy * sy : 0.0;
        const double k2 = has2 ? -cp.c[4][g] * sy : 0.0;
        My[e] = fma(k2, D[a * lp + k], k22 * D2[a * lp + k]);
      }
      if (k == 0) {
        K[ri] = has12 ? 2.0 * cp.c[1][g] * sx * sy : 0.0;
        K[ni + ri] = has0 ? -cp.c[5][g] : 0.0;
      }
    }
  } else {
    // r = k11 Dxx w + k22 Dyy w + k12 Dy Dx w + k1 Dx w + k2 Dy w + k0 w, D unscaled
    for (int e = threadIdx.x; e < pp; e += blockDim.x) {
      const size_t g = (size_t)jl * pp + e;
      K[e] = has11 ? cp.c[0][g] * sx * sx : 0.0;
      K[pp + e] = has22 ? cp.c[2][g] * sy * sy : 0.0;
      K[2 * pp + e] = has12 ? 2.0 * cp.c[1][g] * sx * sy : 0.0;
      K[3 * pp + e] = has1 ? -cp.c[3][g] * sx : 0.0;
      K[4 * pp + e] = has2 ? -cp.c[4][g] * sy : 0.0;
      K[5 * pp + e] = has0 ? -cp.c[5][g] : 0.0;
    }
  }
  // right-hand sides in blocks of rb; threads take (node, right-hand side) pairs
  for (int r0 = 0; r0 < nrhs; r0 += rb) {
    const int nb = min(rb, nrhs - r0);
    __syncthreads();
    if constexpr (kFromY) {
      for (int e = threadIdx.x; e < pp * nb; e += blockDim.x) {
        const int g = r0 + e / pp, node = e % pp, a = node / p, b = node % p;
        double v = 0.0;
        if (a > 0 && a < p - 1 && b > 0 && b < p - 1) {
          v = (double)Ysrc[(size_t)jl * ys + (a - 1) * pi + (b - 1) + (size_t)g * ni];
        } else {  // column g is Gauss node k of side s: L1's entry at this node
          const int s = g / q, k = g % q;
          int j = -1;
          if (s == 0 && a == 0) j = b;
          if (s == 2 && a == p - 1) j = b;
          if (s == 1 && b == p - 1) j = a;
          if (s == 3 && b == 0) j = a;
          if (j >= 0) v = ((j == 0 || j == p - 1) ? 0.5 : 1.0) * Pg[j * q + k];
        }
        W[e] = v;
      }
    } else {
      for (int e = threadIdx.x; e < pp * nb; e += blockDim.x)
        W[e] = wl[(size_t)(r0 + e / pp) * wstride + e % pp];
    }
    __syncthreads();
    if (has12) {  // Dx w at every node: the mixed term differentiates it along y
      for (int e = threadIdx.x; e < pp * nb; e += blockDim.x) {
        const int node = e % pp, a = node / p, b = node % p;
        const double* Wr = W + (e / pp) * pp;
        double s = 0.0;
        for (int d = 0; d < p; ++d) s = fma(D[b * lp + d], Wr[a * p + d], s);
        Wx[e] = s;
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < ni * nb; e += blockDim.x) {
      const int ri = e % ni, rr = e / ni;
      const int a = ri / pi + 1, b = ri % pi + 1, node = a * p + b;
      const double* Wr = W + rr * pp;
      double dxy = 0.0;
      if (has12) {
        const double* Wxr = Wx + rr * pp;
        for (int k = 0; k < p; ++k) dxy = fma(D[a * lp + k], Wxr[k * p + b], dxy);
      }
      double r = 0.0;
      if constexpr (kMerged) {
        double sxv = 0.0, syv = 0.0;
        if (hasx)
          for (int k = 0; k < p; ++k) sxv = fma(Mx[k * ni + ri], Wr[a * p + k], sxv);
        if (hasy)
          for (int k = 0; k < p; ++k) syv = fma(My[k * ni + ri], Wr[k * p + b], syv);
        r = sxv + syv;
        if (has12) r = fma(K[ri], dxy, r);
        if (has0) r = fma(K[ni + ri], Wr[node], r);
      } else {
        double dxx = 0.0, dyy = 0.0, dx = 0.0, dy = 0.0;
        for (int k = 0; k < p; ++k) {
          dxx = fma(D2[b * lp + k], Wr[a * p + k], dxx);
          dyy = fma(D2[a * lp + k], Wr[k * p + b], dyy);
        }
        if (has1) {
          if (has12) {
            dx = Wx[rr * pp + node];
          } else {
            for (int k = 0; k < p; ++k) dx = fma(D[b * lp + k], Wr[a * p + k], dx);
          }
        }
        if (has2)
          for (int k = 0; k < p; ++k) dy = fma(D[a * lp + k], Wr[k * p + b], dy);
        if (has11) r = fma(K[node], dxx, r);
        if (has22) r = fma(K[pp + node], dyy, r);
        if (has12) r = fma(K[2 * pp + node], dxy, r);
        if (has1) r = fma(K[3 * pp + node], dx, r);
        if (has2) r = fma(K[4 * pp + node], dy, r);
        if (has0) r = fma(K[5 * pp + node], Wr[node], r);
      }
      rl[ri + (size_t)(r0 + rr) * ni] = (R)r;
    }
  }
}

namespace {

// Shared launcher of k_leaf_residual: kFromY takes the grids from a leaf's
// [L1 ; Y] (nrhs = 4q), otherwise from wptr / wrs.
template <typename R, bool kFromY>
void launch_residual(const double* const* coef, int l0, int nl, int p, int q,
                     const double2* hsc, const double* d_D, double* const* wptr,
                     const int64_t* wrs, int nrhs, R* rbuf, const R* Y, int64_t ys,
                     const double* d_Pg2c, const char* name, cudaStream_t st) {
  if (nl <= 0 || nrhs <= 0) return;
  CoefPtrs cp;
  for (int k = 0; k < 6; ++k) cp.c[k] = coef[k];
  const int pp = p * p;
  const int lp = p + 1;
  const int ni = (p - 2) * (p - 2);
  constexpr int kCap = 200 * 1024 / 8;  // doubles of shared memory
  const int extra = kFromY ? p * q : 0;
  // merged rows when a direction has both orders and they fit beside D, D^2
  // and one right-hand side
  const int fixed_m = 2 * p * lp + 2 * ni + 2 * p * ni + extra;
  const bool merged = ((coef[0] && coef[3]) || (coef[2] && coef[4])) && fixed_m + 2 * pp <= kCap;
  // right-hand sides per block: up to 4, as many as fit
  const int fixed = merged ? fixed_m : 2 * p * lp + 6 * pp + extra;
  const int rb = std::max(1, std::min(4, (kCap - fixed) / (2 * pp)));
  const size_t smem = (size_t)(fixed + 2 * rb * pp) * sizeof(double);
  const void* kern = merged ? reinterpret_cast<const void*>(&k_leaf_residual<R, true, kFromY>)
                            : reinterpret_cast<const void*>(&k_leaf_residual<R, false, kFromY>);
  if (!opt_in_smem(kern, 200 * 1024)) return;  // reported by the caller's launch check
  const double ppd = (double)pp, nid = (double)ni;
  // FP64 flops actually issued per leaf and right-hand side: merged, p FMAs
  // per direction present and interior node (plus the rows once per leaf);
  // else Dxx and Dyy always and Dx, Dy for the first-order terms present; the
  // mixed term adds Dx w everywhere and Dy of it at the interior nodes
  const bool hx = coef[0] || coef[3], hy = coef[2] || coef[4];
  double per, once = 2.0 * p * ppd;  // D^2
  if (merged) {
    per = 2.0 * ((hx ? 1 : 0) + (hy ? 1 : 0)) * nid * p + nid;
    once += 3.0 * ((hx ? 1 : 0) + (hy ? 1 : 0)) * nid * p;
    if (coef[1]) per += 2.0 * ppd * p + 2.0 * nid * p + 2.0 * nid;
  } else {
    per = 4.0 * nid * p;
    if (coef[1]) per += 2.0 * ppd * p + 2.0 * nid * p;
    else if (coef[3]) per += 2.0 * nid * p;
    if (coef[4]) per += 2.0 * nid * p;
  }
  const double in_bytes = kFromY ? nid * sizeof(R) : ppd * 8.0;
  prof::Scope sc(name, st, (double)nl * (nrhs * per + once),
                 (double)nl * (nrhs * (in_bytes + nid * sizeof(R)) + 6.0 * ppd * 8.0));
  if (merged)
    k_leaf_residual<R, true, kFromY><<<nl, 256, smem, st>>>(cp, l0, p, rb, hsc, d_D, wptr, wrs,
                                                            nrhs, rbuf, Y, ys, q, d_Pg2c);
  else
    k_leaf_residual<R, false, kFromY><<<nl, 256, smem, st>>>(cp, l0, p, rb, hsc, d_D, wptr, wrs,
                                                             nrhs, rbuf, Y, ys, q, d_Pg2c);
}

}  // namespace

template <typename R>
void leaf_residual(const double* const* coef, int l0, int nl, int p, const double2* hsc,
                   const double* d_D, double* const* wptr, const int64_t* wrs, int nrhs, R* rbuf,
                   cudaStream_t st) {
  launch_residual<R, false>(coef, l0, nl, p, 1, hsc, d_D, wptr, wrs, nrhs, rbuf, nullptr, 0,
                            nullptr, "leaf_residual<f64>", st);
}

// --------------------------- FP64 residual and fluxes by even and odd parts
// For operators without the mixed term (c12 absent), the FP64 residual
// r = -(A w)_i and, optionally, the side fluxes v = L4 L3 w (Section 3.2,
// Steps 3-4) of the same grids, in one pass over w.
//
// The Chebyshev extreme points are symmetric about the leaf's centre, so D is
// anti-centrosymmetric and D^2 centrosymmetric.  A grid line w_0 .. w_{p-1}
// is split into e_k = w_k + w_{p-1-k} and o_k = w_k - w_{p-1-k} (k < h =
// floor(p/2)); for a row i < h of D^2
//   (D^2 w)_i         = sum_k E_ik e_k + O_ik o_k (+ C_i w_c),
//   (D^2 w)_{p-1-i}   = sum_k E_ik e_k - O_ik o_k (+ C_i w_c),
// with E_ik = (D^2_ik + D^2_{i,p-1-k}) / 2, O_ik = (D^2_ik - D^2_{i,p-1-k}) / 2
// and, for odd p, the centre c = h (C_i = D^2_ic).  For D the even part
// changes sign instead: (D w)_{p-1-i} = -(sum E e + C w_c) + sum O o.  The
// tables hold the off-diagonal entries only; each node adds its own diagonal
// entry times its value, so the diagonal (where the rounding of D^2 reaches
// the smooth part of the solution most) is applied exactly as stored, by
// every path.  Each
// mirrored pair of derivatives then costs p FMAs instead of 2p, which halves
// the FP64 work of the derivatives (the FP64 pipe, 2 FMAs per clock per SM,
// bounds this kernel).  A thread takes a symmetric quad of interior nodes
// (a, b), (a, b'), (a', b), (a', b') with a' = p-1-a, b' = p-1-b: two row pairs
// along x and two column pairs along y.  The fluxes take the pair of rows 0
// and p-1 (S and N: d/dy), or of columns 0 and p-1 (W and E: d/dx), from the
// same e/o lines, then the side interpolant at the q Gauss points.
//
// kFromY: the grids are the columns of [L1 ; Y] of each leaf (the residual of
// the leaf systems A_ii Y = -A_ie L1), nrhs = 4q; no fluxes.
// kFlux: hp[r * ext_total + leaf_off[l] + g] = (L4 L3 w)_g (FP64, stored).
template <typename R, bool kFromY, bool kFlux>
__global__ void __launch_bounds__(256) k_leaf_resflux(
    CoefPtrs cp, int l0, int p, int q, int rb, const double2* __restrict__ hsc,
    const double* __restrict__ gD, const double* __restrict__ gPc2g,
    const double* __restrict__ gPg2c, double* const* __restrict__ wptr,
    const int64_t* __restrict__ wrs, int nrhs, R* __restrict__ rbuf, const R* __restrict__ Ysrc,
    int64_t ys, const int64_t* __restrict__ leaf_off, int64_t ext_total,
    double* __restrict__ hp) {
  extern __shared__ __align__(16) double sm[];
  const int pp = p * p, pi = p - 2, ni = pi * pi;
  const int h = p / 2, odd = p & 1, c = h;  // c: the centre index when p is odd
  const int npair = h + odd;                // row pairs 0..h-1, then the centre
  const int tw = 2 * h + 3;                 // table row: E (h), O (h), C, diag(i), diag(p-1-i)
  const int lp = p + 1;                     // padded pitch of the grid and the column parts
  const int hq = h + 1;                     // padded pitch of the row parts
  double* D = sm;                           // p x p
  double* D2 = D + pp;                      // p x p
  double* T2 = D2 + pp;                     // npair x tw: D^2 by even / odd parts
  double* T1 = T2 + npair * tw;             // npair x tw: D
  double* Pc = T1 + npair * tw;             // q x p (kFlux)
  double* Pg = Pc + (kFlux ? q * p : 0);    // p x q (kFromY)
  // per-grid strides, odd so that consecutive grids start in other banks
  const int sW = p * lp + 1, sX = p * hq + 1, sY = h * lp + 1;
  double* K = Pg + (kFromY ? p * q : 0);    // 6 x pp: k11, k22, k1, k2, k0, kd per node
  double* W = K + 6 * pp;                   // rb x sW: grid (p x lp)
  double* XE = W + rb * sW;                 // rb x sX: row parts (along x), p x hq
  double* XO = XE + rb * sX;
  double* YE = XO + rb * sX;                // rb x sY: column parts (along y), h x lp
  double* YO = YE + rb * sY;
  double* Fs = YO + rb * sY;                // rb x 4 x p: side fluxes at the Chebyshev points
  const int jl = blockIdx.x, l = l0 + jl;  // group-local and global leaf
  const double sx = hsc[l].x, sy = hsc[l].y;
  const double* wl = kFromY ? nullptr : wptr[l];
  const int64_t wstride = kFromY ? 0 : wrs[l];
  const bool has11 = cp.c[0] != nullptr, has22 = cp.c[2] != nullptr, has1 = cp.c[3] != nullptr,
             has2 = cp.c[4] != nullptr, has0 = cp.c[5] != nullptr;
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D[e] = gD[e];
  if constexpr (kFlux)
    for (int e = threadIdx.x; e < q * p; e += blockDim.x) Pc[e] = gPc2g[e];
  if constexpr (kFromY)
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) Pg[e] = gPg2c[e];
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    const size_t g = (size_t)jl * pp + e;
    K[e] = has11 ? cp.c[0][g] * sx * sx : 0.0;
    K[pp + e] = has22 ? cp.c[2][g] * sy * sy : 0.0;
    K[2 * pp + e] = has1 ? -cp.c[3][g] * sx : 0.0;
    K[3 * pp + e] = has2 ? -cp.c[4][g] * sy : 0.0;
    K[4 * pp + e] = has0 ? -cp.c[5][g] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D2[e] = gD[pp + e];  // D^2 follows D
  __syncthreads();
  for (int e = threadIdx.x; e < npair * tw; e += blockDim.x) {
    const int i = e / tw, t = e % tw;  // pair i: row i (i < h) or the centre row
    // off-diagonal entries of row i (its diagonal counted as 0)
    auto od2 = [&](int k) { return k == i ? 0.0 : D2[i * p + k]; };
    auto od1 = [&](int k) { return k == i ? 0.0 : D[i * p + k]; };
    double v2, v1;
    if (t < h) {
      v2 = 0.5 * (od2(t) + od2(p - 1 - t));
      v1 = 0.5 * (od1(t) + od1(p - 1 - t));
    } else if (t < 2 * h) {
      v2 = 0.5 * (od2(t - h) - od2(p - 1 - (t - h)));
      v1 = 0.5 * (od1(t - h) - od1(p - 1 - (t - h)));
    } else if (t == 2 * h) {
      v2 = odd ? od2(c) : 0.0;
      v1 = odd ? od1(c) : 0.0;
    } else if (t == 2 * h + 1) {
      v2 = D2[i * p + i];
      v1 = D[i * p + i];
    } else {
      v2 = D2[(p - 1 - i) * p + (p - 1 - i)];
      v1 = D[(p - 1 - i) * p + (p - 1 - i)];
    }
    T2[e] = v2;
    T1[e] = v1;
  }
  // every diagonal contribution of node (a, b) in one coefficient:
  // kd = k11 D^2_bb + k22 D^2_aa + k1 D_bb + k2 D_aa + k0 (times w(a, b))
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    const int a = e / p, b = e % p;
    double kd = K[4 * pp + e];
    kd = fma(K[e], D2[b * p + b], kd);
    kd = fma(K[pp + e], D2[a * p + a], kd);
    kd = fma(K[2 * pp + e], D[b * p + b], kd);
    kd = fma(K[3 * pp + e], D[a * p + a], kd);
    K[5 * pp + e] = kd;
  }
  const int nint = (h - 1) + odd;  // interior pairs: rows 1 .. h-1, then the centre
  const int64_t off = kFlux ? leaf_off[l] : 0;
  for (int r0 = 0; r0 < nrhs; r0 += rb) {
    const int nb = min(rb, nrhs - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * pp; e += blockDim.x) {
      const int gi = e / pp, node = e % pp, a = node / p, b = node % p;
      double v = 0.0;
      if constexpr (kFromY) {
        const int g = r0 + gi;
        if (a > 0 && a < p - 1 && b > 0 && b < p - 1) {
          v = (double)Ysrc[(size_t)jl * ys + (a - 1) * pi + (b - 1) + (size_t)g * ni];
        } else {  // column g is Gauss node k of side s: L1's entry at this node
          const int s = g / q, k = g % q;
          int j = -1;
          if (s == 0 && a == 0) j = b;
          if (s == 2 && a == p - 1) j = b;
          if (s == 1 && b == p - 1) j = a;
          if (s == 3 && b == 0) j = a;
          if (j >= 0) v = ((j == 0 || j == p - 1) ? 0.5 : 1.0) * Pg[j * q + k];
        }
      } else {
        v = wl[(size_t)(r0 + gi) * wstride + node];
      }
      W[gi * sW + a * lp + b] = v;
    }
    __syncthreads();
    // even and odd parts of every row (along x) and every column (along y)
    for (int e = threadIdx.x; e < nb * p * h; e += blockDim.x) {
      const int gi = e / (p * h), rem = e % (p * h), line = rem / h, k = rem % h;
      const double* Wg = W + gi * sW;
      const double x0 = Wg[line * lp + k], x1 = Wg[line * lp + p - 1 - k];
      XE[gi * sX + line * hq + k] = x0 + x1;
      XO[gi * sX + line * hq + k] = x0 - x1;
      const double y0 = Wg[k * lp + line], y1 = Wg[(p - 1 - k) * lp + line];
      YE[gi * sY + k * lp + line] = y0 + y1;
      YO[gi * sY + k * lp + line] = y0 - y1;
    }
    __syncthreads();
    // residual: one symmetric quad of interior nodes per thread and item
    for (int e = threadIdx.x; e < nb * nint * nint; e += blockDim.x) {
      const int gi = e / (nint * nint), qd = e % (nint * nint);
      const int ia = qd / nint, ib = qd % nint;
      const int a0 = ia < h - 1 ? ia + 1 : c, b0 = ib < h - 1 ? ib + 1 : c;
      const int a1 = p - 1 - a0, b1 = p - 1 - b0;
      const double* Wg = W + gi * sW;
      const double* t2a = T2 + a0 * tw;
      const double* t2b = T2 + b0 * tw;
      const double* t1a = T1 + a0 * tw;
      const double* t1b = T1 + b0 * tw;
      const double* xe0 = XE + gi * sX + a0 * hq;
      const double* xo0 = XO + gi * sX + a0 * hq;
      const double* xe1 = XE + gi * sX + a1 * hq;
      const double* xo1 = XO + gi * sX + a1 * hq;
      const double* ye = YE + gi * sY;
      const double* yo = YO + gi * sY;
      // second derivatives: even / odd sums of rows a0, a1 (x) and columns b0, b1 (y)
      double ex0 = 0.0, ox0 = 0.0, ex1 = 0.0, ox1 = 0.0;
      double ey0 = 0.0, oy0 = 0.0, ey1 = 0.0, oy1 = 0.0;
      for (int k = 0; k < h; ++k) {
        const double Eb = t2b[k], Ob = t2b[h + k], Ea = t2a[k], Oa = t2a[h + k];
        ex0 = fma(Eb, xe0[k], ex0);
        ox0 = fma(Ob, xo0[k], ox0);
        ex1 = fma(Eb, xe1[k], ex1);
        ox1 = fma(Ob, xo1[k], ox1);
        ey0 = fma(Ea, ye[k * lp + b0], ey0);
        oy0 = fma(Oa, yo[k * lp + b0], oy0);
        ey1 = fma(Ea, ye[k * lp + b1], ey1);
        oy1 = fma(Oa, yo[k * lp + b1], oy1);
      }
      if (odd) {
        ex0 = fma(t2b[2 * h], Wg[a0 * lp + c], ex0);
        ex1 = fma(t2b[2 * h], Wg[a1 * lp + c], ex1);
        ey0 = fma(t2a[2 * h], Wg[c * lp + b0], ey0);
        ey1 = fma(t2a[2 * h], Wg[c * lp + b1], ey1);
      }
      // first derivatives where the operator has them (warp-uniform branches)
      double fx0 = 0.0, gx0 = 0.0, fx1 = 0.0, gx1 = 0.0;
      double fy0 = 0.0, gy0 = 0.0, fy1 = 0.0, gy1 = 0.0;
      if (has1) {
        for (int k = 0; k < h; ++k) {
          const double Eb = t1b[k], Ob = t1b[h + k];
          fx0 = fma(Eb, xe0[k], fx0);
          gx0 = fma(Ob, xo0[k], gx0);
          fx1 = fma(Eb, xe1[k], fx1);
          gx1 = fma(Ob, xo1[k], gx1);
        }
        if (odd) {
          fx0 = fma(t1b[2 * h], Wg[a0 * lp + c], fx0);
          fx1 = fma(t1b[2 * h], Wg[a1 * lp + c], fx1);
        }
      }
      if (has2) {
        for (int k = 0; k < h; ++k) {
          const double Ea = t1a[k], Oa = t1a[h + k];
          fy0 = fma(Ea, ye[k * lp + b0], fy0);
          gy0 = fma(Oa, yo[k * lp + b0], gy0);
          fy1 = fma(Ea, ye[k * lp + b1], fy1);
          gy1 = fma(Oa, yo[k * lp + b1], gy1);
        }
        if (odd) {
          fy0 = fma(t1a[2 * h], Wg[c * lp + b0], fy0);
          fy1 = fma(t1a[2 * h], Wg[c * lp + b1], fy1);
        }
      }
      R* rl = rbuf + (size_t)jl * ni * nrhs + (size_t)(r0 + gi) * ni;
      // node (a, b): r = k11 X + k22 Y + k1 FX + k2 FY + kd w, with X, Y, FX,
      // FY the off-diagonal parts of Dxx w, Dyy w, Dx w, Dy w; the mirrored
      // node of a pair takes the odd part with the other sign (for D, the even
      // part), the centre of odd p only the even part
      auto put = [&](int a, int b, double X, double Y) {
        const int node = a * p + b;
        double r = K[5 * pp + node] * Wg[a * lp + b];
        if (has11) r = fma(K[node], X, r);
        if (has22) r = fma(K[pp + node], Y, r);
        return r;
      };
      auto out = [&](int a, int b, double r) { rl[(a - 1) * pi + (b - 1)] = (R)r; };
      if (!has1 && !has2) {
        out(a0, b0, put(a0, b0, ex0 + ox0, ey0 + oy0));
        if (b1 != b0) out(a0, b1, put(a0, b1, ex0 - ox0, ey1 + oy1));
        if (a1 != a0) out(a1, b0, put(a1, b0, ex1 + ox1, ey0 - oy0));
        if (a1 != a0 && b1 != b0) out(a1, b1, put(a1, b1, ex1 - ox1, ey1 - oy1));
      } else {
        auto first = [&](int a, int b, double r, double FX, double FY) {
          const int node = a * p + b;
          if (has1) r = fma(K[2 * pp + node], FX, r);
          if (has2) r = fma(K[3 * pp + node], FY, r);
          out(a, b, r);
        };
        first(a0, b0, put(a0, b0, ex0 + ox0, ey0 + oy0), fx0 + gx0, fy0 + gy0);
        if (b1 != b0) first(a0, b1, put(a0, b1, ex0 - ox0, ey1 + oy1), gx0 - fx0, fy1 + gy1);
        if (a1 != a0) first(a1, b0, put(a1, b0, ex1 + ox1, ey0 - oy0), fx1 + gx1, gy0 - fy0);
        if (a1 != a0 && b1 != b0)
          first(a1, b1, put(a1, b1, ex1 - ox1, ey1 - oy1), gx1 - fx1, gy1 - fy1);
      }
    }
    if constexpr (kFlux) {
      __syncthreads();
      // side derivatives at the Chebyshev points: columns j give d/dy at rows 0
      // (S) and p-1 (N), rows j give d/dx at columns 0 (W) and p-1 (E); the
      // direction is uniform over each half of the items
      for (int e = threadIdx.x; e < 2 * nb * p; e += blockDim.x) {
        const int dir = e / (nb * p), rem = e % (nb * p), gi = rem / p, j = rem % p;
        const double* Wg = W + gi * sW;
        double ev = 0.0, od = 0.0;
        if (dir == 0) {
          const double* ye = YE + gi * sY;
          const double* yo = YO + gi * sY;
          for (int k = 0; k < h; ++k) {
            ev = fma(T1[k], ye[k * lp + j], ev);
            od = fma(T1[h + k], yo[k * lp + j], od);
          }
          if (odd) ev = fma(T1[2 * h], Wg[c * lp + j], ev);
          Fs[(gi * 4 + 0) * p + j] = sy * fma(T1[2 * h + 1], Wg[j], ev + od);
          Fs[(gi * 4 + 2) * p + j] = sy * fma(T1[2 * h + 2], Wg[(p - 1) * lp + j], od - ev);
        } else {
          const double* xe = XE + gi * sX + j * hq;
          const double* xo = XO + gi * sX + j * hq;
          for (int k = 0; k < h; ++k) {
            ev = fma(T1[k], xe[k], ev);
            od = fma(T1[h + k], xo[k], od);
          }
          if (odd) ev = fma(T1[2 * h], Wg[j * lp + c], ev);
          Fs[(gi * 4 + 3) * p + j] = sx * fma(T1[2 * h + 1], Wg[j * lp], ev + od);
          Fs[(gi * 4 + 1) * p + j] = sx * fma(T1[2 * h + 2], Wg[j * lp + p - 1], od - ev);
        }
      }
      __syncthreads();
      // Step 4: the side interpolants at the q Gauss points, sides S, E, N, W
      for (int e = threadIdx.x; e < nb * 4 * q; e += blockDim.x) {
        const int gi = e / (4 * q), g = e % (4 * q), s = g / q, k = g % q;
        const double* F = Fs + (gi * 4 + s) * p;
        double acc = 0.0;
        for (int j = 0; j < p; ++j) acc = fma(Pc[k * p + j], F[j], acc);
        hp[(size_t)(r0 + gi) * ext_total + off + g] = acc;
      }
    }
  }
}

namespace {

// Grids per block of k_leaf_resflux: as many as fit in sm_cap doubles, chosen
// so that the quads of a block fill the CTA's threads evenly.
int resflux_block(int p, int q, bool from_y, bool flux, int nrhs, int sm_cap, size_t* smem) {
  const int pp = p * p, h = p / 2, odd = p & 1, npair = h + odd, tw = 2 * h + 3;
  const int nint = (h - 1) + odd;
  const int fixed = 2 * pp + 2 * npair * tw + (flux ? q * p : 0) + (from_y ? p * q : 0) + 6 * pp;
  const int per = (p * (p + 1) + 1) + 2 * (p * (h + 1) + 1) + 2 * (h * (p + 1) + 1) + 4 * p;
  const int rbmax = std::max(1, std::min(nrhs, (sm_cap - fixed) / per));
  int best = 1;
  double best_eff = 0.0;
  for (int rb = 1; rb <= rbmax; ++rb) {
    const int items = rb * nint * nint;
    const double eff = (double)items / (double)(((items + 255) / 256) * 256);
    if (eff >= best_eff - 1e-9) {
      best_eff = eff;
      best = rb;
    }
  }
  *smem = (size_t)(fixed + best * per) * sizeof(double);
  return best;
}

template <typename R, bool kFromY, bool kFlux>
void launch_resflux(const double* const* coef, int l0, int nl, int p, int q, const double2* hsc,
                    const double* d_D, const double* d_Pc2g, const double* d_Pg2c,
                    double* const* wptr, const int64_t* wrs, int nrhs, R* rbuf, const R* Y,
                    int64_t ys, const int64_t* leaf_off, int64_t ext_total, double* hp,
                    const char* name, cudaStream_t st) {
  if (nl <= 0 || nrhs <= 0) return;
  CoefPtrs cp;
  for (int k = 0; k < 6; ++k) cp.c[k] = coef[k];
  size_t smem = 0;
  // about 100 KB, so that two CTAs share an SM
  const int rb = resflux_block(p, q, kFromY, kFlux, nrhs, 100 * 1024 / 8, &smem);
  const void* kern = reinterpret_cast<const void*>(&k_leaf_resflux<R, kFromY, kFlux>);
  // the attribute is a ceiling (cached per kernel); a launch asking for more
  // than it fails, and the caller's launch check reports that
  if (!opt_in_smem(kern, 200 * 1024)) return;  // reported by the caller's launch check
  // FP64 flops per grid, counted as issued: the even / odd parts (2 p h adds
  // per direction), the h-term sums of each mirrored pair per derivative
  // (direction and order) present, per node and derivative an add (even and
  // odd parts) and an FMA, and the diagonal coefficient times w; the fluxes'
  // side pairs (2h-term sums, their diagonals and scalings) and the Gauss
  // interpolation
  const int h = p / 2, odd = p & 1, nint = (h - 1) + odd;
  const double nid = (double)(p - 2) * (p - 2);
  const int orders = (coef[0] ? 1 : 0) + (coef[2] ? 1 : 0) + (coef[3] ? 1 : 0) + (coef[4] ? 1 : 0);
  double per = 4.0 * p * h + (double)nint * nint * orders * 8.0 * (h + odd) +
               nid * (3.0 * orders + 1.0);
  if (kFlux) per += 2.0 * p * (4.0 * (h + odd) + 8.0) + 4.0 * q * 2.0 * p;
  const double in_bytes = kFromY ? nid * sizeof(R) : (double)p * p * 8.0;
  prof::Scope sc(name, st, (double)nl * nrhs * per,
                 (double)nl * (nrhs * (in_bytes + nid * sizeof(R) + (kFlux ? 32.0 * q : 0.0)) +
                               5.0 * p * p * 8.0));
  k_leaf_resflux<R, kFromY, kFlux><<<nl, 256, smem, st>>>(cp, l0, p, q, rb, hsc, d_D, d_Pc2g,
                                                          d_Pg2c, wptr, wrs, nrhs, rbuf, Y, ys,
                                                          leaf_off, ext_total, hp);
}

}  // namespace

template <typename R>
void leaf_resflux(const double* const* coef, int l0, int nl, int p, int q, const double2* hsc,
                  const double* d_D, const double* d_Pc2g, double* const* wptr,
                  const int64_t* wrs, int nrhs, R* rbuf, const int64_t* leaf_off,
                  int64_t ext_total, double* hp, cudaStream_t st) {
  launch_resflux<R, false, true>(coef, l0, nl, p, q, hsc, d_D, d_Pc2g, nullptr, wptr, wrs, nrhs,
                                 rbuf, nullptr, 0, leaf_off, ext_total, hp, "leaf_resflux<f64>",
                                 st);
}

template <typename R>
void leaf_y_residual(const double* const* coef, int l0, int nl, int p, int q,
                     const double2* hsc, const double* d_D, const double* d_Pg2c, const R* Y,
                     int64_t ys, R* rbuf, cudaStream_t st) {
  if (coef[1])  // the mixed term: the direct form (no even / odd split of Dy Dx w)
    launch_residual<R, true>(coef, l0, nl, p, q, hsc, d_D, nullptr, nullptr, 4 * q, rbuf, Y, ys,
                             d_Pg2c, "leaf_yresid<f64>", st);
  else
    launch_resflux<R, true, false>(coef, l0, nl, p, q, hsc, d_D, nullptr, d_Pg2c, nullptr,
                                   nullptr, 4 * q, rbuf, Y, ys, nullptr, 0, nullptr,
                                   "leaf_yresid<f64>", st);
}

// ------------------------------------------------- flux offsets of the leaves
// h[g] = (L4 L3 (w_full + [0 ; z]))[g]: the side fluxes, at the Gauss nodes,
// of the current iterate plus the interior particular solution z = A_ii^{-1} r.
// Written to the leaf's exterior slot of the flux pool hp (FP64).
template <typename R>
__global__ void __launch_bounds__(256) k_leaf_flux(double* const* __restrict__ wptr,
                                                   const int64_t* __restrict__ wrs,
                                                   const R* __restrict__ z, int l0, int p, int q,
                                                   int nrhs, int rb,
                                                   const double2* __restrict__ hsc,
                                                   const double* __restrict__ gD,
                                                   const double* __restrict__ gPc2g,
                                                   const int64_t* __restrict__ leaf_off,
                                                   int64_t ext_total, double* __restrict__ hp) {
  extern __shared__ __align__(16) double sm[];
  const int pp = p * p, pi = p - 2, ni = pi * pi, nq = 4 * q;
  const int lp = p + 1;      // padded row pitch: column walks hit distinct banks
  const int vs = p * lp;     // one right-hand side's grid
  double* D = sm;
  double* Pc = D + pp;       // q x p, pitch lp
  double* V = Pc + q * lp;   // rb x (p x p), pitch lp
  double* F = V + rb * vs;   // rb x 4p
  const int l = blockIdx.x;  // group-local leaf
  const double sx = hsc[l0 + l].x, sy = hsc[l0 + l].y;
  const double* wl = wptr[l0 + l];
  const int64_t wstride = wrs[l0 + l];
  for (int e = threadIdx.x; e < pp; e += blockDim.x) D[e] = gD[e];
  for (int e = threadIdx.x; e < q * p; e += blockDim.x) Pc[(e / p) * lp + e % p] = gPc2g[e];
  const R* zl = z ? z + (size_t)l * ni * nrhs : nullptr;
  const int64_t off = leaf_off[l0 + l];
  // right-hand sides in blocks of rb, so every phase keeps the CTA busy
  for (int r0 = 0; r0 < nrhs; r0 += rb) {
    const int nb = min(rb, nrhs - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < pp * nb; e += blockDim.x) {
      const int r = r0 + e / pp, node = e % pp, a = node / p, b = node % p;
      double v = wl[(size_t)r * wstride + node];
      if (zl && a > 0 && a < p - 1 && b > 0 && b < p - 1)
        v += (double)zl[(a - 1) * pi + (b - 1) + (size_t)r * ni];
      V[(e / pp) * vs + a * lp + b] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * p * nb; e += blockDim.x) {
      // sides in the order S, N, E, W: a warp's lanes take one branch
      const int sj = e % (4 * p), s = side_order(sj / p), j = sj % p;
      const double* Vr = V + (e / (4 * p)) * vs;
      double acc = 0.0;
      if (s == 0 || s == 2) {
        const int row = (s == 0) ? 0 : p - 1;
        for (int a = 0; a < p; ++a) acc = fma(D[row * p + a], Vr[a * lp + j], acc);
        acc *= sy;
      } else {
        const int col = (s == 1) ? p - 1 : 0;
        for (int b = 0; b < p; ++b) acc = fma(D[col * p + b], Vr[j * lp + b], acc);
        acc *= sx;
      }
      F[(e / (4 * p)) * 4 * p + s * p + j] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nq * nb; e += blockDim.x) {
      const int g = e % nq, rr = e / nq, s = g / q, k = g % q;
      const double* Fr = F + rr * 4 * p;
      double acc = 0.0;
      for (int j = 0; j < p; ++j) acc = fma(Pc[k * lp + j], Fr[s * p + j], acc);
      hp[(size_t)(r0 + rr) * ext_total + off + g] = acc;
    }
  }
}

template <typename R>
void leaf_flux(double* const* wptr, const int64_t* wrs, const R* z, int l0, int nl, int p, int q,
               int nrhs, const double2* hsc, const double* d_D, const double* d_Pc2g,
               const int64_t* leaf_off, int64_t ext_total, double* hp, cudaStream_t st) {
  if (nl <= 0 || nrhs <= 0) return;
  const int pp = p * p;
  const int lp = p + 1;
  const int cap = (int)((200 * 1024 / 8 - pp - q * lp) / (p * lp + 4 * p));
  const int rb = std::max(1, std::min(8, cap));
  const size_t smem = (size_t)(pp + q * lp + rb * (p * lp + 4 * p)) * sizeof(double);
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_leaf_flux<R>), 200 * 1024))
    return;  // reported by the caller's launch check
  prof::Scope sc("leaf_flux<f64>", st, (double)nl * nrhs * (8.0 * p * p + 8.0 * q * p),
                 (double)nl * nrhs * ((double)p * p * 8.0 + (p - 2.0) * (p - 2.0) * sizeof(R) +
                                      4.0 * q * 8.0));
  k_leaf_flux<R><<<nl, 256, smem, st>>>(wptr, wrs, z, l0, p, q, nrhs, rb, hsc, d_D, d_Pc2g,
                                        leaf_off, ext_total, hp);
}

#define HPS_INST_LEAF(R)                                                                        \
  template void leaf_assemble<R>(const double* const*, int, int, int, int, const double2*,       \
                                 const double*, const double*, R*, R*, int64_t, int,            \
                                 cudaStream_t);                                                 \
  template void leaf_dtn<R>(R*, int64_t, int, int, int, int, const double2*, const double*,       \
                            const double*, const double*, R*, cudaStream_t, const R*, int64_t); \
  template void leaf_post<R>(const R*, int64_t, int, const double*, const int64_t*, int64_t, int, \
                             int, int, int, const double*, double* const*, const int64_t*,      \
                             cudaStream_t, const R*, int, const double*);                       \
  template void leaf_residual<R>(const double* const*, int, int, int, const double2*,           \
                                 const double*, double* const*, const int64_t*, int, R*,        \
                                 cudaStream_t);                                                 \
  template void leaf_y_residual<R>(const double* const*, int, int, int, int, const double2*,     \
                                   const double*, const double*, const R*, int64_t, R*,         \
                                   cudaStream_t);                                               \
  template void leaf_resflux<R>(const double* const*, int, int, int, int, const double2*,        \
                                const double*, const double*, double* const*, const int64_t*,   \
                                int, R*, const int64_t*, int64_t, double*, cudaStream_t);       \
  template void leaf_flux<R>(double* const*, const int64_t*, const R*, int, int, int, int, int,  \
                             const double2*, const double*, const double*, const int64_t*,      \
                             int64_t, double*, cudaStream_t);
HPS_INST_LEAF(double)
HPS_INST_LEAF(float)

}  // namespace hps
