// Device-side descriptors and launchers of libhps.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace hps {

// One dense system A X = B solved in place by LU with partial (row) pivoting:
// A (m x m, column-major, lda) is overwritten by its factors P A = L U, ipiv
// receives the pivot rows (absolute, 0-based, LAPACK order), B (m x nrhs, ldb)
// is overwritten by A^{-1} B.  A bad pivot (zero or not finite) records box+1
// in the status word.
template <typename R>
struct LuDesc {
  R* A;
  int* ipiv;
  R* B;
  int m, lda, nrhs, ldb;
  int box;
};

// C = beta C + alpha A B, all column-major (element types may differ from the
// compute type of the launch).
template <typename TA, typename TB = TA, typename TC = TA>
struct GemmDesc {
  const TA* A;
  const TB* B;
  TC* C;
  int M, N, K, lda, ldb, ldc;
};

// Gather of one merge (Section 4, eq. U_parent and eq. merge):
//   Aw = T33^a - T33^b (m x m), S = [-T31^a | T32^b] (m x ne, parent column order),
//   Cw = [T13^a ; T23^b] (ne x m, parent row order), Tp = diag(T11^a, T22^b).
// The children's T are read in their own precision (ta64 / tb64: double or float).
template <typename R>
struct MergeDesc {
  const void* Ta;
  const void* Tb;
  int ta64, tb64;
  R* Aw;
  R* S;
  R* Cw;
  R* Tp;       // may be null (root DtN not formed)
  R* W;        // may be null; else an m x m identity is written there (ld m)
  const int* src;
  int na, nb, m, ne, j3a, j3b;
};

// Downward pass of one merge (Algorithm 2, line 3): u3 = S u_parent, then the
// children's exterior vectors from the parent's and u3.
struct SolveScatterDesc {
  int64_t par_off, a_off, b_off;  // exterior-pool offsets (in nodes)
  const int* cmap_a;
  const int* cmap_b;
  int64_t u3_off;                 // offset of this merge's u3 block (in nodes)
  int na, nb, m;
};

// Body-load pass of one merge (correction equation of iterative refinement):
// z = (T33^a - T33^b)^{-1} (h3^b - h3^a), h^tau = [h1^a; h2^b] + [T13^a; T23^b] z,
// and in the downward pass u3 = S u_parent + z.  Offsets index the exterior
// pool (flux offsets h and values u share its layout), the u3 pool, and this
// merge's block of its level's z buffer (z_off * nrhs elements in, ld m).
struct BodyDesc {
  int64_t par_off, a_off, b_off, u3_off, z_off;
  const int* src;
  int j3a, j3b, m, ne;
};

// ---- dense engine (hps_linalg.cu)
// mode: kLuFactor (factor and solve; the factors are left partly unswapped),
// kLuFactorKeep (factor and solve, leaving P A = L U in LAPACK form for later
// solves), kLuSolveOnly (solve with factors from an earlier kLuFactorKeep).
// h_m / h_nrhs: host copies of each descriptor's m and nrhs (launch accounting
// only; null means every descriptor has the maximum sizes).
constexpr int kLuFactor = 0, kLuFactorKeep = 1, kLuSolveOnly = 2;
constexpr int kLeafGjN = 196;  // the order leaf_gj_inverse takes (p = 16)
// A^{-1} of n x n FP32 leaf systems (n = kLeafGjN only; false otherwise) by
// Gauss-Jordan elimination, one CTA per matrix: per descriptor A (ld n) is
// read and then overwritten by B's first nq columns; B's columns nq .. nq+n-1
// (ld n) receive A^{-1}.  Bad pivots as for the LU.
bool leaf_gj_inverse(const LuDesc<float>* d_desc, int nd, int n, int nq, int* status,
                     cudaStream_t st);
template <typename R>
void lu_solve_batched(const LuDesc<R>* d_desc, int ndesc, int max_m, int max_nrhs, int mode,
                      int* d_status, cudaStream_t st, const int* h_m, const int* h_nrhs);
// Two-level blocked LU (FP64, kLuFactor semantics) for large systems: outer
// block columns of kLuOuter are factored by the one-level steps restricted to
// the block, then the block's interchanges and unit-lower solve reach the far
// columns and one rank-kLuOuter product updates the trailing rows; backward
// substitution is blocked the same way.  The rank-kLuOuter products large
// enough run on the tensor cores (oz_gemm), the rest as FP64 tile GEMMs.
// h: host copies of the descriptors (d_desc their device copy), every one
// lu_tc_eligible.  push copies a host array to device memory that stays valid
// while the stream runs this call.  ws: lu_tc_workspace(h) bytes of scratch.
constexpr int kLuOuter = 256;
inline bool lu_tc_eligible(int m) { return m >= 2 * kLuOuter; }
struct LuDescHost {
  double* A;
  double* B;
  int m, lda, nrhs, ldb;
};
size_t lu_tc_workspace(const std::vector<LuDescHost>& h);
cudaError_t lu_solve_tc(const LuDesc<double>* d_desc, const std::vector<LuDescHost>& h,
                        int* d_status, cudaStream_t st,
                        void* (*push)(void* ctx, const void* src, size_t bytes), void* push_ctx,
                        void* ws, size_t ws_bytes);
// name / flops / bytes: launch accounting (algorithmic work of this launch).
// ws / ws_elems (optional): scratch of element type R.  With a scratch, a
// launch whose largest K exceeds kSplitK splits K into chunks of kSplitK across
// CTAs, writes the partial products to ws and sums them in a fixed order; the
// split of a product depends only on its own K, so its result does not depend
// on what else the launch holds.  Needs nd * ceil(max_K / kSplitK) * max_M *
// max_N elements (split_ws_elems); with less, the launch does not split.
constexpr int kSplitK = 128;
inline size_t split_ws_elems(int nd, int max_M, int max_N, int max_K) {
  return max_K > kSplitK ? (size_t)nd * ((max_K + kSplitK - 1) / kSplitK) * max_M * max_N : 0;
}
// With a status word, FP32 products (A and B in FP32) with M >= 96 and K >= 32
// run on the tensor cores (gemm_tc32), the others on the FP32 tile kernels;
// the choice (and the tensor-core tile width) depends on each product's own
// shape only, never on the other products of the launch.  Without a status
// word all run on the tile kernels.
__host__ __device__ constexpr bool gemm_on_tc(int M, int K) { return M >= 96 && K >= 32; }
template <typename R, typename TA, typename TB, typename TC>
void gemm_batched(const GemmDesc<TA, TB, TC>* d_desc, int ndesc, int max_M, int max_N, R alpha,
                  R beta, cudaStream_t st, const char* name, double flops, double bytes,
                  int max_K = 0, R* ws = nullptr, size_t ws_elems = 0, int* status = nullptr);
// C = beta C + alpha A B in FP32 accuracy on the tensor cores (hps_gemmtc.cu):
// every FP32 operand split exactly into three BF16 terms, six BF16 products
// per K step accumulated in FP32.  A wait that gives up sets *status to -1.
// Products of the list for which gemm_on_tc holds; the others are skipped.
template <typename TB, typename TC>
void gemm_tc32(const GemmDesc<float, TB, TC>* d_desc, int ndesc, int max_M, int max_N,
               float alpha, float beta, int* status, cudaStream_t st);

// ---- leaf kernels (hps_leaf.cu)
// Leaf kernels run on a group of leaves with one (p, q): group-local leaf j is
// global leaf l0 + j.  Per global leaf: hsc[l] = (2/hx, 2/hy) of its problem;
// wptr[l] / wrs[l] = base pointer and right-hand-side stride of its p x p block
// in the caller's u array.  Y of group leaf j starts at Y + j*ys (ni x 4q, ld
// ni); with_identity also writes an ni x ni identity after it, so that the leaf
// solve returns A_ii^{-1} as well.  Coefficient arrays start at the group's first leaf (group-local index j).
template <typename R>
void leaf_assemble(const double* const* coef, int l0, int nleaves, int p, int q,
                   const double2* hsc, const double* d_D, const double* d_Pg2c, R* Aii, R* Y,
                   int64_t ys, int with_identity, cudaStream_t st);
// dY (optional, leaf stride dys): a correction of Y; T is formed from Y + dY
// summed in FP64 and the rounded sum is written back to Y.
template <typename R>
void leaf_dtn(R* Y, int64_t ys, int l0, int nleaves, int p, int q, const double2* hsc,
              const double* d_D, const double* d_Pg2c, const double* d_Pc2g, R* T,
              cudaStream_t st, const R* dY = nullptr, int64_t dys = 0);
template <typename R>
void leaf_post(const R* Y, int64_t ys, int l0, const double* uext, const int64_t* leaf_ext_off,
               int64_t ext_total, int nleaves, int p, int q, int nrhs, const double* d_Pg2c,
               double* const* wptr, const int64_t* wrs, cudaStream_t st, const R* z = nullptr,
               int accumulate = 0, const double* bndv = nullptr);
template <typename R>
void leaf_residual(const double* const* coef, int l0, int nl, int p, const double2* hsc,
                   const double* d_D, double* const* wptr, const int64_t* wrs, int nrhs, R* rbuf,
                   cudaStream_t st);
// FP64 residual of the leaf systems themselves: rbuf (leaf stride ni*4q, ld ni)
// = -A_ie L1 - A_ii Y, Y read from Y + j*ys (ni x 4q, ld ni).
template <typename R>
void leaf_y_residual(const double* const* coef, int l0, int nl, int p, int q,
                     const double2* hsc, const double* d_D, const double* d_Pg2c, const R* Y,
                     int64_t ys, R* rbuf, cudaStream_t st);
// Without the mixed term (c12 absent): the FP64 residual r (as leaf_residual)
// and the fluxes of w itself, hp[r*ext_total + leaf_off[l] + g] = (L4 L3 w)_g,
// in one pass, by even and odd parts of the grid lines.
template <typename R>
void leaf_resflux(const double* const* coef, int l0, int nl, int p, int q, const double2* hsc,
                  const double* d_D, const double* d_Pc2g, double* const* wptr,
                  const int64_t* wrs, int nrhs, R* rbuf, const int64_t* leaf_off,
                  int64_t ext_total, double* hp, cudaStream_t st);
// The same two passes with the derivative products on the tensor cores (exact
// digit products, hps_residtc.cu), for p = 16, q <= 16 and operators without
// the mixed and first-order terms; false (nothing launched) for any other
// shape.  A tensor-core wait that gives up sets *status to -1.
template <typename R>
bool leaf_resflux_tc(const double* const* coef, int l0, int nl, int p, int q, const double2* hsc,
                     const double* d_D, const double* d_Pc2g, double* const* wptr,
                     const int64_t* wrs, int nrhs, R* rbuf, const int64_t* leaf_off,
                     int64_t ext_total, double* hp, int* status, cudaStream_t st);
// The FP64 boundary rows L1 u_e of every leaf and right-hand side on the tensor
// cores: out[((r*nleaves + l)*4 + side)*p + j] = sum_k Pg2c[j][k] u_e[side*q + k]
// (p = 16 and q <= 16 only; false otherwise).
bool leaf_bnd_interp_tc(const double* uext, const int64_t* leaf_ext_off, int l0, int nleaves,
                        int64_t ext_total, int p, int q, int nrhs, const double* d_Pg2c,
                        double* out, int* status, cudaStream_t st);
template <typename R>
bool leaf_y_residual_tc(const double* const* coef, int l0, int nl, int p, int q,
                        const double2* hsc, const double* d_D, const double* d_Pg2c, const R* Y,
                        int64_t ys, R* rbuf, int* status, cudaStream_t st);
template <typename R>
void leaf_flux(double* const* wptr, const int64_t* wrs, const R* z, int l0, int nl, int p, int q,
               int nrhs, const double2* hsc, const double* d_D, const double* d_Pc2g,
               const int64_t* leaf_off, int64_t ext_total, double* hp, cudaStream_t st);

// ---- merge / solve kernels (hps_merge.cu)
template <typename R>
void merge_gather(const MergeDesc<R>* d_desc, int ndesc, int64_t max_work, cudaStream_t st,
                  double bytes);
template <typename R>
void merge_rhs(const BodyDesc* d, int nd, int max_m, const double* hp, int64_t ext_total,
               int nrhs, R* zlev, cudaStream_t st);
void merge_hpar(const BodyDesc* d, int nd, int max_ne, double* hp, int64_t ext_total, int nrhs,
                cudaStream_t st);
template <typename R>
void z_to_u3(const BodyDesc* d, int nd, int max_m, const R* zlev, double* u3, int64_t u3_total,
             int nrhs, cudaStream_t st);
// Root exterior values of every problem from its Dirichlet data f (or zeros
// when f is null): uext[r*ext_total + root_off + k] = f[r*nbnd + rff[k]].
struct RootDesc {
  const double* f;
  const int* rff;
  int64_t root_off;
  int nbnd;
};
void solve_root_scatter(const RootDesc* d, int nprob, int max_nbnd, int nrhs, double* uext,
                        int64_t ext_total, cudaStream_t st);
void solve_child_scatter(const SolveScatterDesc* d_desc, int ndesc, int max_n, const double* u3,
                         int64_t u3_total, double* uext, int64_t ext_total, int nrhs,
                         cudaStream_t st);

// ---- FP64 GEMM on the tensor cores by exact BF16 splitting (hps_ozaki.cu)
// C = alpha A B + beta C, column-major, per descriptor.  oz_plan fills the
// tiling and workspace offsets and returns the workspace bytes; oz_gemm runs
// exponents, splitting and the tensor-core products.  A wait that gives up
// sets *status to -1 (a device error, distinct from pivot failures > 0).
struct OzDesc {
  const double* A;
  const double* B;
  double* C;
  int M, N, K, lda, ldb, ldc;
  int mt = 0, nt = 0, nkb = 0;
  int ea_off = 0, eb_off = 0;
  int64_t a_off = 0, b_off = 0;
};
size_t oz_plan(std::vector<OzDesc>& ds);
cudaError_t oz_gemm(const OzDesc* d_desc, const std::vector<OzDesc>& h, void* work,
                    size_t work_bytes, double alpha, double beta, int* status, cudaStream_t st,
                    const char* name);
// Products worth the splitting: large enough that the tensor-core path beats
// FP64 FMAs (a property of the product alone, so batches keep solo results).
inline bool oz_eligible(int M, int N, int K) {
  return M >= 128 && N >= 128 && K >= 64 && (double)M * N * K >= 8.0e6;
}

// ---- post-processing (hps_post.cu)
// g = T f for a root DtN T (n x n, column-major, FP64) with f and g in Gamma
// order (nrhs columns of n) and rff[k] the Gamma index of root exterior
// position k; ws holds dtn_apply_ws_bytes(n, nrhs) bytes.  A wait of the
// tensor-core path that gives up sets *status to -1.
size_t dtn_apply_ws_bytes(int n, int nrhs);
cudaError_t dtn_apply(const double* T, int n, const int* rff, const double* f, int nrhs,
                      double* g, void* ws, size_t ws_bytes, int* status, cudaStream_t st);
void f32_to_f64(const float* s, double* d, int64_t n, cudaStream_t st);
void f64_to_f32(const double* s, float* d, int64_t n, cudaStream_t st);
// The leaf grid of one problem, for point evaluation.
struct InterpGrid {
  double x0, x1, y0, y1;
  int nx, ny, p;
};
// out[r * npts + i] = u_r(xy_i) from the leaf Chebyshev values u (nrhs blocks
// of nx*ny*p*p); points outside the closed domain give NaN and set *status to 1.
void interp_points(const double* u, int nrhs, const InterpGrid& s, const double* xy,
                   int64_t npts, double* out, int* status, cudaStream_t st);

// ---- accelerated refinement (hps_refine.cu)
constexpr int kAaMaxDepth = 8;               // longest Anderson history
constexpr int kAaChunk = 8192;               // elements per reduction chunk
constexpr int kAaQ = 2 + 2 * kAaMaxDepth;    // partials per chunk
// One right-hand side of one problem: w (the iterate, the caller's u) and the
// column's range [off, off + len) in the work vectors; its chunks are
// ch0 .. ch0 + ceil(len / kAaChunk) - 1.
struct AaCol {
  double* w;
  int64_t off, len, ch0;
};
// Forms dF_new = F - Fprev and G_new = dWlast + dF_new in ring slot slot_new
// (j >= 1), sets Fprev = F, and reduces per column: colsum[c*kAaQ + q] with
// q = 0 max|F|, 1 max|w|, 2 + s <dF_s, F>, 2 + kAaMaxDepth + s <dF_s, dF_new>.
// col_of[b]: the column of chunk b.
void aa_reduce(const AaCol* cols, const int* col_of, int ncol, int64_t nchunks, const double* F,
               double* Fprev,
               const double* dWlast, float* dF, double* G, int64_t nu, int j, int slot_new,
               int nslots, double* part, double* colsum, cudaStream_t st);
// w += F - sum_s gamma_s G_s (mode 1, also dWlast = that update), w += F
// (mode 2) or nothing (mode 0), per column from coef[c*(kAaMaxDepth+1) ...].
void aa_update(const AaCol* cols, const int* col_of, int ncol, int64_t nchunks, const double* F,
               double* dWlast,
               const double* G, int64_t nu, int nslots, const double* coef, cudaStream_t st);

}  // namespace hps
