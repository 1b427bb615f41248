// Device-side descriptors and launchers of libhps.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

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

// C = beta C + alpha A B, all column-major.
template <typename R>
struct GemmDesc {
  const R* A;
  const R* B;
  R* C;
  int M, N, K, lda, ldb, ldc;
};

// Gather of one merge (Section 4, eq. U_parent and eq. merge):
//   Aw = T33^a - T33^b (m x m), S = [-T31^a | T32^b] (m x ne, parent column order),
//   Cw = [T13^a ; T23^b] (ne x m, parent row order), Tp = diag(T11^a, T22^b).
template <typename Rin, typename R>
struct MergeDesc {
  const Rin* Ta;
  const Rin* Tb;
  R* Aw;
  R* S;
  R* Cw;
  R* Tp;       // may be null (root DtN not formed)
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

// ---- dense engine (hps_linalg.cu)
template <typename R>
void lu_solve_batched(const LuDesc<R>* d_desc, int ndesc, int max_m, int max_nrhs, bool swap_left,
                      int* d_status, cudaStream_t st);
template <typename R>
void gemm_batched(const GemmDesc<R>* d_desc, int ndesc, int max_M, int max_N, R alpha, R beta,
                  cudaStream_t st);

// ---- leaf kernels (hps_leaf.cu)
struct LeafConsts;  // device copy of the 1-D constants
template <typename R>
void leaf_assemble(const double* const* coef, int nleaves, int p, int q, double hx, double hy,
                   const double* d_D, const double* d_Pg2c, R* Aii, R* Y, cudaStream_t st);
template <typename R>
void leaf_dtn(const R* Y, int nleaves, int p, int q, double hx, double hy, const double* d_D,
              const double* d_Pg2c, const double* d_Pc2g, R* T, cudaStream_t st);
template <typename R>
void leaf_post(const R* Y, const double* uext, const int64_t* leaf_ext_off, int64_t ext_total,
               int nleaves, int p, int q, int nrhs, const double* d_Pg2c, double* u,
               cudaStream_t st);

// ---- merge / solve kernels (hps_merge.cu)
template <typename Rin, typename R>
void merge_gather(const MergeDesc<Rin, R>* d_desc, int ndesc, int64_t max_work, cudaStream_t st);
void solve_root_scatter(const double* f, const int* root_from_f, int nbnd, int nrhs,
                        double* uext, int64_t root_off, int64_t ext_total, cudaStream_t st);
void solve_child_scatter(const SolveScatterDesc* d_desc, int ndesc, int max_n, const double* u3,
                         int64_t u3_total, double* uext, int64_t ext_total, int nrhs,
                         cudaStream_t st);

}  // namespace hps
