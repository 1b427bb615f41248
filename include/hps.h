/*
 * hps.h -- C ABI of a GB300 (sm_103a) direct solver for variable-coefficient
 * elliptic PDEs on a rectangle, discretised by the composite spectral
 * collocation method of Gillman & Martinsson, "A direct solver with O(N)
 * complexity for variable coefficient elliptic PDEs discretized via a
 * high-order composite spectral collocation method" (arXiv:1307.2665).
 *
 * Problem (Section 1.1, eqs. basic and defA): on Omega = [x0,x1] x [y0,y1],
 *     A u = 0 in Omega,  u = f on the boundary Gamma, with
 *     A u = -c11 u_xx - 2 c12 u_xy - c22 u_yy + c1 u_x + c2 u_y + c u.
 *
 * Discretisation (Sections 2-3): Omega is split into nx-by-ny equal leaves.
 * Each leaf carries a p x p tensor grid of Chebyshev extreme points (the
 * collocation nodes) and q Gauss-Legendre points on each edge (the nodes of
 * the global unknowns).  hps_build runs Algorithm 1 (leaf DtN maps, Section 3;
 * Schur-complement merges, Section 4, eqs. U_parent and merge); hps_solve runs
 * Algorithm 2 (downward pass) and the leaf post-processing of Section 5.3, and
 * returns u at every leaf's p x p Chebyshev grid.
 *
 * Conventions shared by every entry point:
 *   - Leaf l = iy*nx + ix (ix along x).  Within a leaf, node (a, b) has index
 *     a*p + b with a the y index and b the x index, both increasing with the
 *     coordinate ("iy-major").
 *   - Coefficient arrays hold nx*ny*p*p doubles sampled at hps_cheb_nodes().
 *     A NULL coefficient pointer means that coefficient is identically zero.
 *   - Dirichlet data f holds, per right-hand side, the values at the
 *     nbnd = 2*(nx+ny)*q Gauss nodes of Gamma in counter-clockwise order from
 *     (x0, y0): south side (x increasing), east (y increasing), north
 *     (x decreasing), west (y decreasing).  hps_boundary_nodes() returns them.
 *     Layout: f[r*nbnd + i] for right-hand side r.
 *   - The solution u holds u[(r*nx*ny + l)*p*p + a*p + b].
 *   - Every array argument is a HOST pointer unless options.device_ptrs is 1,
 *     in which case coefficient, f and u pointers passed to hps_build /
 *     hps_solve are device pointers on the current CUDA device.
 *   - The caller owns every buffer it passes.  The library copies what it
 *     needs; the handle owns its device memory until hps_free().
 *   - Return value: HPS_OK (0) or a negative status (below).  All argument
 *     validation happens before any device work; on error no handle is
 *     returned and nothing is left allocated.
 */
#ifndef HPS_H
#define HPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPS_OK 0
#define HPS_EINVAL (-1)         /* bad sizes, p < 3, q < 1, q > p, q == p on a grid with
                                   interior vertices (see hps_build), NULL required pointer */
#define HPS_ENOMEM (-2)         /* device or host allocation failed, or over the memory budget */
#define HPS_ESINGULAR (-3)      /* zero or non-finite pivot in a leaf or merge factorisation */
#define HPS_ENOTCONVERGED (-4)  /* iterative refinement did not reach the tolerance */
#define HPS_EDEVICE (-5)        /* CUDA error */

#define HPS_FP64 0   /* every stage in double precision */
#define HPS_MIXED 1  /* FP32 leaves and lower merges, FP64 top merges, FP64 refinement */

typedef struct hps_handle_s* hps_handle;

typedef struct {
  double x0, x1, y0, y1;
} hps_domain;

typedef struct {
  int precision;          /* HPS_FP64 or HPS_MIXED */
  double refine_tol;      /* mixed mode: stop when max|delta| <= tol * max|u| (default 1e-11) */
  int max_refine;         /* mixed mode: iteration cap (default 10; 0: low-precision solve only) */
  int fp64_top_levels;    /* mixed mode: merge levels below the root kept in FP64 (default 2) */
  int device_ptrs;        /* 1: coefficient / f / u pointers are device pointers */
  void* stream;           /* cudaStream_t to run on; NULL: the library's own stream */
  int form_root_dtn;      /* 1: also form the root DtN T^1 (not needed by hps_solve) */
  int refine_depth;       /* mixed mode: Anderson history length of the refinement, 0..8
                             (default 0: plain refinement u += delta, as fast as the
                             accelerated one once the leaf operators are corrected) */
  int leaf_refine;        /* mixed mode: 1 (default) corrects each leaf's FP32 solution
                             operator Y once against its FP64 residual before the leaf
                             DtN map is formed from it; 0: no correction */
} hps_options;

typedef struct {
  int status;             /* HPS_OK or the failing status */
  int iterations;         /* refinement corrections computed, the most over all
                             right-hand sides (0 in FP64 mode) */
  double last_update;     /* largest over right-hand sides of the last max|delta| / max|u|
                             (the last correction applied) */
  int bad_box;            /* box index of a singular pivot, or -1 */
} hps_solve_info;

/* Fill *opt with the defaults above (FP64, host pointers, library stream). */
void hps_default_options(hps_options* opt);

/* Number of Dirichlet nodes on Gamma, 2*(nx+ny)*q. */
int64_t hps_boundary_count(int nx, int ny, int q);

/* Coordinates of every leaf's Chebyshev grid (Section 3.1: p extreme points
 * per direction).  xy: host array of nx*ny*p*p*2 doubles, (x, y) pairs in the
 * node order above. */
int hps_cheb_nodes(hps_domain d, int nx, int ny, int p, double* xy);

/* Coordinates (x, y) of the Gauss nodes on Gamma in the order of f, computed
 * without a handle.  xy: host array of 2*nbnd doubles. */
int hps_boundary_nodes_grid(hps_domain d, int nx, int ny, int q, double* xy);

/* Build stage (Algorithm 1): leaf DtN maps T = L4 L3 L2 L1 (Section 3.2) for
 * every leaf, then the merges of Section 4 up the binary tree, storing each
 * merge's solution operator S (eq. U_parent) and each leaf's interior solution
 * operator Y = -A_ii^{-1} A_ie L1 (eq. leaf_solve, Section 5.3) on the device.
 * The tree splits a box's longer side at floor(n/2) (ties: x), so any nx, ny
 * >= 1 is accepted.  q must be below p when nx > 1 and ny > 1: with q == p the
 * side interpolants of Step 1 are bijective and averaging the two values at a
 * corner leaves one free combination of the four edges at every interior vertex
 * (+a, +a on the two horizontal edges, -a, -a on the two vertical ones), so the
 * composite system is singular and so is every merge whose interface holds an
 * interior vertex.  Returns HPS_ESINGULAR if a pivot is zero or not finite (e.g.
 * a Helmholtz box at a Dirichlet resonance, Remark 1.1). */
int hps_build(hps_domain d, int nx, int ny, int p, int q,
              const double* c11, const double* c12, const double* c22,
              const double* c1, const double* c2, const double* c,
              const hps_options* opt, hps_handle* out);

/* One problem of a batch: the arguments of hps_build. */
typedef struct {
  hps_domain d;
  int nx, ny, p, q;
  const double *c11, *c12, *c22, *c1, *c2, *c;
} hps_problem;

/* Build stage for a batch of independent problems (of uneven size and order p)
 * in one handle.  The leaves of consecutive problems with equal (p, q) run as
 * one launch group, and the merges of all problems are processed height by
 * height (heights counted from the leaves), one launch sequence per height for
 * the whole batch (two in mixed mode: FP32 and FP64 merges).  Every problem's
 * arithmetic is the same as when it is built alone.  Options apply to every
 * problem; fp64_top_levels counts from each problem's own root. */
int hps_build_batch(const hps_problem* probs, int nprob, const hps_options* opt, hps_handle* out);

/* Number of problems held by a handle (1 for hps_build). */
int hps_batch_size(hps_handle h);

/* Solve stage for a batch handle: f[k] (nrhs * nbnd_k) and u[k] (nrhs * nx_k *
 * ny_k * p_k * p_k) for problem k, same layouts as hps_solve; the pointer kind
 * follows options.device_ptrs of the build.  In mixed mode the refinement runs
 * until every problem meets the tolerance. */
int hps_solve_batch(hps_handle h, const double* const* f, int nrhs, double* const* u,
                    hps_solve_info* info);

/* Coordinates of the Gauss nodes on Gamma in the order of f (host array of
 * 2*nbnd doubles); for a batch handle, of its first problem. */
int hps_boundary_nodes(hps_handle h, double* xy);

/* Solve stage (Algorithm 2 and Section 5.3): given nrhs Dirichlet data sets f,
 * compute u at every leaf's Chebyshev grid.  In HPS_MIXED mode this runs
 * iterative refinement against the FP64 residual of the global collocation
 * system: each step solves the correction equation (interior residual as a
 * body load, flux jumps at the interior Gauss nodes) with the low-precision
 * factors, giving a correction delta of the iterate u in FP64.  With
 * refine_depth m > 0 the step is Anderson-accelerated: the new iterate is
 * u + delta minus the least-squares combination of the last m differences of
 * corrections and iterates that best cancels delta (the GMRES iterate of the
 * same Krylov space, for this linear map); with m = 0 it is u + delta.  Every
 * right-hand side of every problem is refined on its own: it stops when its
 * max|delta| <= refine_tol * max|u| (then u += delta), when the last two
 * corrections shrink by a ratio r < 1/4 with r * max|delta| <= refine_tol *
 * max|u| (then u += delta: the next correction, the error left, is predicted
 * below the tolerance and is not computed), when delta no longer
 * shrinks to half of the smaller of the two previous ones (the iterate has
 * reached the accuracy the FP64 residual resolves for this conditioning), or
 * after max_refine corrections, and its result does not depend on the other
 * right-hand sides or problems solved with it.  HPS_ENOTCONVERGED if any
 * right-hand side stopped above refine_tol (u holds the last iterates;
 * info->last_update the largest relative correction).  info may be NULL.
 * f and u follow options.device_ptrs of the build. */
int hps_solve(hps_handle h, const double* f, int nrhs, double* u, hps_solve_info* info);

/* Same as hps_solve with an explicit pointer kind: device_ptrs 0 (host arrays,
 * copies to and from the device inside the call) or 1 (device arrays).
 * hps_solve / hps_solve_ex need a single-problem handle (else HPS_EINVAL). */
int hps_solve_ex(hps_handle h, const double* f, int nrhs, double* u, int device_ptrs,
                 hps_solve_info* info);

/* Sizes of a built handle: number of leaves, p, q (of the first problem),
 * total nbnd, bytes of device memory held.  Any output pointer may be NULL. */
int hps_query(hps_handle h, int* n_leaves, int* p, int* q, int64_t* nbnd, int64_t* device_bytes);

/* Device memory estimates from the plan alone (no device work): build_peak,
 * the most held during hps_build / hps_build_batch of these problems with
 * these options; resident, what the handle keeps afterwards (S and Y, and in
 * mixed mode W, [T13; T23] and the coefficients); solve, the workspace one
 * solve with nrhs right-hand sides adds while it runs (u excluded).  Any
 * output pointer may be NULL.  The serving loop admits work by these. */
int hps_estimate_bytes(const hps_problem* probs, int nprob, const hps_options* opt, int nrhs,
                       int64_t* build_peak, int64_t* resident, int64_t* solve);

/* Apply the DtN map of the whole domain (the root map T^1 of Algorithm 1;
 * Section 9.1 times this as T_apply, Table 1): g = T^1 f for nrhs Dirichlet
 * data sets f (nrhs * nbnd, the layout and Gamma order of hps_solve).  g has
 * the same layout: at each Gamma node, the derivative of the solution in the
 * global direction (d/dx on the west and east sides, d/dy on the south and
 * north sides; the fluxes v of Section 2), not the outward normal derivative.
 * Needs a single-problem handle built with form_root_dtn = 1, which keeps T^1
 * (nbnd^2 doubles) on the device; T^1 is applied as the build formed it
 * (mixed mode: from the FP32 maps of the lower levels, without refinement).
 * f and g: host arrays (device_ptrs 0, copied inside the call) or device
 * arrays (1).  HPS_EINVAL: NULL pointer, nrhs < 1, a batch handle or a handle
 * without T^1. */
int hps_apply_dtn(hps_handle h, const double* f, int nrhs, double* g, int device_ptrs);

/* Evaluate solutions at arbitrary points (Section 5.3): inside a leaf the
 * solution is the tensor-product polynomial interpolant of its p x p
 * Chebyshev values.  u: nrhs solutions in the layout of hps_solve's output;
 * xy: npts (x, y) pairs; out[r * npts + i] = u_r(x_i, y_i).  A point on an
 * edge shared by two leaves takes the leaf to its east (north); a point on the
 * domain's east (north) side takes the last leaf.  Points must lie in the
 * closed domain: with host arrays (device_ptrs 0) any other point makes the
 * call return HPS_EINVAL before device work; with device arrays (1) its outputs
 * are NaN and the call returns HPS_EINVAL.  npts = 0 is a no-op.  Needs a
 * single-problem handle (its grid is all that is used). */
int hps_interpolate(hps_handle h, const double* u, int nrhs, const double* xy, int64_t npts,
                    double* out, int device_ptrs);

/* C = alpha A B + beta C for FP64 device matrices (column-major, leading
 * dimensions lda >= M, ldb >= K, ldc >= M) through the tensor-core engine the
 * FP64 merges use for their Schur-complement products (eq. merge): every row
 * of A and column of B is split exactly into 8 BF16 slices of 7 bits, the 36
 * significant slice products run as tcgen05 MMAs with exact FP32
 * accumulation, and the integer results are combined in 64-bit fixed point;
 * the error is of the order of an FP64 GEMM's rounding.  Synchronous on the
 * current device.  Exposed for testing and measurement; the paper computes
 * these products in plain double precision. */
int hps_dgemm_tc(int M, int N, int K, double alpha, const double* A, int lda, const double* B,
                 int ldb, double beta, double* C, int ldc);

/* C = alpha A B + beta C for FP32 device matrices (column-major, leading
 * dimensions lda >= M, ldb >= K, ldc >= M) through the engine the mixed mode
 * uses for its FP32 products (leaf inverse times residual, Schur complements
 * of the lower merges, Section 4 eq. merge in FP32): with M >= 96 and K >= 32
 * on the tensor cores, every FP32 value split exactly into three BF16 terms
 * and six BF16 products per K step accumulated in FP32 (the error of an FP32
 * GEMM); smaller products on the FP32 tile kernels.  Synchronous on the
 * current device.  Exposed for testing and measurement. */
int hps_sgemm_tc(int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                 int ldb, float beta, float* C, int ldc);

/* One pass of the mixed mode's FP64 residual kernel on raw leaves (Section
 * 3.1's collocation operator A = -c11 d_xx - c22 d_yy + c with the Section 3.2
 * leaf maps): for every leaf l and right-hand side k,
 *   r[(l nrhs + k) (p-2)^2 + i] = -(A w)_i at the interior Chebyshev nodes
 *     (i = (a-1)(p-2) + (b-1), node (a, b) = a p + b, a along y, b along x),
 *   flux[(k nleaves + l) 4q + g] = (L4 L3 w)_g, the side fluxes at the q
 *     Gauss points of the sides S, E, N, W (d/dy on S and N, d/dx on E and W),
 * from w[(k nleaves + l) p^2 + node] and the coefficient samples c11, c22, c
 * (nleaves x p^2 each, leaf-major; null = absent) on leaves of size hx x hy.
 * All arrays are device memory.  tensor_cores = 1: the tensor-core kernel
 * (exact BF16 digit products; p = 16, q <= 16, else HPS_EINVAL); 0: the
 * FP64-pipe kernel (even and odd parts of the grid lines).  A grid holding an
 * infinity or NaN gives NaN at all of its outputs in the tensor-core kernel.
 * Synchronous.  Exposed for testing and measurement. */
int hps_leaf_residual(int p, int q, int nleaves, double hx, double hy, const double* c11,
                      const double* c22, const double* c, const double* w, int nrhs, double* r,
                      double* flux, int tensor_cores);

/* Batched FP32 inverse through the kernel the mixed mode uses for its leaf
 * systems A_ii (Section 3.1; the paper solves them by a dense factorisation):
 * Gauss-Jordan elimination with partial pivoting, one thread block per matrix
 * with the whole matrix in registers.  Ainv[m n^2 ..] = A[m n^2 ..]^{-1} for
 * m < count, every matrix n x n column-major; A and Ainv are 16-byte aligned
 * device memory and must not overlap; A is not modified.  Only n = 196 (the
 * interior of a p = 16 leaf); otherwise, or for overlapping or unaligned
 * arrays, HPS_EINVAL with the reason in hps_last_error().  A zero or non-finite pivot gives HPS_ESINGULAR
 * (hps_last_error() names the first such matrix); Ainv is then written but
 * meaningless for it.  Synchronous.  Exposed for testing and measurement. */
int hps_sinv_gj(int n, int count, const float* A, float* Ainv);

/* Release the solve workspace a handle caches between solves (exterior-value
 * pools, refinement buffers, staging); the next solve allocates it again.
 * Must not overlap a solve on the same handle. */
int hps_release_workspace(hps_handle h);

/* Release every resource of the handle (NULL is accepted). */
int hps_free(hps_handle h);

/* Static text for a status code. */
const char* hps_status_string(int status);

/* Text of the last CUDA error seen by this thread inside the library (empty if
 * none); valid until the next library call on this thread. */
const char* hps_last_error(void);

/* Solve without allocating (the paper has no counterpart: this serves callers
 * that cannot allocate device memory at solve time, e.g. a process with a
 * fixed memory budget reserved up front, or code that must not enter the
 * allocator or synchronise the device while other work runs).  The same
 * result, to rounding, as hps_solve_ex(h, f, nrhs, u, 1, NULL) for an HPS_FP64
 * handle, with f and u device pointers (the downward products sum their
 * columns in another order: no split-K scratch).  Its working memory is a
 * static 16 MiB device array that every GPU loading the library holds until
 * the process exits, so no cudaMalloc / cudaFree or other allocation happens
 * in the call.
 *   - Limit: 8 * nrhs * (exterior-pool + interface) values plus the launch
 *     descriptors must fit in the 16 MiB, and the handle may have at most 256
 *     merge heights; otherwise HPS_EINVAL, with the sizes in hps_last_error().
 *     Mixed-precision handles return HPS_EINVAL.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - Every call copies descriptors from host memory and synchronises the
 *     handle's stream before it returns: do not call it while that stream is
 *     being captured into a CUDA graph.
 *   - Every call shares the one array (its contents are those of the last
 *     call; nothing in it needs to start at zero).  Calls that overlap on the
 *     GPU race: serialise them (the call itself returns only after its work has
 *     finished on the handle's stream). */
int hps_solve_static(hps_handle h, const double* f, int nrhs, double* u);

/* ---- Launch accounting (instrumentation, not part of the method) --------
 * Every kernel launch of the library is counted.  With profiling enabled,
 * each launch is bracketed by CUDA events on its stream and charged, under
 * its kernel name, with the algorithmic flops and bytes of that launch (the
 * dense work the method itself defines, counted from the problem sizes).
 * hps_profile_read synchronises the device, fills up to max_out entries and
 * returns the number of kernel names recorded since the last reset.  The
 * name strings stay valid until the next hps_profile_read or reset. */
typedef struct {
  const char* name;
  int64_t launches;
  double ms;
  double flops;
  double bytes;
} hps_kernel_stat;

int64_t hps_kernel_launches(void);
void hps_profile_enable(int on);
void hps_profile_reset(void);
int hps_profile_read(hps_kernel_stat* out, int max_out);

#ifdef __cplusplus
}
#endif
#endif /* HPS_H */
