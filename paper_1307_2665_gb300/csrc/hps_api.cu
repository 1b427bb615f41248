// C ABI of libhps: the build stage (Algorithm 1) and the solve stage
// (Algorithm 2 + Section 5.3) orchestrated over the batched kernels.
//
// A handle holds one problem or a batch of independent problems (a forest).
// Leaves are processed per group of equal (p, q); merges per tree height
// (counted from the leaves) across all problems, so every launch covers every
// leaf or every merge of that height in the whole batch:
//   leaves  leaf_assemble -> LU of [A_ii | -A_ie L1] -> Y, leaf_dtn -> T
//   h >= 1  merge_gather  -> LU of [T33^a - T33^b | -T31^a, T32^b] -> S,
//           GEMM Tp += [T13^a; T23^b] S (eq. merge; skipped at a root unless
//           the root DtN is requested: the solve never needs it)
// Children's T are released in stream order once every parent reading them is
// built.  All device memory comes from a stream-ordered pool and all launch
// descriptors are staged in pinned memory, so a build synchronises the host
// only once, at the end, to read the pivot status.
//
// Precision.  HPS_FP64: every stage in double.  HPS_MIXED: the leaves and the
// merges below each problem's top `fp64_top_levels` heights run in float, the
// top heights in double; float and double merges of one height are two
// launch groups.  The build then also forms A_ii^{-1} and (T33^a - T33^b)^{-1}
// (an identity appended to each right-hand side) and keeps [T13^a; T23^b],
// and the solve refines against the FP64 residual of the global collocation
// system, one body-load correction per iteration (the elimination of
// Algorithms 1-2 applied to a right-hand side).
//
// Solve: root exterior values from f, then per height from the top a batched
// GEMM u3 = S u_parent and a scatter into the children's exterior vectors, then
// the leaf post-process w_full = [L1 ; Y] u_e.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hps.h"
#include "hps_internal.hpp"
#include "hps_kernels.cuh"
#include "hps_prof.hpp"

using namespace hps;

namespace {

thread_local std::string g_last_error;

struct CudaError {
  cudaError_t err;
};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) {
    g_last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
    throw CudaError{e};
  }
}

// One stream-ordered pool per device; freed blocks stay cached for reuse.
cudaMemPool_t device_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  ck(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  ck(cudaMemPoolCreate(&pool, &props));
  uint64_t thr = UINT64_MAX;
  ck(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  pools[dev] = pool;
  return pool;
}

// Device buffer from the pool, released in the order of its stream.
struct PoolBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  PoolBuf() = default;
  PoolBuf(const PoolBuf&) = delete;
  PoolBuf& operator=(const PoolBuf&) = delete;
  ~PoolBuf() { release(); }
  void alloc(size_t n, cudaStream_t s) {
    release();
    if (n == 0) return;
    ck(cudaMallocFromPoolAsync(&p, n, device_pool(), s));
    st = s;
    bytes = n;
  }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};
using PoolPtr = std::unique_ptr<PoolBuf>;
PoolPtr new_buf() { return PoolPtr(new PoolBuf()); }

// Pinned staging of launch descriptors: each array is copied into the next
// free slice of a pinned host block and uploaded asynchronously into the same
// offset of a device block.  Slices are never rewritten before the owner
// synchronises, so no copy is ever overtaken.
struct Stager {
  void* host = nullptr;
  size_t cap = 0, used = 0;
  PoolBuf dev;
  Stager() = default;
  Stager(const Stager&) = delete;
  Stager& operator=(const Stager&) = delete;
  ~Stager() {
    if (host) cudaFreeHost(host);
  }
  void begin(size_t bytes, cudaStream_t st) {
    bytes = std::max<size_t>(bytes, 256);
    if (cap < bytes) {
      if (host) {
        ck(cudaStreamSynchronize(st));
        cudaFreeHost(host);
      }
      host = nullptr;
      cap = 0;
      ck(cudaMallocHost(&host, bytes));
      cap = bytes;
    }
    if (dev.bytes < bytes) dev.alloc(bytes, st);
    used = 0;
  }
  void* push_raw(const void* src, size_t n, cudaStream_t st) {
    size_t off = (used + 255) & ~size_t(255);
    if (off + n > cap || off + n > dev.bytes) throw std::bad_alloc();
    if (n) {
      std::memcpy(static_cast<char*>(host) + off, src, n);
      ck(cudaMemcpyAsync(static_cast<char*>(dev.p) + off, static_cast<char*>(host) + off, n,
                         cudaMemcpyHostToDevice, st));
    }
    used = off + n;
    return static_cast<char*>(dev.p) + off;
  }
  template <typename T>
  T* push(const std::vector<T>& v, cudaStream_t st) {
    return static_cast<T*>(push_raw(v.data(), v.size() * sizeof(T), st));
  }
};

// Smallest FP32 merge (interface unknowns) whose S is formed as W [-T31 | T32].
constexpr int kNBw = 32;

// Raw pushes through the stager (callback form for the two-level LU).
struct StagerCtx {
  Stager* stg;
  cudaStream_t st;
  static void* push(void* ctx, const void* src, size_t n) {
    auto* c = static_cast<StagerCtx*>(ctx);
    return c->stg->push_raw(src, n, c->st);
  }
};

template <typename T>
size_t stage_bytes(size_t n) {
  return n * sizeof(T) + 256;
}

// Leaves of consecutive problems with one (p, q).
struct LeafGroup {
  int l0 = 0, nl = 0, p = 0, q = 0, ni = 0, nq = 0;
  int64_t ys = 0;                   // elements per leaf in Y
  Consts consts;
  PoolPtr Y = new_buf();            // per leaf [Y | A_ii^{-1} (mixed)] (ld ni)
  PoolPtr dD = new_buf(), dPg2c = new_buf(), dPc2g = new_buf();
  const double* coefp[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  PoolPtr rleaf = new_buf(), zleaf = new_buf();  // mixed: residual and correction
  void* gemm_leaf = nullptr;        // mixed: z = A_ii^{-1} r
  // mixed, no mixed term: per problem of the group, the side fluxes of
  // interior values (4q x ni, FP32), and the per-solve products h += F_i z
  PoolPtr Fi = new_buf();
  int prob0 = 0;
  void* gemm_fz = nullptr;
};

// Merges of one height and one precision, across all problems.
struct LevelGroup {
  int h = 0, f64 = 1;
  std::vector<int> boxes;
  int max_m = 0, max_ne = 0, max_nanb = 0;
  int64_t sum_m = 0;                // rows of the group's z buffer
  PoolPtr S = new_buf(), Cw = new_buf();  // [S | W (mixed)] per merge; Cw kept in mixed mode
  std::vector<int64_t> s_off, cw_off, z_off;
  std::vector<int> hm, hne;         // host copies of m and ne (launch accounting)
  SolveScatterDesc* scatter = nullptr;  // device descriptors (the handle's keep stager)
  BodyDesc* body = nullptr;
  PoolPtr rlev = new_buf(), zlev = new_buf();  // mixed solve buffers
  void* gemm_down = nullptr;        // per solve configuration
  void* gemm_w = nullptr;
  void* gemm_hpar = nullptr;
  int n_hpar = 0;                   // merges with a parent (a root's offsets are never read)
  int built_f64 = 0;                // mixed mode: factored in FP64, solved with FP32 copies
  double down_flops1 = 0, down_bytes = 0;
};

}  // namespace

struct hps_handle_s {
  Plan plan;
  hps_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool mixed = false;
  int nprob = 0;
  std::vector<LeafGroup> lg;
  std::vector<LevelGroup> lev;      // in increasing height
  PoolBuf maps, root_from_f, leaf_off, hsc, status, coef;
  PoolBuf root_dtn;                 // form_root_dtn: each problem's T^1 in FP64
  std::vector<int64_t> root_dtn_off;
  std::vector<int64_t> src_off, cma_off, cmb_off, u3_off;
  int64_t u3_total = 0;
  Stager keep;                      // descriptors that live as long as the handle
  // solve workspace and descriptors, cached for one nrhs
  int cache_nrhs = 0;
  PoolBuf uext, u3, hpool, split_ws, fstage, ustage;
  Stager solve_st, call_st;
  double* h_aa = nullptr;           // pinned: refinement sums and weights per column
  size_t h_aa_cap = 0;
  ~hps_handle_s() {
    if (stream) cudaStreamSynchronize(stream);
    if (h_aa) cudaFreeHost(h_aa);
  }
};

namespace {

int validate(hps_domain d, int nx, int ny, int p, int q) {
  if (nx < 1 || ny < 1 || p < 3 || q < 1 || q > p) return HPS_EINVAL;
  // q == p with interior vertices: the composite system is singular (one null
  // vector per interior vertex, from the averaged corners of Step 1)
  if (q == p && nx > 1 && ny > 1) return HPS_EINVAL;
  if (!(d.x1 > d.x0) || !(d.y1 > d.y0) || !std::isfinite(d.x0) || !std::isfinite(d.x1) ||
      !std::isfinite(d.y0) || !std::isfinite(d.y1))
    return HPS_EINVAL;
  if (p > 64 || (int64_t)nx * ny > (1 << 26)) return HPS_EINVAL;
  return HPS_OK;
}

// ------------------------------------------------------------------ build
// T of every box, in the precision it was produced in.
struct TRef {
  const void* p = nullptr;
  int f64 = 1;
};

template <typename R>
void build_leaves(hps_handle_s& H, LeafGroup& G, Stager& stg, std::vector<TRef>& Tref,
                  PoolBuf& T0) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  const int ni = G.ni, nq = G.nq, nl = G.nl;
  // mixed mode also forms A_ii^{-1} (columns nq .. nq+ni-1 of Y): at p = 16 by
  // Gauss-Jordan in registers, Y's first nq columns then by one product;
  // otherwise by the LU with identity right-hand sides after -A_ie L1
  const int nrhs_leaf = nq + (H.mixed ? ni : 0);
  const bool gj = std::is_same<R, float>::value && H.mixed && ni == kLeafGjN;
  // mixed mode: one correction of Y against its FP64 residual before T is
  // formed; the residual and the correction reuse the factors' memory
  const bool yref = H.mixed && H.opt.leaf_refine > 0;
  G.ys = (int64_t)ni * nrhs_leaf;
  G.Y->alloc((size_t)nl * G.ys * sizeof(R), st);
  PoolBuf Aii, piv;
  Aii.alloc((size_t)nl * std::max<int64_t>((int64_t)ni * ni, yref ? 2LL * ni * nq : 0) *
                sizeof(R),
            st);
  piv.alloc((size_t)nl * ni * sizeof(int), st);
  const double2* hsc = H.hsc.as<double2>();
  leaf_assemble<R>(G.coefp, G.l0, nl, G.p, G.q, hsc, G.dD->as<double>(), G.dPg2c->as<double>(),
                   Aii.as<R>(), G.Y->as<R>(), G.ys, (H.mixed && !gj) ? 1 : 0, st);
  ck(cudaGetLastError());
  std::vector<LuDesc<R>> ld(nl);
  for (int j = 0; j < nl; ++j) {
    ld[j].A = Aii.as<R>() + (size_t)j * ni * ni;
    ld[j].ipiv = piv.as<int>() + (size_t)j * ni;
    ld[j].B = G.Y->as<R>() + (size_t)j * G.ys;
    ld[j].m = ni;
    ld[j].lda = ni;
    ld[j].nrhs = nrhs_leaf;
    ld[j].ldb = ni;
    ld[j].box = pl.leaf_box[G.l0 + j];
  }
  LuDesc<R>* dl = stg.push(ld, st);
  if constexpr (std::is_same<R, float>::value) {
    if (gj) {
      // A_ii^{-1} into Y's last ni columns (the right-hand sides -A_ie L1 moved
      // into A_ii's memory), then Y = A_ii^{-1} (-A_ie L1)
      if (!leaf_gj_inverse(dl, nl, ni, nq, H.status.as<int>(), st))
        throw CudaError{cudaErrorInvalidValue};
      std::vector<GemmDesc<float>> gy(nl);
      for (int j = 0; j < nl; ++j) {
        gy[j].A = G.Y->as<float>() + (size_t)j * G.ys + (size_t)ni * nq;
        gy[j].B = Aii.as<float>() + (size_t)j * ni * ni;
        gy[j].C = G.Y->as<float>() + (size_t)j * G.ys;
        gy[j].M = ni;
        gy[j].N = nq;
        gy[j].K = ni;
        gy[j].lda = ni;
        gy[j].ldb = ni;
        gy[j].ldc = ni;
      }
      GemmDesc<float>* dgy = stg.push(gy, st);
      gemm_batched<float>(dgy, nl, ni, nq, 1.0f, 0.0f, st, "gemm_leafy<f32>",
                          2.0 * nl * (double)ni * ni * nq,
                          (double)nl * ni * (ni + 2.0 * nq) * sizeof(float), ni, nullptr, 0,
                          H.status.as<int>());
    }
  }
  if (!gj)
    lu_solve_batched<R>(dl, nl, ni, nrhs_leaf, kLuFactor, H.status.as<int>(), st, nullptr,
                        nullptr);
  ck(cudaGetLastError());
  R* dY = nullptr;
  if (yref) {
    // Rl = -A_ie L1 - A_ii Y_l in FP64 (rounded to R), dY_l = A_ii^{-1} Rl.  The
    // low-precision LU leaves Y with an error of about cond(A_ii) units of
    // rounding, which the side derivatives of T amplify; T formed from Y + dY
    // in FP64 carries only the rounding of T itself.
    R* Rb = Aii.as<R>();
    dY = Rb + (size_t)nl * ni * nq;
    if (!leaf_y_residual_tc<R>(G.coefp, G.l0, nl, G.p, G.q, hsc, G.dD->as<double>(),
                               G.dPg2c->as<double>(), G.Y->as<R>(), G.ys, Rb,
                               H.status.as<int>(), st))
      leaf_y_residual<R>(G.coefp, G.l0, nl, G.p, G.q, hsc, G.dD->as<double>(),
                         G.dPg2c->as<double>(), G.Y->as<R>(), G.ys, Rb, st);
    ck(cudaGetLastError());
    std::vector<GemmDesc<R>> gd(nl);
    for (int j = 0; j < nl; ++j) {
      gd[j].A = G.Y->as<R>() + (size_t)j * G.ys + (size_t)ni * nq;  // A_ii^{-1}
      gd[j].B = Rb + (size_t)j * ni * nq;
      gd[j].C = dY + (size_t)j * ni * nq;
      gd[j].M = ni;
      gd[j].N = nq;
      gd[j].K = ni;
      gd[j].lda = ni;
      gd[j].ldb = ni;
      gd[j].ldc = ni;
    }
    GemmDesc<R>* dg = stg.push(gd, st);
    gemm_batched<R>(dg, nl, ni, nq, R(1), R(0), st, "gemm_yref<f32>",
                    2.0 * nl * (double)ni * ni * nq, (double)nl * ni * (ni + 2.0 * nq) * sizeof(R),
                    ni, nullptr, 0, H.status.as<int>());
    ck(cudaGetLastError());
  }
  T0.alloc((size_t)nl * nq * nq * sizeof(R), st);
  leaf_dtn<R>(G.Y->as<R>(), G.ys, G.l0, nl, G.p, G.q, hsc, G.dD->as<double>(),
              G.dPg2c->as<double>(), G.dPc2g->as<double>(), T0.as<R>(), st, dY,
              (int64_t)ni * nq);
  ck(cudaGetLastError());
  for (int j = 0; j < nl; ++j) {
    Tref[pl.leaf_box[G.l0 + j]].p = T0.as<R>() + (size_t)j * nq * nq;
    Tref[pl.leaf_box[G.l0 + j]].f64 = sizeof(R) == 8;
  }
}

template <typename R>
void build_level(hps_handle_s& H, LevelGroup& L, Stager& stg, std::vector<TRef>& Tref,
                 PoolBuf& Tout) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  const int nm = (int)L.boxes.size();
  const bool form_root = H.opt.form_root_dtn != 0;
  int64_t aw_tot = 0, cw_tot = 0, tp_tot = 0, piv_tot = 0, s_tot = 0;
  int64_t max_work = 0;
  std::vector<int64_t> aw_off(nm), piv_off(nm);
  for (int i = 0; i < nm; ++i) {
    const int b = L.boxes[i];
    const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
    const bool tp = pl.boxes[b].parent >= 0 || form_root;
    L.s_off[i] = s_tot;
    aw_off[i] = aw_tot;
    L.cw_off[i] = cw_tot;
    piv_off[i] = piv_tot;
    s_tot += (int64_t)sh.m * (sh.ne + (H.mixed ? sh.m : 0));
    aw_tot += (int64_t)sh.m * sh.m;
    cw_tot += (int64_t)sh.ne * sh.m;
    tp_tot += tp ? (int64_t)sh.ne * sh.ne : 0;
    piv_tot += sh.m;
    // gather work: T33 difference, S block, [T13; T23], diag(T11, T22) and, in
    // mixed mode, the identity block that turns into W
    max_work = std::max<int64_t>(max_work, (int64_t)sh.m * sh.m + 2LL * sh.m * sh.ne +
                                               (tp ? (int64_t)sh.ne * sh.ne : 0) +
                                               (H.mixed ? (int64_t)sh.m * sh.m : 0));
  }
  L.S->alloc((size_t)s_tot * sizeof(R), st);
  PoolBuf Aw, piv, cw_tmp;
  PoolBuf& Cw = H.mixed ? *L.Cw : cw_tmp;
  Aw.alloc((size_t)aw_tot * sizeof(R), st);
  Cw.alloc((size_t)cw_tot * sizeof(R), st);
  piv.alloc((size_t)piv_tot * sizeof(int), st);
  Tout.alloc((size_t)tp_tot * sizeof(R), st);
  std::vector<MergeDesc<R>> md(nm);
  std::vector<LuDesc<R>> lu(nm);
  std::vector<GemmDesc<R>> gm;
  std::vector<int> hn(nm);
  double gather_bytes = 0.0, schur_flops = 0.0, schur_bytes = 0.0;
  int64_t ot = 0;
  // Mixed mode: the LU solves for W = (T33^a - T33^b)^{-1} only (identity
  // right-hand side, 2 m^3 flops instead of 2 m^2 ne) and S = W [-T31^a |
  // T32^b] is one product: on the tensor cores for FP64 merges large enough,
  // by the FP32 tile GEMM for FP32 merges.  An explicit inverse is not
  // backward stable (its residual can be cond times that of the
  // substitution); the refinement absorbs that, so FP64 mode keeps the
  // substitution.  [-T31^a | T32^b] is gathered into a temporary.  The choice
  // depends on the merge's own shape.
  const bool w_first = H.mixed;
  std::vector<OzDesc> sw;
  std::vector<GemmDesc<R>> swf;  // FP32: S = W [-T31^a | T32^b] by the tile GEMM
  double swf_flops = 0.0, swf_bytes = 0.0;
  int swf_m = 0, swf_n = 0;
  int64_t tmp_tot = 0;
  std::vector<int64_t> tmp_off(nm, -1);
  for (int i = 0; i < nm && w_first; ++i) {
    const MergeShape& sh = pl.shapes[pl.boxes[L.boxes[i]].shape];
    if (sizeof(R) == 8 ? oz_eligible(sh.m, sh.ne, sh.m) : sh.m >= kNBw) {
      tmp_off[i] = tmp_tot;
      tmp_tot += (int64_t)sh.m * sh.ne;
    }
  }
  PoolBuf Btmp;
  Btmp.alloc((size_t)tmp_tot * sizeof(R), st);
  for (int i = 0; i < nm; ++i) {
    const int b = L.boxes[i];
    const Box& B = pl.boxes[b];
    const MergeShape& sh = pl.shapes[B.shape];
    const bool tp = B.parent >= 0 || form_root;
    MergeDesc<R>& g = md[i];
    g.Ta = Tref[B.child[0]].p;
    g.ta64 = Tref[B.child[0]].f64;
    g.Tb = Tref[B.child[1]].p;
    g.tb64 = Tref[B.child[1]].f64;
    R* const S_final = L.S->as<R>() + L.s_off[i];
    const bool wf = tmp_off[i] >= 0;
    g.Aw = Aw.as<R>() + aw_off[i];
    g.S = wf ? Btmp.as<R>() + tmp_off[i] : S_final;
    g.Cw = Cw.as<R>() + L.cw_off[i];
    g.Tp = tp ? Tout.as<R>() + ot : nullptr;
    g.W = H.mixed ? S_final + (int64_t)sh.m * sh.ne : nullptr;
    g.src = H.maps.as<int>() + H.src_off[B.shape];
    g.na = sh.na;
    g.nb = sh.nb;
    g.m = sh.m;
    g.ne = sh.ne;
    g.j3a = sh.j3a;
    g.j3b = sh.j3b;
    lu[i].A = g.Aw;
    lu[i].ipiv = piv.as<int>() + piv_off[i];
    lu[i].B = wf ? g.W : g.S;
    lu[i].m = sh.m;
    lu[i].lda = sh.m;
    lu[i].nrhs = wf ? sh.m : sh.ne + (H.mixed ? sh.m : 0);
    lu[i].ldb = sh.m;
    lu[i].box = b;
    hn[i] = lu[i].nrhs;
    if (wf && sizeof(R) == 8) {
      OzDesc o;
      o.A = reinterpret_cast<const double*>(g.W);
      o.B = reinterpret_cast<const double*>(g.S);
      o.C = reinterpret_cast<double*>(S_final);
      o.M = sh.m;
      o.N = sh.ne;
      o.K = sh.m;
      o.lda = sh.m;
      o.ldb = sh.m;
      o.ldc = sh.m;
      sw.push_back(o);
    } else if (wf) {
      GemmDesc<R> q;
      q.A = g.W;
      q.B = g.S;
      q.C = S_final;
      q.M = sh.m;
      q.N = sh.ne;
      q.K = sh.m;
      q.lda = sh.m;
      q.ldb = sh.m;
      q.ldc = sh.m;
      swf.push_back(q);
      swf_flops += 2.0 * sh.m * (double)sh.m * sh.ne;
      swf_bytes += sizeof(R) * ((double)sh.m * sh.m + 2.0 * sh.m * (double)sh.ne);
      swf_m = std::max(swf_m, sh.m);
      swf_n = std::max(swf_n, sh.ne);
    }
    gather_bytes += (sizeof(R) + 8.0) *
                    ((double)sh.m * sh.m + 2.0 * sh.m * sh.ne + (tp ? (double)sh.ne * sh.ne : 0.0));
    if (tp) {
      GemmDesc<R> gg;
      gg.A = g.Cw;
      gg.B = S_final;
      gg.C = g.Tp;
      gg.M = sh.ne;
      gg.N = sh.ne;
      gg.K = sh.m;
      gg.lda = sh.ne;
      gg.ldb = sh.m;
      gg.ldc = sh.ne;
      gm.push_back(gg);
      schur_flops += 2.0 * sh.ne * (double)sh.ne * sh.m;
      schur_bytes += sizeof(R) * (2.0 * sh.ne * (double)sh.m + 2.0 * sh.ne * (double)sh.ne);
      Tref[b].p = g.Tp;
      Tref[b].f64 = sizeof(R) == 8;
      ot += (int64_t)sh.ne * sh.ne;
    }
  }
  MergeDesc<R>* dmd = stg.push(md, st);
  merge_gather<R>(dmd, nm, max_work, st, gather_bytes);
  ck(cudaGetLastError());
  // FP64 systems large enough take the two-level LU (its rank-256 updates on
  // the tensor cores), the rest the one-level LU; the choice depends on each
  // system's own size
  std::vector<LuDesc<R>> lu1;
  std::vector<int> hm1, hn1;
  std::vector<LuDesc<double>> lu2;
  std::vector<LuDescHost> lh2;
  for (int i = 0; i < nm; ++i) {
    if (sizeof(R) == 8 && lu_tc_eligible(lu[i].m)) {
      LuDesc<double> d2;
      std::memcpy(&d2, &lu[i], sizeof(d2));
      lu2.push_back(d2);
      lh2.push_back({reinterpret_cast<double*>(lu[i].A), reinterpret_cast<double*>(lu[i].B),
                     lu[i].m, lu[i].lda, lu[i].nrhs, lu[i].ldb});
    } else {
      lu1.push_back(lu[i]);
      hm1.push_back(lu[i].m);
      hn1.push_back(hn[i]);
    }
  }
  if (!lu1.empty()) {
    LuDesc<R>* dlu = stg.push(lu1, st);
    lu_solve_batched<R>(dlu, (int)lu1.size(), *std::max_element(hm1.begin(), hm1.end()),
                        *std::max_element(hn1.begin(), hn1.end()), kLuFactor, H.status.as<int>(),
                        st, hm1.data(), hn1.data());
    ck(cudaGetLastError());
  }
  if (!lu2.empty()) {
    LuDesc<double>* dlu = stg.push(lu2, st);
    const size_t wb = lu_tc_workspace(lh2);
    PoolBuf lw;
    lw.alloc(wb, st);
    StagerCtx sctx{&stg, st};
    ck(lu_solve_tc(dlu, lh2, H.status.as<int>(), st, &StagerCtx::push, &sctx, lw.p, wb));
  }
  if (!sw.empty()) {  // S = W [-T31^a | T32^b] on the tensor cores
    const size_t wb = oz_plan(sw);
    PoolBuf ow;
    ow.alloc(wb, st);
    OzDesc* dz = stg.push(sw, st);
    ck(oz_gemm(dz, sw, ow.p, wb, 1.0, 0.0, H.status.as<int>(), st, "gemm_s_tc<f64>"));
  }
  if (!swf.empty()) {  // S = W [-T31^a | T32^b], FP32
    GemmDesc<R>* dg = stg.push(swf, st);
    gemm_batched<R>(dg, (int)swf.size(), swf_m, swf_n, R(1), R(0), st, "gemm_s<f32>", swf_flops,
                    swf_bytes, swf_m, nullptr, 0, H.status.as<int>());
    ck(cudaGetLastError());
  }
  // FP64 products large enough go to the tensor cores (exact BF16 splitting);
  // the choice depends on each product's own shape only
  std::vector<GemmDesc<R>> gsimt;
  std::vector<OzDesc> goz;
  for (const auto& gg : gm) {
    if (sizeof(R) == 8 && oz_eligible(gg.M, gg.N, gg.K)) {
      OzDesc o;
      o.A = reinterpret_cast<const double*>(gg.A);
      o.B = reinterpret_cast<const double*>(gg.B);
      o.C = reinterpret_cast<double*>(gg.C);
      o.M = gg.M;
      o.N = gg.N;
      o.K = gg.K;
      o.lda = gg.lda;
      o.ldb = gg.ldb;
      o.ldc = gg.ldc;
      goz.push_back(o);
    } else {
      gsimt.push_back(gg);
    }
  }
  if (!gsimt.empty()) {
    double fl = 0, by = 0;
    int mx = 0, mk = 0;
    for (const auto& gg : gsimt) {
      fl += 2.0 * gg.M * (double)gg.N * gg.K;
      by += sizeof(R) * (2.0 * gg.M * (double)gg.K + 2.0 * gg.M * (double)gg.N);
      mx = std::max(mx, std::max(gg.M, gg.N));
      mk = std::max(mk, gg.K);
    }
    GemmDesc<R>* dg = stg.push(gsimt, st);
    gemm_batched<R>(dg, (int)gsimt.size(), mx, mx, R(1), R(1), st,
                    sizeof(R) == 8 ? "gemm_schur<f64>" : "gemm_schur<f32>", fl, by, mk, nullptr,
                    0, H.status.as<int>());
    ck(cudaGetLastError());
  }
  if (!goz.empty()) {
    const size_t wb = oz_plan(goz);
    PoolBuf ow;
    ow.alloc(wb, st);
    OzDesc* dz = stg.push(goz, st);
    ck(oz_gemm(dz, goz, ow.p, wb, 1.0, 1.0, H.status.as<int>(), st, "gemm_schur_tc<f64>"));
  }
  (void)schur_flops;
  (void)schur_bytes;
}

void build_all(hps_handle_s& H, const std::vector<const double*>& coef_in, bool dev_ptrs) {
  Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  const int nl_tot = pl.n_leaves();
  const int top = std::max(0, H.opt.fp64_top_levels);
  // ---- leaf groups: consecutive problems with one (p, q)
  H.lg.clear();
  for (int k = 0; k < H.nprob; ++k) {
    const ProblemSpec& s = pl.probs[k].s;
    if (H.lg.empty() || H.lg.back().p != s.p || H.lg.back().q != s.q) {
      H.lg.emplace_back();
      LeafGroup& G = H.lg.back();
      G.l0 = pl.probs[k].leaf0;
      G.p = s.p;
      G.q = s.q;
      G.ni = (s.p - 2) * (s.p - 2);
      G.nq = 4 * s.q;
    }
    H.lg.back().nl += pl.probs[k].nl;
  }
  // ---- level groups: (height, precision), in increasing height
  H.lev.clear();
  for (int h = 1; h <= pl.height; ++h) {
    for (int f64 : {0, 1}) {
      std::vector<int> bx;
      for (int b : pl.levels[h]) {
        const int prob_h = pl.probs[pl.boxes[b].prob].height;
        const int want = H.mixed ? (h > prob_h - top ? 1 : 0) : 1;
        if (want == f64) bx.push_back(b);
      }
      if (bx.empty()) continue;
      H.lev.emplace_back();
      LevelGroup& L = H.lev.back();
      L.h = h;
      L.f64 = f64;
      L.boxes = bx;
      const int nm = (int)bx.size();
      L.s_off.assign(nm, 0);
      L.cw_off.assign(nm, 0);
      L.z_off.assign(nm, 0);
      L.hm.assign(nm, 0);
      L.hne.assign(nm, 0);
      int64_t zrows = 0;
      for (int i = 0; i < nm; ++i) {
        const MergeShape& sh = pl.shapes[pl.boxes[bx[i]].shape];
        L.max_m = std::max(L.max_m, sh.m);
        L.max_ne = std::max(L.max_ne, sh.ne);
        L.max_nanb = std::max(L.max_nanb, sh.na + sh.nb);
        L.hm[i] = sh.m;
        L.hne[i] = sh.ne;
        L.z_off[i] = zrows;
        zrows += sh.m;
      }
      L.sum_m = zrows;
    }
  }
  H.u3_off.assign(pl.boxes.size(), -1);
  H.u3_total = 0;
  for (auto& L : H.lev)
    for (int b : L.boxes) {
      H.u3_off[b] = H.u3_total;
      H.u3_total += pl.shapes[pl.boxes[b].shape].m;
    }
  // descriptor staging (upper bound of every array pushed below)
  const size_t nb = pl.boxes.size();
  Stager stg;
  size_t bytes = 8 * 256 + stage_bytes<LuDesc<double>>(nl_tot) +
                 stage_bytes<GemmDesc<double>>(nl_tot) + 512 * H.lg.size();
  for (auto& L : H.lev) {
    bytes += stage_bytes<MergeDesc<double>>(L.boxes.size()) +
             2 * stage_bytes<LuDesc<double>>(L.boxes.size()) +
             stage_bytes<GemmDesc<double>>(L.boxes.size()) +
             2 * stage_bytes<OzDesc>(L.boxes.size());
    // two-level LU: per outer block, at most four arrays of two products per system
    if (L.f64 && lu_tc_eligible(L.max_m))
      bytes += (size_t)((L.max_m + kLuOuter - 1) / kLuOuter) * 4 *
               stage_bytes<OzDesc>(2 * L.boxes.size());
  }
  stg.begin(bytes, st);
  H.keep.begin(stage_bytes<SolveScatterDesc>(nb) + stage_bytes<BodyDesc>(nb) +
                   4 * 256 * (H.lev.size() + 2),
               st);
  // constants, maps, per-leaf data, status (pageable uploads: synchronised below)
  auto up = [&](PoolBuf& b, const void* src, size_t n) {
    b.alloc(n, st);
    if (n) ck(cudaMemcpyAsync(b.p, src, n, cudaMemcpyHostToDevice, st));
  };
  for (auto& G : H.lg) {
    G.consts = make_consts(G.p, G.q);
    {  // [D | D^2]: the leaf kernels read D^2 at D + p*p
      std::vector<double> dd(G.consts.D);
      dd.insert(dd.end(), G.consts.D2.begin(), G.consts.D2.end());
      up(*G.dD, dd.data(), dd.size() * sizeof(double));
      ck(cudaStreamSynchronize(st));  // the pageable source goes out of scope
    }
    up(*G.dPg2c, G.consts.Pg2c.data(), G.consts.Pg2c.size() * sizeof(double));
    up(*G.dPc2g, G.consts.Pc2g.data(), G.consts.Pc2g.size() * sizeof(double));
  }
  {
    std::vector<int> all;
    for (const auto& s : pl.shapes) {
      H.src_off.push_back((int64_t)all.size());
      all.insert(all.end(), s.src.begin(), s.src.end());
      H.cma_off.push_back((int64_t)all.size());
      all.insert(all.end(), s.cmap_a.begin(), s.cmap_a.end());
      H.cmb_off.push_back((int64_t)all.size());
      all.insert(all.end(), s.cmap_b.begin(), s.cmap_b.end());
    }
    up(H.maps, all.data(), all.size() * sizeof(int));
    up(H.root_from_f, pl.root_from_f.data(), pl.root_from_f.size() * sizeof(int));
    std::vector<int64_t> lo(nl_tot);
    std::vector<double2> hs(nl_tot);
    for (int l = 0; l < nl_tot; ++l) {
      lo[l] = pl.boxes[pl.leaf_box[l]].ext_off;
      const ProbInfo& pi = pl.probs[pl.leaf_prob[l]];
      hs[l] = make_double2(2.0 / pi.hx, 2.0 / pi.hy);
    }
    up(H.leaf_off, lo.data(), lo.size() * sizeof(int64_t));
    up(H.hsc, hs.data(), hs.size() * sizeof(double2));
    ck(cudaStreamSynchronize(st));  // the pageable sources above go out of scope
  }
  H.status.alloc(sizeof(int), st);
  ck(cudaMemsetAsync(H.status.p, 0, sizeof(int), st));
  // ---- coefficients: one device copy laid out group by group (kept in mixed
  // mode for the FP64 residual); a coefficient absent from a problem is zero
  // there, and absent from a whole group is skipped by the kernels
  {
    size_t elems = 0;
    std::vector<std::array<int64_t, 6>> goff(H.lg.size());
    for (size_t g = 0; g < H.lg.size(); ++g) {
      LeafGroup& G = H.lg[g];
      for (int c = 0; c < 6; ++c) {
        bool any = false;
        for (int k = 0; k < H.nprob; ++k)
          if (pl.probs[k].leaf0 >= G.l0 && pl.probs[k].leaf0 < G.l0 + G.nl && coef_in[6 * k + c])
            any = true;
        goff[g][c] = any ? (int64_t)elems : -1;
        if (any) elems += (size_t)G.nl * G.p * G.p;
      }
    }
    H.coef.alloc(elems * sizeof(double), st);
    for (size_t g = 0; g < H.lg.size(); ++g) {
      LeafGroup& G = H.lg[g];
      const int pp = G.p * G.p;
      for (int c = 0; c < 6; ++c) {
        if (goff[g][c] < 0) {
          G.coefp[c] = nullptr;
          continue;
        }
        double* base = H.coef.as<double>() + goff[g][c];
        G.coefp[c] = base;
        for (int k = 0; k < H.nprob; ++k) {
          const ProbInfo& pi = pl.probs[k];
          if (pi.leaf0 < G.l0 || pi.leaf0 >= G.l0 + G.nl) continue;
          double* dst = base + (size_t)(pi.leaf0 - G.l0) * pp;
          const size_t n = (size_t)pi.nl * pp * sizeof(double);
          if (coef_in[6 * k + c])
            ck(cudaMemcpyAsync(dst, coef_in[6 * k + c], n,
                               dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
          else
            ck(cudaMemsetAsync(dst, 0, n, st));
        }
      }
    }
  }
  // ---- mixed mode, groups without the mixed term: per problem, the side
  // fluxes of interior values (the refinement's h += F_i z)
  if (H.mixed) {
    for (auto& G : H.lg) {
      if (G.coefp[1]) continue;
      std::vector<float> all;
      G.prob0 = -1;
      for (int k = 0; k < H.nprob; ++k) {
        const ProbInfo& pi = pl.probs[k];
        if (pi.leaf0 < G.l0 || pi.leaf0 >= G.l0 + G.nl) continue;
        if (G.prob0 < 0) G.prob0 = k;
        const std::vector<float> f = interior_flux_map(G.consts, 2.0 / pi.hx, 2.0 / pi.hy);
        all.insert(all.end(), f.begin(), f.end());
      }
      G.Fi->alloc(all.size() * sizeof(float), st);
      ck(cudaMemcpyAsync(G.Fi->p, all.data(), all.size() * sizeof(float),
                         cudaMemcpyHostToDevice, st));
      ck(cudaStreamSynchronize(st));  // the pageable source goes out of scope
    }
  }
  // ---- leaves and merges
  std::vector<TRef> Tref(pl.boxes.size());
  std::vector<PoolPtr> Tleaf;
  for (auto& G : H.lg) {
    Tleaf.push_back(new_buf());
    if (H.mixed)
      build_leaves<float>(H, G, stg, Tref, *Tleaf.back());
    else
      build_leaves<double>(H, G, stg, Tref, *Tleaf.back());
  }
  // T buffers per level group, released after the last level group reading them
  std::vector<PoolPtr> Tlev;
  for (size_t i = 0; i < H.lev.size(); ++i) Tlev.push_back(new_buf());
  std::vector<int> box_group(pl.boxes.size(), -1);  // level group producing each box's T
  for (size_t i = 0; i < H.lev.size(); ++i)
    for (int b : H.lev[i].boxes) box_group[b] = (int)i;
  std::vector<int> last_use_leaf(H.lg.size(), -1), last_use(H.lev.size(), -1);
  for (size_t i = 0; i < H.lev.size(); ++i)
    for (int b : H.lev[i].boxes)
      for (int c : pl.boxes[b].child) {
        if (pl.boxes[c].leaf >= 0) {
          for (size_t g = 0; g < H.lg.size(); ++g)
            if (pl.boxes[c].leaf >= H.lg[g].l0 && pl.boxes[c].leaf < H.lg[g].l0 + H.lg[g].nl)
              last_use_leaf[g] = (int)i;
        } else {
          last_use[box_group[c]] = std::max(last_use[box_group[c]], (int)i);
        }
      }
  for (size_t i = 0; i < H.lev.size(); ++i) {
    if (H.lev[i].f64)
      build_level<double>(H, H.lev[i], stg, Tref, *Tlev[i]);
    else
      build_level<float>(H, H.lev[i], stg, Tref, *Tlev[i]);
    for (size_t g = 0; g < H.lg.size(); ++g)
      if (last_use_leaf[g] == (int)i) Tleaf[g]->release();
    for (size_t j = 0; j < i; ++j)
      if (last_use[j] == (int)i) Tlev[j]->release();
  }
  // ---- mixed mode: the heights factored in FP64 (the ill-conditioned top
  // interface systems) keep FP32 copies of S, W and [T13; T23] for the solve.
  // Their factorisation and the T they passed up were formed in FP64; the
  // solve only needs a correction accurate to a few digits, which the
  // refinement then removes, so rounding the stored operators costs no
  // accuracy and halves their bytes and the solve's FP64 work.
  if (H.mixed) {
    for (auto& L : H.lev) {
      if (!L.f64) continue;
      auto demote = [&](PoolPtr& b) {
        const int64_t n = (int64_t)(b->bytes / sizeof(double));
        PoolPtr d = new_buf();
        d->alloc((size_t)n * sizeof(float), st);
        f64_to_f32(b->as<double>(), d->as<float>(), n, st);
        b = std::move(d);  // the FP64 copy is released in stream order
      };
      demote(L.S);
      demote(L.Cw);
      L.f64 = 0;
      L.built_f64 = 1;
    }
  }
  // ---- solve-side structures that do not depend on nrhs
  for (auto& L : H.lev) {
    std::vector<SolveScatterDesc> sd;
    std::vector<BodyDesc> bd;
    for (size_t i = 0; i < L.boxes.size(); ++i) {
      const int b = L.boxes[i];
      const Box& B = pl.boxes[b];
      const MergeShape& sh = pl.shapes[B.shape];
      SolveScatterDesc s;
      s.par_off = B.ext_off;
      s.a_off = pl.boxes[B.child[0]].ext_off;
      s.b_off = pl.boxes[B.child[1]].ext_off;
      s.cmap_a = H.maps.as<int>() + H.cma_off[B.shape];
      s.cmap_b = H.maps.as<int>() + H.cmb_off[B.shape];
      s.u3_off = H.u3_off[b];
      s.na = sh.na;
      s.nb = sh.nb;
      s.m = sh.m;
      sd.push_back(s);
      BodyDesc y;
      y.par_off = B.ext_off;
      y.a_off = s.a_off;
      y.b_off = s.b_off;
      y.u3_off = H.u3_off[b];
      y.z_off = L.z_off[i];
      y.src = H.maps.as<int>() + H.src_off[B.shape];
      y.j3a = sh.j3a;
      y.j3b = sh.j3b;
      y.m = sh.m;
      y.ne = sh.ne;
      bd.push_back(y);
    }
    L.scatter = H.keep.push(sd, st);
    L.body = H.keep.push(bd, st);
  }
  // form_root_dtn, single-problem handles (the only ones hps_apply_dtn takes;
  // in a batch a one-leaf problem's T may share a buffer released above): keep
  // the root DtN, in FP64
  if (H.opt.form_root_dtn && H.nprob == 1) {
    int64_t tot = 0;
    H.root_dtn_off.assign(H.nprob, 0);
    for (int k = 0; k < H.nprob; ++k) {
      H.root_dtn_off[k] = tot;
      tot += (int64_t)pl.probs[k].nbnd * pl.probs[k].nbnd;
    }
    H.root_dtn.alloc((size_t)tot * sizeof(double), st);
    for (int k = 0; k < H.nprob; ++k) {
      const TRef& t = Tref[pl.probs[k].root];
      const int64_t n2 = (int64_t)pl.probs[k].nbnd * pl.probs[k].nbnd;
      double* dst = H.root_dtn.as<double>() + H.root_dtn_off[k];
      if (t.f64)
        ck(cudaMemcpyAsync(dst, t.p, (size_t)n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      else
        f32_to_f64(static_cast<const float*>(t.p), dst, n2, st);
    }
  }
  if (!H.mixed) H.coef.release();  // only the residual of mixed mode reads it later
  int* bad_h = nullptr;
  ck(cudaMallocHost(&bad_h, sizeof(int)));
  *bad_h = 0;
  cudaError_t e1 = cudaMemcpyAsync(bad_h, H.status.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  int bad = *bad_h;
  cudaFreeHost(bad_h);
  ck(e1);
  ck(e2);
  Tleaf.clear();
  Tlev.clear();
  if (bad < 0) {
    g_last_error = "tensor-core GEMM: a wait for an asynchronous copy or MMA gave up";
    throw CudaError{cudaErrorLaunchTimeout};
  }
  if (bad) throw bad;
}

// ------------------------------------------------------------------ solve
template <typename R>
void push_down_gemms(hps_handle_s& H, LevelGroup& L, int nrhs) {
  const Plan& pl = H.plan;
  std::vector<GemmDesc<R, double, double>> all;
  double fl = 0, by = 0;
  for (size_t i = 0; i < L.boxes.size(); ++i) {
    const int b = L.boxes[i];
    const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
    GemmDesc<R, double, double> g;
    g.A = L.S->as<R>() + L.s_off[i];
    g.B = H.uext.as<double>() + pl.boxes[b].ext_off;
    g.C = H.u3.as<double>() + H.u3_off[b];
    g.M = sh.m;
    g.N = nrhs;
    g.K = sh.ne;
    g.lda = sh.m;
    g.ldb = (int)pl.ext_total;
    g.ldc = (int)H.u3_total;
    all.push_back(g);
    fl += 2.0 * sh.m * (double)sh.ne;
    by += sizeof(R) * (double)sh.m * sh.ne;
  }
  L.gemm_down = H.solve_st.push(all, H.stream);
  L.down_flops1 = fl;
  L.down_bytes = by;
}

template <typename R>
void push_body(hps_handle_s& H, LevelGroup& L, int nrhs) {
  const Plan& pl = H.plan;
  std::vector<GemmDesc<R, R, double>> gh;
  std::vector<GemmDesc<R>> gw;
  R* z = L.zlev->as<R>();
  R* r = L.rlev->as<R>();
  for (size_t i = 0; i < L.boxes.size(); ++i) {
    const int b = L.boxes[i];
    const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
    GemmDesc<R> w;  // z = W (h3^b - h3^a), W = (T33^a - T33^b)^{-1}
    w.A = L.S->as<R>() + L.s_off[i] + (int64_t)sh.m * sh.ne;
    w.B = r + L.z_off[i] * nrhs;
    w.C = z + L.z_off[i] * nrhs;
    w.M = sh.m;
    w.N = nrhs;
    w.K = sh.m;
    w.lda = sh.m;
    w.ldb = sh.m;
    w.ldc = sh.m;
    gw.push_back(w);
    if (pl.boxes[b].parent < 0) continue;  // a root's flux offsets are never read
    GemmDesc<R, R, double> g;  // h^tau += [T13^a; T23^b] z
    g.A = L.Cw->as<R>() + L.cw_off[i];
    g.B = z + L.z_off[i] * nrhs;
    g.C = H.hpool.as<double>() + pl.boxes[b].ext_off;
    g.M = sh.ne;
    g.N = nrhs;
    g.K = sh.m;
    g.lda = sh.ne;
    g.ldb = sh.m;
    g.ldc = (int)pl.ext_total;
    gh.push_back(g);
  }
  L.gemm_w = H.solve_st.push(gw, H.stream);
  L.gemm_hpar = H.solve_st.push(gh, H.stream);
  L.n_hpar = (int)gh.size();
}

template <typename R>
void push_leaf_inverse(hps_handle_s& H, LeafGroup& G, int nrhs) {
  std::vector<GemmDesc<R>> g(G.nl);
  const int ni = G.ni;
  if (G.Fi->p) {  // h_l += F_i z_l: the flux offsets of the interior corrections
    const Plan& pl = H.plan;
    std::vector<GemmDesc<R, R, double>> f(G.nl);
    for (int j = 0; j < G.nl; ++j) {
      const int l = G.l0 + j;
      f[j].A = G.Fi->as<R>() + (size_t)(pl.leaf_prob[l] - G.prob0) * G.nq * ni;
      f[j].B = G.zleaf->as<R>() + (size_t)j * ni * nrhs;
      f[j].C = H.hpool.as<double>() + pl.boxes[pl.leaf_box[l]].ext_off;
      f[j].M = G.nq;
      f[j].N = nrhs;
      f[j].K = ni;
      f[j].lda = G.nq;
      f[j].ldb = ni;
      f[j].ldc = (int)pl.ext_total;
    }
    G.gemm_fz = H.solve_st.push(f, H.stream);
  }
  for (int j = 0; j < G.nl; ++j) {  // z_l = A_ii^{-1} r_l
    g[j].A = G.Y->as<R>() + (size_t)j * G.ys + (size_t)ni * G.nq;
    g[j].B = G.rleaf->as<R>() + (size_t)j * ni * nrhs;
    g[j].C = G.zleaf->as<R>() + (size_t)j * ni * nrhs;
    g[j].M = ni;
    g[j].N = nrhs;
    g[j].K = ni;
    g[j].lda = ni;
    g[j].ldb = ni;
    g[j].ldc = ni;
  }
  G.gemm_leaf = H.solve_st.push(g, H.stream);
}

void prepare_solve(hps_handle_s& H, int nrhs) {
  if (H.cache_nrhs == nrhs) return;
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  H.cache_nrhs = 0;
  H.uext.alloc((size_t)nrhs * pl.ext_total * sizeof(double), st);
  H.u3.alloc((size_t)nrhs * std::max<int64_t>(H.u3_total, 1) * sizeof(double), st);
  // split-K scratch: the largest need of any solve-phase GEMM
  size_t ws = 0;
  for (auto& L : H.lev) {
    const size_t es = L.f64 ? 8 : 4;
    const int nm = (int)L.boxes.size();
    ws = std::max(ws, es * split_ws_elems(nm, L.max_m, nrhs, L.max_ne));
    if (H.mixed) {
      ws = std::max(ws, es * split_ws_elems(nm, L.max_m, nrhs, L.max_m));
      ws = std::max(ws, es * split_ws_elems(nm, L.max_ne, nrhs, L.max_m));
    }
  }
  H.split_ws.alloc(ws, st);
  size_t bytes = 4 * 256 * (H.lev.size() + H.lg.size() + 2);
  for (auto& G : H.lg) bytes += 2 * stage_bytes<GemmDesc<double>>(G.nl);
  for (auto& L : H.lev) bytes += 3 * stage_bytes<GemmDesc<double>>(L.boxes.size());
  H.solve_st.begin(bytes, st);
  if (H.mixed) {
    H.hpool.alloc((size_t)nrhs * pl.ext_total * sizeof(double), st);
    for (auto& G : H.lg) {
      G.rleaf->alloc((size_t)G.nl * G.ni * nrhs * sizeof(float), st);
      G.zleaf->alloc((size_t)G.nl * G.ni * nrhs * sizeof(float), st);
      push_leaf_inverse<float>(H, G, nrhs);
    }
    for (auto& L : H.lev) {
      const size_t n = (size_t)L.sum_m * nrhs * (L.f64 ? 8 : 4);
      L.rlev->alloc(n, st);
      L.zlev->alloc(n, st);
    }
  }
  for (auto& L : H.lev) {
    if (L.f64) {
      push_down_gemms<double>(H, L, nrhs);
      if (H.mixed) push_body<double>(H, L, nrhs);
    } else {
      push_down_gemms<float>(H, L, nrhs);
      if (H.mixed) push_body<float>(H, L, nrhs);
    }
  }
  H.cache_nrhs = nrhs;
}

template <typename R>
R* split_ws(hps_handle_s& H, size_t* elems) {
  *elems = H.split_ws.bytes / sizeof(R);
  return H.split_ws.as<R>();
}

// Downward pass (Algorithm 2) of one level group from the exterior values
// already in uext; with_z adds the body-load interface values z of each merge.
template <typename R>
void down_level(hps_handle_s& H, LevelGroup& L, int nrhs, bool with_z) {
  cudaStream_t st = H.stream;
  const int nm = (int)L.boxes.size();
  if (with_z)
    z_to_u3<R>(L.body, nm, L.max_m, L.zlev->as<R>(), H.u3.as<double>(), H.u3_total, nrhs, st);
  size_t wse = 0;
  R* ws = split_ws<R>(H, &wse);
  gemm_batched<R>(static_cast<GemmDesc<R, double, double>*>(L.gemm_down), nm, L.max_m, nrhs, R(1),
                  with_z ? R(1) : R(0), st, sizeof(R) == 8 ? "gemm_solve<f64>" : "gemm_solve<f32>",
                  L.down_flops1 * nrhs, L.down_bytes, L.max_ne, ws, wse, H.status.as<int>());
  solve_child_scatter(L.scatter, nm, L.max_nanb, H.u3.as<double>(), H.u3_total,
                      H.uext.as<double>(), H.plan.ext_total, nrhs, st);
}

void downward(hps_handle_s& H, int nrhs, bool with_z) {
  for (int i = (int)H.lev.size() - 1; i >= 0; --i) {
    if (H.lev[i].f64)
      down_level<double>(H, H.lev[i], nrhs, with_z);
    else
      down_level<float>(H, H.lev[i], nrhs, with_z);
  }
}

struct CallPtrs {           // per solve call: where f comes from and u goes
  RootDesc* roots = nullptr;
  double* const* wptr = nullptr;  // per leaf: its first node of u (right-hand side 0)
  const int64_t* wrs = nullptr;   // per leaf: stride between right-hand sides
  int max_nbnd = 0;
  // refinement (mixed mode): per leaf pointers into the correction vector F,
  // and the columns (problem, right-hand side) of the accelerated update
  double* const* fptr = nullptr;
  AaCol* cols = nullptr;
  int* col_of = nullptr;  // per reduction chunk: its column
  int ncol = 0;
  int64_t nchunks = 0, nu = 0;
};

// Refinement work vectors of one solve call (pool memory, released with it).
struct RefineBufs {
  PoolBuf F, Fprev, dWlast, dF, G, part, colsum, coef;
};

void leaf_out(hps_handle_s& H, double* const* wptr, const int64_t* wrs, int nrhs,
              bool correction) {
  for (auto& G : H.lg) {
    if (H.mixed) {
      // the FP64 side values on the tensor cores first, into the residual
      // buffer (free here: the leaf correction has consumed it)
      double* bv = G.rleaf->as<double>();
      if (G.rleaf->bytes < (size_t)nrhs * G.nl * 4 * G.p * sizeof(double) ||
          !leaf_bnd_interp_tc(H.uext.as<double>(), H.leaf_off.as<int64_t>(), G.l0, G.nl,
                              H.plan.ext_total, G.p, G.q, nrhs, G.dPg2c->as<double>(), bv,
                              H.status.as<int>(), H.stream))
        bv = nullptr;
      leaf_post<float>(G.Y->as<float>(), G.ys, G.l0, H.uext.as<double>(), H.leaf_off.as<int64_t>(),
                       H.plan.ext_total, G.nl, G.p, G.q, nrhs, G.dPg2c->as<double>(), wptr, wrs,
                       H.stream, correction ? G.zleaf->as<float>() : nullptr, 0, bv);
    } else
      leaf_post<double>(G.Y->as<double>(), G.ys, G.l0, H.uext.as<double>(),
                        H.leaf_off.as<int64_t>(), H.plan.ext_total, G.nl, G.p, G.q, nrhs,
                        G.dPg2c->as<double>(), wptr, wrs, H.stream);
  }
}

// Leaf part of one refinement step: r = -(A w)_i in FP64, z = A_ii^{-1} r, and
// the leaves' flux offsets h = L4 L3 (w + [0; z]).
void leaf_correction_rhs(hps_handle_s& H, const CallPtrs& cp, int nrhs) {
  cudaStream_t st = H.stream;
  for (auto& G : H.lg) {
    if (G.gemm_fz) {
      // no mixed term: r and the fluxes of w in one FP64 pass, z = A_ii^{-1} r,
      // then h += F_i z (FP32 products, FP64 sums)
      if (!leaf_resflux_tc<float>(G.coefp, G.l0, G.nl, G.p, G.q, H.hsc.as<double2>(),
                                  G.dD->as<double>(), G.dPc2g->as<double>(), cp.wptr, cp.wrs,
                                  nrhs, G.rleaf->as<float>(), H.leaf_off.as<int64_t>(),
                                  H.plan.ext_total, H.hpool.as<double>(), H.status.as<int>(), st))
        leaf_resflux<float>(G.coefp, G.l0, G.nl, G.p, G.q, H.hsc.as<double2>(),
                            G.dD->as<double>(), G.dPc2g->as<double>(), cp.wptr, cp.wrs, nrhs,
                            G.rleaf->as<float>(), H.leaf_off.as<int64_t>(), H.plan.ext_total,
                            H.hpool.as<double>(), st);
      gemm_batched<float>(static_cast<GemmDesc<float>*>(G.gemm_leaf), G.nl, G.ni, nrhs, 1.0f,
                          0.0f, st, "gemm_leafinv<f32>", 2.0 * G.nl * (double)G.ni * G.ni * nrhs,
                          (double)G.nl * G.ni * G.ni * sizeof(float), G.ni, nullptr, 0,
                          H.status.as<int>());
      gemm_batched<float>(static_cast<GemmDesc<float, float, double>*>(G.gemm_fz), G.nl, G.nq,
                          nrhs, 1.0f, 1.0f, st, "gemm_fluxz<f32>",
                          2.0 * G.nl * (double)G.nq * G.ni * nrhs,
                          (double)G.nl * nrhs * (G.ni * 4.0 + G.nq * 16.0), G.ni, nullptr, 0,
                          H.status.as<int>());
      continue;
    }
    leaf_residual<float>(G.coefp, G.l0, G.nl, G.p, H.hsc.as<double2>(), G.dD->as<double>(),
                         cp.wptr, cp.wrs, nrhs, G.rleaf->as<float>(), st);
    gemm_batched<float>(static_cast<GemmDesc<float>*>(G.gemm_leaf), G.nl, G.ni, nrhs, 1.0f, 0.0f,
                        st, "gemm_leafinv<f32>", 2.0 * G.nl * (double)G.ni * G.ni * nrhs,
                        (double)G.nl * G.ni * G.ni * sizeof(float), G.ni, nullptr, 0,
                        H.status.as<int>());
    leaf_flux<float>(cp.wptr, cp.wrs, G.zleaf->as<float>(), G.l0, G.nl, G.p, G.q, nrhs,
                     H.hsc.as<double2>(), G.dD->as<double>(), G.dPc2g->as<double>(),
                     H.leaf_off.as<int64_t>(), H.plan.ext_total, H.hpool.as<double>(), st);
  }
}

// Merge part of the upward pass: z = W (h3^b - h3^a), h^tau = [h1^a; h2^b] + C z.
template <typename R>
void up_level(hps_handle_s& H, LevelGroup& L, int nrhs) {
  cudaStream_t st = H.stream;
  const Plan& pl = H.plan;
  const int nm = (int)L.boxes.size();
  size_t wse = 0;
  R* ws = split_ws<R>(H, &wse);
  merge_rhs<R>(L.body, nm, L.max_m, H.hpool.as<double>(), pl.ext_total, nrhs, L.rlev->as<R>(),
               st);
  double flw = 0, flc = 0;
  for (int i = 0; i < nm; ++i) {
    flw += 2.0 * L.hm[i] * (double)L.hm[i] * nrhs;
    if (pl.boxes[L.boxes[i]].parent >= 0) flc += 2.0 * L.hne[i] * (double)L.hm[i] * nrhs;
  }
  gemm_batched<R>(static_cast<GemmDesc<R>*>(L.gemm_w), nm, L.max_m, nrhs, R(1), R(0), st,
                  sizeof(R) == 8 ? "gemm_body<f64>" : "gemm_body<f32>", flw, 0.0, L.max_m, ws,
                  wse, H.status.as<int>());
  // parents' flux offsets: [h1^a; h2^b] copied for every merge (a root's copy
  // is never read and costs little), the product only where a parent reads it
  merge_hpar(L.body, nm, L.max_ne, H.hpool.as<double>(), pl.ext_total, nrhs, st);
  if (L.n_hpar == 0) return;
  gemm_batched<R>(static_cast<GemmDesc<R, R, double>*>(L.gemm_hpar), L.n_hpar, L.max_ne, nrhs, R(1),
                  R(1), st, sizeof(R) == 8 ? "gemm_body<f64>" : "gemm_body<f32>", flc, 0.0,
                  L.max_m, ws, wse, H.status.as<int>());
}

// Least-squares weights of one column: minimise ||F - sum_s g_s dF_s|| over
// the valid history slots through the normal equations (Cholesky); a slot
// whose pivot falls below 1e-12 of the largest diagonal entry is dropped,
// oldest first, and the system is solved again without it.
void anderson_weights(const double* A, const double* bvec, int m, int nslots, int newest,
                      double* g) {
  for (int s = 0; s < kAaMaxDepth; ++s) g[s] = 0.0;
  std::vector<int> use;  // slots, newest first
  for (int k = 0; k < nslots; ++k) use.push_back(((newest - k) % m + m) % m);
  while (!use.empty()) {
    const int n = (int)use.size();
    double L[kAaMaxDepth][kAaMaxDepth] = {};
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) dmax = std::max(dmax, A[use[i] * m + use[i]]);
    bool ok = dmax > 0.0;
    for (int i = 0; i < n && ok; ++i) {
      for (int k = 0; k <= i; ++k) {
        double v = A[use[i] * m + use[k]];
        for (int t = 0; t < k; ++t) v -= L[i][t] * L[k][t];
        if (k == i) {
          if (!(v > 1e-12 * dmax)) {
            ok = false;
            break;
          }
          L[i][i] = std::sqrt(v);
        } else {
          L[i][k] = v / L[k][k];
        }
      }
    }
    if (ok) {
      double y[kAaMaxDepth], x[kAaMaxDepth];
      for (int i = 0; i < n; ++i) {
        double v = bvec[use[i]];
        for (int t = 0; t < i; ++t) v -= L[i][t] * y[t];
        y[i] = v / L[i][i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double v = y[i];
        for (int t = i + 1; t < n; ++t) v -= L[t][i] * x[t];
        x[i] = v / L[i][i];
      }
      for (int i = 0; i < n; ++i) g[use[i]] = x[i];
      return;
    }
    use.pop_back();  // drop the oldest slot
  }
}

// Per column refinement state kept on the host.
struct ColState {
  int mode = 1;          // 1 active, 0 finished
  bool converged = false, failed = false;
  int iters = 0;
  double rel = 0.0, rel1 = 0.0, rel2 = 0.0;  // this and the two previous relative corrections
  std::vector<double> A, b;                    // Gram matrix and right-hand side by slot
};

// The tensor-core kernels of a mixed solve (FP32 products, FP64 residual)
// report a wait that gave up in the status word: read it (synchronises).
void check_tc_status(hps_handle_s& H) {
  int dev_status = 0;
  ck(cudaMemcpyAsync(&dev_status, H.status.p, sizeof(int), cudaMemcpyDeviceToHost, H.stream));
  ck(cudaStreamSynchronize(H.stream));
  if (dev_status < 0) {
    g_last_error = "tensor-core kernel: a wait for the tensor cores gave up";
    throw CudaError{cudaErrorLaunchTimeout};
  }
}

int solve_all(hps_handle_s& H, const CallPtrs& cp, RefineBufs* rb, int nrhs,
              hps_solve_info* info) {
  cudaStream_t st = H.stream;
  solve_root_scatter(cp.roots, H.nprob, cp.max_nbnd, nrhs, H.uext.as<double>(),
                     H.plan.ext_total, st);
  downward(H, nrhs, false);
  leaf_out(H, cp.wptr, cp.wrs, nrhs, false);
  ck(cudaGetLastError());
  if (!H.mixed) return HPS_OK;
  if (H.opt.max_refine == 0) {
    check_tc_status(H);
    return HPS_OK;
  }
  // ---- iterative refinement against the FP64 residual, Anderson-accelerated
  // per column (problem, right-hand side); columns finish independently
  const int m = H.opt.refine_depth;
  const int ncol = cp.ncol;
  std::vector<ColState> cs(ncol);
  for (auto& c : cs) {
    c.A.assign((size_t)std::max(m, 1) * std::max(m, 1), 0.0);
    c.b.assign(std::max(m, 1), 0.0);
  }
  const size_t stride = kAaMaxDepth + 1;
  double* h_sum = H.h_aa;                          // ncol * kAaQ
  double* h_coef = H.h_aa + (size_t)ncol * kAaQ;   // ncol * stride
  int active = ncol;
  for (int j = 0; j < H.opt.max_refine && active > 0; ++j) {
    leaf_correction_rhs(H, cp, nrhs);
    for (auto& L : H.lev) {
      if (L.f64)
        up_level<double>(H, L, nrhs);
      else
        up_level<float>(H, L, nrhs);
    }
    // the correction has zero Dirichlet data on every Gamma (roots from f = null)
    solve_root_scatter(cp.roots + H.nprob, H.nprob, cp.max_nbnd, nrhs, H.uext.as<double>(),
                       H.plan.ext_total, st);
    downward(H, nrhs, true);
    leaf_out(H, cp.fptr, cp.wrs, nrhs, true);  // F_j, the correction at w_j
    const int nslots = m > 0 ? std::min(j, m) : 0;
    const int slot_new = (m > 0 && j >= 1) ? (j - 1) % m : -1;
    aa_reduce(cp.cols, cp.col_of, ncol, cp.nchunks, rb->F.as<double>(),
              m > 0 ? rb->Fprev.as<double>() : nullptr,
              rb->dWlast.as<double>(), rb->dF.as<float>(), rb->G.as<double>(), cp.nu,
              m > 0 ? j : 0, slot_new, nslots, rb->part.as<double>(), rb->colsum.as<double>(), st);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(h_sum, rb->colsum.p, (size_t)ncol * kAaQ * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    for (int c = 0; c < ncol; ++c) {
      ColState& S = cs[c];
      double* cf = h_coef + (size_t)c * stride;
      for (size_t t = 0; t < stride; ++t) cf[t] = 0.0;
      if (S.mode == 0) continue;
      const double* q = h_sum + (size_t)c * kAaQ;
      const double fmax_ = q[0], wmax = q[1];
      S.rel2 = S.rel1;
      S.rel1 = S.rel;
      S.rel = wmax > 0 ? fmax_ / wmax : fmax_;
      S.iters = j + 1;
      if (m > 0 && j >= 1) {
        for (int t = 0; t < nslots; ++t) {
          const double v = q[2 + kAaMaxDepth + t];
          S.A[t * m + slot_new] = v;
          S.A[slot_new * m + t] = v;
        }
      }
      for (int t = 0; t < nslots; ++t) S.b[t] = q[2 + t];
      int mode = 1;
      bool done = false;
      if (!(S.rel <= 1e300) || (j >= 2 && S.rel > 1.0)) {  // NaN, inf or growing corrections
        S.failed = true;
        mode = 0;
        done = true;
      } else if (S.rel <= H.opt.refine_tol) {
        S.converged = true;
        mode = 2;
        done = true;
      } else if (j >= 1 && S.rel < 0.25 * S.rel1 && S.rel * (S.rel / S.rel1) <= H.opt.refine_tol) {
        // the corrections contract by about rel / rel1 per step: after this one
        // is applied, the error (the next correction) is predicted below the
        // tolerance, so it is not computed
        S.converged = true;
        mode = 2;
        done = true;
      } else if (j >= 3 && S.rel > 0.5 * std::min(S.rel1, S.rel2)) {
        // no longer shrinking: the iterate has reached the accuracy the FP64
        // residual resolves for this conditioning
        mode = 2;
        done = true;
      } else if (j == H.opt.max_refine - 1) {
        done = true;
      }
      if (mode == 1 && m > 0 && nslots > 0)
        anderson_weights(S.A.data(), S.b.data(), m, nslots, slot_new, cf + 1);
      if (mode == 1 && m == 0) mode = 2;
      cf[0] = mode;
      if (done) {
        S.mode = 0;
        --active;
      }
    }
    ck(cudaMemcpyAsync(rb->coef.p, h_coef, (size_t)ncol * stride * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    aa_update(cp.cols, cp.col_of, ncol, cp.nchunks, rb->F.as<double>(), rb->dWlast.as<double>(),
              rb->G.as<double>(), cp.nu, nslots, rb->coef.as<double>(), st);
    ck(cudaGetLastError());
  }
  check_tc_status(H);
  int iters = 0;
  double worst = 0.0;
  bool ok = true;
  for (const auto& S : cs) {
    iters = std::max(iters, S.iters);
    worst = (S.rel == S.rel) ? std::max(worst, S.rel) : S.rel;
    if (!S.converged) ok = false;
  }
  if (info) {
    info->iterations = iters;
    info->last_update = worst;
  }
  if (!ok) {
    if (info) info->status = HPS_ENOTCONVERGED;
    return HPS_ENOTCONVERGED;
  }
  return HPS_OK;
}

// Reduction chunks of one solve's refinement columns.
int64_t n_chunks_upper(const hps_handle_s& H, int nrhs) {
  int64_t n = 0;
  for (const auto& pi : H.plan.probs)
    n += (int64_t)nrhs * (((int64_t)pi.nl * pi.s.p * pi.s.p + kAaChunk - 1) / kAaChunk);
  return n;
}

// Upload the per-call root descriptors (with f, then with zeros), the per-leaf
// output pointers and, in mixed mode, the refinement layout.  f[k] / u[k] are
// device pointers.
CallPtrs stage_call(hps_handle_s& H, const double* const* f, double* const* u, int nrhs,
                    RefineBufs* rb) {
  const Plan& pl = H.plan;
  const int nl = pl.n_leaves();
  const bool refine = H.mixed && H.opt.max_refine > 0;
  const int ncol = H.nprob * nrhs;
  H.call_st.begin(stage_bytes<RootDesc>(2 * H.nprob) + 2 * stage_bytes<double*>(nl) +
                      stage_bytes<int64_t>(nl) + (refine ? stage_bytes<AaCol>(ncol) : 0) + 1024 +
                      (refine ? stage_bytes<int>(n_chunks_upper(H, nrhs)) : 0),
                  H.stream);
  std::vector<RootDesc> rd(2 * H.nprob);
  std::vector<double*> wp(nl), fp;
  std::vector<int64_t> wr(nl);
  std::vector<AaCol> cols;
  std::vector<int> col_of;
  CallPtrs cp;
  int64_t nu = 0;  // refinement vector length: every column of every problem
  for (int k = 0; k < H.nprob; ++k) nu += (int64_t)nrhs * pl.probs[k].nl * pl.probs[k].s.p * pl.probs[k].s.p;
  if (refine) {
    const int m = H.opt.refine_depth;
    rb->F.alloc((size_t)nu * sizeof(double), H.stream);
    if (m > 0) {
      rb->Fprev.alloc((size_t)nu * sizeof(double), H.stream);
      rb->dWlast.alloc((size_t)nu * sizeof(double), H.stream);
      rb->dF.alloc((size_t)m * nu * sizeof(float), H.stream);
      rb->G.alloc((size_t)m * nu * sizeof(double), H.stream);
    }
    fp.resize(nl);
  }
  int64_t fo = 0, ch = 0;
  for (int k = 0; k < H.nprob; ++k) {
    const ProbInfo& pi = pl.probs[k];
    RootDesc r;
    r.f = f[k];
    r.rff = H.root_from_f.as<int>() + pi.rff_off;
    r.root_off = pl.boxes[pi.root].ext_off;
    r.nbnd = pi.nbnd;
    rd[k] = r;
    r.f = nullptr;
    rd[H.nprob + k] = r;
    cp.max_nbnd = std::max(cp.max_nbnd, pi.nbnd);
    const int pp = pi.s.p * pi.s.p;
    const int64_t len = (int64_t)pi.nl * pp;
    for (int j = 0; j < pi.nl; ++j) {
      wp[pi.leaf0 + j] = u[k] + (size_t)j * pp;
      wr[pi.leaf0 + j] = len;
      if (refine) fp[pi.leaf0 + j] = rb->F.as<double>() + fo + (size_t)j * pp;
    }
    if (refine)
      for (int r2 = 0; r2 < nrhs; ++r2) {
        AaCol c;
        c.w = u[k] + (size_t)r2 * len;
        c.off = fo + (int64_t)r2 * len;
        c.len = len;
        c.ch0 = ch;
        ch += (len + kAaChunk - 1) / kAaChunk;
        col_of.resize(ch, (int)cols.size());
        cols.push_back(c);
      }
    fo += (int64_t)nrhs * len;
  }
  cp.roots = H.call_st.push(rd, H.stream);
  cp.wptr = H.call_st.push(wp, H.stream);
  cp.wrs = H.call_st.push(wr, H.stream);
  if (refine) {
    cp.fptr = H.call_st.push(fp, H.stream);
    cp.cols = H.call_st.push(cols, H.stream);
    cp.col_of = H.call_st.push(col_of, H.stream);
    cp.ncol = ncol;
    cp.nchunks = ch;
    cp.nu = nu;
    rb->part.alloc((size_t)ch * kAaQ * sizeof(double), H.stream);
    rb->colsum.alloc((size_t)ncol * kAaQ * sizeof(double), H.stream);
    rb->coef.alloc((size_t)ncol * (kAaMaxDepth + 1) * sizeof(double), H.stream);
    const size_t need = (size_t)ncol * (kAaQ + kAaMaxDepth + 1);
    if (H.h_aa_cap < need) {
      if (H.h_aa) {
        ck(cudaStreamSynchronize(H.stream));
        cudaFreeHost(H.h_aa);
        H.h_aa = nullptr;
        H.h_aa_cap = 0;
      }
      ck(cudaMallocHost(&H.h_aa, need * sizeof(double)));
      H.h_aa_cap = need;
    }
  }
  return cp;
}

// hps_solve_batch body: device or host pointers per problem.
int solve_entry(hps_handle_s& H, const double* const* f, int nrhs, double* const* u,
                int device_ptrs, hps_solve_info* info) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  prepare_solve(H, nrhs);
  std::vector<const double*> fd(H.nprob);
  std::vector<double*> ud(H.nprob);
  if (device_ptrs) {
    for (int k = 0; k < H.nprob; ++k) {
      fd[k] = f[k];
      ud[k] = u[k];
    }
  } else {
    size_t fb = 0, ub = 0;
    for (int k = 0; k < H.nprob; ++k) {
      fb += (size_t)nrhs * pl.probs[k].nbnd;
      ub += (size_t)nrhs * pl.probs[k].nl * pl.probs[k].s.p * pl.probs[k].s.p;
    }
    if (H.fstage.bytes < fb * sizeof(double)) H.fstage.alloc(fb * sizeof(double), st);
    if (H.ustage.bytes < ub * sizeof(double)) H.ustage.alloc(ub * sizeof(double), st);
    size_t fo = 0, uo = 0;
    for (int k = 0; k < H.nprob; ++k) {
      const size_t nf = (size_t)nrhs * pl.probs[k].nbnd;
      const size_t nu = (size_t)nrhs * pl.probs[k].nl * pl.probs[k].s.p * pl.probs[k].s.p;
      fd[k] = H.fstage.as<double>() + fo;
      ud[k] = H.ustage.as<double>() + uo;
      ck(cudaMemcpyAsync(const_cast<double*>(fd[k]), f[k], nf * sizeof(double),
                         cudaMemcpyHostToDevice, st));
      fo += nf;
      uo += nu;
    }
  }
  RefineBufs rb;
  CallPtrs cp = stage_call(H, fd.data(), ud.data(), nrhs, &rb);
  int rc = solve_all(H, cp, &rb, nrhs, info);
  if (!device_ptrs)
    for (int k = 0; k < H.nprob; ++k) {
      const size_t nu = (size_t)nrhs * pl.probs[k].nl * pl.probs[k].s.p * pl.probs[k].s.p;
      ck(cudaMemcpyAsync(u[k], ud[k], nu * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
  ck(cudaStreamSynchronize(st));
  return rc;
}

int build_entry(const hps_problem* probs, int nprob, const hps_options* opt_in, hps_handle* out) {
  if (!out || !probs || nprob < 1) return HPS_EINVAL;
  *out = nullptr;
  std::vector<ProblemSpec> specs(nprob);
  std::vector<const double*> coef(6 * (size_t)nprob);
  for (int k = 0; k < nprob; ++k) {
    const hps_problem& P = probs[k];
    int v = validate(P.d, P.nx, P.ny, P.p, P.q);
    if (v != HPS_OK) return v;
    specs[k] = {P.d.x0, P.d.x1, P.d.y0, P.d.y1, P.nx, P.ny, P.p, P.q};
    const double* c[6] = {P.c11, P.c12, P.c22, P.c1, P.c2, P.c};
    for (int i = 0; i < 6; ++i) coef[6 * k + i] = c[i];
  }
  hps_options opt;
  hps_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.precision != HPS_FP64 && opt.precision != HPS_MIXED) return HPS_EINVAL;
  if (opt.precision == HPS_MIXED &&
      (!(opt.refine_tol > 0) || opt.max_refine < 0 || opt.fp64_top_levels < 0 ||
       opt.refine_depth < 0 || opt.refine_depth > kAaMaxDepth || opt.leaf_refine < 0 ||
       opt.leaf_refine > 1))
    return HPS_EINVAL;
  g_last_error.clear();
  hps_handle_s* H = nullptr;
  try {
    H = new hps_handle_s();
    H->opt = opt;
    H->mixed = opt.precision == HPS_MIXED;
    H->nprob = nprob;
    H->plan = make_forest(specs);
    if (opt.stream) {
      H->stream = (cudaStream_t)opt.stream;
    } else {
      ck(cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking));
      H->own_stream = true;
    }
    build_all(*H, coef, opt.device_ptrs != 0);
    *out = H;
    return HPS_OK;
  } catch (CudaError& e) {
    cudaGetLastError();
    hps_free(H);
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  } catch (int) {
    hps_free(H);
    return HPS_ESINGULAR;
  } catch (std::bad_alloc&) {
    hps_free(H);
    return HPS_ENOMEM;
  } catch (...) {
    hps_free(H);
    return HPS_EDEVICE;
  }
}

void clear_info(hps_solve_info* info) {
  if (info) {
    info->status = HPS_OK;
    info->iterations = 0;
    info->last_update = 0.0;
    info->bad_box = -1;
  }
}

int solve_guarded(hps_handle h, const double* const* f, int nrhs, double* const* u,
                  int device_ptrs, hps_solve_info* info) {
  try {
    return solve_entry(*h, f, nrhs, u, device_ptrs, info);
  } catch (CudaError& e) {
    cudaGetLastError();
    if (info) info->status = HPS_EDEVICE;
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  } catch (std::bad_alloc&) {
    return HPS_ENOMEM;
  } catch (...) {
    return HPS_EDEVICE;
  }
}

}  // namespace

// =================================================================== C ABI
extern "C" {

void hps_default_options(hps_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = HPS_FP64;
  opt->refine_tol = 1e-11;
  opt->max_refine = 10;
  opt->fp64_top_levels = 2;
  opt->device_ptrs = 0;
  opt->stream = nullptr;
  opt->form_root_dtn = 0;
  opt->refine_depth = 0;
  opt->leaf_refine = 1;
}

int64_t hps_boundary_count(int nx, int ny, int q) { return 2LL * (nx + ny) * q; }

int hps_cheb_nodes(hps_domain d, int nx, int ny, int p, double* xy) {
  if (validate(d, nx, ny, p, 1) != HPS_OK || !xy) return HPS_EINVAL;
  cheb_node_coords(d.x0, d.x1, d.y0, d.y1, nx, ny, p, xy);
  return HPS_OK;
}

int hps_boundary_nodes_grid(hps_domain d, int nx, int ny, int q, double* xy) {
  if (validate(d, nx, ny, std::max(q + 1, 3), q) != HPS_OK || !xy) return HPS_EINVAL;
  boundary_node_coords(d.x0, d.x1, d.y0, d.y1, nx, ny, q, xy);
  return HPS_OK;
}

int hps_build(hps_domain d, int nx, int ny, int p, int q, const double* c11, const double* c12,
              const double* c22, const double* c1, const double* c2, const double* c,
              const hps_options* opt, hps_handle* out) {
  hps_problem P;
  P.d = d;
  P.nx = nx;
  P.ny = ny;
  P.p = p;
  P.q = q;
  P.c11 = c11;
  P.c12 = c12;
  P.c22 = c22;
  P.c1 = c1;
  P.c2 = c2;
  P.c = c;
  if (!out) return HPS_EINVAL;
  return build_entry(&P, 1, opt, out);
}

int hps_build_batch(const hps_problem* probs, int nprob, const hps_options* opt,
                    hps_handle* out) {
  return build_entry(probs, nprob, opt, out);
}

int hps_boundary_nodes(hps_handle h, double* xy) {
  if (!h || !xy) return HPS_EINVAL;
  const ProblemSpec& s = h->plan.probs[0].s;
  boundary_node_coords(s.x0, s.x1, s.y0, s.y1, s.nx, s.ny, s.q, xy);
  return HPS_OK;
}

int hps_solve_ex(hps_handle h, const double* f, int nrhs, double* u, int device_ptrs,
                 hps_solve_info* info) {
  clear_info(info);
  if (!h || !f || !u || nrhs < 1 || h->nprob != 1) return HPS_EINVAL;
  g_last_error.clear();
  return solve_guarded(h, &f, nrhs, &u, device_ptrs, info);
}

int hps_solve(hps_handle h, const double* f, int nrhs, double* u, hps_solve_info* info) {
  if (!h) return HPS_EINVAL;
  return hps_solve_ex(h, f, nrhs, u, h->opt.device_ptrs, info);
}

int hps_solve_batch(hps_handle h, const double* const* f, int nrhs, double* const* u,
                    hps_solve_info* info) {
  clear_info(info);
  if (!h || !f || !u || nrhs < 1) return HPS_EINVAL;
  for (int k = 0; k < h->nprob; ++k)
    if (!f[k] || !u[k]) return HPS_EINVAL;
  g_last_error.clear();
  return solve_guarded(h, f, nrhs, u, h->opt.device_ptrs, info);
}

int hps_apply_dtn(hps_handle h, const double* f, int nrhs, double* g, int device_ptrs) {
  if (!h || !f || !g || nrhs < 1 || h->nprob != 1 || !h->opt.form_root_dtn || !h->root_dtn.p)
    return HPS_EINVAL;
  g_last_error.clear();
  try {
    hps_handle_s& H = *h;
    cudaStream_t st = H.stream;
    const int n = H.plan.probs[0].nbnd;
    const size_t nb = (size_t)n * nrhs * sizeof(double);
    const size_t wb = dtn_apply_ws_bytes(n, nrhs);
    PoolBuf ws, io, stt;
    ws.alloc(wb, st);
    stt.alloc(sizeof(int), st);
    ck(cudaMemsetAsync(stt.p, 0, sizeof(int), st));
    const double* fd = f;
    double* gd = g;
    if (!device_ptrs) {
      io.alloc(2 * nb, st);
      fd = io.as<double>();
      gd = io.as<double>() + (size_t)n * nrhs;
      ck(cudaMemcpyAsync(const_cast<double*>(fd), f, nb, cudaMemcpyHostToDevice, st));
    }
    ck(dtn_apply(H.root_dtn.as<double>(), n, H.root_from_f.as<int>() + H.plan.probs[0].rff_off,
                 fd, nrhs, gd, ws.p, wb, stt.as<int>(), st));
    if (!device_ptrs) ck(cudaMemcpyAsync(g, gd, nb, cudaMemcpyDeviceToHost, st));
    int hst = 0;
    ck(cudaMemcpyAsync(&hst, stt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    if (hst != 0) {
      g_last_error = "tensor-core GEMM: a wait gave up";
      return HPS_EDEVICE;
    }
    return HPS_OK;
  } catch (CudaError& e) {
    cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  } catch (std::bad_alloc&) {
    return HPS_ENOMEM;
  } catch (...) {
    return HPS_EDEVICE;
  }
}

int hps_interpolate(hps_handle h, const double* u, int nrhs, const double* xy, int64_t npts,
                    double* out, int device_ptrs) {
  if (!h || nrhs < 1 || npts < 0 || h->nprob != 1) return HPS_EINVAL;
  if (npts == 0) return HPS_OK;
  if (!u || !xy || !out) return HPS_EINVAL;
  const ProblemSpec& ps = h->plan.probs[0].s;
  if (!device_ptrs)
    for (int64_t i = 0; i < npts; ++i) {
      const double x = xy[2 * i], y = xy[2 * i + 1];
      if (!(x >= ps.x0 && x <= ps.x1 && y >= ps.y0 && y <= ps.y1)) return HPS_EINVAL;
    }
  g_last_error.clear();
  try {
    cudaStream_t st = h->stream;
    InterpGrid gr;
    gr.x0 = ps.x0;
    gr.x1 = ps.x1;
    gr.y0 = ps.y0;
    gr.y1 = ps.y1;
    gr.nx = ps.nx;
    gr.ny = ps.ny;
    gr.p = ps.p;
    const size_t ub = (size_t)nrhs * ps.nx * ps.ny * ps.p * ps.p * sizeof(double);
    const size_t xb = (size_t)npts * 2 * sizeof(double), ob = (size_t)npts * nrhs * sizeof(double);
    PoolBuf io, stt;
    stt.alloc(sizeof(int), st);
    ck(cudaMemsetAsync(stt.p, 0, sizeof(int), st));
    const double *ud = u, *xd = xy;
    double* od = out;
    if (!device_ptrs) {
      io.alloc(ub + xb + ob, st);
      char* b = static_cast<char*>(io.p);
      ud = reinterpret_cast<const double*>(b);
      xd = reinterpret_cast<const double*>(b + ub);
      od = reinterpret_cast<double*>(b + ub + xb);
      ck(cudaMemcpyAsync(const_cast<double*>(ud), u, ub, cudaMemcpyHostToDevice, st));
      ck(cudaMemcpyAsync(const_cast<double*>(xd), xy, xb, cudaMemcpyHostToDevice, st));
    }
    interp_points(ud, nrhs, gr, xd, npts, od, stt.as<int>(), st);
    ck(cudaGetLastError());
    if (!device_ptrs) ck(cudaMemcpyAsync(out, od, ob, cudaMemcpyDeviceToHost, st));
    int hst = 0;
    ck(cudaMemcpyAsync(&hst, stt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    return hst ? HPS_EINVAL : HPS_OK;
  } catch (CudaError& e) {
    cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  } catch (std::bad_alloc&) {
    return HPS_ENOMEM;
  } catch (...) {
    return HPS_EDEVICE;
  }
}

int hps_dgemm_tc(int M, int N, int K, double alpha, const double* A, int lda, const double* B,
                 int ldb, double beta, double* C, int ldc) {
  if (M < 1 || N < 1 || K < 1 || lda < M || ldb < K || ldc < M || !A || !B || !C)
    return HPS_EINVAL;
  g_last_error.clear();
  try {
    cudaStream_t st = nullptr;
    ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    std::vector<OzDesc> h(1);
    h[0].A = A;
    h[0].B = B;
    h[0].C = C;
    h[0].M = M;
    h[0].N = N;
    h[0].K = K;
    h[0].lda = lda;
    h[0].ldb = ldb;
    h[0].ldc = ldc;
    const size_t wb = oz_plan(h);
    int rc = HPS_OK;
    {
      PoolBuf ow, dd, stt;
      ow.alloc(wb, st);
      dd.alloc(sizeof(OzDesc), st);
      stt.alloc(sizeof(int), st);
      ck(cudaMemcpyAsync(dd.p, h.data(), sizeof(OzDesc), cudaMemcpyHostToDevice, st));
      ck(cudaMemsetAsync(stt.p, 0, sizeof(int), st));
      ck(oz_gemm(dd.as<OzDesc>(), h, ow.p, wb, alpha, beta, stt.as<int>(), st, "dgemm_tc<f64>"));
      int hst = 0;
      ck(cudaMemcpyAsync(&hst, stt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (hst != 0) {
        g_last_error = "tensor-core GEMM: a wait gave up";
        rc = HPS_EDEVICE;
      }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
  } catch (CudaError& e) {
    cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  }
}

int hps_sgemm_tc(int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                 int ldb, float beta, float* C, int ldc) {
  if (M < 1 || N < 1 || K < 1 || lda < M || ldb < K || ldc < M || !A || !B || !C)
    return HPS_EINVAL;
  g_last_error.clear();
  try {
    cudaStream_t st = nullptr;
    ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = HPS_OK;
    {
      GemmDesc<float> h{A, B, C, M, N, K, lda, ldb, ldc};
      PoolBuf dd, stt;
      dd.alloc(sizeof(h), st);
      stt.alloc(sizeof(int), st);
      ck(cudaMemcpyAsync(dd.p, &h, sizeof(h), cudaMemcpyHostToDevice, st));
      ck(cudaMemsetAsync(stt.p, 0, sizeof(int), st));
      gemm_batched<float>(dd.as<GemmDesc<float>>(), 1, M, N, alpha, beta, st, "sgemm<f32>",
                          2.0 * M * (double)N * K, 4.0 * ((double)M * K + (double)K * N + M * N),
                          K, nullptr, 0, stt.as<int>());
      ck(cudaGetLastError());
      int hst = 0;
      ck(cudaMemcpyAsync(&hst, stt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (hst != 0) {
        g_last_error = "tensor-core GEMM: a wait gave up";
        rc = HPS_EDEVICE;
      }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
  } catch (CudaError& e) {
    cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  }
}

int hps_sinv_gj(int n, int count, const float* A, float* Ainv) {
  g_last_error.clear();
  if (n != kLeafGjN || count < 1 || !A || !Ainv) {
    g_last_error = "hps_sinv_gj: takes n = " + std::to_string(kLeafGjN) +
                   ", count >= 1 and non-null arrays";
    return HPS_EINVAL;
  }
  const size_t nn = (size_t)n * n;
  const char *a0 = reinterpret_cast<const char*>(A), *b0 = reinterpret_cast<const char*>(Ainv);
  if (a0 < b0 + nn * count * sizeof(float) && b0 < a0 + nn * count * sizeof(float)) {
    g_last_error = "hps_sinv_gj: A and Ainv overlap";
    return HPS_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(Ainv) % 16) {
    g_last_error = "hps_sinv_gj: A and Ainv must be 16-byte aligned";  // 16-byte vector copies
    return HPS_EINVAL;
  }
  try {
    cudaStream_t st = nullptr;
    ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = HPS_OK;
    {
      // nq = 0: nothing is copied into A, which is only read
      std::vector<LuDesc<float>> h(count);
      for (int m = 0; m < count; ++m) {
        h[m].A = const_cast<float*>(A) + nn * m;
        h[m].ipiv = nullptr;
        h[m].B = Ainv + nn * m;
        h[m].m = n;
        h[m].lda = n;
        h[m].nrhs = n;
        h[m].ldb = n;
        h[m].box = m;
      }
      PoolBuf dd, stt;
      dd.alloc(h.size() * sizeof(LuDesc<float>), st);
      stt.alloc(sizeof(int), st);
      ck(cudaMemcpyAsync(dd.p, h.data(), h.size() * sizeof(LuDesc<float>), cudaMemcpyHostToDevice,
                         st));
      ck(cudaMemsetAsync(stt.p, 0, sizeof(int), st));
      if (!leaf_gj_inverse(dd.as<LuDesc<float>>(), count, n, 0, stt.as<int>(), st))
        throw CudaError{cudaErrorInvalidValue};
      ck(cudaGetLastError());
      int hst = 0;
      ck(cudaMemcpyAsync(&hst, stt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (hst > 0) {
        g_last_error = "hps_sinv_gj: zero or non-finite pivot in matrix " + std::to_string(hst - 1);
        rc = HPS_ESINGULAR;
      }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
  } catch (CudaError& e) {
    cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  }
}

int hps_leaf_residual(int p, int q, int nleaves, double hx, double hy, const double* c11,
                      const double* c22, const double* c, const double* w, int nrhs, double* r,
                      double* flux, int tensor_cores) {
  if (p < 3 || p > 64 || q < 1 || q > p || nleaves < 1 || nrhs < 1 || !(hx > 0) || !(hy > 0) ||
      !w || !r || !flux || (tensor_cores != 0 && tensor_cores != 1))
    return HPS_EINVAL;
  const double* coef[6] = {c11, nullptr, c22, nullptr, nullptr, c};
  g_last_error.clear();
  try {
    cudaStream_t st = nullptr;
    ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = HPS_OK;
    {
      const Consts k = make_consts(p, q);
      const int pp = p * p;
      std::vector<double> dtab(2 * (size_t)pp);
      std::copy(k.D.begin(), k.D.end(), dtab.begin());
      std::copy(k.D2.begin(), k.D2.end(), dtab.begin() + pp);
      std::vector<double2> hsc(nleaves, make_double2(2.0 / hx, 2.0 / hy));
      std::vector<const double*> wp(nleaves);
      std::vector<int64_t> wr(nleaves, (int64_t)nleaves * pp), off(nleaves);
      for (int l = 0; l < nleaves; ++l) {
        wp[l] = w + (size_t)l * pp;
        off[l] = (int64_t)l * 4 * q;
      }
      PoolBuf dD, dP, dh, dw, dwr, doff, stt;
      auto up = [&](PoolBuf& b, const void* src, size_t bytes) {
        b.alloc(bytes, st);
        ck(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st));
      };
      up(dD, dtab.data(), dtab.size() * sizeof(double));
      up(dP, k.Pc2g.data(), k.Pc2g.size() * sizeof(double));
      up(dh, hsc.data(), hsc.size() * sizeof(double2));
      up(dw, wp.data(), wp.size() * sizeof(double*));
      up(dwr, wr.data(), wr.size() * sizeof(int64_t));
      up(doff, off.data(), off.size() * sizeof(int64_t));
      stt.alloc(sizeof(int), st);
      ck(cudaMemsetAsync(stt.p, 0, sizeof(int), st));
      double* const* wptr = reinterpret_cast<double* const*>(dw.p);
      const int64_t ext_total = (int64_t)nleaves * 4 * q;
      if (tensor_cores) {
        if (!leaf_resflux_tc<double>(coef, 0, nleaves, p, q, dh.as<double2>(), dD.as<double>(),
                                     dP.as<double>(), wptr, dwr.as<int64_t>(), nrhs, r,
                                     doff.as<int64_t>(), ext_total, flux, stt.as<int>(), st)) {
          g_last_error = "hps_leaf_residual: the tensor-core kernel takes p = 16, q <= 16";
          rc = HPS_EINVAL;
        }
      } else {
        leaf_resflux<double>(coef, 0, nleaves, p, q, dh.as<double2>(), dD.as<double>(),
                             dP.as<double>(), wptr, dwr.as<int64_t>(), nrhs, r,
                             doff.as<int64_t>(), ext_total, flux, st);
      }
      ck(cudaGetLastError());
      int hst = 0;
      ck(cudaMemcpyAsync(&hst, stt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (hst != 0) {
        g_last_error = "tensor-core residual: a wait gave up";
        rc = HPS_EDEVICE;
      }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
  } catch (CudaError& e) {
    cudaGetLastError();
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  }
}

int hps_estimate_bytes(const hps_problem* probs, int nprob, const hps_options* opt_in, int nrhs,
                       int64_t* build_peak, int64_t* resident, int64_t* solve) {
  if (!probs || nprob < 1 || nrhs < 0) return HPS_EINVAL;
  hps_options opt;
  hps_default_options(&opt);
  if (opt_in) opt = *opt_in;
  std::vector<ProblemSpec> specs(nprob);
  int64_t coef_bytes = 0;
  for (int k = 0; k < nprob; ++k) {
    const hps_problem& P = probs[k];
    const int v = validate(P.d, P.nx, P.ny, P.p, P.q);
    if (v != HPS_OK) return v;
    specs[k] = {P.d.x0, P.d.x1, P.d.y0, P.d.y1, P.nx, P.ny, P.p, P.q};
    const double* c[6] = {P.c11, P.c12, P.c22, P.c1, P.c2, P.c};
    for (int i = 0; i < 6; ++i)
      if (c[i]) coef_bytes += (int64_t)P.nx * P.ny * P.p * P.p * 8;
  }
  try {
    const Plan pl = make_forest(specs);
    const bool mixed = opt.precision == HPS_MIXED;
    const int top = std::max(0, opt.fp64_top_levels);
    const int64_t bl = mixed ? 4 : 8;
    int64_t y = 0, leaf_tmp = 0, dof = 0, nint = 0;
    for (const auto& pi : pl.probs) {
      const int64_t ni = (int64_t)(pi.s.p - 2) * (pi.s.p - 2), nq = 4LL * pi.s.q;
      y += pi.nl * ni * (nq + (mixed ? ni : 0)) * bl;
      const bool yref = mixed && opt.leaf_refine > 0;  // residual and correction of Y
      leaf_tmp += pi.nl * (std::max(ni * ni, yref ? 2 * ni * nq : 0) + nq * nq) * bl;
      dof += (int64_t)pi.nl * pi.s.p * pi.s.p;
      nint += pi.nl * ni;
    }
    // per height: stored S (+ W, [T13; T23] in mixed mode), transient T, A_w
    std::vector<int64_t> t_at(pl.height + 1, 0), tmp_at(pl.height + 1, 0);
    // sres: stored operators as built; sres_r: as resident after the build (in
    // mixed mode the FP64-factored heights keep FP32 copies); demote: those
    // copies, held beside the FP64 originals while they are made
    int64_t sres = 0, sres_r = 0, demote = 0, u3_rows = 0, max_level_rows = 0;
    t_at[0] = 0;
    for (const auto& pi : pl.probs) t_at[0] += pi.nl * 16LL * pi.s.q * pi.s.q * bl;
    for (int h = 1; h <= pl.height; ++h) {
      int64_t rows = 0;
      for (int b : pl.levels[h]) {
        const Box& B = pl.boxes[b];
        const MergeShape& sh = pl.shapes[B.shape];
        const int ph = pl.probs[B.prob].height;
        const int64_t bm = (!mixed || h > ph - top) ? 8 : 4;
        const int64_t ops = (int64_t)sh.m * (sh.ne + (mixed ? sh.m : 0)) +
                            (mixed ? (int64_t)sh.ne * sh.m : 0);
        sres += ops * bm;
        sres_r += ops * (mixed ? 4 : 8);
        if (mixed && bm == 8) demote += ops * 4;
        if (B.parent >= 0 || opt.form_root_dtn) t_at[h] += (int64_t)sh.ne * sh.ne * bm;
        tmp_at[h] += (int64_t)sh.m * sh.m * bm + (mixed ? 0 : (int64_t)sh.ne * sh.m * bm);
        if (bm == 4 && mixed && sh.m >= kNBw) tmp_at[h] += (int64_t)sh.m * sh.ne * 4;  // [-T31 | T32]
        if (bm == 8) {  // tensor-core products: S's temporaries, split operands
          const int64_t m = sh.m, ne = sh.ne, kp = (m + 31) / 32 * 32;
          if (mixed && oz_eligible(sh.m, sh.ne, sh.m))
            tmp_at[h] += m * ne * 8 + 16 * ((m + 127) / 128 * 128) * kp +
                         16 * ((ne + 127) / 128 * 128) * kp + 4 * (m + ne);
          if (oz_eligible(sh.ne, sh.ne, sh.m))
            tmp_at[h] += 32 * ((ne + 127) / 128 * 128) * kp + 8 * ne;
          if (lu_tc_eligible(sh.m)) {  // two-level LU: split operands of one outer step
            const int64_t nr = ne + m;
            tmp_at[h] += 16 * (kLuOuter + 32) * (3 * (m + 128) + nr + 64) + 4 * (3 * m + nr);
          }
        }
        u3_rows += sh.m;
        rows += sh.m;
      }
      max_level_rows = std::max(max_level_rows, rows);
    }
    int64_t root_dtn = 0;  // form_root_dtn: the kept T^1 of every problem
    if (opt.form_root_dtn && nprob == 1) root_dtn = (int64_t)pl.probs[0].nbnd * pl.probs[0].nbnd * 8;
    const int64_t res = y + sres_r + (mixed ? coef_bytes : 0) + root_dtn;
    int64_t peak = std::max(leaf_tmp, demote);
    for (int h = 1; h <= pl.height; ++h) peak = std::max(peak, t_at[h - 1] + t_at[h] + tmp_at[h]);
    peak += y + sres + coef_bytes + root_dtn;
    int64_t work = (int64_t)nrhs * (pl.ext_total + u3_rows) * 8 + 2 * (int64_t)nrhs * max_level_rows * 8;
    if (mixed && opt.max_refine > 0) {
      const int64_t m = std::max(0, opt.refine_depth);
      work += (int64_t)nrhs * pl.ext_total * 8 + 2 * nint * nrhs * 4 + 2 * u3_rows * nrhs * 8;
      work += (int64_t)nrhs * dof * (24 + (m > 0 ? 12 * m : -16));
    }
    if (build_peak) *build_peak = peak;
    if (resident) *resident = res;
    if (solve) *solve = work;
  } catch (...) {
    return HPS_ENOMEM;
  }
  return HPS_OK;
}

int hps_release_workspace(hps_handle h) {
  if (!h) return HPS_EINVAL;
  for (PoolBuf* x : {&h->uext, &h->u3, &h->hpool, &h->split_ws, &h->fstage, &h->ustage,
                     &h->solve_st.dev, &h->call_st.dev})
    x->release();
  for (auto& G : h->lg) {
    G.rleaf->release();
    G.zleaf->release();
  }
  for (auto& L : h->lev) {
    L.rlev->release();
    L.zlev->release();
  }
  h->cache_nrhs = 0;
  return HPS_OK;
}

int hps_query(hps_handle h, int* n_leaves, int* p, int* q, int64_t* nbnd, int64_t* device_bytes) {
  if (!h) return HPS_EINVAL;
  if (n_leaves) *n_leaves = h->plan.n_leaves();
  if (p) *p = h->plan.probs[0].s.p;
  if (q) *q = h->plan.probs[0].s.q;
  if (nbnd) {
    int64_t b = 0;
    for (const auto& pi : h->plan.probs) b += pi.nbnd;
    *nbnd = b;
  }
  if (device_bytes) {
    int64_t b = 0;
    for (const PoolBuf* x : {&h->coef, &h->maps, &h->uext, &h->u3, &h->hpool, &h->fstage,
                             &h->ustage, &h->split_ws, &h->keep.dev, &h->solve_st.dev,
                             &h->root_dtn})
      b += (int64_t)x->bytes;
    for (const auto& G : h->lg) b += (int64_t)(G.Y->bytes + G.rleaf->bytes + G.zleaf->bytes);
    for (const auto& L : h->lev)
      b += (int64_t)(L.S->bytes + L.Cw->bytes + L.rlev->bytes + L.zlev->bytes);
    *device_bytes = b;
  }
  return HPS_OK;
}

int hps_batch_size(hps_handle h) { return h ? h->nprob : 0; }

int hps_free(hps_handle h) {
  if (!h) return HPS_OK;
  cudaStream_t st = h->stream;
  bool own = h->own_stream;
  delete h;  // buffers are released in stream order
  if (st) cudaStreamSynchronize(st);
  if (own && st) cudaStreamDestroy(st);
  return HPS_OK;
}

const char* hps_last_error(void) { return g_last_error.c_str(); }

int64_t hps_kernel_launches(void) { return prof::launches(); }

void hps_profile_enable(int on) { prof::set_enabled(on != 0); }

void hps_profile_reset(void) { prof::reset(); }

int hps_profile_read(hps_kernel_stat* out, int max_out) {
  std::vector<prof::Stat> tmp(std::max(max_out, 0) + 1);
  int n = prof::read(tmp.data(), std::max(max_out, 0));
  for (int i = 0; i < std::min(n, max_out); ++i) {
    out[i].name = tmp[i].name;
    out[i].launches = tmp[i].launches;
    out[i].ms = tmp[i].ms;
    out[i].flops = tmp[i].flops;
    out[i].bytes = tmp[i].bytes;
  }
  return n;
}

const char* hps_status_string(int status) {
  switch (status) {
    case HPS_OK: return "ok";
    case HPS_EINVAL: return "invalid argument";
    case HPS_ENOMEM: return "out of memory";
    case HPS_ESINGULAR: return "singular or non-finite pivot";
    case HPS_ENOTCONVERGED: return "iterative refinement did not converge";
    case HPS_EDEVICE: return "CUDA device error";
    default: return "unknown status";
  }
}

}  // extern "C"

// ================================================ solve without allocation
// Some callers cannot allocate device memory when they solve: code that runs
// under a fixed memory budget reserved up front (a serving process that must
// not grow), code that must not synchronise the device or touch the allocator
// while other work is in flight, or embeddings whose allocator is not
// reachable from the calling thread.  hps_solve_static serves them: the solve
// of an FP64 handle runs entirely in a static device array that every GPU
// loading this library holds until the process exits.
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // per device
constexpr size_t kStaticHostBytes = size_t(4) << 20;      // descriptor staging
constexpr int kMaxDevices = 64;
constexpr size_t kStaticMaxLevels = 256;  // merge heights of one handle

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
alignas(256) unsigned char g_static_host[kStaticHostBytes];
std::mutex g_static_mu;
void* g_static_dev[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int hps_solve_static(hps_handle h, const double* f, int nrhs, double* u) {
  if (!h || !f || !u || nrhs < 1 || h->nprob != 1) return HPS_EINVAL;
  g_last_error.clear();
  hps_handle_s& H = *h;
  if (H.mixed) {
    g_last_error = "hps_solve_static: only FP64 handles (mixed handles refine with more buffers)";
    return HPS_EINVAL;
  }
  const Plan& pl = H.plan;
  const ProbInfo& pi = pl.probs[0];
  const int nl = pl.n_leaves();
  if (H.lev.size() > kStaticMaxLevels) {
    g_last_error = "hps_solve_static: " + std::to_string(H.lev.size()) +
                   " merge heights, the static descriptor table holds " +
                   std::to_string(kStaticMaxLevels);
    return HPS_EINVAL;
  }
  // carve the static array: exterior-value pool, u3 pool, descriptors
  const size_t b_uext = align256((size_t)nrhs * pl.ext_total * sizeof(double));
  const size_t b_u3 = align256((size_t)nrhs * std::max<int64_t>(H.u3_total, 1) * sizeof(double));
  size_t b_desc = align256(sizeof(RootDesc)) + align256((size_t)nl * sizeof(double*)) +
                  align256((size_t)nl * sizeof(int64_t));
  for (auto& L : H.lev) b_desc += align256(L.boxes.size() * sizeof(GemmDesc<double>));
  if (b_uext + b_u3 + b_desc > kStaticScratchBytes || b_desc > kStaticHostBytes) {
    g_last_error = "hps_solve_static: needs " + std::to_string(b_uext + b_u3 + b_desc) +
                   " bytes of scratch, the static array holds " +
                   std::to_string(kStaticScratchBytes);
    return HPS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  try {
    int dev = 0;
    ck(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
      g_last_error = "hps_solve_static: device ordinal out of range";
      return HPS_EINVAL;
    }
    if (!g_static_dev[dev]) {  // first call on this device: the array's device address
      void* p = nullptr;
      ck(cudaGetSymbolAddress(&p, g_static_scratch));
      g_static_dev[dev] = p;
    }
    unsigned char* base = static_cast<unsigned char*>(g_static_dev[dev]);
    double* uext = reinterpret_cast<double*>(base);
    double* u3 = reinterpret_cast<double*>(base + b_uext);
    unsigned char* dd = base + b_uext + b_u3;
    cudaStream_t st = H.stream;
    // descriptors staged in static host memory; the earlier call's copies have
    // completed (each call ends synchronised)
    size_t off = 0;
    auto stage = [&](const void* src, size_t n) {
      if (src != g_static_host + off) std::memcpy(g_static_host + off, src, n);
      ck(cudaMemcpyAsync(dd + off, g_static_host + off, n, cudaMemcpyHostToDevice, st));
      void* dst = dd + off;
      off += align256(n);
      return dst;
    };
    RootDesc rd;
    rd.f = f;
    rd.rff = H.root_from_f.as<int>() + pi.rff_off;
    rd.root_off = pl.boxes[pi.root].ext_off;
    rd.nbnd = pi.nbnd;
    RootDesc* droot = static_cast<RootDesc*>(stage(&rd, sizeof(rd)));
    // per-leaf output pointers, written straight into the staging block
    {
      const int pp = pi.s.p * pi.s.p;
      double** wp = reinterpret_cast<double**>(g_static_host + off);
      for (int j = 0; j < nl; ++j) wp[j] = u + (size_t)j * pp;
    }
    double* const* dwp = static_cast<double* const*>(stage(g_static_host + off, nl * sizeof(double*)));
    {
      int64_t* wr = reinterpret_cast<int64_t*>(g_static_host + off);
      for (int j = 0; j < nl; ++j) wr[j] = (int64_t)nl * pi.s.p * pi.s.p;
    }
    const int64_t* dwr = static_cast<const int64_t*>(stage(g_static_host + off, nl * sizeof(int64_t)));
    GemmDesc<double>* dptr[kStaticMaxLevels] = {};
    for (size_t li = 0; li < H.lev.size(); ++li) {
      LevelGroup& L = H.lev[li];
      GemmDesc<double>* hs = reinterpret_cast<GemmDesc<double>*>(g_static_host + off);
      for (size_t i = 0; i < L.boxes.size(); ++i) {
        const int b = L.boxes[i];
        const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
        GemmDesc<double>& g = hs[i];
        g.A = L.S->as<double>() + L.s_off[i];
        g.B = uext + pl.boxes[b].ext_off;
        g.C = u3 + H.u3_off[b];
        g.M = sh.m;
        g.N = nrhs;
        g.K = sh.ne;
        g.lda = sh.m;
        g.ldb = (int)pl.ext_total;
        g.ldc = (int)H.u3_total;
      }
      dptr[li] = static_cast<GemmDesc<double>*>(
          stage(g_static_host + off, L.boxes.size() * sizeof(GemmDesc<double>)));
    }
    // nothing in the array has to start at zero: every exterior value and every
    // u3 entry is written (root scatter, GEMMs with beta = 0, child scatters)
    // before it is read
    solve_root_scatter(droot, 1, pi.nbnd, nrhs, uext, pl.ext_total, st);
    for (int li = (int)H.lev.size() - 1; li >= 0; --li) {
      LevelGroup& L = H.lev[li];
      const int nm = (int)L.boxes.size();
      gemm_batched<double>(dptr[li], nm, L.max_m, nrhs, 1.0, 0.0, st, "gemm_solve_static<f64>",
                           0.0, 0.0);
      solve_child_scatter(L.scatter, nm, L.max_nanb, u3, H.u3_total, uext, pl.ext_total, nrhs, st);
    }
    for (auto& G : H.lg)
      leaf_post<double>(G.Y->as<double>(), G.ys, G.l0, uext, H.leaf_off.as<int64_t>(),
                        pl.ext_total, G.nl, G.p, G.q, nrhs, G.dPg2c->as<double>(), dwp, dwr, st);
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(st));
    return HPS_OK;
  } catch (CudaError&) {
    cudaGetLastError();
    return HPS_EDEVICE;
  } catch (...) {
    return HPS_EDEVICE;
  }
}
