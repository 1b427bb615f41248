// C ABI of libhps: the build stage (Algorithm 1) and the solve stage
// (Algorithm 2 + Section 4.3) orchestrated over the batched kernels.
//
// Build, per tree height h (h = 0: the leaves), one batched launch sequence per
// height covering every leaf / merge of that height:
//   h = 0   leaf_assemble -> LU of [A_ii | -A_ie L1] -> Y, leaf_dtn -> T
//   h >= 1  merge_gather  -> LU of [T33^a - T33^b | -T31^a, T32^b] -> S,
//           GEMM Tp += [T13^a; T23^b] S (eq. merge; skipped at the root unless
//           the root DtN is requested: the solve never needs it)
// Children's T are released in stream order once every parent reading them is
// built.  All device memory comes from a stream-ordered pool and all launch
// descriptors are staged in pinned memory, so a build synchronises the host
// only once, at the end, to read the pivot status.
//
// Precision.  HPS_FP64: every stage in double.  HPS_MIXED: the leaves and the
// merges below the top `fp64_top_levels` heights run in float (their LU
// factors, pivots and [T13^a; T23^b] blocks are kept), the top heights in
// double; the solve then refines against the FP64 residual of the global
// collocation system, one body-load correction per iteration (the elimination
// of Algorithms 1-2 applied to a right-hand side).
//
// Solve: root exterior values from f, then per height from the top a batched
// GEMM u3 = S u_parent and a scatter into the children's exterior vectors, then
// the leaf post-process w_full = [L1 ; Y] u_e.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
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
    dev.alloc(bytes, st);
    used = 0;
  }
  template <typename T>
  T* push(const std::vector<T>& v, cudaStream_t st) {
    size_t off = (used + 255) & ~size_t(255);
    size_t n = v.size() * sizeof(T);
    if (off + n > cap || off + n > dev.bytes) throw std::bad_alloc();
    if (n) {
      std::memcpy(static_cast<char*>(host) + off, v.data(), n);
      ck(cudaMemcpyAsync(static_cast<char*>(dev.p) + off, static_cast<char*>(host) + off, n,
                         cudaMemcpyHostToDevice, st));
    }
    used = off + n;
    return reinterpret_cast<T*>(static_cast<char*>(dev.p) + off);
  }
};

template <typename T>
size_t stage_bytes(size_t n) {
  return n * sizeof(T) + 256;
}

struct LevelOps {
  int f64 = 1;                    // precision of this height's merges
  std::vector<int> boxes;
  int max_m = 0, max_ne = 0, max_nanb = 0;
  int64_t sum_m = 0;              // rows of the height's z buffer
  std::unique_ptr<PoolBuf> S, Cw;  // [S | W (mixed)] per merge; Cw kept in mixed mode
  std::vector<int64_t> s_off, aw_off, cw_off, piv_off, z_off;
  std::vector<int> hm, hne;       // host copies of m and ne (launch accounting)
  SolveScatterDesc* scatter = nullptr;  // device descriptors (the handle's stager)
  BodyDesc* body = nullptr;
  LevelOps() : S(new PoolBuf()), Cw(new PoolBuf()) {}
};

}  // namespace

struct hps_handle_s {
  Plan plan;
  Consts consts;
  hps_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int ni = 0, nq = 0, nl = 0, nbnd = 0;
  bool mixed = false;
  int leaf_f64 = 1;
  double hx = 0, hy = 0;
  PoolBuf dD, dPg2c, dPc2g, maps, root_from_f, leaf_off, status;
  std::vector<int64_t> src_off, cma_off, cmb_off;
  PoolBuf coef;                    // FP64 coefficient copy (mixed mode: the residual)
  const double* coefp[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  PoolBuf Y;                       // per leaf [Y | A_ii^{-1} (mixed mode)], stride ys
  int64_t ys = 0;
  std::vector<LevelOps> levels;    // index = height (0 unused)
  std::vector<int64_t> u3_off;
  int64_t u3_total = 0;
  Stager keep;                     // descriptors that live as long as the handle
  // solve workspace and descriptors, cached for one nrhs
  int cache_nrhs = 0;
  PoolBuf uext, u3, hpool, rleaf, zleaf, fstage, ustage, maxabs, split_ws;
  std::vector<std::unique_ptr<PoolBuf>> rlev, zlev;
  Stager solve_st;
  std::vector<void*> gemm_down;    // per height: GemmDesc array (typed by level)
  std::vector<void*> gemm_hpar;    // per height (mixed)
  std::vector<void*> gemm_w;       // per height (mixed): z = W rhs
  void* gemm_leaf = nullptr;       // (mixed): z = A_ii^{-1} r
  std::vector<double> down_flops1, down_bytes;
  unsigned long long* h_maxabs = nullptr;  // pinned
  ~hps_handle_s() {
    if (stream) cudaStreamSynchronize(stream);
    if (h_maxabs) cudaFreeHost(h_maxabs);
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
void build_leaves(hps_handle_s& H, Stager& stg, std::vector<TRef>& Tref, PoolBuf& T0) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  const int p = pl.p, q = pl.q, ni = H.ni, nq = H.nq, nl = H.nl;
  // mixed mode also solves for A_ii^{-1} (identity columns after -A_ie L1)
  const int nrhs_leaf = nq + (H.mixed ? ni : 0);
  H.ys = (int64_t)ni * nrhs_leaf;
  H.Y.alloc((size_t)nl * H.ys * sizeof(R), st);
  PoolBuf Aii, piv;
  Aii.alloc((size_t)nl * ni * ni * sizeof(R), st);
  piv.alloc((size_t)nl * ni * sizeof(int), st);
  leaf_assemble<R>(H.coefp, nl, p, q, H.hx, H.hy, H.dD.as<double>(), H.dPg2c.as<double>(),
                   Aii.as<R>(), H.Y.as<R>(), H.ys, H.mixed ? 1 : 0, st);
  ck(cudaGetLastError());
  std::vector<LuDesc<R>> ld(nl);
  for (int l = 0; l < nl; ++l) {
    ld[l].A = Aii.as<R>() + (size_t)l * ni * ni;
    ld[l].ipiv = piv.as<int>() + (size_t)l * ni;
    ld[l].B = H.Y.as<R>() + (size_t)l * H.ys;
    ld[l].m = ni;
    ld[l].lda = ni;
    ld[l].nrhs = nrhs_leaf;
    ld[l].ldb = ni;
    ld[l].box = pl.leaf_box[l];
  }
  LuDesc<R>* dl = stg.push(ld, st);
  lu_solve_batched<R>(dl, nl, ni, nrhs_leaf, kLuFactor, H.status.as<int>(), st, nullptr, nullptr);
  ck(cudaGetLastError());
  T0.alloc((size_t)nl * nq * nq * sizeof(R), st);
  leaf_dtn<R>(H.Y.as<R>(), H.ys, nl, p, q, H.hx, H.hy, H.dD.as<double>(), H.dPg2c.as<double>(),
              H.dPc2g.as<double>(), T0.as<R>(), st);
  ck(cudaGetLastError());
  for (int l = 0; l < nl; ++l) {
    Tref[pl.leaf_box[l]].p = T0.as<R>() + (size_t)l * nq * nq;
    Tref[pl.leaf_box[l]].f64 = sizeof(R) == 8;
  }
}

template <typename R>
void build_level(hps_handle_s& H, int h, Stager& stg, std::vector<TRef>& Tref, PoolBuf& Tout) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  LevelOps& L = H.levels[h];
  const int nm = (int)L.boxes.size();
  const bool form_root = H.opt.form_root_dtn != 0;
  int64_t aw_tot = 0, cw_tot = 0, tp_tot = 0, piv_tot = 0, s_tot = 0;
  int64_t max_work = 0;
  for (int i = 0; i < nm; ++i) {
    const int b = L.boxes[i];
    const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
    const bool tp = (b != 0) || form_root;
    L.s_off[i] = s_tot;
    L.aw_off[i] = aw_tot;
    L.cw_off[i] = cw_tot;
    L.piv_off[i] = piv_tot;
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
  double gather_bytes = 0.0, schur_flops = 0.0, schur_bytes = 0.0;
  int64_t ot = 0;
  for (int i = 0; i < nm; ++i) {
    const int b = L.boxes[i];
    const Box& B = pl.boxes[b];
    const MergeShape& sh = pl.shapes[B.shape];
    const bool tp = (b != 0) || form_root;
    MergeDesc<R>& g = md[i];
    g.Ta = Tref[B.child[0]].p;
    g.ta64 = Tref[B.child[0]].f64;
    g.Tb = Tref[B.child[1]].p;
    g.tb64 = Tref[B.child[1]].f64;
    g.Aw = Aw.as<R>() + L.aw_off[i];
    g.S = L.S->as<R>() + L.s_off[i];
    g.Cw = Cw.as<R>() + L.cw_off[i];
    g.Tp = tp ? Tout.as<R>() + ot : nullptr;
    g.W = H.mixed ? g.S + (int64_t)sh.m * sh.ne : nullptr;
    g.src = H.maps.as<int>() + H.src_off[B.shape];
    g.na = sh.na;
    g.nb = sh.nb;
    g.m = sh.m;
    g.ne = sh.ne;
    g.j3a = sh.j3a;
    g.j3b = sh.j3b;
    lu[i].A = g.Aw;
    lu[i].ipiv = piv.as<int>() + L.piv_off[i];
    lu[i].B = g.S;
    lu[i].m = sh.m;
    lu[i].lda = sh.m;
    lu[i].nrhs = sh.ne + (H.mixed ? sh.m : 0);
    lu[i].ldb = sh.m;
    lu[i].box = b;
    gather_bytes += (sizeof(R) + 8.0) *
                    ((double)sh.m * sh.m + 2.0 * sh.m * sh.ne + (tp ? (double)sh.ne * sh.ne : 0.0));
    if (tp) {
      GemmDesc<R> gg;
      gg.A = g.Cw;
      gg.B = g.S;
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
  LuDesc<R>* dlu = stg.push(lu, st);
  merge_gather<R>(dmd, nm, max_work, st, gather_bytes);
  ck(cudaGetLastError());
  std::vector<int> hn(nm);
  for (int i = 0; i < nm; ++i) hn[i] = L.hne[i] + (H.mixed ? L.hm[i] : 0);
  lu_solve_batched<R>(dlu, nm, L.max_m, L.max_ne + (H.mixed ? L.max_m : 0), kLuFactor,
                      H.status.as<int>(), st, L.hm.data(), hn.data());
  ck(cudaGetLastError());
  if (!gm.empty()) {
    GemmDesc<R>* dg = stg.push(gm, st);
    gemm_batched<R>(dg, (int)gm.size(), L.max_ne, L.max_ne, R(1), R(1), st,
                    sizeof(R) == 8 ? "gemm_schur<f64>" : "gemm_schur<f32>", schur_flops,
                    schur_bytes);
    ck(cudaGetLastError());
  }
}

void build_all(hps_handle_s& H, const double* const coef_in[6], bool dev_ptrs) {
  Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  const int p = pl.p, pp = p * p, nl = H.nl;
  // precision of each height
  H.levels.clear();
  H.levels.resize(pl.height + 1);
  const int top = std::max(0, H.opt.fp64_top_levels);
  H.leaf_f64 = H.mixed ? 0 : 1;
  for (int h = 1; h <= pl.height; ++h) {
    LevelOps& L = H.levels[h];
    L.f64 = H.mixed ? (h > pl.height - top ? 1 : 0) : 1;
    L.boxes = pl.levels[h];
    const int nm = (int)L.boxes.size();
    L.s_off.assign(nm, 0);
    L.aw_off.assign(nm, 0);
    L.cw_off.assign(nm, 0);
    L.piv_off.assign(nm, 0);
    L.z_off.assign(nm, 0);
    L.hm.assign(nm, 0);
    L.hne.assign(nm, 0);
    int64_t zrows = 0;
    for (int i = 0; i < nm; ++i) {
      const MergeShape& sh = pl.shapes[pl.boxes[L.boxes[i]].shape];
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
  H.u3_off.assign(pl.boxes.size(), -1);
  H.u3_total = 0;
  for (int h = 1; h <= pl.height; ++h)
    for (int b : pl.levels[h]) {
      H.u3_off[b] = H.u3_total;
      H.u3_total += pl.shapes[pl.boxes[b].shape].m;
    }
  // descriptor staging (upper bound of every array pushed below)
  size_t nb = pl.boxes.size();
  Stager stg;
  size_t bytes = stage_bytes<LuDesc<double>>(nl) + 8 * 256;
  for (int h = 1; h <= pl.height; ++h) {
    size_t nm = H.levels[h].boxes.size();
    bytes += stage_bytes<MergeDesc<double>>(nm) + stage_bytes<LuDesc<double>>(nm) +
             stage_bytes<GemmDesc<double>>(nm);
  }
  stg.begin(bytes, st);
  H.keep.begin(stage_bytes<SolveScatterDesc>(nb) + stage_bytes<BodyDesc>(nb) +
                   4 * 256 * (pl.height + 2),
               st);
  // constants, maps, status
  auto up = [&](PoolBuf& b, const void* src, size_t n) {
    b.alloc(n, st);
    if (n) ck(cudaMemcpyAsync(b.p, src, n, cudaMemcpyHostToDevice, st));
  };
  up(H.dD, H.consts.D.data(), H.consts.D.size() * sizeof(double));
  up(H.dPg2c, H.consts.Pg2c.data(), H.consts.Pg2c.size() * sizeof(double));
  up(H.dPc2g, H.consts.Pc2g.data(), H.consts.Pc2g.size() * sizeof(double));
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
    std::vector<int64_t> lo(nl);
    for (int l = 0; l < nl; ++l) lo[l] = pl.boxes[pl.leaf_box[l]].ext_off;
    up(H.leaf_off, lo.data(), lo.size() * sizeof(int64_t));
    ck(cudaStreamSynchronize(st));  // the pageable sources above go out of scope
  }
  H.status.alloc(sizeof(int), st);
  ck(cudaMemsetAsync(H.status.p, 0, sizeof(int), st));
  // coefficients on the device (kept in mixed mode for the FP64 residual)
  PoolBuf coef_tmp;
  {
    int npresent = 0;
    for (int k = 0; k < 6; ++k) npresent += coef_in[k] != nullptr;
    PoolBuf& cb = H.mixed ? H.coef : coef_tmp;
    const bool copy = !dev_ptrs || H.mixed;
    if (copy && npresent) cb.alloc((size_t)npresent * nl * pp * sizeof(double), st);
    int slot = 0;
    for (int k = 0; k < 6; ++k) {
      if (!coef_in[k]) {
        H.coefp[k] = nullptr;
      } else if (!copy) {
        H.coefp[k] = coef_in[k];
      } else {
        double* dst = cb.as<double>() + (size_t)slot * nl * pp;
        ck(cudaMemcpyAsync(dst, coef_in[k], (size_t)nl * pp * sizeof(double),
                           dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        H.coefp[k] = dst;
        ++slot;
      }
    }
  }
  // ---- leaves and merges
  std::vector<TRef> Tref(pl.boxes.size());
  std::vector<std::unique_ptr<PoolBuf>> Tbuf(pl.height + 1);
  for (auto& t : Tbuf) t.reset(new PoolBuf());
  if (H.leaf_f64)
    build_leaves<double>(H, stg, Tref, *Tbuf[0]);
  else
    build_leaves<float>(H, stg, Tref, *Tbuf[0]);
  std::vector<int> last_use(pl.height + 1, -1);
  for (const auto& bx : pl.boxes)
    if (bx.parent >= 0)
      last_use[bx.height] = std::max(last_use[bx.height], pl.boxes[bx.parent].height);
  for (int h = 1; h <= pl.height; ++h) {
    if (H.levels[h].f64)
      build_level<double>(H, h, stg, Tref, *Tbuf[h]);
    else
      build_level<float>(H, h, stg, Tref, *Tbuf[h]);
    for (int hh = 0; hh < h; ++hh)
      if (last_use[hh] == h) Tbuf[hh]->release();
  }
  // ---- solve-side structures that do not depend on nrhs
  for (int h = 1; h <= pl.height; ++h) {
    LevelOps& L = H.levels[h];
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
  int* bad_h = nullptr;
  ck(cudaMallocHost(&bad_h, sizeof(int)));
  *bad_h = 0;
  cudaError_t e1 = cudaMemcpyAsync(bad_h, H.status.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  int bad = *bad_h;
  cudaFreeHost(bad_h);
  ck(e1);
  ck(e2);
  for (auto& t : Tbuf) t->release();
  if (bad) throw bad;
}

// ------------------------------------------------------------------ solve
template <typename R>
void push_down_gemms(hps_handle_s& H, int h, int nrhs) {
  const Plan& pl = H.plan;
  LevelOps& L = H.levels[h];
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
  H.gemm_down[h] = H.solve_st.push(all, H.stream);
  H.down_flops1[h] = fl;
  H.down_bytes[h] = by;
}

template <typename R>
void push_body(hps_handle_s& H, int h, int nrhs) {
  const Plan& pl = H.plan;
  LevelOps& L = H.levels[h];
  std::vector<GemmDesc<R, R, double>> gh;
  std::vector<GemmDesc<R>> gw;
  R* z = H.zlev[h]->as<R>();
  R* r = H.rlev[h]->as<R>();
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
  H.gemm_w[h] = H.solve_st.push(gw, H.stream);
  H.gemm_hpar[h] = H.solve_st.push(gh, H.stream);
}

template <typename R>
void push_leaf_inverse(hps_handle_s& H, int nrhs) {
  std::vector<GemmDesc<R>> g(H.nl);
  const int ni = H.ni;
  for (int l = 0; l < H.nl; ++l) {  // z_l = A_ii^{-1} r_l
    g[l].A = H.Y.as<R>() + (size_t)l * H.ys + (size_t)ni * H.nq;
    g[l].B = H.rleaf.as<R>() + (size_t)l * ni * nrhs;
    g[l].C = H.zleaf.as<R>() + (size_t)l * ni * nrhs;
    g[l].M = ni;
    g[l].N = nrhs;
    g[l].K = ni;
    g[l].lda = ni;
    g[l].ldb = ni;
    g[l].ldc = ni;
  }
  H.gemm_leaf = H.solve_st.push(g, H.stream);
}

void prepare_solve(hps_handle_s& H, int nrhs) {
  if (H.cache_nrhs == nrhs) return;
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  H.cache_nrhs = 0;
  H.uext.alloc((size_t)nrhs * pl.ext_total * sizeof(double), st);
  H.u3.alloc((size_t)nrhs * std::max<int64_t>(H.u3_total, 1) * sizeof(double), st);
  H.split_ws.alloc((size_t)64 << 20, st);
  H.gemm_down.assign(pl.height + 1, nullptr);
  H.gemm_hpar.assign(pl.height + 1, nullptr);
  H.gemm_w.assign(pl.height + 1, nullptr);
  H.down_flops1.assign(pl.height + 1, 0.0);
  H.down_bytes.assign(pl.height + 1, 0.0);
  size_t bytes = 4 * 256 * (pl.height + 2) + stage_bytes<GemmDesc<double>>(H.nl);
  for (int h = 1; h <= pl.height; ++h) bytes += 3 * stage_bytes<GemmDesc<double>>(H.levels[h].boxes.size());
  H.solve_st.begin(bytes, st);
  if (H.mixed) {
    H.hpool.alloc((size_t)nrhs * pl.ext_total * sizeof(double), st);
    const size_t es = H.leaf_f64 ? 8 : 4;
    H.rleaf.alloc((size_t)H.nl * H.ni * nrhs * es, st);
    H.zleaf.alloc((size_t)H.nl * H.ni * nrhs * es, st);
    H.rlev.clear();
    H.zlev.clear();
    for (int h = 0; h <= pl.height; ++h) {
      H.rlev.emplace_back(new PoolBuf());
      H.zlev.emplace_back(new PoolBuf());
      if (h >= 1) {
        const size_t n = (size_t)H.levels[h].sum_m * nrhs * (H.levels[h].f64 ? 8 : 4);
        H.rlev[h]->alloc(n, st);
        H.zlev[h]->alloc(n, st);
      }
    }
    H.maxabs.alloc(2 * sizeof(unsigned long long), st);
    if (!H.h_maxabs) ck(cudaMallocHost(&H.h_maxabs, 2 * sizeof(unsigned long long)));
    if (H.leaf_f64)
      push_leaf_inverse<double>(H, nrhs);
    else
      push_leaf_inverse<float>(H, nrhs);
  }
  for (int h = 1; h <= pl.height; ++h) {
    if (H.levels[h].f64) {
      push_down_gemms<double>(H, h, nrhs);
      if (H.mixed) push_body<double>(H, h, nrhs);
    } else {
      push_down_gemms<float>(H, h, nrhs);
      if (H.mixed) push_body<float>(H, h, nrhs);
    }
  }
  H.cache_nrhs = nrhs;
}

template <typename R>
R* split_ws(hps_handle_s& H, size_t* elems) {
  *elems = H.split_ws.bytes / sizeof(R);
  return H.split_ws.as<R>();
}

// Downward pass (Algorithm 2) from the root exterior values already in uext;
// with_z adds the body-load interface values z of each merge.
template <typename R>
void down_level(hps_handle_s& H, int h, int nrhs, bool with_z) {
  LevelOps& L = H.levels[h];
  cudaStream_t st = H.stream;
  const int nm = (int)L.boxes.size();
  if (with_z)
    z_to_u3<R>(L.body, nm, L.max_m, H.zlev[h]->as<R>(), H.u3.as<double>(), H.u3_total, nrhs, st);
  size_t wse = 0;
  R* ws = split_ws<R>(H, &wse);
  gemm_batched<R>(static_cast<GemmDesc<R, double, double>*>(H.gemm_down[h]), nm, L.max_m, nrhs,
                  R(1), with_z ? R(1) : R(0), st,
                  sizeof(R) == 8 ? "gemm_solve<f64>" : "gemm_solve<f32>",
                  H.down_flops1[h] * nrhs, H.down_bytes[h], L.max_ne, ws, wse);
  solve_child_scatter(L.scatter, nm, L.max_nanb, H.u3.as<double>(), H.u3_total,
                      H.uext.as<double>(), H.plan.ext_total, nrhs, st);
}

void downward(hps_handle_s& H, int nrhs, bool with_z) {
  for (int h = H.plan.height; h >= 1; --h) {
    if (H.levels[h].f64)
      down_level<double>(H, h, nrhs, with_z);
    else
      down_level<float>(H, h, nrhs, with_z);
  }
}

template <typename R>
void leaf_out(hps_handle_s& H, int nrhs, double* u, bool correction) {
  const Plan& pl = H.plan;
  leaf_post<R>(H.Y.as<R>(), H.ys, H.uext.as<double>(), H.leaf_off.as<int64_t>(), pl.ext_total, H.nl,
               pl.p, pl.q, nrhs, H.dPg2c.as<double>(), u, H.stream,
               correction ? H.zleaf.as<R>() : nullptr, correction ? 1 : 0,
               correction ? H.maxabs.as<unsigned long long>() : nullptr);
}

// Leaf part of one refinement step: r = -(A w)_i in FP64, z = A_ii^{-1} r, and
// the leaves' flux offsets h = L4 L3 (w + [0; z]).
template <typename RL>
void leaf_correction_rhs(hps_handle_s& H, int nrhs, const double* u) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  leaf_residual<RL>(H.coefp, H.nl, pl.p, H.hx, H.hy, H.dD.as<double>(), u, nrhs,
                    H.rleaf.as<RL>(), st);
  gemm_batched<RL>(static_cast<GemmDesc<RL>*>(H.gemm_leaf), H.nl, H.ni, nrhs, RL(1), RL(0), st,
                   sizeof(RL) == 8 ? "gemm_leafinv<f64>" : "gemm_leafinv<f32>",
                   2.0 * H.nl * (double)H.ni * H.ni * nrhs, (double)H.nl * H.ni * H.ni * sizeof(RL));
  leaf_flux<RL>(u, H.zleaf.as<RL>(), H.nl, pl.p, pl.q, nrhs, H.hx, H.hy, H.dD.as<double>(),
                H.dPc2g.as<double>(), H.leaf_off.as<int64_t>(), pl.ext_total,
                H.hpool.as<double>(), st);
}

// Merge part of the upward pass: z = W (h3^b - h3^a), h^tau = [h1^a; h2^b] + C z.
template <typename R>
void up_level(hps_handle_s& H, int h, int nrhs) {
  LevelOps& L = H.levels[h];
  cudaStream_t st = H.stream;
  const Plan& pl = H.plan;
  const int nm = (int)L.boxes.size();
  size_t wse = 0;
  R* ws = split_ws<R>(H, &wse);
  merge_rhs<R>(L.body, nm, L.max_m, H.hpool.as<double>(), pl.ext_total, nrhs,
               H.rlev[h]->as<R>(), st);
  double flw = 0, flc = 0;
  for (int i = 0; i < nm; ++i) {
    flw += 2.0 * L.hm[i] * (double)L.hm[i] * nrhs;
    flc += 2.0 * L.hne[i] * (double)L.hm[i] * nrhs;
  }
  gemm_batched<R>(static_cast<GemmDesc<R>*>(H.gemm_w[h]), nm, L.max_m, nrhs, R(1), R(0), st,
                  sizeof(R) == 8 ? "gemm_body<f64>" : "gemm_body<f32>", flw, 0.0, L.max_m, ws,
                  wse);
  if (h < pl.height) {  // the root's flux offsets are not needed
    merge_hpar(L.body, nm, L.max_ne, H.hpool.as<double>(), pl.ext_total, nrhs, st);
    gemm_batched<R>(static_cast<GemmDesc<R, R, double>*>(H.gemm_hpar[h]), nm, L.max_ne, nrhs,
                    R(1), R(1), st, sizeof(R) == 8 ? "gemm_body<f64>" : "gemm_body<f32>", flc,
                    0.0, L.max_m, ws, wse);
  }
}

int solve_all(hps_handle_s& H, const double* f_dev, int nrhs, double* u_dev,
              hps_solve_info* info) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  prepare_solve(H, nrhs);
  solve_root_scatter(f_dev, H.root_from_f.as<int>(), H.nbnd, nrhs, H.uext.as<double>(),
                     pl.boxes[0].ext_off, pl.ext_total, st);
  downward(H, nrhs, false);
  if (H.leaf_f64)
    leaf_out<double>(H, nrhs, u_dev, false);
  else
    leaf_out<float>(H, nrhs, u_dev, false);
  ck(cudaGetLastError());
  if (!H.mixed || H.opt.max_refine == 0) return HPS_OK;
  // ---- iterative refinement against the FP64 residual
  double last = 0.0;
  int it = 0;
  for (it = 1; it <= H.opt.max_refine; ++it) {
    if (H.leaf_f64)
      leaf_correction_rhs<double>(H, nrhs, u_dev);
    else
      leaf_correction_rhs<float>(H, nrhs, u_dev);
    for (int h = 1; h <= pl.height; ++h) {
      if (H.levels[h].f64)
        up_level<double>(H, h, nrhs);
      else
        up_level<float>(H, h, nrhs);
    }
    // the correction has zero Dirichlet data on Gamma
    ck(cudaMemset2DAsync(H.uext.as<double>() + pl.boxes[0].ext_off, pl.ext_total * sizeof(double),
                         0, pl.boxes[0].ne * sizeof(double), nrhs, st));
    downward(H, nrhs, true);
    ck(cudaMemsetAsync(H.maxabs.p, 0, 2 * sizeof(unsigned long long), st));
    if (H.leaf_f64)
      leaf_out<double>(H, nrhs, u_dev, true);
    else
      leaf_out<float>(H, nrhs, u_dev, true);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(H.h_maxabs, H.maxabs.p, 2 * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    double dmax, umax;
    std::memcpy(&dmax, &H.h_maxabs[0], sizeof(double));
    std::memcpy(&umax, &H.h_maxabs[1], sizeof(double));
    const double prev = last;
    last = umax > 0 ? dmax / umax : dmax;
    if (!(last <= 1.0)) break;  // NaN or divergence
    if (last <= H.opt.refine_tol) break;
    // stagnation: the update no longer shrinks, i.e. the iterate has reached
    // the accuracy the FP64 residual can resolve for this conditioning
    if (it >= 3 && last > 0.5 * prev) break;
  }
  if (info) {
    info->iterations = std::min(it, H.opt.max_refine);
    info->last_update = last;
  }
  if (!(last <= H.opt.refine_tol)) {
    if (info) info->status = HPS_ENOTCONVERGED;
    return HPS_ENOTCONVERGED;
  }
  return HPS_OK;
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
              const hps_options* opt_in, hps_handle* out) {
  if (!out) return HPS_EINVAL;
  *out = nullptr;
  int v = validate(d, nx, ny, p, q);
  if (v != HPS_OK) return v;
  hps_options opt;
  hps_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.precision != HPS_FP64 && opt.precision != HPS_MIXED) return HPS_EINVAL;
  if (opt.precision == HPS_MIXED &&
      (!(opt.refine_tol > 0) || opt.max_refine < 0 || opt.fp64_top_levels < 0))
    return HPS_EINVAL;
  g_last_error.clear();
  hps_handle_s* H = nullptr;
  try {
    H = new hps_handle_s();
    H->opt = opt;
    H->mixed = opt.precision == HPS_MIXED;
    H->plan = make_plan(d.x0, d.x1, d.y0, d.y1, nx, ny, p, q);
    H->consts = make_consts(p, q);
    H->ni = (p - 2) * (p - 2);
    H->nq = 4 * q;
    H->nl = nx * ny;
    H->nbnd = 2 * (nx + ny) * q;
    H->hx = (d.x1 - d.x0) / nx;
    H->hy = (d.y1 - d.y0) / ny;
    if (opt.stream) {
      H->stream = (cudaStream_t)opt.stream;
    } else {
      ck(cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking));
      H->own_stream = true;
    }
    const double* coef[6] = {c11, c12, c22, c1, c2, c};
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

int hps_boundary_nodes(hps_handle h, double* xy) {
  if (!h || !xy) return HPS_EINVAL;
  const Plan& pl = h->plan;
  boundary_node_coords(pl.x0, pl.x1, pl.y0, pl.y1, pl.nx, pl.ny, pl.q, xy);
  return HPS_OK;
}

int hps_solve_ex(hps_handle h, const double* f, int nrhs, double* u, int device_ptrs,
                 hps_solve_info* info) {
  if (info) {
    info->status = HPS_OK;
    info->iterations = 0;
    info->last_update = 0.0;
    info->bad_box = -1;
  }
  if (!h || !f || !u || nrhs < 1) return HPS_EINVAL;
  g_last_error.clear();
  try {
    hps_handle_s& H = *h;
    cudaStream_t st = H.stream;
    const size_t fb = (size_t)nrhs * H.nbnd * sizeof(double);
    const size_t ub = (size_t)nrhs * H.nl * H.plan.p * H.plan.p * sizeof(double);
    const double* fd = f;
    double* ud = u;
    if (!device_ptrs) {
      if (H.fstage.bytes < fb) H.fstage.alloc(fb, st);
      if (H.ustage.bytes < ub) H.ustage.alloc(ub, st);
      ck(cudaMemcpyAsync(H.fstage.p, f, fb, cudaMemcpyHostToDevice, st));
      fd = H.fstage.as<double>();
      ud = H.ustage.as<double>();
    }
    int rc = solve_all(H, fd, nrhs, ud, info);
    if (!device_ptrs) ck(cudaMemcpyAsync(u, ud, ub, cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    return rc;
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

int hps_solve(hps_handle h, const double* f, int nrhs, double* u, hps_solve_info* info) {
  if (!h) return HPS_EINVAL;
  return hps_solve_ex(h, f, nrhs, u, h->opt.device_ptrs, info);
}

int hps_query(hps_handle h, int* n_leaves, int* p, int* q, int64_t* nbnd, int64_t* device_bytes) {
  if (!h) return HPS_EINVAL;
  if (n_leaves) *n_leaves = h->nl;
  if (p) *p = h->plan.p;
  if (q) *q = h->plan.q;
  if (nbnd) *nbnd = h->nbnd;
  if (device_bytes) {
    int64_t b = 0;
    for (const PoolBuf* x : {&h->Y, &h->coef, &h->maps, &h->uext, &h->u3, &h->hpool, &h->rleaf,
                             &h->zleaf, &h->fstage, &h->ustage, &h->split_ws, &h->keep.dev,
                             &h->solve_st.dev})
      b += (int64_t)x->bytes;
    for (const auto& L : h->levels) b += (int64_t)(L.S->bytes + L.Cw->bytes);
    for (const auto& z : h->zlev) b += (int64_t)z->bytes;
    for (const auto& r : h->rlev) b += (int64_t)r->bytes;
    *device_bytes = b;
  }
  return HPS_OK;
}

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

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
alignas(256) unsigned char g_static_host[kStaticHostBytes];
std::mutex g_static_mu;
void* g_static_dev[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int hps_solve_static(hps_handle h, const double* f, int nrhs, double* u) {
  if (!h || !f || !u || nrhs < 1) return HPS_EINVAL;
  g_last_error.clear();
  hps_handle_s& H = *h;
  if (H.mixed) {
    g_last_error = "hps_solve_static: only FP64 handles (mixed handles refine with more buffers)";
    return HPS_EINVAL;
  }
  const Plan& pl = H.plan;
  // carve the static array: exterior-value pool, u3 pool, GEMM descriptors
  const size_t b_uext = align256((size_t)nrhs * pl.ext_total * sizeof(double));
  const size_t b_u3 = align256((size_t)nrhs * std::max<int64_t>(H.u3_total, 1) * sizeof(double));
  size_t b_desc = 0;
  for (int hh = 1; hh <= pl.height; ++hh)
    b_desc += align256(H.levels[hh].boxes.size() * sizeof(GemmDesc<double>));
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
    // descriptors of the downward GEMMs, staged in static host memory; the
    // earlier call's copies have completed (each call ends synchronised)
    GemmDesc<double>* dptr[128] = {};  // tree heights stay far below 128 (nx * ny <= 2^26)
    if (pl.height >= 128) return HPS_EINVAL;
    size_t off = 0;
    for (int hh = 1; hh <= pl.height; ++hh) {
      LevelOps& L = H.levels[hh];
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
      const size_t n = L.boxes.size() * sizeof(GemmDesc<double>);
      ck(cudaMemcpyAsync(dd + off, g_static_host + off, n, cudaMemcpyHostToDevice, st));
      dptr[hh] = reinterpret_cast<GemmDesc<double>*>(dd + off);
      off += align256(n);
    }
    // nothing in the array has to start at zero: every exterior value and every
    // u3 entry is written (root scatter, GEMMs with beta = 0, child scatters)
    // before it is read
    solve_root_scatter(f, H.root_from_f.as<int>(), H.nbnd, nrhs, uext, pl.boxes[0].ext_off,
                       pl.ext_total, st);
    for (int hh = pl.height; hh >= 1; --hh) {
      LevelOps& L = H.levels[hh];
      const int nm = (int)L.boxes.size();
      gemm_batched<double>(dptr[hh], nm, L.max_m, nrhs, 1.0, 0.0, st, "gemm_solve_static<f64>",
                           0.0, 0.0);
      solve_child_scatter(L.scatter, nm, L.max_nanb, u3, H.u3_total, uext, pl.ext_total, nrhs, st);
    }
    leaf_post<double>(H.Y.as<double>(), H.ys, uext, H.leaf_off.as<int64_t>(), pl.ext_total, H.nl,
                      pl.p, pl.q, nrhs, H.dPg2c.as<double>(), u, st);
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
