// C ABI of libhps: the build stage (Algorithm 1) and the solve stage
// (Algorithm 2 + Section 4.3) orchestrated over the batched kernels.
//
// Build, per tree height h (h = 0: the leaves):
//   h = 0   leaf_assemble -> batched LU of [A_ii | -A_ie L1] -> Y, leaf_dtn -> T
//   h >= 1  merge_gather  -> batched LU of [T33^a - T33^b | -T31^a, T32^b] -> S
//           GEMM Tp += [T13^a; T23^b] S  (eq. merge; skipped at the root unless
//           the root DtN is requested: the solve never needs it)
// The children's T are released once every parent that reads them is built.
// Solve: root exterior values from f, then per height from the top a batched
// GEMM u3 = S u_parent and a scatter into the children's exterior vectors,
// then the leaf post-process w_full = [L1 ; Y] u_e.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "../../include/hps.h"
#include "hps_internal.hpp"
#include "hps_kernels.cuh"

using namespace hps;

namespace {

struct CudaError {
  cudaError_t err;
};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaError{e};
}

// Device allocation that is released with its owner.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  void alloc(size_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (n == 0) return;
    ck(cudaMalloc(&p, n));
    bytes = n;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

template <typename T>
void upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  b.alloc(v.size() * sizeof(T));
  if (!v.empty()) ck(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

}  // namespace

struct hps_handle_s {
  Plan plan;
  Consts consts;
  hps_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int ni = 0, nq = 0, nl = 0, nbnd = 0;
  // constants on the device
  DevBuf dD, dPg2c, dPc2g;
  // operators kept for the solve
  DevBuf Y;                       // nl * ni * nq, FP64
  DevBuf S;                       // all merges' S, FP64
  std::vector<int64_t> S_off;     // per box (parents), element offset into S
  // index maps on the device
  DevBuf maps;                    // src / cmap_a / cmap_b of every shape
  std::vector<int64_t> src_off, cma_off, cmb_off;
  DevBuf root_from_f, leaf_ext_off;
  // solve structures
  std::vector<int64_t> u3_off;    // per box (parents)
  int64_t u3_total = 0;
  std::vector<std::unique_ptr<DevBuf>> solve_scatter;  // per height
  std::vector<int> solve_max_n;
  DevBuf solve_gemm;              // all heights' GEMM descriptors
  std::vector<int> gemm_first, gemm_count, gemm_maxM;
  int gemm_nrhs = -1;
  DevBuf uext, u3, fstage, ustage;
  int ws_nrhs = 0;
  size_t fstage_bytes = 0, ustage_bytes = 0;
  DevBuf status;
  int64_t persistent_bytes = 0;
  ~hps_handle_s() {
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

int validate(hps_domain d, int nx, int ny, int p, int q) {
  if (nx < 1 || ny < 1 || p < 3 || q < 1 || q > p) return HPS_EINVAL;
  if (!(d.x1 > d.x0) || !(d.y1 > d.y0) || !std::isfinite(d.x0) || !std::isfinite(d.x1) ||
      !std::isfinite(d.y0) || !std::isfinite(d.y1))
    return HPS_EINVAL;
  if (p > 64 || (int64_t)nx * ny > (1 << 26)) return HPS_EINVAL;
  return HPS_OK;
}

// ------------------------------------------------------------------ build
void build_fp64(hps_handle_s& H, const double* const coef_in[6], bool dev_ptrs) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  const int p = pl.p, q = pl.q, pp = p * p, ni = H.ni, nq = H.nq, nl = H.nl;
  const double hx = (pl.x1 - pl.x0) / pl.nx, hy = (pl.y1 - pl.y0) / pl.ny;
  // constants
  upload(H.dD, H.consts.D, st);
  upload(H.dPg2c, H.consts.Pg2c, st);
  upload(H.dPc2g, H.consts.Pc2g, st);
  H.status.alloc(sizeof(int));
  ck(cudaMemsetAsync(H.status.p, 0, sizeof(int), st));
  // coefficients on the device
  DevBuf coefbuf;
  const double* coef[6];
  {
    int npresent = 0;
    for (int k = 0; k < 6; ++k) npresent += coef_in[k] != nullptr;
    if (!dev_ptrs && npresent) coefbuf.alloc((size_t)npresent * nl * pp * sizeof(double));
    int slot = 0;
    for (int k = 0; k < 6; ++k) {
      if (!coef_in[k]) {
        coef[k] = nullptr;
      } else if (dev_ptrs) {
        coef[k] = coef_in[k];
      } else {
        double* dst = coefbuf.as<double>() + (size_t)slot * nl * pp;
        ck(cudaMemcpyAsync(dst, coef_in[k], (size_t)nl * pp * sizeof(double),
                           cudaMemcpyHostToDevice, st));
        coef[k] = dst;
        ++slot;
      }
    }
  }
  // index maps
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
    upload(H.maps, all, st);
    upload(H.root_from_f, pl.root_from_f, st);
    std::vector<int64_t> lo(nl);
    for (int l = 0; l < nl; ++l) lo[l] = pl.boxes[pl.leaf_box[l]].ext_off;
    upload(H.leaf_ext_off, lo, st);
  }
  // ---- leaves
  H.Y.alloc((size_t)nl * ni * nq * sizeof(double));
  std::vector<const double*> Tptr(pl.boxes.size(), nullptr);
  std::vector<std::unique_ptr<DevBuf>> Tbuf(pl.height + 1);
  {
    DevBuf Aii, piv, desc;
    Aii.alloc((size_t)nl * ni * ni * sizeof(double));
    piv.alloc((size_t)nl * ni * sizeof(int));
    leaf_assemble<double>(coef, nl, p, q, hx, hy, H.dD.as<double>(), H.dPg2c.as<double>(),
                          Aii.as<double>(), H.Y.as<double>(), st);
    ck(cudaGetLastError());
    std::vector<LuDesc<double>> ld(nl);
    for (int l = 0; l < nl; ++l) {
      ld[l].A = Aii.as<double>() + (size_t)l * ni * ni;
      ld[l].ipiv = piv.as<int>() + (size_t)l * ni;
      ld[l].B = H.Y.as<double>() + (size_t)l * ni * nq;
      ld[l].m = ni;
      ld[l].lda = ni;
      ld[l].nrhs = nq;
      ld[l].ldb = ni;
      ld[l].box = pl.leaf_box[l];
    }
    upload(desc, ld, st);
    lu_solve_batched<double>(desc.as<LuDesc<double>>(), nl, ni, nq, false, H.status.as<int>(), st);
    ck(cudaGetLastError());
    Tbuf[0].reset(new DevBuf());
    Tbuf[0]->alloc((size_t)nl * nq * nq * sizeof(double));
    leaf_dtn<double>(H.Y.as<double>(), nl, p, q, hx, hy, H.dD.as<double>(), H.dPg2c.as<double>(),
                     H.dPc2g.as<double>(), Tbuf[0]->as<double>(), st);
    ck(cudaGetLastError());
    for (int l = 0; l < nl; ++l) Tptr[pl.leaf_box[l]] = Tbuf[0]->as<double>() + (size_t)l * nq * nq;
    ck(cudaStreamSynchronize(st));  // Aii / piv / desc are released at scope exit
  }
  // ---- merges
  // S storage for every parent, laid out by height
  int64_t s_total = 0;
  H.S_off.assign(pl.boxes.size(), -1);
  H.u3_off.assign(pl.boxes.size(), -1);
  H.u3_total = 0;
  for (int h = 1; h <= pl.height; ++h)
    for (int b : pl.levels[h]) {
      const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
      H.S_off[b] = s_total;
      s_total += (int64_t)sh.m * sh.ne;
      H.u3_off[b] = H.u3_total;
      H.u3_total += sh.m;
    }
  H.S.alloc((size_t)s_total * sizeof(double));
  // last height that reads the T of boxes of height h
  std::vector<int> last_use(pl.height + 1, -1);
  for (const auto& bx : pl.boxes)
    if (bx.parent >= 0)
      last_use[bx.height] = std::max(last_use[bx.height], pl.boxes[bx.parent].height);
  const bool form_root = H.opt.form_root_dtn != 0;
  for (int h = 1; h <= pl.height; ++h) {
    const auto& lev = pl.levels[h];
    const int nm = (int)lev.size();
    int64_t aw_tot = 0, cw_tot = 0, tp_tot = 0, piv_tot = 0;
    int max_m = 0, max_ne = 0;
    int64_t max_work = 0;
    for (int b : lev) {
      const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
      const bool tp = (b != 0) || form_root;
      aw_tot += (int64_t)sh.m * sh.m;
      cw_tot += (int64_t)sh.ne * sh.m;
      tp_tot += tp ? (int64_t)sh.ne * sh.ne : 0;
      piv_tot += sh.m;
      max_m = std::max(max_m, sh.m);
      max_ne = std::max(max_ne, sh.ne);
      max_work = std::max<int64_t>(max_work, (int64_t)sh.m * sh.m + 2LL * sh.m * sh.ne +
                                        (tp ? (int64_t)sh.ne * sh.ne : 0));
    }
    DevBuf Aw, Cw, piv, mdesc, ldesc, gdesc;
    Aw.alloc((size_t)aw_tot * sizeof(double));
    Cw.alloc((size_t)cw_tot * sizeof(double));
    piv.alloc((size_t)piv_tot * sizeof(int));
    Tbuf[h].reset(new DevBuf());
    Tbuf[h]->alloc((size_t)tp_tot * sizeof(double));
    std::vector<MergeDesc<double, double>> md(nm);
    std::vector<LuDesc<double>> lu(nm);
    std::vector<GemmDesc<double>> gm;
    int64_t oa = 0, oc = 0, ot = 0, op = 0;
    for (int i = 0; i < nm; ++i) {
      const int b = lev[i];
      const Box& B = pl.boxes[b];
      const MergeShape& sh = pl.shapes[B.shape];
      const bool tp = (b != 0) || form_root;
      MergeDesc<double, double>& g = md[i];
      g.Ta = Tptr[B.child[0]];
      g.Tb = Tptr[B.child[1]];
      g.Aw = Aw.as<double>() + oa;
      g.S = H.S.as<double>() + H.S_off[b];
      g.Cw = Cw.as<double>() + oc;
      g.Tp = tp ? Tbuf[h]->as<double>() + ot : nullptr;
      g.src = H.maps.as<int>() + H.src_off[B.shape];
      g.na = sh.na;
      g.nb = sh.nb;
      g.m = sh.m;
      g.ne = sh.ne;
      g.j3a = sh.j3a;
      g.j3b = sh.j3b;
      lu[i].A = g.Aw;
      lu[i].ipiv = piv.as<int>() + op;
      lu[i].B = g.S;
      lu[i].m = sh.m;
      lu[i].lda = sh.m;
      lu[i].nrhs = sh.ne;
      lu[i].ldb = sh.m;
      lu[i].box = b;
      if (tp) {
        GemmDesc<double> gg;
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
        Tptr[b] = g.Tp;
      }
      oa += (int64_t)sh.m * sh.m;
      oc += (int64_t)sh.ne * sh.m;
      ot += tp ? (int64_t)sh.ne * sh.ne : 0;
      op += sh.m;
    }
    upload(mdesc, md, st);
    upload(ldesc, lu, st);
    merge_gather<double, double>(mdesc.as<MergeDesc<double, double>>(), nm, max_work, st);
    ck(cudaGetLastError());
    lu_solve_batched<double>(ldesc.as<LuDesc<double>>(), nm, max_m, max_ne, false,
                             H.status.as<int>(), st);
    ck(cudaGetLastError());
    if (!gm.empty()) {
      upload(gdesc, gm, st);
      gemm_batched<double>(gdesc.as<GemmDesc<double>>(), (int)gm.size(), max_ne, max_ne, 1.0, 1.0,
                           st);
      ck(cudaGetLastError());
    }
    ck(cudaStreamSynchronize(st));  // level workspaces are released at scope exit
    for (int hh = 0; hh < h; ++hh)
      if (last_use[hh] == h && Tbuf[hh]) Tbuf[hh].reset();
  }
  // ---- solve-side structures
  H.solve_scatter.clear();
  for (int h = 0; h <= pl.height; ++h) H.solve_scatter.emplace_back(new DevBuf());
  H.solve_max_n.assign(pl.height + 1, 0);
  for (int h = 1; h <= pl.height; ++h) {
    std::vector<SolveScatterDesc> sd;
    for (int b : pl.levels[h]) {
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
      H.solve_max_n[h] = std::max(H.solve_max_n[h], sh.na + sh.nb);
    }
    upload(*H.solve_scatter[h], sd, st);
  }
  ck(cudaStreamSynchronize(st));
  int bad = 0;
  ck(cudaMemcpy(&bad, H.status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) throw bad;
}

// ------------------------------------------------------------------ solve
void ensure_workspace(hps_handle_s& H, int nrhs) {
  if (nrhs <= H.ws_nrhs) return;
  H.uext.alloc((size_t)nrhs * H.plan.ext_total * sizeof(double));
  H.u3.alloc((size_t)nrhs * std::max<int64_t>(H.u3_total, 1) * sizeof(double));
  H.ws_nrhs = nrhs;
  H.gemm_nrhs = -1;
}

void prepare_solve_gemms(hps_handle_s& H, int nrhs) {
  if (H.gemm_nrhs == nrhs) return;
  const Plan& pl = H.plan;
  std::vector<GemmDesc<double>> all;
  H.gemm_first.assign(pl.height + 1, 0);
  H.gemm_count.assign(pl.height + 1, 0);
  H.gemm_maxM.assign(pl.height + 1, 0);
  for (int h = 1; h <= pl.height; ++h) {
    H.gemm_first[h] = (int)all.size();
    for (int b : pl.levels[h]) {
      const MergeShape& sh = pl.shapes[pl.boxes[b].shape];
      GemmDesc<double> g;
      g.A = H.S.as<double>() + H.S_off[b];
      g.B = H.uext.as<double>() + pl.boxes[b].ext_off;
      g.C = H.u3.as<double>() + H.u3_off[b];
      g.M = sh.m;
      g.N = nrhs;
      g.K = sh.ne;
      g.lda = sh.m;
      g.ldb = (int)pl.ext_total;
      g.ldc = (int)H.u3_total;
      all.push_back(g);
      H.gemm_maxM[h] = std::max(H.gemm_maxM[h], sh.m);
    }
    H.gemm_count[h] = (int)all.size() - H.gemm_first[h];
  }
  upload(H.solve_gemm, all, H.stream);
  H.gemm_nrhs = nrhs;
}

void solve_fp64(hps_handle_s& H, const double* f_dev, int nrhs, double* u_dev) {
  const Plan& pl = H.plan;
  cudaStream_t st = H.stream;
  ensure_workspace(H, nrhs);
  prepare_solve_gemms(H, nrhs);
  solve_root_scatter(f_dev, H.root_from_f.as<int>(), H.nbnd, nrhs, H.uext.as<double>(),
                     pl.boxes[0].ext_off, pl.ext_total, st);
  for (int h = pl.height; h >= 1; --h) {
    gemm_batched<double>(H.solve_gemm.as<GemmDesc<double>>() + H.gemm_first[h], H.gemm_count[h],
                         H.gemm_maxM[h], nrhs, 1.0, 0.0, st);
    solve_child_scatter(H.solve_scatter[h]->as<SolveScatterDesc>(), (int)pl.levels[h].size(),
                        H.solve_max_n[h], H.u3.as<double>(), H.u3_total, H.uext.as<double>(),
                        pl.ext_total, nrhs, st);
  }
  leaf_post<double>(H.Y.as<double>(), H.uext.as<double>(), H.leaf_ext_off.as<int64_t>(),
                    pl.ext_total, H.nl, pl.p, pl.q, nrhs, H.dPg2c.as<double>(), u_dev, st);
  ck(cudaGetLastError());
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
  if (validate(d, nx, ny, std::max(q, 3), q) != HPS_OK || !xy) return HPS_EINVAL;
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
  if (opt.precision == HPS_MIXED) return HPS_EINVAL;  // not available in this build
  hps_handle_s* H = nullptr;
  try {
    H = new hps_handle_s();
    H->opt = opt;
    H->plan = make_plan(d.x0, d.x1, d.y0, d.y1, nx, ny, p, q);
    H->consts = make_consts(p, q);
    H->ni = (p - 2) * (p - 2);
    H->nq = 4 * q;
    H->nl = nx * ny;
    H->nbnd = 2 * (nx + ny) * q;
    if (opt.stream) {
      H->stream = (cudaStream_t)opt.stream;
    } else {
      ck(cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking));
      H->own_stream = true;
    }
    const double* coef[6] = {c11, c12, c22, c1, c2, c};
    build_fp64(*H, coef, opt.device_ptrs != 0);
    *out = H;
    return HPS_OK;
  } catch (CudaError& e) {
    delete H;
    return e.err == cudaErrorMemoryAllocation ? HPS_ENOMEM : HPS_EDEVICE;
  } catch (int) {
    delete H;
    return HPS_ESINGULAR;
  } catch (std::bad_alloc&) {
    delete H;
    return HPS_ENOMEM;
  } catch (...) {
    delete H;
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
  try {
    hps_handle_s& H = *h;
    cudaStream_t st = H.stream;
    const size_t fb = (size_t)nrhs * H.nbnd * sizeof(double);
    const size_t ub = (size_t)nrhs * H.nl * H.plan.p * H.plan.p * sizeof(double);
    const double* fd = f;
    double* ud = u;
    if (!device_ptrs) {
      if (H.fstage_bytes < fb) {
        H.fstage.alloc(fb);
        H.fstage_bytes = fb;
      }
      if (H.ustage_bytes < ub) {
        H.ustage.alloc(ub);
        H.ustage_bytes = ub;
      }
      ck(cudaMemcpyAsync(H.fstage.p, f, fb, cudaMemcpyHostToDevice, st));
      fd = H.fstage.as<double>();
      ud = H.ustage.as<double>();
    }
    solve_fp64(H, fd, nrhs, ud);
    if (!device_ptrs) ck(cudaMemcpyAsync(u, ud, ub, cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    return HPS_OK;
  } catch (CudaError& e) {
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
    int64_t b = (int64_t)(h->Y.bytes + h->S.bytes + h->maps.bytes + h->uext.bytes + h->u3.bytes +
                          h->fstage.bytes + h->ustage.bytes + h->solve_gemm.bytes);
    for (auto& s : h->solve_scatter) b += (int64_t)s->bytes;
    *device_bytes = b;
  }
  return HPS_OK;
}

int hps_free(hps_handle h) {
  if (!h) return HPS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  delete h;
  return HPS_OK;
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
