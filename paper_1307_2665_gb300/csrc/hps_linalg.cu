// Batched dense linear algebra for the leaf eliminations (eq. leaf_solve) and
// the merge factorisations (eq. U_parent): right-looking blocked LU with
// partial pivoting applied to the augmented system [A | B], then blocked
// backward substitution, and a tiled batched GEMM for every rank-nb update and
// for the Schur-complement products of eq. merge.
//
// Every kernel walks an array of per-problem descriptors, so one launch covers
// all leaves or all merges of a tree level (of one or of many problems).
//
// Panel factorisation: one CTA per matrix; the panel (rows k0..m-1, nb columns)
// is staged in shared memory when it fits, the pivot search is a warp-shuffle
// argmax, and the scale + rank-1 update of each column is fused.  Row swaps and
// the unit-lower triangular solve of the block row run one warp per column with
// the block row held in registers (lane = row).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <cstdint>
#include <cstdio>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"

namespace hps {

constexpr int kNB = 32;  // panel width == warp width (lane = row of the block row)
constexpr int kTrsmCols = 64;  // columns (threads) per CTA of the diagonal-block solve

template <typename R>
struct TName;
template <>
struct TName<double> {
  static const char* panel() { return "lu_panel<f64>"; }
  static const char* swap() { return "lu_swap_trsm<f64>"; }
  static const char* update() { return "lu_update<f64>"; }
  static const char* trsm() { return "trsm_upper<f64>"; }
  static const char* backsub() { return "backsub_update<f64>"; }
};
template <>
struct TName<float> {
  static const char* panel() { return "lu_panel<f32>"; }
  static const char* swap() { return "lu_swap_trsm<f32>"; }
  static const char* update() { return "lu_update<f32>"; }
  static const char* trsm() { return "trsm_upper<f32>"; }
  static const char* backsub() { return "backsub_update<f32>"; }
};

// ------------------------------------------------------------------- GEMM tile
// C[m0:m0+BM, n0:n0+BN] = beta C + alpha A[m0:, 0:K] B[0:K, n0:], computed in R.
// A, B and C may have other element types (converted on load and store).
// Threads: (BM/TM) x (BN/TN); thread t covers TM consecutive rows and TN
// consecutive columns, the column-tile index varying fastest, so one warp owns
// a contiguous band of rows and a ragged tail of rows idles whole warps (no
// FMAs on padding rows: the FP64 kernels are DFMA-bound).  The epilogue moves
// each thread's TM rows of a column as 16-byte vectors when aligned, so the
// adjacent row groups of a warp fill whole 32-byte sectors.
// Pipelining: the K tiles are double-buffered in shared memory; the global
// loads of tile k+1 are issued into registers before the FMAs of tile k and
// stored after them, so one __syncthreads per K tile and the load latency
// overlaps the arithmetic.  Every element's FMA chain runs over k in order,
// whatever the tile shape or the launch.
template <typename R, int BM_, int BN_, int BK_, int TM_, int TN_>
struct Tile {
  static constexpr int BM = BM_, BN = BN_, BK = BK_, TM = TM_, TN = TN_;
  static constexpr int NTN = BN / TN;
  static constexpr int NTM = BM / TM;
  static constexpr int NT = NTN * NTM;
  static constexpr int LA = BM * BK / NT;  // A elements per thread and K tile
  static constexpr int LB = BK * BN / NT;  // B elements per thread and K tile
  // FP32 tiles of 4k x 4k per thread read their A and B values as float4
  static constexpr bool kVec = sizeof(R) == 4 && TM % 4 == 0 && TN % 4 == 0;
  // padded row of the B stage: the transposed store of a column hits distinct
  // banks (a multiple of 4 for the vector reads)
  static constexpr int BNP = kVec ? BN + 4 : BN + 1;
  static constexpr int STAGE = BK * BM + BK * BNP;
  static constexpr int SMEM = 2 * STAGE * (int)sizeof(R);
  static_assert(BM * BK % NT == 0 && BK * BN % NT == 0, "tile loads must divide evenly");

  // 4 consecutive elements of one column (16-byte aligned)
  __device__ static void load4(const float* cp, float* v) {
    const float4 q = *reinterpret_cast<const float4*>(cp);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  }
  __device__ static void load4(const double* cp, double* v) {
    const double2 lo = reinterpret_cast<const double2*>(cp)[0];
    const double2 hi = reinterpret_cast<const double2*>(cp)[1];
    v[0] = lo.x;
    v[1] = lo.y;
    v[2] = hi.x;
    v[3] = hi.y;
  }
  __device__ static void save4(float* cp, const float* v) {
    *reinterpret_cast<float4*>(cp) = make_float4(v[0], v[1], v[2], v[3]);
  }
  __device__ static void save4(double* cp, const double* v) {
    reinterpret_cast<double2*>(cp)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(cp)[1] = make_double2(v[2], v[3]);
  }

  template <typename TA, typename TB, typename TC>
  __device__ static void run(int M, int N, int K, R alpha, const TA* __restrict__ A, int lda,
                             const TB* B, int ldb, R beta, TC* C, int ldc, int m0, int n0, R* sm) {
    const int t = threadIdx.x;
    const int tn = t % NTN, tm = t / NTN;
    const int r0 = tm * TM, c0 = tn * TN;
    // first row of this warp's band; the band is idle when it starts past M
    const bool warp_live = (m0 + (((t / 32) * 32) / NTN) * TM) < M;
    R acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = R(0);
    R ra[LA], rb[LB];
    auto gload = [&](int k0) {
#pragma unroll
      for (int l = 0; l < LA; ++l) {
        const int e = t + l * NT, i = e % BM, k = e / BM;
        const int gi = m0 + i, gk = k0 + k;
        ra[l] = (gi < M && gk < K) ? (R)A[gi + (size_t)gk * lda] : R(0);
      }
#pragma unroll
      for (int l = 0; l < LB; ++l) {
        const int e = t + l * NT, k = e % BK, j = e / BK;
        const int gk = k0 + k, gj = n0 + j;
        rb[l] = (gk < K && gj < N) ? (R)B[gk + (size_t)gj * ldb] : R(0);
      }
    };
    auto sstore = [&](R* st) {
#pragma unroll
      for (int l = 0; l < LA; ++l) {
        const int e = t + l * NT;
        st[e] = ra[l];  // [k][i], i = e % BM, k = e / BM
      }
#pragma unroll
      for (int l = 0; l < LB; ++l) {
        const int e = t + l * NT;
        st[BK * BM + (e % BK) * BNP + e / BK] = rb[l];
      }
    };
    if (K > 0) {
      gload(0);
      sstore(sm);
    }
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
      const bool more = k0 + BK < K;
      if (more) gload(k0 + BK);
      const R* As = sm + buf * STAGE;
      const R* Bs = As + BK * BM;
#pragma unroll 4
      for (int k = 0; k < (warp_live ? BK : 0); ++k) {
        R a[TM], b[TN];
        if constexpr (kVec) {
#pragma unroll
          for (int i = 0; i < TM; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(As + k * BM + r0 + i);
            a[i] = v.x;
            a[i + 1] = v.y;
            a[i + 2] = v.z;
            a[i + 3] = v.w;
          }
#pragma unroll
          for (int j = 0; j < TN; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(Bs + k * BNP + c0 + j);
            b[j] = v.x;
            b[j + 1] = v.y;
            b[j + 2] = v.z;
            b[j + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[k * BM + r0 + i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = Bs[k * BNP + c0 + j];
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (more) sstore(sm + (buf ^ 1) * STAGE);
      __syncthreads();
      buf ^= 1;
    }
    const int gi0 = m0 + r0;
    if (gi0 >= M) return;
    // the C values of kJB columns are all loaded before any of them is stored:
    // for all the compiler knows the stores alias the loads, which would
    // otherwise cost one memory round trip per column (kJB caps the values
    // held at 128 bytes per thread)
    constexpr int kJB0 = 128 / (TM * (int)sizeof(TC));
    constexpr int kJB = kJB0 < 1 ? 1 : (kJB0 > TN ? TN : kJB0);
    static_assert(TN % kJB == 0, "column batches divide the tile");
    const bool rows_in = gi0 + TM <= M;
    auto vec_ok = [&](const TC* cp) {
      return TM % 4 == 0 && rows_in && (reinterpret_cast<uintptr_t>(cp) & 15) == 0;
    };
#pragma unroll
    for (int j0 = 0; j0 < TN; j0 += kJB) {
      TC cv[kJB][TM];
      if (beta != R(0)) {
#pragma unroll
        for (int jj = 0; jj < kJB; ++jj) {
          const int gj = n0 + c0 + j0 + jj;
          const TC* cp = C + gi0 + (size_t)gj * ldc;
          if (gj < N && vec_ok(cp)) {
#pragma unroll
            for (int i = 0; i < TM; i += 4) load4(cp + i, &cv[jj][i]);
          } else {
#pragma unroll
            for (int i = 0; i < TM; ++i) cv[jj][i] = (gj < N && gi0 + i < M) ? cp[i] : TC(0);
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < kJB; ++jj) {
        const int j = j0 + jj, gj = n0 + c0 + j;
        if (gj >= N) continue;
        TC* cp = C + gi0 + (size_t)gj * ldc;
        TC out[TM];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          if (beta == R(0))
            out[i] = (TC)(alpha * acc[i][j]);
          else  // accumulate in the wider of the two types
            out[i] = (TC)fma((TC)alpha, (TC)acc[i][j], (TC)beta * cv[jj][i]);
        }
        if (vec_ok(cp)) {
#pragma unroll
          for (int i = 0; i < TM; i += 4) save4(cp + i, &out[i]);
        } else {
#pragma unroll
          for (int i = 0; i < TM; ++i)
            if (gi0 + i < M) cp[i] = out[i];
        }
      }
    }
  }
};

template <typename R>
using TileSq = Tile<R, 64, 64, 16, 4, 4>;
template <typename R>
using TileNarrow = Tile<R, 128, 16, 16, 4, 4>;
// FP32 products with K >= kWideK and M >= kWideM: 8 x 8 outputs per thread
// read with float4, half the shared-memory reads per FMA of the 4 x 4 tile
// (whose two LDS per FMA pair cap it near half the FFMA rate); shorter
// products would leave most of its 128 rows idle
using TileWideF = Tile<float, 128, 64, 16, 8, 8>;
constexpr int kWideK = 64, kWideM = 96;
// The profiler name of a product on the tensor cores: the name with "_tc"
// before its type suffix ("gemm_body<f32>" -> "gemm_body_tc<f32>").
const char* tc_name(const char* name) {
  static std::mutex mu;
  static std::unordered_map<std::string, std::string> names;
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(name);
  if (it == names.end()) {
    std::string n(name);
    const size_t lt = n.find('<');
    n = lt == std::string::npos ? n + "_tc" : n.substr(0, lt) + "_tc" + n.substr(lt);
    it = names.emplace(std::string(name), n).first;
  }
  return it->second.c_str();
}

// ------------------------------------------------------------ explicit GEMMs
template <typename R, class TL, typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(TL::NT) k_gemm(const GemmDesc<TA, TB, TC>* __restrict__ d,
                                                 int tpm, int tpn, R alpha, R beta, int skip_tc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int per = tpm * tpn;
  const GemmDesc<TA, TB, TC> g = d[blockIdx.x / per];
  const int tile = blockIdx.x % per;
  const int m0 = (tile % tpm) * TL::BM, n0 = (tile / tpm) * TL::BN;
  if (m0 >= g.M || n0 >= g.N || (skip_tc && gemm_on_tc(g.M, g.K))) return;
  TL::run(g.M, g.N, g.K, alpha, g.A, g.lda, g.B, g.ldb, beta, g.C, g.ldc, m0, n0,
          reinterpret_cast<R*>(smraw));
}

// Split-K: CTA (desc, tile, split) computes the partial product over its K
// range into ws[(desc*splits + split)] (max_M x max_N blocks, ld max_M); the
// reduction adds the partials in split order.
template <typename R, class TL, typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(TL::NT) k_gemm_split(const GemmDesc<TA, TB, TC>* __restrict__ d,
                                                       int tpm, int tpn, int splits, int kc,
                                                       R* __restrict__ ws, int wsM, int wsN,
                                                       int skip_tc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int per = tpm * tpn * splits;
  const int di = blockIdx.x / per;
  const GemmDesc<TA, TB, TC> g = d[di];
  const int rem = blockIdx.x % per;
  const int sp = rem / (tpm * tpn), tile = rem % (tpm * tpn);
  const int m0 = (tile % tpm) * TL::BM, n0 = (tile / tpm) * TL::BN;
  const int k0 = sp * kc;
  if (m0 >= g.M || n0 >= g.N || k0 >= g.K || (skip_tc && gemm_on_tc(g.M, g.K))) return;
  const int kn = min(kc, g.K - k0);
  R* wp = ws + ((size_t)di * splits + sp) * wsM * wsN;
  TL::run(g.M, g.N, kn, R(1), g.A + (size_t)k0 * g.lda, g.lda, g.B + k0, g.ldb, R(0), wp, wsM, m0,
          n0, reinterpret_cast<R*>(smraw));
}

template <typename R, typename TA, typename TB, typename TC>
__global__ void k_gemm_split_reduce(const GemmDesc<TA, TB, TC>* __restrict__ d, int splits, int kc,
                                    const R* __restrict__ ws, int wsM, int wsN, int chunks,
                                    R alpha, R beta, int skip_tc) {
  const int di = blockIdx.x / chunks;
  const GemmDesc<TA, TB, TC> g = d[di];
  if (skip_tc && gemm_on_tc(g.M, g.K)) return;
  const int ns = min(splits, (g.K + kc - 1) / kc);
  const int64_t n = (int64_t)g.M * g.N;
  for (int64_t e = (int64_t)(blockIdx.x % chunks) * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)chunks * blockDim.x) {
    const int i = (int)(e % g.M), j = (int)(e / g.M);
    R acc = R(0);
    for (int s = 0; s < ns; ++s) acc += ws[((size_t)di * splits + s) * wsM * wsN + i + (size_t)j * wsM];
    TC* cp = g.C + i + (size_t)j * g.ldc;
    if (beta == R(0))
      *cp = (TC)(alpha * acc);
    else
      *cp = (TC)fma((TC)alpha, (TC)acc, (TC)beta * *cp);
  }
}

template <typename R, class TL, typename TA, typename TB, typename TC>
static void launch_gemm(const GemmDesc<TA, TB, TC>* d, int nd, int max_M, int max_N, int max_K,
                        R alpha, R beta, cudaStream_t st, const char* name, double flops,
                        double bytes, R* ws, size_t ws_elems, int skip_tc) {
  int tpm = (max_M + TL::BM - 1) / TL::BM, tpn = (max_N + TL::BN - 1) / TL::BN;
  if (nd <= 0 || tpm <= 0 || tpn <= 0) return;
  long long tiles = (long long)nd * tpm * tpn;
  prof::Scope sc(name, st, flops, bytes);
  // split K in fixed chunks of kSplitK: the split of a product depends only on
  // its own K, never on the other products of the launch
  const int splits = (ws && max_K > kSplitK) ? (max_K + kSplitK - 1) / kSplitK : 1;
  if (splits < 2 || (size_t)nd * splits * max_M * max_N > ws_elems) {
    k_gemm<R, TL, TA, TB, TC><<<(unsigned)tiles, TL::NT, TL::SMEM, st>>>(d, tpm, tpn, alpha, beta,
                                                                       skip_tc);
    return;
  }
  const int kc = kSplitK;
  k_gemm_split<R, TL, TA, TB, TC><<<(unsigned)(tiles * splits), TL::NT, TL::SMEM, st>>>(
      d, tpm, tpn, splits, kc, ws, max_M, max_N, skip_tc);
  int chunks = (int)std::min<long long>(((long long)max_M * max_N + 255) / 256, 256);
  k_gemm_split_reduce<R, TA, TB, TC><<<(unsigned)((long long)nd * chunks), 256, 0, st>>>(
      d, splits, kc, ws, max_M, max_N, chunks, alpha, beta, skip_tc);
}

template <typename R, typename TA, typename TB, typename TC>
void gemm_batched(const GemmDesc<TA, TB, TC>* d_desc, int ndesc, int max_M, int max_N, R alpha,
                  R beta, cudaStream_t st, const char* name, double flops, double bytes,
                  int max_K, R* ws, size_t ws_elems, int* status) {
  int skip_tc = 0;
  // (FP64 B operands, converted per element as they are loaded, stay on the
  // tile kernels: measured faster there)
  if constexpr (std::is_same<R, float>::value && std::is_same<TA, float>::value &&
                std::is_same<TB, float>::value) {
    if (status && ndesc > 0 && gemm_on_tc(max_M, max_K)) {
      // the products gemm_on_tc takes; the tile kernels below run the others
      // (only the launch's maxima are known here, so they always launch; the
      // profiler counts the flops and bytes under the tensor-core entry)
      {
        prof::Scope sc(tc_name(name), st, flops, bytes);
        gemm_tc32<TB, TC>(d_desc, ndesc, max_M, max_N, alpha, beta, status, st);
      }
      skip_tc = 1;
      flops = 0.0;
      bytes = 0.0;
    }
  }
  if (max_N <= 16)
    launch_gemm<R, TileNarrow<R>>(d_desc, ndesc, max_M, max_N, max_K, alpha, beta, st, name,
                                  flops, bytes, ws, ws_elems, skip_tc);
  else if constexpr (sizeof(R) == 4) {
    if (max_K >= kWideK && max_M >= kWideM)
      launch_gemm<R, TileWideF>(d_desc, ndesc, max_M, max_N, max_K, alpha, beta, st, name, flops,
                                bytes, ws, ws_elems, skip_tc);
    else
      launch_gemm<R, TileSq<R>>(d_desc, ndesc, max_M, max_N, max_K, alpha, beta, st, name,
                                flops, bytes, ws, ws_elems, skip_tc);
  } else {
    launch_gemm<R, TileSq<R>>(d_desc, ndesc, max_M, max_N, max_K, alpha, beta, st, name, flops,
                              bytes, ws, ws_elems, skip_tc);
  }
}

// ------------------------------------------------------------ LU: the panel
// Pivot keys: |x| as its bit pattern, which orders non-negative values as the
// values do, so the argmax runs on integer compares (FP64 compares share the
// FP64 pipe, 2 per clock per SM).  A NaN pattern sorts above every number: a
// NaN in the column becomes the pivot and is reported as a bad pivot.
__device__ __forceinline__ long long pivot_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}
__device__ __forceinline__ int pivot_key(float x) { return __float_as_int(x) & 0x7fffffff; }
template <typename R>
using PivotKey = decltype(pivot_key(R(0)));

// Factor columns k0..k0+nbk-1 (rows k0..m-1) of one matrix per CTA.
template <typename R>
__global__ void __launch_bounds__(512) k_lu_panel(const LuDesc<R>* __restrict__ d, int k0,
                                                  int smem_elems, int* status) {
  const LuDesc<R> D = d[blockIdx.x];
  const int m = D.m;
  if (k0 >= m) return;
  const int nbk = min(kNB, m - k0);
  const int rows = m - k0;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  using Key = PivotKey<R>;
  __shared__ Key red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_piv;
  __shared__ R s_inv;
  const bool staged = rows * nbk <= smem_elems;
  R* A0 = D.A + k0 + (size_t)k0 * D.lda;
  R* P = staged ? sm : A0;
  const int ldp = staged ? rows : D.lda;
  if (staged) {
    for (int e = threadIdx.x; e < rows * nbk; e += blockDim.x) {
      int i = e % rows, c = e / rows;
      P[i + c * ldp] = A0[i + (size_t)c * D.lda];
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int jj = 0; jj < nbk; ++jj) {
    // pivot search: largest |P(i, jj)| over i >= jj, ties to the smaller row
    Key best = -1;
    int bi = jj;
    for (int i = jj + threadIdx.x; i < rows; i += blockDim.x) {
      const Key v = pivot_key(P[i + jj * ldp]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Key ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[wid] = best;
      red_i[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {
      best = lane < nw ? red_v[lane] : -1;
      bi = lane < nw ? red_i[lane] : jj;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const Key ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_piv = bi;
        D.ipiv[k0 + jj] = k0 + bi;
        // the pivot value (row bi before the swap) and its reciprocal, once
        const R pv = P[bi + jj * ldp];
        const bool bad = !(pv != R(0)) || !isfinite(pv);
        if (bad && status) atomicCAS(status, 0, D.box + 1);
        s_inv = bad ? R(0) : R(1) / pv;
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != jj) {
      for (int c = threadIdx.x; c < nbk; c += blockDim.x) {
        R a = P[jj + c * ldp];
        P[jj + c * ldp] = P[piv + c * ldp];
        P[piv + c * ldp] = a;
      }
      __syncthreads();
    }
    const R inv = s_inv;
    for (int i = jj + 1 + threadIdx.x; i < rows; i += blockDim.x) {
      R l = P[i + jj * ldp] * inv;
      P[i + jj * ldp] = l;
      for (int c = jj + 1; c < nbk; ++c) P[i + c * ldp] = fma(-l, P[jj + c * ldp], P[i + c * ldp]);
    }
    __syncthreads();
  }
  if (staged) {
    for (int e = threadIdx.x; e < rows * nbk; e += blockDim.x) {
      int i = e % rows, c = e / rows;
      A0[i + (size_t)c * D.lda] = P[i + c * ldp];
    }
  }
}

// Tall panels: one thread-block cluster of kPanelCl CTAs per matrix, the
// panel's rows split into kPanelCl slices, each staged in its CTA's shared
// memory, so the rank-1 updates of a column run on kPanelCl SMs (FP64 FMAs are
// 2 per clock per SM: one SM bounds a tall panel).  Per column: every CTA
// offers its best row (pivot key, row, value), one lane per CTA reads the
// offers over distributed shared memory and the lanes reduce them by shuffles,
// so all CTAs take the same pivot and form the same reciprocal; every CTA
// reads the pivot row, the owner of the pivot row also reads row jj, and after
// one cluster barrier (only when rows are interchanged) the two owners write
// the rows back swapped.  A thread owns the same rows in the argmax and in the
// update, so no block barrier separates them.  Same pivots, same reciprocal,
// same FMAs in the same order per element: the factors equal k_lu_panel's bit
// for bit.  Cluster barriers: one per column, two when rows are swapped, and
// one before exit (no CTA leaves while others may still read its memory).
constexpr int kPanelCl = 8;

template <typename R>
__global__ void __cluster_dims__(kPanelCl, 1, 1) __launch_bounds__(256)
    k_lu_panel_cl(const LuDesc<R>* __restrict__ d, int k0, int chunk_max, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const LuDesc<R> D = d[blockIdx.x / kPanelCl];
  const int m = D.m;
  if (k0 >= m) return;  // the whole cluster
  const int nbk = min(kNB, m - k0);
  const int rows = m - k0;
  const int chunk = (rows + kPanelCl - 1) / kPanelCl;  // <= chunk_max
  const int r0 = min(rows, rank * chunk), r1 = min(rows, r0 + chunk);
  extern __shared__ __align__(16) unsigned char smraw[];
  R* P = reinterpret_cast<R*>(smraw);  // own rows r0..r1-1 (relative to k0), column-major, ld chunk
  using Key = PivotKey<R>;
  __shared__ Key cand_v[2];  // this CTA's offer per column parity: pivot key, row, value
  __shared__ int cand_i[2];
  __shared__ R cand_x[2];
  __shared__ Key red_v[8];
  __shared__ int red_i[8];
  __shared__ int s_piv;
  __shared__ R s_inv;
  __shared__ R prow[kNB];
  R* A0 = D.A + k0 + (size_t)k0 * D.lda;
  const int nown = r1 - r0;
  for (int e = threadIdx.x; e < nown * nbk; e += blockDim.x) {
    const int i = e % nown, c = e / nown;
    P[i + c * chunk] = A0[(r0 + i) + (size_t)c * D.lda];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int jj = 0; jj < nbk; ++jj) {
    const int par = jj & 1;
    Key best = -1;
    int bi = jj;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      if (i < jj) continue;
      const Key v = pivot_key(P[(i - r0) + jj * chunk]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Key ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[wid] = best;
      red_i[wid] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Key bv = red_v[0];
      int bx = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bx)) {
          bv = red_v[w];
          bx = red_i[w];
        }
      cand_v[par] = bv;
      cand_i[par] = bx;
      // the offered row's value (any own row when this CTA has none left)
      cand_x[par] = bv >= 0 ? P[(bx - r0) + jj * chunk] : R(0);
    }
    cl.sync();  // offers visible
    if (wid == 0) {  // lane r reads rank r's offer; the 8 lanes reduce
      Key bv = -1;
      int bx = 0x7fffffff;
      R xv = R(0);
      if (lane < kPanelCl) {
        bv = *cl.map_shared_rank(&cand_v[par], lane);
        bx = *cl.map_shared_rank(&cand_i[par], lane);
        xv = *cl.map_shared_rank(&cand_x[par], lane);
      }
#pragma unroll
      for (int o = kPanelCl / 2; o > 0; o >>= 1) {
        const Key ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int ox = __shfl_xor_sync(0xffffffffu, bx, o);
        const R oxv = __shfl_xor_sync(0xffffffffu, xv, o);
        if (ov > bv || (ov == bv && ox < bx)) {
          bv = ov;
          bx = ox;
          xv = oxv;
        }
      }
      if (lane == 0) {
        // a CTA without rows >= jj offers key -1, which every real row beats
        s_piv = bx;
        if (rank == 0) D.ipiv[k0 + jj] = k0 + bx;
        const bool bad = !(xv != R(0)) || !isfinite(xv);
        if (bad && rank == 0 && status) atomicCAS(status, 0, D.box + 1);
        s_inv = bad ? R(0) : R(1) / xv;
      }
    }
    __syncthreads();
    const int piv = s_piv;
    const int og = jj / chunk;  // owner of row jj
    const int op = piv / chunk;  // owner of the pivot row
    R vg = R(0), vp = R(0);
    if (threadIdx.x < nbk) {
      const int c = threadIdx.x;
      vp = cl.map_shared_rank(P, op)[(piv - op * chunk) + c * chunk];
      prow[c] = vp;  // the pivot row becomes row jj
      if (piv != jj && rank == op) vg = cl.map_shared_rank(P, og)[(jj - og * chunk) + c * chunk];
    }
    if (piv != jj) {  // the same decision in every CTA
      cl.sync();  // both rows read everywhere before either is written
      if (threadIdx.x < nbk) {
        const int c = threadIdx.x;
        if (rank == og) P[(jj - r0) + c * chunk] = vp;
        if (rank == op) P[(piv - r0) + c * chunk] = vg;
      }
    }
    __syncthreads();
    const R inv = s_inv;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      if (i <= jj) continue;
      const int li = i - r0;
      R l = P[li + jj * chunk] * inv;
      P[li + jj * chunk] = l;
      for (int c = jj + 1; c < nbk; ++c) P[li + c * chunk] = fma(-l, prow[c], P[li + c * chunk]);
    }
    // no block barrier: each thread's rows are its own in the next argmax,
    // and prow / the offers are rewritten only after the next barriers
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nown * nbk; e += blockDim.x) {
    const int i = e % nown, c = e / nown;
    A0[(r0 + i) + (size_t)c * D.lda] = P[i + c * chunk];
  }
  cl.sync();  // no CTA exits while another may still read its shared memory
}

// One panel launch: a cluster per matrix for tall panels of few matrices (the
// top merges), from 256 rows in FP64 and 512 in FP32 (below, the cluster
// barriers cost what spreading the FMAs saves), else one CTA per matrix.  Both
// give the same factors.
template <typename R>
bool launch_panel(const LuDesc<R>* d_desc, int nd, int max_m, int k0, int* d_status,
                  cudaStream_t st, double fl, double by) {
  const int rows = max_m - k0;
  const int smem_max = 224 * 1024;
  const int chunk = (rows + kPanelCl - 1) / kPanelCl;
  const long long cl_bytes = (long long)chunk * std::min(kNB, rows) * (long long)sizeof(R);
  prof::Scope sc(TName<R>::panel(), st, fl, by);
  // the opt-in is cached per kernel: always ask for the same (largest) size
  if (rows >= (sizeof(R) == 8 ? 256 : 512) && nd <= 32) {
    if (cl_bytes <= smem_max &&
      opt_in_smem(reinterpret_cast<const void*>(&k_lu_panel_cl<R>), smem_max)) {
      k_lu_panel_cl<R><<<(unsigned)(nd * kPanelCl), 256, (size_t)cl_bytes, st>>>(d_desc, k0,
                                                                               chunk, d_status);
      return true;
    }
  }
  const long long need = (long long)rows * std::min(kNB, rows) * (long long)sizeof(R);
  const int smem_bytes = (int)std::min<long long>(need, smem_max);
  const int threads = rows > 512 ? 512 : 256;
  k_lu_panel<R><<<nd, threads, smem_bytes, st>>>(d_desc, k0, smem_bytes / (int)sizeof(R), d_status);
  return true;
}

// ----------------------------------------- LU: swaps + unit-lower block solve
// The interchanges of one panel (rows k0.., pivots ipiv[k0..k0+nbk)) move at
// most 2*nb rows: rows_inv lists them (relative to k0; the block rows first,
// then the other pivot rows in order of first use) and slot t takes the old
// value of slot src_of[t].  Built by one warp in parallel: lane j holds
// interchange j; the external pivot rows are deduplicated with
// __match_any_sync and numbered by a ballot; the interchanges are then
// replayed on the slot contents (lane t holds slots t and t + 32) with
// shuffles.  Returns the number of rows involved.
__device__ int panel_perm_warp(const int* ipiv, int k0, int nbk, int* rows_inv, int* src_of,
                               int lane) {
  const int pr = lane < nbk ? ipiv[k0 + lane] - k0 : -1;
  const bool ext = lane < nbk && pr >= nbk;
  const unsigned same = __match_any_sync(0xffffffffu, ext ? pr : -1 - lane);
  const int lead = __ffs(same) - 1;  // first lane with this pivot row
  const bool first = ext && lead == lane;
  const unsigned firsts = __ballot_sync(0xffffffffu, first);
  const int nr = nbk + __popc(firsts);
  const int slot = !ext ? (lane < nbk ? pr : 0) : nbk + __popc(firsts & ((1u << lead) - 1u));
  if (lane < nbk) rows_inv[lane] = lane;
  if (first) rows_inv[slot] = pr;
  int c0 = lane, c1 = lane + 32;
  for (int j = 0; j < nbk; ++j) {
    const int tp = __shfl_sync(0xffffffffu, slot, j);
    const int vj = __shfl_sync(0xffffffffu, c0, j);
    const int vt = __shfl_sync(0xffffffffu, tp < 32 ? c0 : c1, tp & 31);
    if (lane == j) c0 = vt;
    if (tp < 32) {
      if (lane == tp) c0 = vj;
    } else if (lane == (tp & 31)) {
      c1 = vj;
    }
  }
  if (lane < nr) src_of[lane] = c0;
  if (lane + 32 < nr) src_of[lane + 32] = c1;
  return nr;
}

// One warp applies a panel's interchanges to column x (rows relative to k0)
// and returns, in lanes < nbk, the new block-row values (not yet stored).
template <typename R>
__device__ __forceinline__ R warp_permute(R* x, const int* rows_inv, const int* src_of, int nr,
                                          int lane) {
  // gather the involved rows (lane holds slots lane and lane+32)
  R v0 = lane < nr ? x[rows_inv[lane]] : R(0);
  R v1 = (lane + 32) < nr ? x[rows_inv[lane + 32]] : R(0);
  // permuted values: slot t takes the old value of slot src_of[t]
  int s0 = lane < nr ? src_of[lane] : 0;
  int s1 = (lane + 32) < nr ? src_of[lane + 32] : 0;
  R n0a = __shfl_sync(0xffffffffu, v0, s0 & 31);
  R n0b = __shfl_sync(0xffffffffu, v1, s0 & 31);
  R n1a = __shfl_sync(0xffffffffu, v0, s1 & 31);
  R n1b = __shfl_sync(0xffffffffu, v1, s1 & 31);
  R w0 = s0 < 32 ? n0a : n0b;
  R w1 = s1 < 32 ? n1a : n1b;
  if ((lane + 32) < nr) x[rows_inv[lane + 32]] = w1;
  return w0;
}

// Columns a panel's interchanges and block solve act on.  part < 0 (one-level
// LU): the trailing columns of A and the columns of B, plus the columns left of
// the panel when swap_left.  Two-level LU (outer block column [K0, oe), oe =
// min(K0 + kLuOuter, m)): part 0 is the outer block itself, its columns left of
// the panel (interchanges only) and right of it; part 1 is the far columns,
// A's [oe, m) and B, solved only (their interchanges were applied before).
struct SwapCols {
  int nleft, left0, a_lo, a_hi, nb;
};
__device__ __forceinline__ SwapCols swap_cols(int part, int K0, int k0, int nbk, int m, int nrhs,
                                              int swap_left, int b_only) {
  SwapCols c;
  if (part < 0) {
    c.nleft = (swap_left && !b_only) ? k0 : 0;
    c.left0 = 0;
    c.a_lo = k0 + nbk;
    c.a_hi = b_only ? c.a_lo : m;
    c.nb = nrhs;
  } else {
    const int oe = min(K0 + kLuOuter, m);
    c.nleft = part == 0 ? k0 - K0 : 0;
    c.left0 = K0;
    c.a_lo = part == 0 ? k0 + nbk : oe;
    c.a_hi = part == 0 ? oe : m;
    c.nb = part == 0 ? 0 : nrhs;
  }
  return c;
}

// For every column of the region: apply the panel's row interchanges (unless
// part 1), then (all but the left columns) solve with the unit-lower L11.
// One warp per column.
template <typename R>
__global__ void __launch_bounds__(256) k_lu_swap_trsm(const LuDesc<R>* __restrict__ d, int k0,
                                                      int chunks, int cols_per_cta,
                                                      int swap_left, int b_only, int part,
                                                      int K0) {
  const LuDesc<R> D = d[blockIdx.x / chunks];
  const int chunk = blockIdx.x % chunks;
  const int m = D.m;
  if (k0 >= m) return;
  const int nbk = min(kNB, m - k0);
  const SwapCols sc = swap_cols(part, K0, k0, nbk, m, D.nrhs, swap_left, b_only);
  const int nleft = sc.nleft, ntr = sc.a_hi - sc.a_lo;
  const int total = nleft + ntr + sc.nb;
  const int cbeg = chunk * cols_per_cta;
  if (cbeg >= total) return;
  const int cend = min(total, cbeg + cols_per_cta);
  const bool do_swap = part != 1;
  __shared__ R L11[kNB * kNB];
  __shared__ int rows_inv[2 * kNB];  // involved rows (relative to k0)
  __shared__ int src_of[2 * kNB];    // new value of rows_inv[t] comes from rows_inv[src_of[t]]
  __shared__ int s_nr;
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e % nbk, j = e / nbk;
    L11[i + j * kNB] = D.A[(k0 + i) + (size_t)(k0 + j) * D.lda];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (wid == 0) {
    const int n = do_swap ? panel_perm_warp(D.ipiv, k0, nbk, rows_inv, src_of, lane) : nbk;
    if (lane == 0) s_nr = n;
  }
  __syncthreads();
  const int nr = s_nr;
  for (int col = cbeg + wid; col < cend; col += nw) {
    R* x;
    bool solve;
    if (col < nleft) {
      x = D.A + k0 + (size_t)(sc.left0 + col) * D.lda;
      solve = false;
    } else if (col < nleft + ntr) {
      x = D.A + k0 + (size_t)(sc.a_lo + (col - nleft)) * D.lda;
      solve = true;
    } else {
      x = D.B + k0 + (size_t)(col - nleft - ntr) * D.ldb;
      solve = true;
    }
    R w0;
    if (do_swap)
      w0 = warp_permute(x, rows_inv, src_of, nr, lane);
    else
      w0 = lane < nbk ? x[lane] : R(0);
    // w0 of lanes < nbk is the block row; solve with unit-lower L11
    if (solve) {
      for (int j = 0; j < nbk - 1; ++j) {
        R xj = __shfl_sync(0xffffffffu, w0, j);
        if (lane > j && lane < nbk) w0 = fma(-L11[lane + j * kNB], xj, w0);
      }
    }
    if (lane < nr) x[do_swap ? rows_inv[lane] : lane] = w0;
  }
}

// Two-level LU: the interchanges of every panel of the outer block column
// [K0, oe), in panel order, applied to the far columns (A's [oe, m) and B).
// One warp per column; the panels' permutations are computed in parallel.
template <typename R>
__global__ void __launch_bounds__(256) k_lu_swap_far(const LuDesc<R>* __restrict__ d, int K0,
                                                     int chunks, int cols_per_cta) {
  constexpr int kP = kLuOuter / kNB;
  const LuDesc<R> D = d[blockIdx.x / chunks];
  const int chunk = blockIdx.x % chunks;
  const int m = D.m;
  if (K0 >= m) return;
  const int oe = min(K0 + kLuOuter, m);
  const int nfa = m - oe, total = nfa + D.nrhs;
  const int cbeg = chunk * cols_per_cta;
  if (cbeg >= total) return;
  const int cend = min(total, cbeg + cols_per_cta);
  const int np = (oe - K0 + kNB - 1) / kNB;
  __shared__ int rows_inv[kP][2 * kNB];
  __shared__ int src_of[kP][2 * kNB];
  __shared__ int s_nr[kP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = wid; b < np; b += nw) {  // one warp per panel
    const int k0 = K0 + b * kNB;
    const int n = panel_perm_warp(D.ipiv, k0, min(kNB, m - k0), rows_inv[b], src_of[b], lane);
    if (lane == 0) s_nr[b] = n;
  }
  __syncthreads();
  for (int col = cbeg + wid; col < cend; col += nw) {
    R* x0 = col < nfa ? D.A + (size_t)(oe + col) * D.lda : D.B + (size_t)(col - nfa) * D.ldb;
    for (int p = 0; p < np; ++p) {
      R* x = x0 + K0 + p * kNB;
      const int nr = s_nr[p];
      const R w0 = warp_permute(x, rows_inv[p], src_of[p], nr, lane);
      if (lane < nr) x[rows_inv[p][lane]] = w0;
      __syncwarp();  // the next panel's gather reads rows other lanes wrote
    }
  }
}

// ------------------------------------------------------ LU: trailing update
// (rows, columns of A, columns of B) -= L21 * U12 over the panel's nbk columns:
//   part < 0: rows k0+nbk..m-1, A columns k0+nbk..m-1 and B (one-level LU);
//   part 0:   rows k0+nbk..m-1, A columns k0+nbk..oe-1 (two-level: inside the
//             outer block column [K0, oe));
//   part 1:   rows k0+nbk..oe-1, A columns oe..m-1 and B (the far columns'
//             block-row solve).
template <typename R, class TL>
__global__ void __launch_bounds__(TL::NT) k_lu_update(const LuDesc<R>* __restrict__ d, int k0,
                                                      int tpm, int tpnA, int tpnB, int part,
                                                      int K0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int per = tpm * (tpnA + tpnB);
  const LuDesc<R> D = d[blockIdx.x / per];
  const int tile = blockIdx.x % per;
  const int m = D.m;
  if (k0 >= m) return;
  const int nbk = min(kNB, m - k0);
  const int r0 = k0 + nbk;
  const int oe = part < 0 ? m : min(K0 + kLuOuter, m);
  const int r_hi = part == 1 ? oe : m;
  const int c_lo = part == 1 ? oe : r0, c_hi = part == 0 ? oe : m;
  const bool with_b = part != 0;
  const int M = r_hi - r0;
  if (M <= 0) return;
  const int tmi = tile % tpm, tni = tile / tpm;
  const R* L21 = D.A + r0 + (size_t)k0 * D.lda;
  if (tni < tpnA) {
    const int N = c_hi - c_lo;
    const int m0 = tmi * TL::BM, n0 = tni * TL::BN;
    if (m0 >= M || n0 >= N) return;
    TL::run(M, N, nbk, R(-1), L21, D.lda, D.A + k0 + (size_t)c_lo * D.lda, D.lda, R(1),
            D.A + r0 + (size_t)c_lo * D.lda, D.lda, m0, n0, reinterpret_cast<R*>(smraw));
  } else {
    if (!with_b) return;
    const int N = D.nrhs;
    const int m0 = tmi * TL::BM, n0 = (tni - tpnA) * TL::BN;
    if (m0 >= M || n0 >= N) return;
    TL::run(M, N, nbk, R(-1), L21, D.lda, D.B + k0, D.ldb, R(1), D.B + r0, D.ldb, m0, n0,
            reinterpret_cast<R*>(smraw));
  }
}

// ------------------------------------------- back substitution: diagonal block
// Rows kb0..kb0+nbk-1 of B := U11^{-1} (those rows) by column-sweep back
// substitution: one thread per column, the nbk values in registers, U11 and the
// reciprocals of its diagonal in shared memory (broadcast reads).
template <typename R>
__global__ void __launch_bounds__(256) k_trsm_upper(const LuDesc<R>* __restrict__ d, int kb0,
                                                    int chunks) {
  const LuDesc<R> D = d[blockIdx.x / chunks];
  const int chunk = blockIdx.x % chunks;
  const int m = D.m;
  if (kb0 >= m || chunk * (int)blockDim.x >= D.nrhs) return;
  const int nbk = min(kNB, m - kb0);
  __shared__ R U[kNB][kNB + 1];
  __shared__ R rd[kNB];
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int i = e % kNB, j = e / kNB;
    U[i][j] = (i < nbk && j < nbk) ? D.A[(kb0 + i) + (size_t)(kb0 + j) * D.lda] : R(0);
  }
  __syncthreads();
  if (threadIdx.x < kNB) {
    R dj = U[threadIdx.x][threadIdx.x];
    rd[threadIdx.x] = (dj != R(0)) ? R(1) / dj : R(0);
  }
  __syncthreads();
  const int col = chunk * blockDim.x + threadIdx.x;
  if (col >= D.nrhs) return;
  R* x = D.B + kb0 + (size_t)col * D.ldb;
  R v[kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i) v[i] = (i < nbk) ? x[i] : R(0);
#pragma unroll
  for (int j = kNB - 1; j >= 0; --j) {
    if (j < nbk) {
      v[j] *= rd[j];
#pragma unroll
      for (int i = 0; i < j; ++i) v[i] = fma(-U[i][j], v[j], v[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < nbk) x[i] = v[i];
}

// ---------------------------------------------- back substitution: update
// Rows rlo..kb0-1 of B -= U[rlo:kb0, kb0:kb0+nbk] * B[kb0:kb0+nbk, :]
// (rlo = 0 in the one-level LU, the outer block's first row in the two-level).
template <typename R, class TL>
__global__ void __launch_bounds__(TL::NT) k_backsub_update(const LuDesc<R>* __restrict__ d,
                                                           int kb0, int tpm, int tpn, int rlo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int per = tpm * tpn;
  const LuDesc<R> D = d[blockIdx.x / per];
  const int tile = blockIdx.x % per;
  if (kb0 >= D.m || kb0 <= rlo) return;
  const int nbk = min(kNB, D.m - kb0);
  const int M = kb0 - rlo;
  const int m0 = (tile % tpm) * TL::BM, n0 = (tile / tpm) * TL::BN;
  if (m0 >= M || n0 >= D.nrhs) return;
  TL::run(M, D.nrhs, nbk, R(-1), D.A + rlo + (size_t)kb0 * D.lda, D.lda, D.B + kb0, D.ldb, R(1),
          D.B + rlo, D.ldb, m0, n0, reinterpret_cast<R*>(smraw));
}

// ------------------------------------------------ leaf inverse, Gauss-Jordan
// The leaf systems of a mixed build at p = 16 (n = 196 interior nodes): A^{-1}
// by Gauss-Jordan elimination with partial pivoting (the inverse of Section
// 3.1's A_ii, from which the solution operator Y = A_ii^{-1} (-A_ie L1) and the
// refinement's interior corrections follow by products), the whole matrix in
// registers: one CTA per leaf, thread (tr, tc) of 28 x 14 holding rows
// tr + 28a (a < 7) and columns tc + 14b (b < 14); 24 more threads make the
// last warp whole and hold nothing.  Rows are never interchanged: step k
// takes as pivot row p_k the largest |entry| of column k among the rows not
// yet used (ties: the lower row), scales row p_k by 1/pivot (its column-k
// entry becoming 1/pivot) and subtracts multiples of it from every other row
// (their column-k entries becoming -entry/pivot), one FMA per entry.  After n
// steps entry (i, k) of the array is A^{-1}(s(i), p_k), s(i) the step at which
// row i was pivot; the inverse is written un-permuted through shared memory.
// The pivot search of step k+1 runs in the warps that hold column k+1 while
// the others still update for step k (they update that column first).
// Per descriptor: A (n x n, ld n) is read and then receives a copy of B's
// first nq columns (ld n); B's columns nq .. nq + n - 1 receive A^{-1}.  A zero
// or non-finite pivot records box+1 in *status (first error wins) and the
// elimination goes on with a zero reciprocal, as the LU's does.
constexpr int kGjN = kLeafGjN, kGjTr = 28, kGjTc = 14, kGjR = 7, kGjC = 14;
constexpr int kGjOwners = kGjTr * kGjTc, kGjThreads = (kGjOwners + 31) / 32 * 32;
static_assert(kGjTr * kGjR == kGjN && kGjTc * kGjC == kGjN, "the tiles cover the matrix");

// Pivot order: |v| (its bit pattern), then the lower row; a row not yet used
// always has a non-zero key.
__device__ __forceinline__ unsigned long long gj_key(float v, int row) {
  return ((unsigned long long)(__float_as_uint(v) & 0x7fffffffu) << 32) | (1u << 17) |
         (0xffffu - (uint32_t)row);
}

__global__ void __launch_bounds__(kGjThreads, 1)
    k_leaf_gj_inverse(const LuDesc<float>* __restrict__ d, int nq, int* status) {
  extern __shared__ __align__(16) float sinv[];  // n x n: the inverse, un-permuted
  __shared__ float prow[kGjN], pcol[kGjN];
  __shared__ unsigned long long cand[2];
  __shared__ float crcp[2];
  __shared__ int rowstep[kGjN], steprow[kGjN];
  constexpr int n = kGjN, Tr = kGjTr, Tc = kGjTc, R = kGjR, C = kGjC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool owner = tid < kGjOwners;
  const int tc = owner ? tid / Tr : -1, tr = owner ? tid - (tid / Tr) * Tr : -1;
  for (int i = tid; i < n; i += kGjThreads) rowstep[i] = steprow[i] = 0;
  float x[R][C];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < C; ++b) x[a][b] = 0.0f;
  {
    // the descriptor is read again where needed, not held through the steps
    float* const A = d[blockIdx.x].A;
    if (owner) {
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < C; ++b) x[a][b] = A[(tr + Tr * a) + (size_t)(tc + Tc * b) * n];
    }
    __syncthreads();  // every read of A precedes the copy into it
    const float4* src = reinterpret_cast<const float4*>(d[blockIdx.x].B);
    float4* dst = reinterpret_cast<float4*>(A);
    for (int e = tid; e < n * nq / 4; e += kGjThreads) dst[e] = src[e];
  }
  uint32_t used = 0;  // bit a: row tr + 28a has been a pivot row
  // Candidates for column (slot B, group kcn) from its owners (threads
  // 28kcn .. 28kcn+27, in warps w0n and w1n): per warp the largest |entry|
  // among unused rows (as bit pattern + 1, so that an unused zero beats a used
  // row), then the lowest row holding it; that lane publishes the 64-bit key
  // and the reciprocal of its entry (zero for a bad pivot).
  auto candidates = [&](auto Bc, int kcn) {
    constexpr int B = decltype(Bc)::value;
    const int w0n = (kcn * Tr) >> 5, w1n = (kcn * Tr + Tr - 1) >> 5;
    uint32_t mk = 0;
    int mrow = 0xffff;
    float mv = 0.0f;
    if (tc == kcn) {
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const float v = x[a][B];
        const uint32_t m = ((used >> a) & 1u) ? 0u : (__float_as_uint(v) & 0x7fffffffu) + 1u;
        if (m > mk) mk = m, mrow = tr + Tr * a, mv = v;  // rows ascend with a
      }
    }
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, mk);
    const uint32_t wrow = __reduce_min_sync(0xffffffffu, mk == wmax ? (uint32_t)mrow : 0xffffu);
    if (lane == 0 && wmax == 0u) cand[warp - w0n] = 0;
    if (wmax != 0u && mk == wmax && (uint32_t)mrow == wrow) {
      const bool bad = !(mv != 0.0f) || !isfinite(mv);
      cand[warp - w0n] = gj_key(mv, mrow);
      crcp[warp - w0n] = bad ? 0.0f : 1.0f / mv;
    }
    if (lane == 0 && w0n == w1n) cand[1] = 0;
  };
  if (warp == 0) candidates(std::integral_constant<int, 0>{}, 0);  // column 0: threads 0 .. 27
  // the steps of columns 14kb .. 14kb + 13 (slot kb of groups tc = 0 .. 13),
  // kb a constant
  auto block = [&](auto KB) {
    constexpr int kb = decltype(KB)::value;
#pragma unroll 1
    for (int kc = 0; kc < Tc; ++kc) {
      const int k = kc + Tc * kb;  // column k = group kc, slot kb
      __syncthreads();  // the candidates of column k are in
      // ---- the pivot, decoded alike by every thread
      const unsigned long long c0 = cand[0], c1 = cand[1];
      const unsigned long long best = max(c0, c1);
      const float rp = crcp[c1 > c0 ? 1 : 0];
      const int p = min(0xffff - (int)(best & 0xffffu), n - 1);  // a row not yet used
      const int tp = p % Tr, ap = p / Tr;
      if (tid == 0) {
        steprow[k] = p;
        rowstep[p] = k;
        const float piv = __uint_as_float((uint32_t)(best >> 32));  // |pivot|
        if ((!(piv != 0.0f) || !isfinite(piv)) && status)
          atomicCAS(status, 0, d[blockIdx.x].box + 1);
      }
      if (tr == tp) {  // the pivot row, scaled (its column-k entry 1/pivot), then cleared
        used |= 1u << ap;
        switch (ap) {
#define HPS_GJ_PROW(A)                                                      \
  case A:                                                                   \
    _Pragma("unroll") for (int b = 0; b < C; ++b) {                         \
      prow[tc + Tc * b] = (b == kb && tc == kc) ? rp : x[A][b] * rp;        \
      x[A][b] = 0.0f;                                                       \
    }                                                                       \
    break;
          HPS_GJ_PROW(0) HPS_GJ_PROW(1) HPS_GJ_PROW(2) HPS_GJ_PROW(3) HPS_GJ_PROW(4)
          HPS_GJ_PROW(5) HPS_GJ_PROW(6)
#undef HPS_GJ_PROW
        }
      }
      if (tc == kc) {  // the multipliers (-1 for the pivot row); column k cleared
#pragma unroll
        for (int a = 0; a < R; ++a) {
          pcol[tr + Tr * a] = (tr + Tr * a == p) ? -1.0f : x[a][kb];
          x[a][kb] = 0.0f;
        }
      }
      __syncthreads();
      // ---- the update: entry -= multiplier x scaled pivot row (the pivot row,
      // cleared, with multiplier -1 becomes the scaled row itself).  The warps
      // holding column k+1 update it first and find its candidates while the
      // other warps update.
      auto update_col = [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        if (owner) {
          const float pb = prow[tc + Tc * B];
#pragma unroll
          for (int a = 0; a < R; ++a) x[a][B] = fmaf(-pcol[tr + Tr * a], pb, x[a][B]);
        }
      };
      auto update_rest = [&](auto Bc) {  // every column slot but B (B = C: all)
        constexpr int B = decltype(Bc)::value;
        if (owner) {
          float f[R];
#pragma unroll
          for (int a = 0; a < R; ++a) f[a] = pcol[tr + Tr * a];
#pragma unroll
          for (int b = 0; b < C; ++b) {
            if (b == B) continue;
            const float pb = prow[tc + Tc * b];
#pragma unroll
            for (int a = 0; a < R; ++a) x[a][b] = fmaf(-f[a], pb, x[a][b]);
          }
        }
      };
      const int kcn = kc + 1 < Tc ? kc + 1 : 0;
      const bool next = k + 1 < n;
      const bool cw = next && (warp == (kcn * Tr) >> 5 || warp == (kcn * Tr + Tr - 1) >> 5);
      if (!cw) {
        update_rest(std::integral_constant<int, C>{});
      } else if (kc + 1 < Tc) {
        update_col(std::integral_constant<int, kb>{});
        candidates(std::integral_constant<int, kb>{}, kcn);
        update_rest(std::integral_constant<int, kb>{});
      } else if constexpr (kb + 1 < C) {
        update_col(std::integral_constant<int, kb + 1>{});
        candidates(std::integral_constant<int, kb + 1>{}, kcn);
        update_rest(std::integral_constant<int, kb + 1>{});
      }
    }
  };
  block(std::integral_constant<int, 0>{});
  block(std::integral_constant<int, 1>{});
  block(std::integral_constant<int, 2>{});
  block(std::integral_constant<int, 3>{});
  block(std::integral_constant<int, 4>{});
  block(std::integral_constant<int, 5>{});
  block(std::integral_constant<int, 6>{});
  block(std::integral_constant<int, 7>{});
  block(std::integral_constant<int, 8>{});
  block(std::integral_constant<int, 9>{});
  block(std::integral_constant<int, 10>{});
  block(std::integral_constant<int, 11>{});
  block(std::integral_constant<int, 12>{});
  block(std::integral_constant<int, 13>{});
  static_assert(kGjC == 14, "one call per column slot");
  // ---- A^{-1}(s(i), p_k) = entry (i, k), through shared memory
  __syncthreads();
  if (owner) {
    int rs[R];
#pragma unroll
    for (int a = 0; a < R; ++a) rs[a] = rowstep[tr + Tr * a];
#pragma unroll
    for (int b = 0; b < C; ++b) {
      const int col = steprow[tc + Tc * b];
#pragma unroll
      for (int a = 0; a < R; ++a) sinv[rs[a] + col * n] = x[a][b];
    }
  }
  __syncthreads();
  {
    const float4* src = reinterpret_cast<const float4*>(sinv);
    float4* dst = reinterpret_cast<float4*>(d[blockIdx.x].B + (size_t)nq * n);
    for (int e = tid; e < n * n / 4; e += kGjThreads) dst[e] = src[e];
  }
}

bool leaf_gj_inverse(const LuDesc<float>* d_desc, int nd, int n, int nq, int* status,
                     cudaStream_t st) {
  if (n != kGjN || nq < 0 || nq > n) return false;
  if (nd <= 0) return true;
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_leaf_gj_inverse), 200 * 1024)) return false;
  prof::Scope sc("leaf_gj_inverse<f32>", st, 2.0 * nd * (double)n * n * n,
                 (double)nd * (2.0 * n * n + 2.0 * n * nq) * sizeof(float));
  k_leaf_gj_inverse<<<nd, kGjThreads, (size_t)n * n * sizeof(float), st>>>(d_desc, nq, status);
  return true;
}

// ------------------------------------------------------------------ driver
template <typename R>
void lu_solve_batched(const LuDesc<R>* d_desc, int nd, int max_m, int max_nrhs, int mode,
                      int* d_status, cudaStream_t st, const int* h_m, const int* h_nrhs) {
  if (nd <= 0 || max_m <= 0) return;
  const bool factor = mode != kLuSolveOnly;
  const bool swap_left = mode == kLuFactorKeep;
  const double es = (double)sizeof(R);
  // algorithmic flops / bytes of each launch, from the host copy of the sizes
  auto sum = [&](auto fn) {
    double t = 0.0;
    for (int i = 0; i < nd; ++i) t += fn(h_m ? h_m[i] : max_m, h_nrhs ? h_nrhs[i] : max_nrhs);
    return t;
  };
  using TL = TileSq<R>;
  using TN = TileNarrow<R>;
  // panel staging: as much shared memory as the tallest panel needs, up to the
  // per-CTA maximum less the kernel's static shared arrays (taller panels are
  // factored in global memory)
  const int smem_max = 224 * 1024;
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_lu_panel<R>), smem_max))
    return;  // reported by the caller's launch check
  // few matrices: narrower column chunks, so the FP64 interchange and solve
  // work spreads over more SMs
  const int cols_per_cta = nd >= 64 ? 64 : 16;
  for (int k0 = 0; k0 < max_m; k0 += kNB) {
    if (factor) {
      double fl = sum([&](int m, int nr) {
        if (k0 >= m) return 0.0;
        int nbk = std::min(kNB, m - k0), rows = m - k0;
        double t = 0.0;
        for (int jj = 0; jj < nbk; ++jj) t += (double)(rows - jj - 1) * (2.0 * (nbk - jj - 1) + 1.0);
        return t;
      });
      double by = sum([&](int m, int nr) {
        return k0 < m ? 2.0 * (m - k0) * std::min(kNB, m - k0) * es : 0.0;
      });
      launch_panel<R>(d_desc, nd, max_m, k0, d_status, st, fl, by);
    }
    int total_cols = (factor ? (swap_left ? k0 : 0) + max_m : 0) + max_nrhs;
    int chunks = (total_cols + cols_per_cta - 1) / cols_per_cta;
    {
      double fl = sum([&](int m, int nr) {
        if (k0 >= m) return 0.0;
        int nbk = std::min(kNB, m - k0);
        return (double)nbk * (nbk - 1) * ((factor ? m - k0 - nbk : 0) + nr);
      });
      double by = sum([&](int m, int nr) {
        if (k0 >= m) return 0.0;
        int nbk = std::min(kNB, m - k0);
        return 2.0 * nbk * ((swap_left ? k0 : 0) + (factor ? m - k0 - nbk : 0) + nr) * es;
      });
      prof::Scope sc(TName<R>::swap(), st, fl, by);
      k_lu_swap_trsm<R><<<(unsigned)((long long)nd * chunks), 256, 0, st>>>(
          d_desc, k0, chunks, cols_per_cta, swap_left ? 1 : 0, factor ? 0 : 1, -1, 0);
    }
    int rem = max_m - k0 - kNB;
    if (rem > 0) {
      int tpm = (rem + TL::BM - 1) / TL::BM;
      int tpnA = factor ? (rem + TL::BN - 1) / TL::BN : 0;
      int tpnB = (max_nrhs + TL::BN - 1) / TL::BN;
      long long blocks = (long long)nd * tpm * (tpnA + tpnB);
      double fl = sum([&](int m, int nr) {
        if (k0 >= m) return 0.0;
        int nbk = std::min(kNB, m - k0);
        double M = m - k0 - nbk, N = (factor ? m - k0 - nbk : 0) + nr;
        return 2.0 * M * N * nbk;
      });
      double by = sum([&](int m, int nr) {
        if (k0 >= m) return 0.0;
        int nbk = std::min(kNB, m - k0);
        double M = m - k0 - nbk, N = (factor ? m - k0 - nbk : 0) + nr;
        return (M * nbk + nbk * N + 2.0 * M * N) * es;
      });
      prof::Scope sc(TName<R>::update(), st, fl, by);
      k_lu_update<R, TL><<<(unsigned)blocks, TL::NT, TL::SMEM, st>>>(d_desc, k0, tpm, tpnA, tpnB,
                                                                    -1, 0);
    }
  }
  const int last = ((max_m - 1) / kNB) * kNB;
  for (int kb0 = last; kb0 >= 0; kb0 -= kNB) {
    {
      double fl = sum([&](int m, int nr) {
        if (kb0 >= m) return 0.0;
        int nbk = std::min(kNB, m - kb0);
        return (double)nbk * nbk * nr;
      });
      double by = sum([&](int m, int nr) {
        if (kb0 >= m) return 0.0;
        int nbk = std::min(kNB, m - kb0);
        return (2.0 * nbk * nr + 0.5 * nbk * nbk) * es;
      });
      prof::Scope sc(TName<R>::trsm(), st, fl, by);
      int chunks = (max_nrhs + kTrsmCols - 1) / kTrsmCols;
      k_trsm_upper<R><<<(unsigned)((long long)nd * chunks), kTrsmCols, 0, st>>>(d_desc, kb0, chunks);
    }
    if (kb0 > 0) {
      double fl = sum([&](int m, int nr) {
        if (kb0 >= m) return 0.0;
        return 2.0 * kb0 * nr * std::min(kNB, m - kb0);
      });
      double by = sum([&](int m, int nr) {
        if (kb0 >= m) return 0.0;
        int nbk = std::min(kNB, m - kb0);
        return ((double)kb0 * nbk + nbk * nr + 2.0 * kb0 * nr) * es;
      });
      prof::Scope sc(TName<R>::backsub(), st, fl, by);
      if (max_nrhs <= 16) {
        int tpm = (kb0 + TN::BM - 1) / TN::BM, tpn = (max_nrhs + TN::BN - 1) / TN::BN;
        k_backsub_update<R, TN><<<(unsigned)((long long)nd * tpm * tpn), TN::NT, TN::SMEM, st>>>(
            d_desc, kb0, tpm, tpn, 0);
      } else {
        int tpm = (kb0 + TL::BM - 1) / TL::BM, tpn = (max_nrhs + TL::BN - 1) / TL::BN;
        k_backsub_update<R, TL><<<(unsigned)((long long)nd * tpm * tpn), TL::NT, TL::SMEM, st>>>(
            d_desc, kb0, tpm, tpn, 0);
      }
    }
  }
}

// ------------------------------------------------------- two-level blocked LU
namespace {

// The rank-kLuOuter products of one outer step: those worth the splitting on
// the tensor cores, the rest as FP64 tile GEMMs.  C -= A B for each.
struct TcStep {
  std::vector<OzDesc> oz;
  std::vector<GemmDesc<double>> simt;
  int maxM = 0, maxN = 0, maxK = 0;
  double simt_flops = 0.0, simt_bytes = 0.0;
  void add(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int M, int N,
           int K) {
    if (M <= 0 || N <= 0 || K <= 0) return;
    if (oz_eligible(M, N, K)) {
      OzDesc o;
      o.A = A;
      o.B = B;
      o.C = C;
      o.M = M;
      o.N = N;
      o.K = K;
      o.lda = lda;
      o.ldb = ldb;
      o.ldc = ldc;
      oz.push_back(o);
      return;
    }
    GemmDesc<double> g;
    g.A = A;
    g.B = B;
    g.C = C;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    simt.push_back(g);
    maxM = std::max(maxM, M);
    maxN = std::max(maxN, N);
    maxK = std::max(maxK, K);
    simt_flops += 2.0 * M * (double)N * K;
    simt_bytes += 8.0 * ((double)M * K + (double)K * N + 2.0 * M * N);
  }
};

// Forward, after the outer block column [K0, oe) is factored and its block row
// solved: rows oe..m-1 of A's columns oe..m-1 and of B -= L21 U12, with
// L21 = A[oe:m, K0:oe] and U12 the block row of those columns.
TcStep fwd_step(const std::vector<LuDescHost>& h, int K0) {
  TcStep s;
  for (const auto& d : h) {
    if (K0 >= d.m) continue;
    const int oe = std::min(K0 + kLuOuter, d.m), M = d.m - oe, K = oe - K0;
    const double* L21 = d.A + oe + (size_t)K0 * d.lda;
    s.add(L21, d.lda, d.A + K0 + (size_t)oe * d.lda, d.lda, d.A + oe + (size_t)oe * d.lda, d.lda,
          M, d.m - oe, K);
    s.add(L21, d.lda, d.B + K0, d.ldb, d.B + oe, d.ldb, M, d.nrhs, K);
  }
  return s;
}

// Backward, once rows K0..oe-1 of B hold the solution: rows 0..K0-1 of B -=
// U[0:K0, K0:oe] B[K0:oe, :].
TcStep bwd_step(const std::vector<LuDescHost>& h, int K0) {
  TcStep s;
  for (const auto& d : h) {
    if (K0 >= d.m || K0 == 0) continue;
    const int oe = std::min(K0 + kLuOuter, d.m);
    s.add(d.A + (size_t)K0 * d.lda, d.lda, d.B + K0, d.ldb, d.B, d.ldb, K0, d.nrhs, oe - K0);
  }
  return s;
}

}  // namespace

size_t lu_tc_workspace(const std::vector<LuDescHost>& h) {
  int max_m = 0;
  for (const auto& d : h) max_m = std::max(max_m, d.m);
  size_t w = 0;
  for (int K0 = 0; K0 < max_m; K0 += kLuOuter) {
    TcStep f = fwd_step(h, K0), b = bwd_step(h, K0);
    w = std::max(w, oz_plan(f.oz));
    w = std::max(w, oz_plan(b.oz));
  }
  return w;
}

cudaError_t lu_solve_tc(const LuDesc<double>* d_desc, const std::vector<LuDescHost>& h,
                        int* d_status, cudaStream_t st,
                        void* (*push)(void* ctx, const void* src, size_t bytes), void* push_ctx,
                        void* ws, size_t ws_bytes) {
  using R = double;
  using TL = TileSq<R>;
  const int nd = (int)h.size();
  if (nd == 0) return cudaSuccess;
  int max_m = 0, max_nrhs = 0;
  for (const auto& d : h) {
    max_m = std::max(max_m, d.m);
    max_nrhs = std::max(max_nrhs, d.nrhs);
  }
  const int smem_max = 224 * 1024;
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_lu_panel<R>), smem_max))
    return cudaErrorInvalidValue;
  const int cpc = nd >= 64 ? 64 : 16;  // columns per CTA of the interchange kernels
  const double es = 8.0;
  // per-descriptor maxima and sums over the descriptors that reach panel k0
  auto over = [&](int k0, auto fn) {
    for (const auto& d : h)
      if (k0 < d.m) fn(d.m, d.nrhs, std::min(kNB, d.m - k0));
  };
  auto run_step = [&](TcStep& s, const char* tc_name, const char* simt_name) -> cudaError_t {
    if (!s.oz.empty()) {
      if (oz_plan(s.oz) > ws_bytes) return cudaErrorInvalidValue;
      auto* dz = static_cast<const OzDesc*>(push(push_ctx, s.oz.data(), s.oz.size() * sizeof(OzDesc)));
      const cudaError_t e = oz_gemm(dz, s.oz, ws, ws_bytes, -1.0, 1.0, d_status, st, tc_name);
      if (e != cudaSuccess) return e;
    }
    if (!s.simt.empty()) {
      auto* dg = static_cast<const GemmDesc<double>*>(
          push(push_ctx, s.simt.data(), s.simt.size() * sizeof(GemmDesc<double>)));
      gemm_batched<R>(dg, (int)s.simt.size(), s.maxM, s.maxN, R(-1), R(1), st, simt_name,
                      s.simt_flops, s.simt_bytes, s.maxK);
    }
    return cudaGetLastError();
  };
  for (int K0 = 0; K0 < max_m; K0 += kLuOuter) {
    const int kend = std::min(K0 + kLuOuter, max_m);
    // 1. the outer block column: one-level steps restricted to it
    for (int k0 = K0; k0 < kend; k0 += kNB) {
      {
        double fl = 0.0, by = 0.0;
        over(k0, [&](int m, int, int nbk) {
          const int rows = m - k0;
          for (int jj = 0; jj < nbk; ++jj) fl += (double)(rows - jj - 1) * (2.0 * (nbk - jj - 1) + 1.0);
          by += 2.0 * rows * nbk * es;
        });
        launch_panel<R>(d_desc, nd, max_m, k0, d_status, st, fl, by);
      }
      int cols = 0, Mx = 0, Nx = 0;
      double fl = 0.0, by = 0.0, flu = 0.0, byu = 0.0;
      over(k0, [&](int m, int, int nbk) {
        const int oe = std::min(K0 + kLuOuter, m), right = oe - k0 - nbk, M = m - k0 - nbk;
        cols = std::max(cols, (k0 - K0) + right);
        Mx = std::max(Mx, M);
        Nx = std::max(Nx, right);
        fl += (double)nbk * (nbk - 1) * right;
        by += 2.0 * nbk * ((k0 - K0) + right) * es;
        flu += 2.0 * M * (double)right * nbk;
        byu += ((double)M * nbk + (double)nbk * right + 2.0 * M * right) * es;
      });
      if (cols > 0) {
        const int chunks = (cols + cpc - 1) / cpc;
        prof::Scope sc(TName<R>::swap(), st, fl, by);
        k_lu_swap_trsm<R><<<(unsigned)((long long)nd * chunks), 256, 0, st>>>(d_desc, k0, chunks,
                                                                            cpc, 0, 0, 0, K0);
      }
      if (Mx > 0 && Nx > 0) {
        const int tpm = (Mx + TL::BM - 1) / TL::BM, tpn = (Nx + TL::BN - 1) / TL::BN;
        prof::Scope sc(TName<R>::update(), st, flu, byu);
        k_lu_update<R, TL><<<(unsigned)((long long)nd * tpm * tpn), TL::NT, TL::SMEM, st>>>(
            d_desc, k0, tpm, tpn, 0, 0, K0);
      }
    }
    // 2. the far columns: the block's interchanges, then its unit-lower solve
    {
      int cols = 0;
      double by = 0.0;
      over(K0, [&](int m, int nrhs, int) {
        const int oe = std::min(K0 + kLuOuter, m);
        cols = std::max(cols, m - oe + nrhs);
        by += 2.0 * 2.0 * (oe - K0) * (double)(m - oe + nrhs) * es;
      });
      if (cols > 0) {
        const int chunks = (cols + cpc - 1) / cpc;
        prof::Scope sc(TName<R>::swap(), st, 0.0, by);
        k_lu_swap_far<R><<<(unsigned)((long long)nd * chunks), 256, 0, st>>>(d_desc, K0, chunks,
                                                                           cpc);
      }
    }
    for (int k0 = K0; k0 < kend; k0 += kNB) {
      int cols = 0, Mx = 0, NA = 0, NB = 0;
      double fl = 0.0, by = 0.0, flu = 0.0, byu = 0.0;
      over(k0, [&](int m, int nrhs, int nbk) {
        const int oe = std::min(K0 + kLuOuter, m), far = m - oe + nrhs, M = oe - k0 - nbk;
        cols = std::max(cols, far);
        fl += (double)nbk * (nbk - 1) * far;
        by += 2.0 * nbk * far * es;
        if (M > 0) {
          Mx = std::max(Mx, M);
          NA = std::max(NA, m - oe);
          NB = std::max(NB, nrhs);
          flu += 2.0 * M * (double)far * nbk;
          byu += ((double)M * nbk + (double)nbk * far + 2.0 * M * far) * es;
        }
      });
      if (cols > 0) {
        const int chunks = (cols + cpc - 1) / cpc;
        prof::Scope sc(TName<R>::swap(), st, fl, by);
        k_lu_swap_trsm<R><<<(unsigned)((long long)nd * chunks), 256, 0, st>>>(d_desc, k0, chunks,
                                                                            cpc, 0, 0, 1, K0);
      }
      if (Mx > 0 && NA + NB > 0) {
        const int tpm = (Mx + TL::BM - 1) / TL::BM;
        const int tpnA = (NA + TL::BN - 1) / TL::BN, tpnB = (NB + TL::BN - 1) / TL::BN;
        prof::Scope sc(TName<R>::update(), st, flu, byu);
        k_lu_update<R, TL><<<(unsigned)((long long)nd * tpm * (tpnA + tpnB)), TL::NT, TL::SMEM,
                             st>>>(d_desc, k0, tpm, tpnA, tpnB, 1, K0);
      }
    }
    // 3. the trailing rows: one rank-kLuOuter product
    TcStep f = fwd_step(h, K0);
    const cudaError_t e = run_step(f, "lu_update_tc<f64>", TName<R>::update());
    if (e != cudaSuccess) return e;
  }
  // backward substitution, blocked the same way
  const int lastK0 = ((max_m - 1) / kLuOuter) * kLuOuter;
  for (int K0 = lastK0; K0 >= 0; K0 -= kLuOuter) {
    const int kend = std::min(K0 + kLuOuter, max_m);
    for (int kb0 = K0 + ((kend - 1 - K0) / kNB) * kNB; kb0 >= K0; kb0 -= kNB) {
      {
        double fl = 0.0, by = 0.0;
        over(kb0, [&](int, int nrhs, int nbk) {
          fl += (double)nbk * nbk * nrhs;
          by += (2.0 * nbk * nrhs + 0.5 * nbk * nbk) * es;
        });
        const int chunks = (max_nrhs + kTrsmCols - 1) / kTrsmCols;
        prof::Scope sc(TName<R>::trsm(), st, fl, by);
        k_trsm_upper<R><<<(unsigned)((long long)nd * chunks), kTrsmCols, 0, st>>>(d_desc, kb0,
                                                                                chunks);
      }
      if (kb0 > K0) {
        double fl = 0.0, by = 0.0;
        const int M = kb0 - K0;
        over(kb0, [&](int, int nrhs, int nbk) {
          fl += 2.0 * M * (double)nrhs * nbk;
          by += ((double)M * nbk + (double)nbk * nrhs + 2.0 * M * nrhs) * es;
        });
        const int tpm = (M + TL::BM - 1) / TL::BM, tpn = (max_nrhs + TL::BN - 1) / TL::BN;
        prof::Scope sc(TName<R>::backsub(), st, fl, by);
        k_backsub_update<R, TL><<<(unsigned)((long long)nd * tpm * tpn), TL::NT, TL::SMEM, st>>>(
            d_desc, kb0, tpm, tpn, K0);
      }
    }
    if (K0 > 0) {
      TcStep b = bwd_step(h, K0);
      const cudaError_t e = run_step(b, "backsub_tc<f64>", TName<R>::backsub());
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template void lu_solve_batched<double>(const LuDesc<double>*, int, int, int, int, int*,
                                       cudaStream_t, const int*, const int*);
template void lu_solve_batched<float>(const LuDesc<float>*, int, int, int, int, int*,
                                      cudaStream_t, const int*, const int*);
#define HPS_INST_GEMM(R, TA, TB, TC)                                                            \
  template void gemm_batched<R, TA, TB, TC>(const GemmDesc<TA, TB, TC>*, int, int, int, R, R,   \
                                            cudaStream_t, const char*, double, double, int, R*, \
                                            size_t, int*);
HPS_INST_GEMM(double, double, double, double)
HPS_INST_GEMM(float, float, float, float)
HPS_INST_GEMM(float, float, double, double)
HPS_INST_GEMM(float, float, float, double)
HPS_INST_GEMM(double, double, double, float)

}  // namespace hps
