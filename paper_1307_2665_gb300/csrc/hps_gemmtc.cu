// Batched FP32 GEMM on the tensor cores: C = beta C + alpha A B (column-major,
// A in FP32, B and C in FP32 or FP64), the low-precision products of the
// mixed-precision build and solve (Section 6's FP32 leaf and merge algebra).
//
// Every FP32 operand x is split exactly into three BF16 terms by rounding to
// nearest: x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2) (each
// remainder is exact in FP32 and the three terms carry all 24 bits).  A
// product a b is then sum_{i + j <= 4} a_i b_j (six tcgen05 BF16 MMAs per K
// step of 16, each product exact in FP32); the dropped terms a2 b3, a3 b2,
// a3 b3 weigh about 2^-24 of |a b|.  The tensor cores' FP32 accumulation aligns
// its addends and drops low bits, an error that grows with every MMA into one
// accumulator: so each K block of 32 sums into fresh accumulators, the leading
// term a1 b1 apart from the five smaller ones, and the block sums are added in
// FP32 registers (round to nearest).  The result carries the rounding of an
// FP32 FMA chain.
//
// A CTA computes a 128 x BN tile of one product: per K block of 32 its 256
// threads load the FP32 tiles (the next block's loads are in flight during
// this block's products), split them into the two-stage shared-memory ring in
// the K-major no-swizzle layout, and thread 0 issues 2 x 6 MMAs into the
// block's two accumulators (double-buffered in tensor memory) and commits them
// to the stage's mbarrier; while they run, all eight warps add the previous
// block's sums into registers.  Waits are bounded: a CTA whose wait gives up sets
// *status to -1, waits (bounded again) for its products in flight and frees
// its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"
#include "hps_tc.cuh"

namespace hps {

namespace {

constexpr int kGM = 128;           // tile rows (TMEM lanes)
constexpr int kGKB = 32;           // K per block (two MMA steps of 16)
constexpr int kGThreads = 256;
constexpr int kGSub = kGM * 16 * 2;  // bytes of one A sub-tile: 128 rows x 16 k (BF16)
constexpr long kGSpin = 1L << 22;  // bound of every wait (iterations)

using tc::g_off;
using tc::split8;
using tc::st16;

template <int BN>
struct GTile {
  static constexpr int kBSub = BN * 16 * 2;                  // bytes of one B sub-tile
  static constexpr int kStage = 3 * 2 * (kGSub + kBSub);     // 3 terms x 2 sub-tiles
  static constexpr int kSmem = 2 * kStage;
  static constexpr int kAPer = kGM * kGKB / kGThreads;       // A values per thread: 16
  static constexpr int kBPer = BN * kGKB / kGThreads;        // B values per thread
  static_assert(kAPer == 16 && (kBPer == 8 || kBPer == 16), "load split");
};

// CTA (descriptor, m tile, n tile).  The launch with BN = 64 takes the
// products with N <= 64, the one with BN = 128 the wider ones (each product's
// own N decides).  Per K block of 32: the threads split the block's FP32
// values (loaded during the previous block) into the block's operand stage
// and start the loads of the next block; thread 0 issues 2 x 6 MMAs into the
// block's two accumulators (double-buffered in tensor memory) and commits
// them; meanwhile the previous block's sums are added into registers.
template <typename TB, typename TC, int BN>
__global__ void __launch_bounds__(kGThreads, BN == 64 ? 2 : 1) k_gemm_tc32(
    const GemmDesc<float, TB, TC>* __restrict__ d, int tpm, int tpn, float alpha, float beta,
    int* __restrict__ status) {
  using T = GTile<BN>;
  constexpr int kCols = 4 * BN;  // two blocks' accumulators (leading, small)
  const int per = tpm * tpn;
  const GemmDesc<float, TB, TC> g = d[blockIdx.x / per];
  const int tile = blockIdx.x % per;
  const int m0 = (tile % tpm) * kGM, n0 = (tile / tpm) * BN;
  // uniform, before any allocation: this product's tile on this launch?
  if (!gemm_on_tc(g.M, g.K) || (BN == 64) != (g.N <= 64)) return;
  if (m0 >= g.M || n0 >= g.N) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int M = g.M, N = g.N, K = g.K;
  const int nkb = (K + kGKB - 1) / kGKB;
  // A: row am = tid % 128 of the tile, k chunks (tid / 128) and + 2 of 8 each
  const int am = tid & (kGM - 1), ac = tid >> 7;
  // B: row bn of the tile (an output column), kBPer / 8 chunks of 8 k from bc0
  constexpr int kBChunks = kGKB / 8;                   // 4 chunks of 8 k per block
  constexpr int kBcPer = T::kBPer / 8;
  const int bn = tid / (kBChunks / kBcPer), bc0 = (tid % (kBChunks / kBcPer)) * kBcPer;
  float av[16], bv[T::kBPer];
  auto fetch = [&](int kb) {
    const int k0 = kb * kGKB;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + (ac + 2 * c) * 8 + j, m = m0 + am;
        av[c * 8 + j] = (m < M && k < K) ? g.A[m + (size_t)k * g.lda] : 0.0f;
      }
#pragma unroll
    for (int c = 0; c < kBcPer; ++c)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + (bc0 + c) * 8 + j, n = n0 + bn;
        bv[c * 8 + j] = (n < N && k < K) ? (float)g.B[k + (size_t)n * g.ldb] : 0.0f;
      }
  };
  bool fail = false;
  int ncommit = 0;  // thread 0: committed blocks (block b on stage b & 1, phase b >> 1)
  // this thread's share of the tile: lane r of quadrant warp % 4, columns
  // cb .. cb + BN/2 - 1; block sums added in FP32 (round to nearest)
  const int r = 32 * (warp & 3) + lane;
  const int cb = (warp >> 2) * (BN / 2);
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  float acc[BN / 2];
#pragma unroll
  for (int j = 0; j < BN / 2; ++j) acc[j] = 0.0f;
  // block b's accumulators: columns (b & 1) * 2 BN (leading term a1 b1) and
  // + BN (the five smaller terms)
  auto drain_block = [&](int b) {
    const uint32_t base = tl + (uint32_t)((b & 1) * 2 * BN + cb);
#pragma unroll
    for (int c16 = 0; c16 < BN / 2; c16 += 16) {
      uint32_t vb[16], vs[16];
      tc::ld16(base + (uint32_t)c16, vb);
      tc::ld16(base + (uint32_t)(BN + c16), vs);
      tc::wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        acc[c16 + j] += __uint_as_float(vb[j]) + __uint_as_float(vs[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };
  if (nkb > 0) fetch(0);
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    // stage s and accumulator buffer s were last used by block kb - 2, whose
    // products were waited for and drained in the previous iteration
    unsigned char* As = smraw + s * T::kStage;    // 3 terms x 2 sub-tiles of A
    unsigned char* Bs = As + 3 * 2 * kGSub;       // 3 terms x 2 sub-tiles of B
    {
      uint32_t w[3][4];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int kc = ac + 2 * c;  // chunk of 8 k: sub-tile kc / 2, k half kc % 2
        split8(av + c * 8, w);
#pragma unroll
        for (int t = 0; t < 3; ++t)
          st16(tc::smem_u32(As + (t * 2 + (kc >> 1)) * kGSub + g_off(am, (kc & 1) * 8) * 2), w[t]);
      }
#pragma unroll
      for (int c = 0; c < kBcPer; ++c) {
        const int kc = bc0 + c;
        split8(bv + c * 8, w);
#pragma unroll
        for (int t = 0; t < 3; ++t)
          st16(tc::smem_u32(Bs + (t * 2 + (kc >> 1)) * T::kBSub + g_off(bn, (kc & 1) * 8) * 2),
               w[t]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (kb + 1 < nkb) fetch(kb + 1);  // in flight during this block's products
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr uint32_t idesc = tc::idesc_bf16(kGM, BN);
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
      const uint32_t big = tmem + (uint32_t)(s * 2 * BN), small = big + (uint32_t)BN;
#pragma unroll
      for (int sub = 0; sub < 2; ++sub)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          // term pairs (i, j) with i + j <= 2 (0-based): (0,0) into the leading
          // accumulator, the others into the small one
          const int ti = p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 1 : 2;
          const int tj = p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 2 : p == 4 ? 1 : 0;
          const uint64_t da = tc::desc_kmajor(a0 + (uint32_t)((ti * 2 + sub) * kGSub), 128, 256);
          const uint64_t db = tc::desc_kmajor(b0 + (uint32_t)((tj * 2 + sub) * T::kBSub), 128, 256);
          tc::mma_bf16(p == 0 ? big : small, da, db, idesc, (sub > 0 || p > 1) ? 1u : 0u);
        }
      tc::commit(&bar[s]);
      ++ncommit;
    }
    if (kb >= 1) {  // block kb - 1: wait for its products, add its sums
      const bool ok = tc::mbar_wait(&bar[s ^ 1], (uint32_t)(((kb - 1) >> 1) & 1), kGSpin);
      if (__syncthreads_or(!ok)) {
        fail = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      drain_block(kb - 1);
    }
  }
  if (!fail && nkb > 0) {
    const int b = nkb - 1;
    const bool ok = tc::mbar_wait(&bar[b & 1], (uint32_t)((b >> 1) & 1), kGSpin);
    if (__syncthreads_or(!ok)) {
      fail = true;
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      drain_block(b);
    }
  }
  if (!fail) {
    const int m = m0 + r;
    if (m < M) {
      TC* crow = g.C + m + (size_t)(n0 + cb) * g.ldc;
      const int nn = min(BN / 2, N - (n0 + cb));
      if (beta == 0.0f) {
#pragma unroll
        for (int j = 0; j < BN / 2; ++j)
          if (j < nn) crow[(size_t)j * g.ldc] = (TC)(alpha * acc[j]);
      } else {
        // per 16 columns every load of C first, then the stores (a few memory
        // round trips instead of one per element)
#pragma unroll
        for (int j0 = 0; j0 < BN / 2; j0 += 16) {
          TC cv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cv[j] = j0 + j < nn ? crow[(size_t)(j0 + j) * g.ldc] : TC(0);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j0 + j < nn)
              crow[(size_t)(j0 + j) * g.ldc] =
                  (TC)fma((TC)alpha, (TC)acc[j0 + j], (TC)beta * cv[j]);
        }
      }
    }
  } else if (tid == 0) {
    // the last committed block of each stage (and all before it) finishes
    // (bounded) before tensor memory is freed
    for (int b = max(0, ncommit - 2); b < ncommit; ++b)
      tc::mbar_wait(&bar[b & 1], (uint32_t)((b >> 1) & 1), kGSpin);
    if (status) atomicCAS(status, 0, -1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

template <typename TB, typename TC, int BN>
void launch_tc32(const GemmDesc<float, TB, TC>* d, int nd, int max_M, int max_N, float alpha,
                 float beta, int* status, cudaStream_t st) {
  const int tpm = (max_M + kGM - 1) / kGM, tpn = (max_N + BN - 1) / BN;
  const void* kern = reinterpret_cast<const void*>(&k_gemm_tc32<TB, TC, BN>);
  if (!opt_in_smem(kern, GTile<BN>::kSmem)) return;  // reported by the caller's launch check
  k_gemm_tc32<TB, TC, BN><<<(unsigned)((long long)nd * tpm * tpn), kGThreads, GTile<BN>::kSmem,
                            st>>>(d, tpm, tpn, alpha, beta, status);
}

}  // namespace

template <typename TB, typename TC>
void gemm_tc32(const GemmDesc<float, TB, TC>* d_desc, int ndesc, int max_M, int max_N,
               float alpha, float beta, int* status, cudaStream_t st) {
  if (ndesc <= 0 || max_M <= 0 || max_N <= 0) return;
  launch_tc32<TB, TC, 64>(d_desc, ndesc, max_M, std::min(max_N, 64), alpha, beta, status, st);
  if (max_N > 64)
    launch_tc32<TB, TC, 128>(d_desc, ndesc, max_M, max_N, alpha, beta, status, st);
}

template void gemm_tc32<float, float>(const GemmDesc<float, float, float>*, int, int, int, float,
                                      float, int*, cudaStream_t);
template void gemm_tc32<float, double>(const GemmDesc<float, float, double>*, int, int, int, float,
                                       float, int*, cudaStream_t);
template void gemm_tc32<double, double>(const GemmDesc<float, double, double>*, int, int, int,
                                        float, float, int*, cudaStream_t);

}  // namespace hps
