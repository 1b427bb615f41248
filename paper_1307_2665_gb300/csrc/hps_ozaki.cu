// FP64 GEMM on the 5th-generation tensor cores by exact splitting (Ozaki's
// scheme; Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012).
//
// GB300 runs FP64 FMAs at 1/64 of the FP32 rate and its FP64 tensor path is no
// faster, while BF16 tensor MMAs with FP32 accumulation run ~1000x faster.
// C (+)= A B with A, B in FP64 is computed here as follows.
//   1. Split.  Every row i of A gets an exponent eA_i with max_k |A_ik| < 2^eA_i
//      and is cut into S = 8 signed 7-bit integer slices:
//        A_ik = 2^eA_i sum_s a^(s)_ik 2^(-7 s) + r_ik,  |a^(s)| <= 127,
//        |r_ik| < 2^(eA_i - 56),
//      (the 56-bit fixed-point value of |A_ik| / 2^eA_i, cut in 7-bit groups,
//      with the sign of A_ik); the same for every column j of B with eB_j.
//      Slices are integers of at most 8 significant bits, exact in BF16.
//   2. Multiply.  For every slice pair (s, t) with s + t <= 9 (the dropped
//      pairs weigh at most 2^-70 of |A| |B|), P = a^(s) b^(t) on the tensor
//      cores, the pairs of equal d = s + t accumulated together in FP32 in
//      tensor memory, one 128-wide K group at a time: at most 8 pairs share a
//      d, so every partial sum is an integer of magnitude
//      <= 8 * 128 * 127^2 = 16 516 096 < 2^24, hence exact (checked at compile
//      time below).
//   3. Combine.  Per output, the exact integers P_st of equal d = s + t are
//      summed in two 64-bit fixed-point accumulators,
//        U_hi = sum_{d=2..5} P_d 2^(7 (5 - d)),  U_lo = sum_{d=6..9} P_d 2^(7 (9 - d)),
//      (each < 2^50, exact in FP64), and
//        C_ij (+)= 2^(eA_i + eB_j) (U_hi 2^-35 + U_lo 2^-63)
//      with one FP64 rounding for the sum; the blocks' integers add exactly.
// The error is at most ~2^-55 K max|A_i.| max|B_.j| per entry, the order of an
// FP64 GEMM's own rounding bound, and the result depends only on the operands
// (no atomics, fixed order), so a product gives the same bits in any batch.
//
// Kernels: k_oz_exp_rows / k_oz_exp_cols (exponents), k_oz_split (slices in the
// tensor cores' shared-memory operand layout: K-major, 8x8-element core
// matrices, no swizzle), k_oz_gemm (one CTA per 128 x 64 tile of C: bulk
// asynchronous copies of all slices of a K block into shared memory,
// tcgen05.mma issued by one thread into eight diagonal TMEM accumulators, all
// eight warps draining them with tcgen05.ld while the next block's copies run).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "hps_kernels.cuh"
#include "hps_prof.hpp"

namespace hps {

namespace {

constexpr int kS = 8;          // slices per operand
constexpr int kBeta = 7;       // bits per slice
constexpr int kTM = 128;       // tile rows (UMMA M)
constexpr int kTN = 64;        // tile columns (UMMA N)
constexpr int kKB = 32;        // K per operand block (4 core matrices)
constexpr int kGroup = 4;      // blocks per exact accumulation (K = 128)
constexpr int kABlock = kTM * kKB;  // BF16 elements of an A block (8 KB)
constexpr int kBBlock = kTN * kKB;  // BF16 elements of a B block (4 KB)
constexpr int kStage = kS * (kABlock + kBBlock);  // all slices of one block (96 KB)
constexpr int kThreads = 256;
constexpr int kNoExp = (int)0x80808080;  // exponent of an all-zero row / column (bytes 0x80)
constexpr long kSpin = 1L << 20;    // bound of every wait (iterations)
// Exactness of the FP32 tensor-memory sums: at most kS slice pairs share a
// diagonal, each adding kGroup * kKB products of magnitude <= 127^2 before the
// accumulator is drained, and FP32 holds every integer below 2^24.
static_assert((long)kS * kGroup * kKB * 127 * 127 < (1L << 24),
              "slice products of one K group must sum exactly in FP32");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// exponent e with |x| < 2^e for the largest |x| of a row / column
__device__ __forceinline__ int exp_of(double mx) { return mx > 0.0 ? ilogb(mx) + 1 : kNoExp; }
// the exponent a row / column is scaled by (an all-zero one is scaled by 1)
__device__ __forceinline__ int exp_at(const int* ework, int i) {
  const int e = ework[i];
  return e == kNoExp ? 0 : e;
}

}  // namespace

// ------------------------------------------------------------------ split
// Exponents: each thread (rows of A) or warp (columns of B) takes a chunk of K
// and folds its exponent in with an integer atomicMax (order-independent).
// ework starts at kNoExp.
__global__ void k_oz_exp_rows(const OzDesc* __restrict__ d, int* __restrict__ ework) {
  const OzDesc g = d[blockIdx.z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * 64;
  if (i >= g.M || k0 >= g.K) return;
  double mx = 0.0;
  for (int k = k0; k < min(g.K, k0 + 64); ++k) mx = fmax(mx, fabs(g.A[i + (size_t)k * g.lda]));
  if (mx > 0.0) atomicMax(&ework[g.ea_off + i], exp_of(mx));
}

__global__ void k_oz_exp_cols(const OzDesc* __restrict__ d, int* __restrict__ ework) {
  const OzDesc g = d[blockIdx.z];
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  const int k0 = blockIdx.y * 256;
  if (j >= g.N || k0 >= g.K) return;
  double mx = 0.0;
  for (int k = k0 + lane; k < min(g.K, k0 + 256); k += 32)
    mx = fmax(mx, fabs(g.B[k + (size_t)j * g.ldb]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.0) atomicMax(&ework[g.eb_off + j], exp_of(mx));
}

// The 8 slices of x relative to 2^e: sign * ((F >> (56 - 7 s)) & 127), F the
// 56-bit fixed-point value floor(|x| 2^(56 - e)) (integer arithmetic on the
// bits of x; x is exact in it to 2^(e - 56)).
__device__ __forceinline__ void slice8(double x, int e, int* q) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & 0xfffffffffffffULL;
  int E;  // x = m 2^E
  if (ex == 0) {
    E = -1074;
  } else {
    m |= 1ULL << 52;
    E = ex - 1075;
  }
  const int sh = E + 56 - e;
  unsigned long long F = 0;
  if (m != 0 && sh > -64) F = sh >= 0 ? (m << sh) : (m >> (-sh));
  const int sg = (bits >> 63) ? -1 : 1;
#pragma unroll
  for (int s = 1; s <= kS; ++s) q[s - 1] = sg * (int)((F >> (56 - kBeta * s)) & 127ULL);
}

// One CTA per (descriptor, tile, K block) of A (side 0, 128-row tiles) or B
// (side 1, 64-row tiles of B^T); writes all 8 slices of the block.  The FP64
// block is read coalesced into shared memory, then slices are written in the
// order of the operand layout (consecutive threads, consecutive elements).
__global__ void __launch_bounds__(kThreads) k_oz_split(const OzDesc* __restrict__ d, int side,
                                                       const int* __restrict__ ework,
                                                       __nv_bfloat16* __restrict__ work) {
  const OzDesc g = d[blockIdx.z];
  const int tile = blockIdx.x, kb = blockIdx.y;
  const int rows = side == 0 ? kTM : kTN;
  const int ntiles = side == 0 ? g.mt : g.nt;
  if (tile >= ntiles || kb >= g.nkb) return;
  __shared__ double X[kKB * (kTM + 1)];  // X[k * (rows + 1) + r]
  __shared__ int ex[kTM];
  const int ld = rows + 1;
  for (int e = threadIdx.x; e < rows * kKB; e += kThreads) {
    int r, k;
    if (side == 0) {  // A: consecutive threads, consecutive rows (contiguous)
      r = e % rows;
      k = e / rows;
    } else {          // B: consecutive threads, consecutive k of one column
      k = e % kKB;
      r = e / kKB;
    }
    const int gi = tile * rows + r, gk = kb * kKB + k;
    double x = 0.0;
    if (side == 0 ? (gi < g.M && gk < g.K) : (gi < g.N && gk < g.K))
      x = side == 0 ? g.A[gi + (size_t)gk * g.lda] : g.B[gk + (size_t)gi * g.ldb];
    X[k * ld + r] = x;
  }
  for (int r = threadIdx.x; r < rows; r += kThreads) {
    const int gi = tile * rows + r;
    const bool in = side == 0 ? gi < g.M : gi < g.N;
    ex[r] = in ? exp_at(ework, (side == 0 ? g.ea_off : g.eb_off) + gi) : 0;
  }
  __syncthreads();
  // block-major: the 8 slices of one (tile, K block) are contiguous, so the
  // GEMM fetches a block's operand with one bulk copy
  const int blk = side == 0 ? kABlock : kBBlock;
  const int64_t base =
      (side == 0 ? g.a_off : g.b_off) + ((int64_t)tile * g.nkb + kb) * kS * (int64_t)blk;
  for (int o = threadIdx.x; o < blk; o += kThreads) {
    // operand layout: core (r / 8, k / 8) of 64 elements, rows of 8 k
    const int core = o >> 6, w = o & 63;
    const int r = (core / (kKB / 8)) * 8 + (w >> 3), k = (core % (kKB / 8)) * 8 + (w & 7);
    int q[kS];
    slice8(X[k * ld + r], ex[r], q);
#pragma unroll
    for (int s = 0; s < kS; ++s) work[base + s * blk + o] = __float2bfloat16_rn((float)q[s]);
  }
}

// ------------------------------------------------------------------ GEMM
namespace {

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // K-major, no swizzle: LBO = 128 B between core matrices along K, SBO =
  // (kKB / 8) * 128 B between 8-row groups.  Advancing the operand by X bytes
  // adds X >> 4 to the descriptor (the start address is its low field).
  uint64_t dsc = (uint64_t)((saddr >> 4) & 0x3FFF);
  dsc |= (uint64_t)(128 >> 4) << 16;
  dsc |= (uint64_t)((kKB / 8) * 128 >> 4) << 32;
  dsc |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
  return dsc;
}

// kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

// bounded wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (long it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

}  // namespace

// grid: (nt, mt, descriptor); 256 threads.  Two stages of shared memory each
// hold all 8 A slices (8 x 8 KB) and all 8 B slices (8 x 4 KB) of one K block
// of 32, filled by two bulk copies (the slices of a block are contiguous in
// the workspace) on the stage's barrier; the copies of block
// kb + 1 run while block kb multiplies.  Thread 0 issues the 36 pair products
// of a block into 8 TMEM accumulators, one per diagonal d = s + t (8 x 64
// columns: all of tensor memory), accumulating over groups of 4 blocks (a
// diagonal's sums stay below 8 * 128 * 127^2 < 2^24, exact in FP32); after
// each group the eight warps drain the accumulators into 64-bit sums.
__global__ void __launch_bounds__(kThreads, 1) k_oz_gemm(const OzDesc* __restrict__ d,
                                                         const int* __restrict__ ework,
                                                         const __nv_bfloat16* __restrict__ work,
                                                         double alpha, double beta,
                                                         int* __restrict__ status) {
  const OzDesc g = d[blockIdx.z];
  const int tn = blockIdx.x, tm = blockIdx.y;
  if (tn >= g.nt || tm >= g.mt) return;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __nv_bfloat16* stage[2] = {reinterpret_cast<__nv_bfloat16*>(smraw),
                             reinterpret_cast<__nv_bfloat16*>(smraw) + kStage};
  // bar_ld[b]: copies into stage b; bar_mma[b]: products reading stage b are
  // done (thread 0 waits on it every block); bar_grp: a group's products are
  // done (one commit per group: the drain waits on it once per group, so no
  // waiter is ever two phases from the barrier)
  __shared__ __align__(8) uint64_t bar_ld[2], bar_mma[2], bar_grp;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kCols = kS * kTN;  // 8 diagonal accumulators x 64 columns = 512
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bar_ld[0], 1);
    mbar_init(&bar_ld[1], 1);
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    mbar_init(&bar_grp, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int r = 32 * (warp & 3) + lane;
  const int c0 = 32 * (warp >> 2);
  long long uhi[32], ulo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) uhi[j] = ulo[j] = 0;
  bool gfail = false;
  bool pfail = false;  // thread 0 only
  // thread 0 only: blocks whose copies / products were issued, and how many of
  // each are known complete (what a failed CTA must still wait for)
  int ld_issued = 0, ld_done = 0, mma_issued = 0, mma_done = 0;

  auto load_block = [&](int kb) {  // thread 0: all slices of block kb into stage kb & 1
    const int b = kb & 1;
    __nv_bfloat16* As = stage[b];
    __nv_bfloat16* Bs = stage[b] + kS * kABlock;
    expect_tx(&bar_ld[b], (uint32_t)(kStage * 2));
    bulk_load(As, work + g.a_off + ((int64_t)tm * g.nkb + kb) * kS * kABlock,
              (uint32_t)(kS * kABlock * 2), &bar_ld[b]);
    bulk_load(Bs, work + g.b_off + ((int64_t)tn * g.nkb + kb) * kS * kBBlock,
              (uint32_t)(kS * kBBlock * 2), &bar_ld[b]);
    ++ld_issued;
  };
  if (tid == 0) {
    load_block(0);
    if (g.nkb > 1) load_block(1);
  }
  for (int kb = 0; kb < g.nkb; ++kb) {
    const int b = kb & 1;
    const uint32_t par = (uint32_t)((kb >> 1) & 1);  // phase of this stage's barriers
    const bool group_start = (kb % kGroup) == 0;
    const bool group_end = (kb % kGroup) == kGroup - 1 || kb == g.nkb - 1;
    // ---- products of block kb (thread 0)
    if (tid == 0 && !pfail) {
      // first refill the other stage with block kb + 1, once block kb - 1 (which
      // used it) has finished multiplying: the copy then runs while block kb's
      // products execute, however long their issue takes
      if (kb >= 1 && kb + 1 < g.nkb) {
        const int ob = (kb - 1) & 1;
        if (!mbar_wait(&bar_mma[ob], (uint32_t)(((kb - 1) >> 1) & 1))) pfail = true;
        else mma_done = kb;  // products complete in issue order
        if (!pfail) load_block(kb + 1);
      }
      if (!pfail && !mbar_wait(&bar_ld[b], par)) pfail = true;
      if (!pfail) ld_done = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!pfail) {
        const uint64_t da0 = smem_desc(smem_u32(stage[b]));
        const uint64_t db0 = smem_desc(smem_u32(stage[b] + kS * kABlock));
        for (int si = 1; si <= kS; ++si)
          for (int ti = 1; si + ti <= kS + 1; ++ti) {
            const uint32_t acc = tmem + (uint32_t)((si + ti - 2) * kTN);
#pragma unroll
            for (int k16 = 0; k16 < kKB / 16; ++k16) {
              // operand advance: slice (si - 1) blocks, k16 * 2 core matrices
              const uint64_t da = da0 + (uint64_t)(((si - 1) * kABlock * 2 + k16 * 256) >> 4);
              const uint64_t db = db0 + (uint64_t)(((ti - 1) * kBBlock * 2 + k16 * 256) >> 4);
              // the first product of a diagonal in a group starts its accumulator
              const uint32_t en = (!group_start || si > 1 || k16 > 0) ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                  "l"(da), "l"(db), "r"(kIdesc), "r"(en)
                  : "memory");
            }
          }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar_mma[b]))
            : "memory");
        mma_issued = kb + 1;
        if (group_end)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(&bar_grp))
              : "memory");
      }
      if (pfail) s_fail = 1;
    }
    // ---- at the end of a group: wait for its products, drain the accumulators
    if (group_end) {
      const uint32_t gpar = (uint32_t)((kb / kGroup) & 1);
      const bool ok = !gfail && __all_sync(0xffffffffu, mbar_wait(&bar_grp, gpar));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok && tid == 0) mma_done = kb + 1;
      if (ok) {
#pragma unroll 1
        for (int dd = 2; dd <= kS + 1; ++dd) {
          const uint32_t addr = tmem + (uint32_t)((dd - 2) * kTN) +
                                ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
          uint32_t v[32];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
              "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                "=r"(v[30]), "=r"(v[31])
              : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (dd <= 5) {
            const int sh = kBeta * (5 - dd);
#pragma unroll
            for (int j = 0; j < 32; ++j)
              uhi[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
          } else {
            const int sh = kBeta * (9 - dd);
#pragma unroll
            for (int j = 0; j < 32; ++j)
              ulo[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
          }
        }
      } else if (lane == 0) {
        atomicExch(&s_fail, 1);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // accumulators drained: the next group may overwrite them
      gfail = s_fail != 0;
    }
  }
  // ---- epilogue: C = alpha 2^(eA+eB) (U_hi 2^-35 + U_lo 2^-63) + beta C
  if (!gfail) {
    const int gi = tm * kTM + r;
    if (gi < g.M) {
      const int ea = exp_at(ework, g.ea_off + gi);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int gj = tn * kTN + c0 + j;
        if (gj >= g.N) break;
        const int ee = ea + exp_at(ework, g.eb_off + gj);
        const double v = ldexp((double)uhi[j], ee - 35) + ldexp((double)ulo[j], ee - 63);
        double* cp = g.C + gi + (size_t)gj * g.ldc;
        *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
      }
    }
  } else if (tid == 0) {
    // a wait gave up: before this CTA's shared and tensor memory are released,
    // let its own copies and products still in flight finish (each wait is
    // bounded again), then report a device error
    for (int j = ld_done; j < ld_issued; ++j) mbar_wait(&bar_ld[j & 1], (uint32_t)((j >> 1) & 1));
    for (int j = mma_done; j < mma_issued; ++j)
      mbar_wait(&bar_mma[j & 1], (uint32_t)((j >> 1) & 1));
    if (status) atomicCAS(status, 0, -1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// ------------------------------------------------------------------ host
size_t oz_plan(std::vector<OzDesc>& ds) {
  int64_t slice_elems = 0, exps = 0;
  for (auto& g : ds) {
    g.mt = (g.M + kTM - 1) / kTM;
    g.nt = (g.N + kTN - 1) / kTN;
    g.nkb = (g.K + kKB - 1) / kKB;
    g.a_off = slice_elems;
    slice_elems += (int64_t)kS * g.mt * g.nkb * kABlock;
    g.b_off = slice_elems;
    slice_elems += (int64_t)kS * g.nt * g.nkb * kBBlock;
    g.ea_off = (int)exps;
    exps += g.M;
    g.eb_off = (int)exps;
    exps += g.N;
  }
  // slices (BF16) then exponents (int), 256-byte aligned
  const size_t sb = ((size_t)slice_elems * 2 + 255) & ~size_t(255);
  return sb + (size_t)exps * sizeof(int);
}

cudaError_t oz_gemm(const OzDesc* d_desc, const std::vector<OzDesc>& h, void* work,
                    size_t work_bytes, double alpha, double beta, int* status, cudaStream_t st,
                    const char* name) {
  const int nd = (int)h.size();
  if (nd == 0) return cudaSuccess;
  int64_t slice_elems = 0;
  int maxM = 0, maxN = 0, max_mt = 0, max_nt = 0, max_kb = 0;
  double flops = 0, bytes = 0;
  for (const auto& g : h) {
    slice_elems = std::max(slice_elems, g.b_off + (int64_t)kS * g.nt * g.nkb * kBBlock);
    maxM = std::max(maxM, g.M);
    maxN = std::max(maxN, g.N);
    max_mt = std::max(max_mt, g.mt);
    max_nt = std::max(max_nt, g.nt);
    max_kb = std::max(max_kb, g.nkb);
    flops += 2.0 * g.M * (double)g.N * g.K;
    bytes += 8.0 * ((double)g.M * g.K + (double)g.K * g.N + 2.0 * g.M * g.N);
  }
  const size_t sb = ((size_t)slice_elems * 2 + 255) & ~size_t(255);
  __nv_bfloat16* slices = static_cast<__nv_bfloat16*>(work);
  int* ew = reinterpret_cast<int*>(static_cast<char*>(work) + sb);
  (void)work_bytes;
  int maxK = 0;
  int64_t nexp = 0;
  for (const auto& g : h) {
    maxK = std::max(maxK, g.K);
    nexp = std::max<int64_t>(nexp, (int64_t)g.eb_off + g.N);
  }
  prof::Scope sc(name, st, flops, bytes);
  cudaError_t e = cudaMemsetAsync(ew, 0x80, (size_t)nexp * sizeof(int), st);  // kNoExp bytes
  if (e != cudaSuccess) return e;
  k_oz_exp_rows<<<dim3((maxM + 127) / 128, (maxK + 63) / 64, nd), 128, 0, st>>>(d_desc, ew);
  k_oz_exp_cols<<<dim3((maxN + 7) / 8, (maxK + 255) / 256, nd), 256, 0, st>>>(d_desc, ew);
  k_oz_split<<<dim3(max_mt, max_kb, nd), kThreads, 0, st>>>(d_desc, 0, ew, slices);
  k_oz_split<<<dim3(max_nt, max_kb, nd), kThreads, 0, st>>>(d_desc, 1, ew, slices);
  const int smem = 2 * kStage * 2;
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_oz_gemm), smem)) return cudaErrorInvalidValue;
  k_oz_gemm<<<dim3(max_nt, max_mt, nd), kThreads, smem, st>>>(d_desc, ew, slices, alpha, beta,
                                                               status);
  return cudaGetLastError();
}

}  // namespace hps
