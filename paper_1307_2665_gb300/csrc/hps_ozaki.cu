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
//      cores, accumulated in FP32 in tensor memory.  Every partial sum is an
//      integer of magnitude < K 127^2 < 2^23 for K <= 448, hence exact.
//   3. Combine.  Per output, the exact integers P_st of equal d = s + t are
//      summed in two 64-bit fixed-point accumulators,
//        U_hi = sum_{d=2..5} P_d 2^(7 (5 - d)),  U_lo = sum_{d=6..9} P_d 2^(7 (9 - d)),
//      (each < 2^50, exact in FP64), and
//        C_ij (+)= 2^(eA_i + eB_j) (U_hi 2^-35 + U_lo 2^-63)
//      with one FP64 rounding for the sum.  Longer K is processed in chunks of
//      448 whose integers add exactly.
// The error is at most ~2^-55 K max|A_i.| max|B_.j| per entry, the order of an
// FP64 GEMM's own rounding bound, and the result depends only on the operands
// (no atomics, fixed order), so a product gives the same bits in any batch.
//
// Kernels: k_oz_exp_rows / k_oz_exp_cols (exponents), k_oz_split (slices in the
// tensor cores' shared-memory operand layout: K-major, 8x8-element core
// matrices, no swizzle), k_oz_gemm (one CTA per 128 x 64 tile of C: bulk
// asynchronous copies of whole operand blocks into shared memory, tcgen05.mma
// issued by one thread into two alternating TMEM accumulators, all eight warps
// draining the previous pair with tcgen05.ld while the next pair multiplies).
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
constexpr int kKB = 64;        // K per operand block (8 core matrices)
constexpr int kChunkKB = 7;    // blocks per exact K chunk (448)
constexpr int kABlock = kTM * kKB;  // BF16 elements of an A block (16 KB)
constexpr int kBBlock = kTN * kKB;  // BF16 elements of a B block (8 KB)
constexpr int kThreads = 256;
constexpr long kSpin = 1L << 20;    // bound of every wait (iterations)

__host__ __device__ constexpr int n_pairs() { return kS * (kS + 1) / 2; }  // s + t <= S + 1

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Element (r, k) of a block with `rows` rows and kKB columns, K-major core
// matrices: core (r / 8, k / 8) holds 8 rows of 8 consecutive k (16 bytes each).
__device__ __forceinline__ int canon(int r, int k) {
  return ((r >> 3) * (kKB / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// exponent e with |x| < 2^e for the largest |x| of a row / column
__device__ __forceinline__ int exp_of(double mx) { return mx > 0.0 ? ilogb(mx) + 1 : 0; }

}  // namespace

// ------------------------------------------------------------------ split
__global__ void k_oz_exp_rows(const OzDesc* __restrict__ d, int* __restrict__ ework) {
  const OzDesc g = d[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.M) return;
  double mx = 0.0;
  for (int k = 0; k < g.K; ++k) mx = fmax(mx, fabs(g.A[i + (size_t)k * g.lda]));
  ework[g.ea_off + i] = exp_of(mx);
}

__global__ void k_oz_exp_cols(const OzDesc* __restrict__ d, int* __restrict__ ework) {
  const OzDesc g = d[blockIdx.y];
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (j >= g.N) return;
  double mx = 0.0;
  for (int k = lane; k < g.K; k += 32) mx = fmax(mx, fabs(g.B[k + (size_t)j * g.ldb]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) ework[g.eb_off + j] = exp_of(mx);
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
// (side 1, 64-row tiles of B^T); writes all 8 slices of the block.
__global__ void __launch_bounds__(kThreads) k_oz_split(const OzDesc* __restrict__ d, int side,
                                                       const int* __restrict__ ework,
                                                       __nv_bfloat16* __restrict__ work) {
  const OzDesc g = d[blockIdx.z];
  const int tile = blockIdx.x, kb = blockIdx.y;
  const int rows = side == 0 ? kTM : kTN;
  const int ntiles = side == 0 ? g.mt : g.nt;
  if (tile >= ntiles || kb >= g.nkb) return;
  const int blk = side == 0 ? kABlock : kBBlock;
  // slice s, tile, block: work[off + ((s * ntiles + tile) * nkb + kb) * blk]
  const int64_t base = (side == 0 ? g.a_off : g.b_off) + ((int64_t)tile * g.nkb + kb) * blk;
  const int64_t sstride = (int64_t)ntiles * g.nkb * blk;
  for (int e = threadIdx.x; e < rows * kKB; e += kThreads) {
    // side 0: consecutive threads take consecutive rows of A (contiguous);
    // side 1: consecutive threads take consecutive k of a column of B
    int r, k;
    if (side == 0) {
      r = e % rows;
      k = e / rows;
    } else {
      k = e % kKB;
      r = e / kKB;
    }
    const int gi = tile * rows + r, gk = kb * kKB + k;
    double x = 0.0;
    int ex = 0;
    if (side == 0) {
      if (gi < g.M && gk < g.K) {
        x = g.A[gi + (size_t)gk * g.lda];
        ex = ework[g.ea_off + gi];
      }
    } else {
      if (gi < g.N && gk < g.K) {
        x = g.B[gk + (size_t)gi * g.ldb];
        ex = ework[g.eb_off + gi];
      }
    }
    int q[kS];
    slice8(x, ex, q);
    const int o = canon(r, k);
#pragma unroll
    for (int s = 0; s < kS; ++s) work[base + s * sstride + o] = __float2bfloat16_rn((float)q[s]);
  }
}

// ------------------------------------------------------------------ GEMM
namespace {

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // K-major, no swizzle: LBO = 128 B between core matrices along K, SBO =
  // 1024 B between 8-row groups (8 core matrices of 128 B per group)
  uint64_t dsc = (uint64_t)((saddr >> 4) & 0x3FFF);
  dsc |= (uint64_t)(128 >> 4) << 16;
  dsc |= (uint64_t)(1024 >> 4) << 32;
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

// pair q of the s-major list of (s, t), s + t <= S + 1 (1-based)
__device__ __forceinline__ void pair_of(int q, int& s, int& t) {
  s = 1;
  int n = kS;
  while (q >= n) {
    q -= n;
    ++s;
    --n;
  }
  t = q + 1;
}

}  // namespace

// grid: (nt, mt, descriptor); 256 threads; shared memory: the 7 A blocks of
// one slice and two buffers of 7 B blocks (224 KB in all) + barriers.
__global__ void __launch_bounds__(kThreads, 1) k_oz_gemm(const OzDesc* __restrict__ d,
                                                         const int* __restrict__ ework,
                                                         const __nv_bfloat16* __restrict__ work,
                                                         double alpha, double beta,
                                                         int* __restrict__ status) {
  const OzDesc g = d[blockIdx.z];
  const int tn = blockIdx.x, tm = blockIdx.y;
  if (tn >= g.nt || tm >= g.mt) return;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smraw);     // kChunkKB A blocks
  __nv_bfloat16* Bs[2] = {As + kChunkKB * kABlock, As + kChunkKB * kABlock + kChunkKB * kBBlock};
  __shared__ __align__(8) uint64_t bar_a, bar_b[2], bar_full[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(2 * kTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bar_a, 1);
    mbar_init(&bar_b[0], 1);
    mbar_init(&bar_b[1], 1);
    mbar_init(&bar_full[0], 1);
    mbar_init(&bar_full[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int nchunks = (g.nkb + kChunkKB - 1) / kChunkKB;
  const int npair = n_pairs();
  const int Q = nchunks * npair;
  const int64_t a_sstride = (int64_t)g.mt * g.nkb * kABlock;
  const int64_t b_sstride = (int64_t)g.nt * g.nkb * kBBlock;
  // per-thread accumulators: row r of the tile, 32 columns
  const int r = 32 * (warp & 3) + lane;
  const int c0 = 32 * (warp >> 2);
  long long uhi[32], ulo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) uhi[j] = ulo[j] = 0;
  uint32_t n_a = 0, n_b[2] = {0, 0}, n_full[2] = {0, 0};  // completed phases per barrier
  bool fail = false;   // producer (thread 0): one of its waits gave up
  bool gfail = false;  // the whole CTA knows a wait gave up (uniform, refreshed per pair)

  // producer helpers (thread 0)
  auto load_a = [&](int chunk, int s) {
    const int kb0 = chunk * kChunkKB, nb = min(kChunkKB, g.nkb - kb0);
    const __nv_bfloat16* src = work + g.a_off + (s - 1) * a_sstride + ((int64_t)tm * g.nkb + kb0) * kABlock;
    expect_tx(&bar_a, (uint32_t)(nb * kABlock * 2));
    bulk_load(As, src, (uint32_t)(nb * kABlock * 2), &bar_a);
  };
  auto load_b = [&](int chunk, int t, int buf) {
    const int kb0 = chunk * kChunkKB, nb = min(kChunkKB, g.nkb - kb0);
    const __nv_bfloat16* src = work + g.b_off + (t - 1) * b_sstride + ((int64_t)tn * g.nkb + kb0) * kBBlock;
    expect_tx(&bar_b[buf], (uint32_t)(nb * kBBlock * 2));
    bulk_load(Bs[buf], src, (uint32_t)(nb * kBBlock * 2), &bar_b[buf]);
  };
  auto pair_at = [&](int qq, int& chunk, int& s, int& t) {
    chunk = qq / npair;
    pair_of(qq % npair, s, t);
  };

  if (tid == 0) {
    int ch, s, t;
    pair_at(0, ch, s, t);
    load_a(ch, s);
    load_b(ch, t, 0);
  }
  for (int q = 0; q <= Q; ++q) {
    // ---- issue pair q (thread 0)
    if (q < Q && tid == 0 && !fail) {
      int ch, s, t;
      pair_at(q, ch, s, t);
      const bool new_a = q == 0 || (q % npair) == 0 || t == 1;
      if (new_a) {
        if (!mbar_wait(&bar_a, n_a & 1)) fail = true;
        ++n_a;
      }
      if (!mbar_wait(&bar_b[q & 1], n_b[q & 1] & 1)) fail = true;
      ++n_b[q & 1];
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (fail) s_fail = 1;
      if (!fail) {
        const int nb = min(kChunkKB, g.nkb - ch * kChunkKB);
        const uint32_t acc = tmem + (uint32_t)((q & 1) * kTN);
        for (int kb = 0; kb < nb; ++kb)
#pragma unroll
          for (int k16 = 0; k16 < kKB / 16; ++k16) {
            const uint64_t da = smem_desc(smem_u32(As + kb * kABlock) + k16 * 256);
            const uint64_t db = smem_desc(smem_u32(Bs[q & 1] + kb * kBBlock) + k16 * 256);
            const uint32_t en = (kb | k16) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                "l"(da), "l"(db), "r"(kIdesc), "r"(en)
                : "memory");
          }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar_full[q & 1]))
            : "memory");
      }
    }
    // ---- drain pair q - 1 (all threads)
    if (q >= 1) {
      const int p = q - 1;
      // warp-uniform: every lane waits on the same barrier phase
      const bool ok =
          !gfail && __all_sync(0xffffffffu, mbar_wait(&bar_full[p & 1], n_full[p & 1] & 1));
      ++n_full[p & 1];
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) {
        int ch, s, t;
        pair_at(p, ch, s, t);
        const int dd = s + t;
        const uint32_t addr = tmem + (uint32_t)((p & 1) * kTN) + ((uint32_t)(32 * (warp & 3)) << 16) +
                              (uint32_t)c0;
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
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
      if (!ok && lane == 0) atomicExch(&s_fail, 1);
    }
    // ---- prefetch pair q + 1 (thread 0): B into the buffer pair q - 1 used
    // (its MMAs are complete), A once the MMAs of pair q are complete
    if (q + 1 < Q && tid == 0 && !fail) {
      int ch, s, t;
      pair_at(q + 1, ch, s, t);
      const bool new_a = ((q + 1) % npair) == 0 || t == 1;
      if (new_a) {
        if (!mbar_wait(&bar_full[q & 1], n_full[q & 1] & 1)) fail = true;
        if (!fail) load_a(ch, s);
      }
      if (!fail) load_b(ch, t, (q + 1) & 1);
    }
    if (fail && tid == 0) s_fail = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    gfail = s_fail != 0;
  }
  // ---- epilogue: C = alpha 2^(eA+eB) (U_hi 2^-35 + U_lo 2^-63) + beta C
  if (!gfail) {
    const int gi = tm * kTM + r;
    if (gi < g.M) {
      const int ea = ework[g.ea_off + gi];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int gj = tn * kTN + c0 + j;
        if (gj >= g.N) break;
        const int ee = ea + ework[g.eb_off + gj];
        const double v = ldexp((double)uhi[j], ee - 35) + ldexp((double)ulo[j], ee - 63);
        double* cp = g.C + gi + (size_t)gj * g.ldc;
        *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
      }
    }
  } else if (tid == 0 && status) {
    atomicCAS(status, 0, -1);  // a wait gave up: reported as a device error
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTN));
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
  prof::Scope sc(name, st, flops, bytes);
  k_oz_exp_rows<<<dim3((maxM + 255) / 256, nd), 256, 0, st>>>(d_desc, ew);
  k_oz_exp_cols<<<dim3((maxN + 7) / 8, nd), 256, 0, st>>>(d_desc, ew);
  k_oz_split<<<dim3(max_mt, max_kb, nd), kThreads, 0, st>>>(d_desc, 0, ew, slices);
  k_oz_split<<<dim3(max_nt, max_kb, nd), kThreads, 0, st>>>(d_desc, 1, ew, slices);
  const int smem = (kChunkKB * kABlock + 2 * kChunkKB * kBBlock) * 2;
  if (!opt_in_smem(reinterpret_cast<const void*>(&k_oz_gemm), smem)) return cudaErrorInvalidValue;
  k_oz_gemm<<<dim3(max_nt, max_mt, nd), kThreads, smem, st>>>(d_desc, ew, slices, alpha, beta,
                                                               status);
  return cudaGetLastError();
}

}  // namespace hps
