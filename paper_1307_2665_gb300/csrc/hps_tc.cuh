// Small helpers for kernels that issue 5th-generation tensor-core MMAs
// (tcgen05) from shared-memory operands written by the CTA itself.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hps {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; lbo = bytes between core matrices adjacent in K, sbo =
// bytes between 8-row groups.  Advancing the operand by X bytes adds X >> 4.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
  return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

// Bounded wait for the phase of the given parity; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long bound) {
  for (long it = 0; it < bound; ++it) {
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

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

// 2 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld2(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(v[0]), "=r"(v[1])
               : "r"(taddr));
}

__device__ __forceinline__ void wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Offset (elements) of operand element (row r, k) of a 16-wide K sub-tile in
// the K-major no-swizzle layout: core matrices of 8 rows x 8 k (128 bytes),
// LBO 128 B (the two K cores), SBO 256 B (row groups).
__device__ __forceinline__ int g_off(int r, int k) {
  return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// The exact three-term BF16 split of 8 floats (x1 = bf16(x), x2 = bf16(x - x1),
// x3 = bf16(x - x1 - x2), rounding to nearest: the remainders are exact in
// FP32 and the three terms carry all 24 bits), packed as three 16-byte rows.
__device__ __forceinline__ void split8(const float* x, uint32_t (*w)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float a = x[2 * j], b = x[2 * j + 1];
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(a, b);
    const float ra = a - __low2float(h1), rb = b - __high2float(h1);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(ra, rb);
    const float sa = ra - __low2float(h2), sb = rb - __high2float(h2);
    const __nv_bfloat162 h3 = __floats2bfloat162_rn(sa, sb);
    w[0][j] = *reinterpret_cast<const uint32_t*>(&h1);
    w[1][j] = *reinterpret_cast<const uint32_t*>(&h2);
    w[2][j] = *reinterpret_cast<const uint32_t*>(&h3);
  }
}

__device__ __forceinline__ void st16(uint32_t saddr, const uint32_t* w) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(saddr), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3])
               : "memory");
}

}  // namespace tc
}  // namespace hps
