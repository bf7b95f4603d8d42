// 5th-generation tensor-core building blocks (sm_103a): tcgen05.mma of kind::f16 with
// bfloat16 operands in shared memory and an FP32 accumulator in tensor memory (TMEM).
//
// Operand layout: the canonical K-major layout without swizzle.  The operand is cut into
// core matrices of 8 rows x 16 bytes (8 bfloat16 along K); a core matrix is stored as 128
// contiguous bytes, row i at byte 16 i.  The shared-memory descriptor gives the start
// address, the leading-dimension byte offset (LBO: the distance between the two core
// matrices adjacent along K that one K = 16 instruction reads) and the stride-dimension
// byte offset (SBO: the distance between core matrices adjacent along M or N, i.e. from
// one group of 8 rows to the next).
//
// Descriptor fields (64 bits): start >> 4 in bits 0-13, LBO >> 4 in bits 16-29, SBO >> 4 in
// bits 32-45, the fixed version value 1 in bits 46-47, base offset 0 (bits 49-51), relative
// LBO mode (bit 52 = 0), swizzle mode 0 = none (bits 61-63).
//
// Instruction descriptor of kind::f16 (32 bits): dense; accumulator format FP32 (bits 4-5 =
// 1); A and B format bfloat16 (bits 7-9 = 1, bits 10-12 = 1); no negation; A and B K-major
// (bits 15, 16 = 0); N >> 3 in bits 17-22; M >> 4 in bits 24-28.
#pragma once
#include <cstdint>

#include "odmd_internal.cuh"

namespace odmd {
namespace tc {

constexpr int kCoreBytes = 128;  // one core matrix: 8 rows x 16 bytes

__host__ __device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__host__ __device__ constexpr uint32_t instr_desc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (row, k) of an operand tile whose core matrices are placed with
// the K direction fastest: core (row / 8, k / 8) at ((row / 8) * kcores + k / 8) * 128,
// kcores = K extent of the tile / 8.  LBO = 128, SBO = kcores * 128.
__host__ __device__ inline int kmajor_off(int row, int k, int kcores) {
  return ((row >> 3) * kcores + (k >> 3)) * kCoreBytes + (row & 7) * 16 + (k & 7) * 2;
}

// TMEM allocation by one full warp; the base address is written to *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A B, one instruction, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the mbarrier gets one arrival once every tcgen05.mma issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (lane = thread), then wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace odmd
