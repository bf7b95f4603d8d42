// Self-test of the tensor-core building block the split-precision contractions rest on:
// one CTA computes D (128 x 64, FP32 in tensor memory) = reps * A (128 x 64) B (64 x 64),
// A and B bfloat16 in the canonical K-major layout without swizzle (tc.cuh), by four
// tcgen05.mma of K = 16 per repetition issued by one thread into one accumulator, then
// reads D back with tcgen05.ld.  The test compares D with the float64 product on the host;
// with integer operands it also checks that FP32 accumulation of integer products is exact
// below 2^24, which the split contractions need.
//
// Every shared-memory address the descriptors can reach lies inside the operand's own
// tile (checked at compile time below for either assignment of the two byte offsets to
// the two directions).  Waits are bounded (2 s): on a timeout the status word is set, the
// products in flight get a further bounded wait, and the tensor memory is still freed.
#include <cstdint>

#include "../../include/odmd.h"
#include "odmd_internal.cuh"
#include "tc.cuh"

namespace odmd {
namespace tcst {

constexpr int kM = 128, kN = 64, kK = 64, kKStep = 16, kKCores = kK / 8;
constexpr int kABytes = kM * kK * 2, kBBytes = kN * kK * 2;
constexpr uint32_t kLBO = tc::kCoreBytes, kSBO = kKCores * tc::kCoreBytes;

// highest byte an instruction of K step ks can touch: 2 core matrices along K, rows / 8
// along M or N, whichever offset the hardware applies to which direction
constexpr int top(int rows, int ks, uint32_t along_k, uint32_t along_rows) {
  return 2 * ks * tc::kCoreBytes + (int)along_k + (rows / 8 - 1) * (int)along_rows + tc::kCoreBytes;
}
static_assert(top(kM, kK / kKStep - 1, kLBO, kSBO) <= kABytes && top(kM, kK / kKStep - 1, kSBO, kLBO) <= kABytes,
              "A descriptors stay inside the A tile");
static_assert(top(kN, kK / kKStep - 1, kLBO, kSBO) <= kBBytes && top(kN, kK / kKStep - 1, kSBO, kLBO) <= kBBytes,
              "B descriptors stay inside the B tile");

__global__ void __launch_bounds__(128, 1) k_tc_selftest(const uint16_t* A, const uint16_t* B, float* D, int reps,
                                                        int* status) {
  extern __shared__ __align__(1024) unsigned char st_smem[];
  unsigned char* sA = st_smem;
  unsigned char* sB = st_smem + kABytes;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < kM * kK; e += blockDim.x)
    *reinterpret_cast<uint16_t*>(sA + tc::kmajor_off(e / kK, e % kK, kKCores)) = A[e];
  for (int e = tid; e < kN * kK; e += blockDim.x)
    *reinterpret_cast<uint16_t*>(sB + tc::kmajor_off(e / kK, e % kK, kKCores)) = B[e];
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  tc::fence_proxy_async();
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint32_t idesc = tc::instr_desc_bf16_f32(kM, kN);
    for (int rep = 0; rep < reps; ++rep)
      for (int ks = 0; ks < kK / kKStep; ++ks) {
        const uint32_t off = (uint32_t)(2 * ks * tc::kCoreBytes);
        const uint64_t ad = tc::smem_desc(smem_addr(sA) + off, kLBO, kSBO);
        const uint64_t bd = tc::smem_desc(smem_addr(sB) + off, kLBO, kSBO);
        tc::mma_bf16(tmem, ad, bd, idesc, (rep > 0 || ks > 0) ? 1u : 0u);
      }
    tc::mma_commit(&bar);
  }
  const bool ok = mbar_wait(&bar, 0, status);
  if (!ok) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(&bar, 0))
      if (global_ns() - t0 > 500000000ull) break;
  }
  tc::fence_after_sync();
  if (__all_sync(0xffffffffu, ok)) {
    for (int c0 = 0; c0 < kN; c0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) D[(size_t)(32 * warp + lane) * kN + c0 + j] = __uint_as_float(r[j]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kN);
}

}  // namespace tcst
}  // namespace odmd

extern "C" {

odmd_status odmd_tc_selftest(const void* a_dev, const void* b_dev, void* d_dev, int32_t* status_dev, int32_t reps) {
  using namespace odmd::tcst;
  if (!a_dev || !b_dev || !d_dev || !status_dev || reps < 1 || reps > 4096) return ODMD_ERR_ARG;
  const int smem = kABytes + kBBytes;
  if (cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return ODMD_ERR_CUDA;
  if (cudaMemset(status_dev, 0, sizeof(int32_t)) != cudaSuccess) return ODMD_ERR_CUDA;
  k_tc_selftest<<<1, 128, smem>>>(static_cast<const uint16_t*>(a_dev), static_cast<const uint16_t*>(b_dev),
                                  static_cast<float*>(d_dev), reps, status_dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t hs = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hs, status_dev, sizeof hs, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ODMD_ERR_CUDA;
  return hs ? ODMD_ERR_TIMEOUT : ODMD_OK;
}

}  // extern "C"
