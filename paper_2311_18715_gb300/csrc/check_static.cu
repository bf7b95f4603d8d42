// Credibility check of a prediction the caller already holds, for callers that must not
// allocate memory.  The paper has no counterpart: this is a library convenience beside
// odmd_check.
//
// Who needs it: code that runs where a device allocation is not allowed or not safe --
// a callback inside a host solver's time loop whose memory is owned by the solver's own
// pool allocator, a process running under a hard device-memory cap, or a section that
// must not pay the implicit device synchronisation a cudaMalloc/cudaFree may cause.
// Such a caller holds the predicted state (from odmd_predict, written into its own
// buffer) and the FOM state, and wants the relative L2 distance between them.
//
// The reduction is the same as that of the fused check pass: per-CTA partial sums of
// ||pred - x_fom||^2 and ||x_fom||^2, then the last CTA to finish adds the partials in
// CTA order (deterministic).  Its scratch (the partials, a ticket counter and the two
// totals) lives in one file-scope device array of fixed size, so a call allocates
// nothing.  The array is shared by every call in the process on that GPU.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "odmd.h"
#include "odmd_internal.cuh"

namespace {

constexpr int kStaticThreads = 256;
constexpr int64_t kStaticChunk = 8192;  // elements per CTA
constexpr int kStaticSlots = 4096;      // per-CTA partial-sum slots, so n <= 4096 * 8192
constexpr int64_t kStaticMaxN = (int64_t)kStaticSlots * kStaticChunk;  // 33,554,432
constexpr size_t kStaticHeader = 256;   // ticket (4 bytes) and the two totals at offset 8
constexpr size_t kStaticBytes = kStaticHeader + (size_t)kStaticSlots * 2 * sizeof(double);  // 64 KiB + 256

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_check_scratch[kStaticBytes];

__global__ void __launch_bounds__(kStaticThreads)
    k_check_static(const double* __restrict__ pred, const double* __restrict__ fom, int64_t n,
                   unsigned char* scratch) {
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  double* total = reinterpret_cast<double*>(scratch + 8);
  double* part = reinterpret_cast<double*>(scratch + kStaticHeader);
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kStaticChunk;
  const int64_t end = base + kStaticChunk < n ? base + kStaticChunk : n;
  double num = 0.0, den = 0.0;
  for (int64_t i = base + tid; i < end; i += kStaticThreads) {
    const double y = __ldcs(fom + i);
    const double d = __ldcs(pred + i) - y;
    num = fma(d, d, num);
    den = fma(y, y, den);
  }
  __shared__ double sn[kStaticThreads / 32], sd[kStaticThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((tid & 31) == 0) {
    sn[tid >> 5] = num;
    sd[tid >> 5] = den;
  }
  __syncthreads();
  __shared__ unsigned last;
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kStaticThreads / 32; ++w) {
      a += sn[w];
      b += sd[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA: thread t sums slots t, t + 256, ...; then a fixed-order combine
  double a = 0.0, b = 0.0;
  for (int s = tid; s < (int)gridDim.x; s += kStaticThreads) {
    a += __ldcg(part + 2 * s);
    b += __ldcg(part + 2 * s + 1);
  }
  __shared__ double ra[kStaticThreads], rb[kStaticThreads];
  ra[tid] = a;
  rb[tid] = b;
  __syncthreads();
  for (int h = kStaticThreads / 2; h > 0; h >>= 1) {
    if (tid < h) {
      ra[tid] += ra[tid + h];
      rb[tid] += rb[tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) {
    total[0] = ra[0];
    total[1] = rb[0];
  }
}

// Device address of g_check_scratch per device, looked up once with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" odmd_status odmd_check_noalloc(const double* pred_dev, const double* x_fom_dev, int64_t n,
                                          double tol, void* stream, double* rel_err, int32_t* pass) {
  using odmd::report_global_error;
  if (!pred_dev || !x_fom_dev) return report_global_error(ODMD_ERR_ARG, "odmd_check_noalloc: NULL input");
  if (n < 1) return report_global_error(ODMD_ERR_ARG, "odmd_check_noalloc: n must be >= 1");
  if (n > kStaticMaxN)
    return report_global_error(ODMD_ERR_ARG,
                               "odmd_check_noalloc: n = " + std::to_string(n) + " exceeds the limit of " +
                                   std::to_string(kStaticMaxN) + " elements set by its fixed scratch array");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return report_global_error(ODMD_ERR_CUDA, std::string("odmd_check_noalloc: cudaGetDevice: ") +
                                                  cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_global_error(ODMD_ERR_ARG, "odmd_check_noalloc: device index too large");
  unsigned char* scratch = nullptr;
  {
    // first call on this device: look up the array's device address (the host-side name
    // g_check_scratch is only a stand-in and must never be passed to a kernel)
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_check_scratch);
      if (e != cudaSuccess)
        return report_global_error(ODMD_ERR_CUDA, std::string("odmd_check_noalloc: cudaGetSymbolAddress: ") +
                                                      cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the ticket and the totals must start at zero; the partial slots are always written
  // before they are read
  e = cudaMemsetAsync(scratch, 0, kStaticHeader, s);
  const int blocks = (int)((n + kStaticChunk - 1) / kStaticChunk);
  if (e == cudaSuccess) {
    k_check_static<<<blocks, kStaticThreads, 0, s>>>(pred_dev, x_fom_dev, n, scratch);
    e = cudaGetLastError();
  }
  double tot[2] = {0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot, scratch + 8, sizeof tot, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return report_global_error(ODMD_ERR_CUDA, std::string("odmd_check_noalloc: ") + cudaGetErrorString(e));
  if (!std::isfinite(tot[0]) || !std::isfinite(tot[1]))
    return report_global_error(ODMD_ERR_NUMERIC, "odmd_check_noalloc: non-finite input");
  double rel;
  if (tot[1] > 0.0)
    rel = std::sqrt(tot[0]) / std::sqrt(tot[1]);
  else
    rel = tot[0] > 0.0 ? INFINITY : 0.0;
  const double t = tol > 0.0 ? tol : 1e-5;
  if (rel_err) *rel_err = rel;
  if (pass) *pass = rel <= t ? 1 : 0;
  return ODMD_OK;
}
