// Relative residual of the FOM's discrete system at a predicted state, ||r|| / ||b|| with
// r = b - A u (Sec. 2.2 of the paper: the prediction is credible when it is below the
// tolerance).  The caller's callback forms r and b; this kernel reduces them: FP64
// partial sums per CTA, then the last CTA adds the partials in CTA order (deterministic)
// and writes the two totals to ws.out2 for the host.
#include "odmd_internal.cuh"

namespace odmd {

constexpr int kResThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kResThreads) k_norm_ratio(Ws ws, const T* __restrict__ r, const T* __restrict__ b) {
  const int tid = threadIdx.x;
  double num = 0.0, den = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kResThreads + tid; i < ws.n; i += (int64_t)gridDim.x * kResThreads) {
    const double ri = (double)r[i], bi = (double)b[i];
    num = fma(ri, ri, num);
    den = fma(bi, bi, den);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  __shared__ double sn[kResThreads / 32], sd[kResThreads / 32];
  if ((tid & 31) == 0) {
    sn[tid >> 5] = num;
    sd[tid >> 5] = den;
  }
  __syncthreads();
  double* part = reinterpret_cast<double*>(ws.part);
  __shared__ unsigned ticket;
  if (tid == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) {
      a += sn[w];
      c += sd[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = c;
    __threadfence();
    ticket = atomicAdd(&ws.ctl->ticket_r, 1u);
  }
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  if (tid == 0) {
    __threadfence();
    double a = 0.0, c = 0.0;
    for (unsigned blk = 0; blk < gridDim.x; ++blk) {
      a += __ldcg(part + 2 * blk);
      c += __ldcg(part + 2 * blk + 1);
    }
    double* out = reinterpret_cast<double*>(ws.out2);
    out[0] = a;
    out[1] = c;
    if (!isfinite(a) || !isfinite(c)) atomicOr(&ws.ctl->status, DEV_NONFINITE);
    ws.ctl->ticket_r = 0u;
  }
}

cudaError_t launch_norm_ratio(const Ws& ws, const void* r, const void* b, cudaStream_t s) {
  const int64_t blocks = (ws.n + kResThreads - 1) / kResThreads;
  const int grid = (int)(blocks < ws.gridA ? blocks : ws.gridA);  // ws.part holds gridA x 2 doubles
  if (ws.prec == ST_DD)
    k_norm_ratio<double><<<grid, kResThreads, 0, s>>>(ws, static_cast<const double*>(r), static_cast<const double*>(b));
  else
    k_norm_ratio<float><<<grid, kResThreads, 0, s>>>(ws, static_cast<const float*>(r), static_cast<const float*>(b));
  return cudaGetLastError();
}

}  // namespace odmd
