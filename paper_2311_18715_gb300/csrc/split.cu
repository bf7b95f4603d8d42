// Multi-horizon rollout X = L0 C on the tensor cores (Sec. 2.3: u(t) = Phi Lambda^t b for
// many t at once is a tall N x r0 basis times a small r0 x k coefficient block), exact to the
// double-float level through a split of both operands into 7-bit digits (Ozaki's scheme:
// an error-free splitting into slices whose products a lower-precision unit sums exactly).
//
// Each row i of L0 (double-float hi + lo) is written on its own power-of-two grid,
// a_ik = sum_{s=1..7} d_iks 2^(e_i - 7 s), and each column j of C on its own,
// c_kj = sum_{t=1..7} d'_kjt 2^(f_j - 7 t), with integer digits |d| <= 128 (exact in
// bfloat16); what is left after seven digits is below 2^-49 of the row (column) maximum.
// Products of digits with s + t = g are integers on the common grid 2^(e_i + f_j - 7 g): the
// 28 digit pairs with g <= 8 are bfloat16 products (tcgen05.mma kind::f16, M = 128, N = 64,
// K = 16) into seven FP32 accumulators in tensor memory, one per g.  A group adds at most
// 7 K products of |d d'| <= 2^14 with K <= 64, below 2^24, so every partial sum is an
// integer the FP32 accumulator holds exactly; pairs with g >= 9 are below 2^-49 K of
// max|a_i| max|c_j| and are left out.  The epilogue adds the seven group sums, scaled by
// 2^(56 - 7 g) (all exact floats), in double-float and scales the result by 2^(e_i + f_j -
// 56), which is the double-float accuracy of the CUDA-core path.
//
// One persistent CTA of 256 threads per SM (the seven accumulators take 448 of the SM's 512
// tensor-memory columns).  C's digits are formed once per CTA.  A 128-row tile of L0 (both
// planes) arrives by two bulk copies into a staging buffer; two threads per row form its
// digits, 32 basis columns (two K chunks) at a time, into the K-major core-matrix layout
// the descriptors describe (tc.cuh); one thread issues the chunk's 28 MMAs and commits them
// to an mbarrier; once the last digits of a tile are formed the staging buffer takes the
// next tile while the products and the epilogue of this one run.  Every wait is bounded
// (2 s): a timeout sets DEV_TIMEOUT, waits (bounded) for the work in flight, and frees the
// tensor memory before the CTA returns.
#include <cstdint>

#include "dd.cuh"
#include "odmd_internal.cuh"
#include "tc.cuh"

namespace odmd {
namespace split {

constexpr int kTM = 128;        // rows per tile (MMA M)
constexpr int kNJ = 64;         // MMA N: horizons of one launch, padded with zero columns
constexpr int kKC = 16;         // K of one MMA
constexpr int kSlices = 7;      // digits per value
constexpr int kGroups = 7;      // g = s + t = 2 .. 8
constexpr int kMaxK = 64;       // basis columns this path takes (4 K chunks)
constexpr int kBufK = 32;       // K columns of L0 digits held at once (two chunks)
constexpr int kThreadsS = 256;
constexpr uint32_t kTmemCols = 512;
constexpr int kASlice = kTM * kBufK * 2;   // bytes of one digit slice of the L0 buffer
constexpr int kBSlice = kNJ * kMaxK * 2;   // bytes of one digit slice of C (K padded to 64)
static_assert(kGroups * kNJ <= (int)kTmemCols, "seven accumulators fit the tensor memory");
// a group sums at most 7 digit pairs over K <= 64 columns of products |d d'| <= 2^14
static_assert(7 * kMaxK * (1 << 14) < (1 << 24), "group sums stay below 2^24");

__host__ __device__ inline int stage_bytes(int rs) { return ((2 * kTM * rs + 1023) / 1024) * 1024; }
__host__ __device__ inline int smem_bytes(int rs) { return stage_bytes(rs) + kSlices * kASlice + kSlices * kBSlice; }

// exponent e with |v| < 2^e for every v of a set with maximum mx (0 for mx = 0)
__device__ __forceinline__ int grid_exp(float mx) {
  if (!(mx > 0.f)) return 0;
  int e;
  frexpf(mx, &e);
  return e;
}

// the seven digits of v = h + l on the grid 2^(e - 7 s), s = 1..7, as bfloat16 bits: with
// w = v 2^-e (|w| < 1), each step takes q = rint(128 w) and keeps 128 w - q (exact)
__device__ __forceinline__ void digits7(float h, float l, int e, uint16_t (&d)[kSlices]) {
  float wh = ldexpf(h, -e), wl = ldexpf(l, -e);
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const float th = wh * 128.f, tl = wl * 128.f;
    const float q = rintf(th);
    const dd r = fast_two_sum(th - q, tl);
    wh = r.h;
    wl = r.l;
    d[s] = __bfloat16_as_ushort(__float2bfloat16_rn(q));
  }
}

__device__ __forceinline__ void issue_tile(const Ws& ws, unsigned char* stage, int rs, int64_t tile, uint64_t* bar) {
  const int64_t row0 = tile * kTM;
  const int64_t rows = (ws.npad - row0) < kTM ? (ws.npad - row0) : kTM;
  const uint32_t bytes = (uint32_t)(rows * rs);
  mbar_arrive_expect_tx(bar, 2 * bytes);
  bulk_g2s(stage, reinterpret_cast<const unsigned char*>(ws.Lh) + row0 * rs, bytes, bar);
  bulk_g2s(stage + (size_t)kTM * rs, reinterpret_cast<const unsigned char*>(ws.Ll) + row0 * rs, bytes, bar);
}

__global__ void __launch_bounds__(kThreadsS, 1) k_split_rollout(Ws ws, int kcols, double* out, int64_t ld) {
  extern __shared__ __align__(1024) unsigned char sp[];
  Ctl* ctl = ws.ctl;
  const StateBuf st = ws.st[ctl->cur];
  const int r0 = st.hdr->r0, qld = ws.cap + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rs = ws.ldg * 4;
  const int kpad = (r0 + kKC - 1) / kKC * kKC;
  const int nchunk = kpad / kKC;
  unsigned char* stage = sp;
  unsigned char* adig = sp + stage_bytes(rs);
  unsigned char* bdig = adig + kSlices * kASlice;
  __shared__ int fexp[kNJ];
  __shared__ int erow[kTM];
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;

  // ---- digits of C: column j of the coefficients is row j of the B operand (K-major)
  for (int j = warp; j < kNJ; j += kThreadsS / 32) {
    float mx = 0.f;
    if (j < kcols)
      for (int k = lane; k < r0; k += 32) mx = fmaxf(mx, fabsf(ws.sm.coef[(size_t)j * qld + k].x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) fexp[j] = grid_exp(mx);
  }
  __syncthreads();
  for (int o = tid; o < kNJ * kMaxK; o += kThreadsS) {
    const int j = o / kMaxK, k = o % kMaxK;
    float h = 0.f, l = 0.f;
    if (j < kcols && k < r0) {
      const float2 q = ws.sm.coef[(size_t)j * qld + k];
      h = q.x;
      l = q.y;
    }
    uint16_t d[kSlices];
    digits7(h, l, fexp[j], d);
    const int off = tc::kmajor_off(j, k, kMaxK / 8);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) *reinterpret_cast<uint16_t*>(bdig + s * kBSlice + off) = d[s];
  }
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  const int64_t ntiles = (ws.n + kTM - 1) / kTM;
  const int G = gridDim.x;
  const int my_tiles = (int)((ntiles - blockIdx.x + G - 1) / G);
  if (tid == 0 && my_tiles > 0) issue_tile(ws, stage, rs, blockIdx.x, &bar_tma);
  const uint32_t idesc = tc::instr_desc_bf16_f32(kTM, kNJ);
  uint32_t par_tma = 0, par_mma = 0;
  // work in flight that a timeout must still wait for (the same in every thread)
  bool tma_out = my_tiles > 0, mma_out = false;
  const int row = tid >> 1, half = tid & 1;  // digit phase: two threads per row
  const float* sh = reinterpret_cast<const float*>(stage) + (size_t)row * (rs / 4);
  const float* sl = reinterpret_cast<const float*>(stage + (size_t)kTM * rs) + (size_t)row * (rs / 4);
  bool ok = true;

  for (int li = 0; li < my_tiles && ok; ++li) {
    const int64_t tile = blockIdx.x + (int64_t)li * G;
    const int64_t row0 = tile * kTM;
    ok = mbar_wait(&bar_tma, par_tma, &ctl->status);
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    par_tma ^= 1u;
    tma_out = false;
    // the row's exponent: max |hi| over its r0 columns, half of them per thread
    const bool live = row0 + row < ws.n;
    {
      float mx = 0.f;
      if (live)
        for (int k = half; k < r0; k += 2) mx = fmaxf(mx, fabsf(sh[k]));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      if (half == 0) erow[row] = grid_exp(mx);
    }
    __syncwarp();
    const int my_e = erow[row];
    for (int c0 = 0; c0 < nchunk; c0 += 2) {
      // digits of chunk c0 + half (16 columns of this row) into the buffer slot `half`
      const int c = c0 + half;
      if (c < nchunk) {
#pragma unroll 2
        for (int kk = 0; kk < kKC; ++kk) {
          const int k = c * kKC + kk;
          float h = 0.f, l = 0.f;
          if (live && k < r0) {
            h = sh[k];
            l = sl[k];
          }
          uint16_t d[kSlices];
          digits7(h, l, my_e, d);
          const int off = tc::kmajor_off(row, half * kKC + kk, kBufK / 8);
#pragma unroll
          for (int s = 0; s < kSlices; ++s) *reinterpret_cast<uint16_t*>(adig + s * kASlice + off) = d[s];
        }
      }
      tc::fence_proxy_async();
      __syncthreads();
      const bool last_digits = c0 + 2 >= nchunk;
      if (last_digits && li + 1 < my_tiles) tma_out = true;
      mma_out = true;
      if (tid == 0) {
        // the staging buffer is free once the tile's last digits are formed: next tile
        if (last_digits && li + 1 < my_tiles) issue_tile(ws, stage, rs, tile + G, &bar_tma);
        tc::fence_after_sync();
        for (int cc = c0; cc < c0 + 2 && cc < nchunk; ++cc) {
          const uint32_t aoff = (uint32_t)((cc - c0) * 2 * tc::kCoreBytes);
          const uint32_t boff = (uint32_t)(cc * 2 * tc::kCoreBytes);
          for (int gs = 2; gs <= 8; ++gs)
            for (int s = 1; s < gs && s <= kSlices; ++s) {
              const int t = gs - s;
              if (t > kSlices) continue;
              const uint64_t ad = tc::smem_desc(smem_addr(adig + (s - 1) * kASlice) + aoff, tc::kCoreBytes,
                                                (kBufK / 8) * tc::kCoreBytes);
              const uint64_t bd = tc::smem_desc(smem_addr(bdig + (t - 1) * kBSlice) + boff, tc::kCoreBytes,
                                                (kMaxK / 8) * tc::kCoreBytes);
              const uint32_t acc = (cc > 0 || s > 1) ? 1u : 0u;
              tc::mma_bf16(tmem + (uint32_t)((gs - 2) * kNJ), ad, bd, idesc, acc);
            }
        }
        tc::mma_commit(&bar_mma);
      }
      // the buffer is rewritten (next chunks) or the accumulators read (epilogue) only
      // once these products are done
      const bool done = mbar_wait(&bar_mma, par_mma, &ctl->status);
      if (__syncthreads_or(!done)) {
        ok = false;
        break;
      }
      par_mma ^= 1u;
      mma_out = false;
      tc::fence_after_sync();
    }
    if (!ok) break;
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the 32
    // columns of its half; X = sum_g G_g 2^(56 - 7 g), then 2^(e_i + f_j - 56)
    {
      const int trow = 32 * (warp & 3) + lane;
      const int64_t orow = row0 + trow;
      const int er = erow[trow];
      const int jb = 32 * (warp >> 2);
      for (int c8 = 0; c8 < 32; c8 += 8) {
        uint32_t g[kGroups][8];
#pragma unroll
        for (int q = 0; q < kGroups; ++q) {
          const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(q * kNJ + jb + c8);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                       : "=r"(g[q][0]), "=r"(g[q][1]), "=r"(g[q][2]), "=r"(g[q][3]), "=r"(g[q][4]), "=r"(g[q][5]),
                         "=r"(g[q][6]), "=r"(g[q][7])
                       : "r"(taddr));
        }
        tc::tmem_ld_wait();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = jb + c8 + u;
          if (j >= kcols || orow >= ws.n) continue;
          // smallest group first; every term G_g 2^(56 - 7 g) is an exact float
          dd sum = dd{ldexpf(__uint_as_float(g[kGroups - 1][u]), 0), 0.f};
#pragma unroll
          for (int q = kGroups - 2; q >= 0; --q) sum = sum + dd{ldexpf(__uint_as_float(g[q][u]), 7 * (kGroups - 1 - q)), 0.f};
          const int sc = er + fexp[j] - 56;
          out[(size_t)j * ld + orow] = ldexp((double)sum.h, sc) + ldexp((double)sum.l, sc);
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (!ok && tid == 0) {
    // a wait ran out (DEV_TIMEOUT is set): give the copy and the products still in flight a
    // bounded wait before the shared and tensor memory are released
    const uint64_t t0 = global_ns();
    while (tma_out && !mbar_try_wait(&bar_tma, par_tma) && global_ns() - t0 < 500000000ull) {
    }
    while (mma_out && !mbar_try_wait(&bar_mma, par_mma) && global_ns() - t0 < 1000000000ull) {
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace split

// The tensor-core rollout takes double-float storage, 8 to 64 horizons and at most 64 basis
// columns (its shared memory holds C's digits for K <= 64 and one staged 128-row tile).
bool split_rollout_ok(const Ws& ws, int kcols) {
  // r0 <= cap for every committed state, so cap <= 64 bounds the basis columns
  return ws.prec == ST_DD && kcols >= 8 && kcols <= split::kNJ && ws.cap <= split::kMaxK &&
         split::smem_bytes(ws.ldg * 4) <= 227 * 1024;
}

cudaError_t prepare_split(const Ws& ws) {
  if (ws.prec != ST_DD || split::smem_bytes(ws.ldg * 4) > 227 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(split::k_split_rollout, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              split::smem_bytes(ws.ldg * 4));
}

cudaError_t launch_split_rollout(const Ws& ws, int kcols, double* out, int64_t ld, int sms, cudaStream_t s) {
  const int64_t ntiles = (ws.n + split::kTM - 1) / split::kTM;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  split::k_split_rollout<<<grid, split::kThreadsS, split::smem_bytes(ws.ldg * 4), s>>>(ws, kcols, out, ld);
  return cudaGetLastError();
}

}  // namespace odmd
