// Tall x small products of the basis (double-float, or FP32 storage) on the tensor cores,
// exact to the double-float level through a split of both operands into 8-bit digits
// (Ozaki's scheme: an error-free splitting into slices whose products a lower-precision unit
// sums exactly):
//   rollout     X = L0 C: u(t) = Phi Lambda^t b for many t at once (Sec. 2.3) is the tall
//               N x r0 basis times a small r0 x k coefficient block; X in doubles;
//   compaction  L0 <- [L0 j0] Q_B of the product-form update (Sec. 2.3, Brand's rank-1
//               append kept as L = L0 Q): the new column j0 = (e - L0 s) / rho0 is formed per
//               row from the stored residual, and the product is written back in place.
//
// Each row i of L0 (double-float hi + lo, or an FP32 value with lo = 0; |a_ik| < 2^e_i) is
// put on the fixed-point grid
// 2^(e_i - 54): the integer I = round(hi 2^(54 - e_i)) + round(lo 2^(54 - e_i)) (within one
// unit, 2^-53 of the row maximum; |I| < 2^54).  Adding 0x80 to each of its seven bytes makes
// every byte b of I + 0x80808080808080 a balanced digit d = b - 128, |d| <= 128 (exact in
// bfloat16, the top one |d| <= 64): a_ik = sum_{s=1..7} d_iks 2^(e_i - 54 + 8 (7 - s)), formed
// by integer shifts and byte moves.  Each column j of C is written the same way on its own
// grid 2^(f_j - 54).  Products of digits with s + t = g are integers on the common grid
// 2^(e_i + f_j - 108 + 8 (14 - g)): the 28 digit pairs with g <= 8 are bfloat16 products
// (tcgen05.mma kind::f16, M = 128, N = 64, K = 16) into seven FP32 accumulators in tensor
// memory, one per g.  A group adds at most 7 K products of |d d'| <= 2^14 with K <= 64
// (double-float storage) or 96 (FP32 storage), below 2^24, so every partial sum is an integer
// the FP32 accumulator holds exactly; pairs with
// g >= 9 are below 2^-48 K of max|a_i| max|c_j| and are left out.  The epilogue adds the
// seven group sums, scaled by 2^(8 (8 - g)) (all exact floats), in double-float (two
// outputs per FP32x2 instruction) and scales the result by 2^(e_i + f_j - 60), which is the
// double-float accuracy of the CUDA-core path; a rollout's doubles are assembled from the
// pair by integer operations (pair2d.cuh: FP64 conversions run at the FP64 rate on this
// GPU).
//
// One persistent CTA per SM (the seven accumulators take 448 of the SM's 512 tensor-memory
// columns) with two roles.  Sixteen worker warps: C's digits once per CTA; for each 128-row
// tile of L0 (its planes staged by bulk copies), four threads per row form its digits
// one 16-column K chunk at a time into one of two buffers (the K-major core-matrix layout
// the descriptors describe, tc.cuh), and read the accumulators in the epilogue.  One issuer
// warp: the tile copies and, per chunk, the 28 MMAs and their commit.  They hand over by
// mbarriers (a buffer's digits are complete; a buffer's products are done), so the workers
// form chunk c + 1 while the tensor core multiplies chunk c and never wait while the issuing
// thread is held by the tensor core's queue; the staging buffer takes the next tile once the
// tile's last digits are formed.  Every wait is bounded (2 s): a timeout sets DEV_TIMEOUT
// and each role stops at its next check; the issuer waits (bounded) for the copies and
// products it issued before the tensor memory is freed.
#include <cstdint>

#include "dd.cuh"
#include "odmd_internal.cuh"
#include "pair2d.cuh"
#include "tc.cuh"

namespace odmd {
namespace split {

constexpr int kTM = 128;        // rows per tile (MMA M)
constexpr int kNJ = 64;         // MMA N: horizons of one launch, padded with zero columns
constexpr int kKC = 16;         // K of one MMA
constexpr int kSlices = 7;      // digits per value
constexpr int kGroups = 7;      // g = s + t = 2 .. 8
constexpr int kBufK = 16;       // K columns of L0 digits in one buffer (one chunk); two buffers
constexpr int kWorkerWarps = 16;  // 4 threads per row in the digit phase, 4 warps per TMEM lane quarter
constexpr int kWorkers = 32 * kWorkerWarps;
constexpr int kThreadsS = kWorkers + 32;  // and one warp that issues the copies and the products
constexpr uint32_t kTmemCols = 512;
constexpr int kASlice = kTM * kBufK * 2;   // bytes of one digit slice of an L0 buffer
constexpr int kABuf = kSlices * kASlice;   // bytes of one L0 digit buffer (one chunk, all slices)
static_assert(kGroups * kNJ <= (int)kTmemCols, "seven accumulators fit the tensor memory");
// Per storage format: the basis columns this path takes (K padded to whole chunks) and the
// planes staged per row.  Four K chunks for the double-float basis (two planes); six for
// FP32 storage, whose single plane leaves room for the larger digit block of the small
// operand.
template <int ST>
struct Geo {
  static constexpr int kPlanes = ST == ST_DD ? 2 : 1;
  static constexpr int kMaxK = ST == ST_DD ? 64 : 96;
  static constexpr int kBSlice = kNJ * kMaxK * 2;  // bytes of one digit slice of the small operand
};
// a group sums at most 7 digit pairs over K columns of products |d d'| <= 2^14
static_assert(7 * Geo<ST_F32>::kMaxK * (1 << 14) < (1 << 24), "group sums stay below 2^24");
static_assert(7 * Geo<ST_DD>::kMaxK * (1 << 14) < (1 << 24), "group sums stay below 2^24");

// staging buffer: the basis planes of a tile, then the tile's stored residual (8 bytes a row)
// 2^(8 (6 - q)): the scale of group g = q + 2 relative to the smallest group (g = 8)
__device__ __forceinline__ float group_scale(int q) { return __int_as_float((127 + 8 * (6 - q)) << 23); }
constexpr int kGridBits = 54;  // values on the grid 2^(e - 54): |I| < 2^54, seven bytes
constexpr long long kDigitBias = 0x80808080808080ll;

template <int ST>
__host__ __device__ constexpr int stage_bytes(int rs) {
  return ((Geo<ST>::kPlanes * kTM * rs + kTM * 8 + 1023) / 1024) * 1024;
}
template <int ST>
__host__ __device__ constexpr int smem_bytes(int rs) {
  return stage_bytes<ST>(rs) + 2 * kABuf + kSlices * Geo<ST>::kBSlice;
}

// a barrier of the worker warps alone (named barrier 1; the issuer warp is not in it) that
// also returns whether v held in any of them
__device__ __forceinline__ bool workers_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.cta.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kWorkers)
      : "memory");
  return r != 0;
}

// exponent e with |v| < 2^e for every double-float v of a set whose largest |hi| is mx (from
// the bits of mx; 0 for mx = 0): |hi + lo| < 2^e as well, since |lo| <= ulp(hi) / 2
__device__ __forceinline__ int grid_exp(float mx) {
  const int ex = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
  return mx > 0.f ? (ex ? ex : 1) - 126 : 0;
}

// round(x 2^k) as an integer, by shifting the significand (|x| < 2^(54 - k) keeps it below 2^54)
__device__ __forceinline__ long long fixed_part(float x, int k) {
  const uint32_t ux = __float_as_uint(x);
  const int ex = (int)((ux >> 23) & 0xFFu);
  const uint32_t m = (ux & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
  const int sh = (ex ? ex : 1) - 150 + k;
  long long v = 0;
  if (sh >= 0)
    v = (long long)m << sh;
  else if (sh > -32)
    v = (long long)((m + (1u << (-sh - 1))) >> (-sh));
  return (ux >> 31) ? -v : v;
}

// the biased fixed-point value of h + l on the grid 2^(e - 54): its byte s (from the top)
// less 128 is digit s
__device__ __forceinline__ unsigned long long biased_fixed(float h, float l, int e) {
  const int k = kGridBits - e;
  return (unsigned long long)(fixed_part(h, k) + fixed_part(l, k) + kDigitBias);
}

// digit s = 1..7 (most significant first) of a biased fixed-point value, as an exact float:
// the byte is moved under the exponent of 2^23 (a float 2^23 + b), then 2^23 + 128 is taken off
template <int S>
__device__ __forceinline__ float digit_f(unsigned long long u) {
  constexpr int byte = 7 - S;  // byte 6 holds digit 1
  const uint32_t w = byte >= 4 ? (uint32_t)(u >> 32) : (uint32_t)u;
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (byte & 3))) - 8388736.0f;
}

// two values' digit s as a bfloat16 pair (the first value in the low half)
template <int S>
__device__ __forceinline__ uint32_t digit_pair(unsigned long long u0, unsigned long long u1) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(digit_f<S>(u0), digit_f<S>(u1));
  return *reinterpret_cast<const uint32_t*>(&p);
}

// the tile's rows of both planes (and of the stored residual e when `with_e`) into the stage;
// npad is a multiple of 64 rows, so every copy is a whole number of 16-byte units
template <int ST>
__device__ __forceinline__ void issue_tile(const Ws& ws, unsigned char* stage, int rs, int64_t tile, bool with_e,
                                           uint64_t* bar) {
  constexpr int P = Geo<ST>::kPlanes;
  const int64_t row0 = tile * kTM;
  const int64_t rows = (ws.npad - row0) < kTM ? (ws.npad - row0) : kTM;
  const uint32_t bytes = (uint32_t)(rows * rs);
  mbar_arrive_expect_tx(bar, P * bytes + (with_e ? (uint32_t)(rows * 8) : 0u));
  bulk_g2s(stage, reinterpret_cast<const unsigned char*>(ws.Lh) + row0 * rs, bytes, bar);
  if constexpr (P == 2)
    bulk_g2s(stage + (size_t)kTM * rs, reinterpret_cast<const unsigned char*>(ws.Ll) + row0 * rs, bytes, bar);
  if (with_e) bulk_g2s(stage + (size_t)P * kTM * rs, ws.ebuf + row0, (uint32_t)(rows * 8), bar);
}

// COMPACT = false: X[:, j] = L0[:, :r0] coef[:, j] for j < kcols, X column-major in the
// snapshot type (doubles with double-float storage, floats with FP32 storage);
// a pending basis column (its residual stored by the last update) is formed on the way and
// written to L0, so no separate pass over the basis is needed before a prediction.
// COMPACT = true: when the update in flight compacts, L0[:, :rnew] <- [L0[:, :r0] j0] Q_B in
// place (the tile's rows are staged before they are overwritten, by the CTA that read them).
// ST: the basis storage, double-float (two planes) or FP32 (one plane: its elements enter
// with a zero lo part, and the columns written back are rounded to FP32 as stored).
template <bool COMPACT, int ST>
__device__ __forceinline__ void split_body(const Ws& ws, CtaPos cp, int kcols, double* out, int64_t ld) {
  constexpr int kMaxK = Geo<ST>::kMaxK;
  constexpr int kBSlice = Geo<ST>::kBSlice;
  constexpr int kPlanes = Geo<ST>::kPlanes;
  if constexpr (COMPACT) {
    pdl_wait();
    if (ws.ctl->mode != PB_COMPACT) return;  // most updates: nothing to do
  }
  extern __shared__ __align__(1024) unsigned char sp[];
  Ctl* ctl = ws.ctl;
  const int qld = ws.cap + 1;
  // K: columns of the tall operand (j0 last when appended, or the pending column of a
  // rollout), J: output columns; r0 of them come from the staged rows
  int r0, K, J, append = 0;
  const float2* bsrc;  // the small operand, column j at bsrc + j qld
  const StateBuf st = ws.st[ctl->cur];
  if constexpr (COMPACT) {
    append = ctl->append;
    r0 = ctl->r0e - append;
    K = r0 + append;
    J = ctl->rnew;
    bsrc = ws.sm.QB;
  } else {
    // column r0 - 1 of L0 may still be pending (its residual stored, the column not yet
    // written): the rollout forms it per row, uses it and writes it back
    append = st.hdr->pend;
    K = st.hdr->r0;
    r0 = K - append;
    J = kcols;
    bsrc = ws.sm.coef;
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rs = ws.ldg * 4;
  const int kpad = (K + kKC - 1) / kKC * kKC;
  const int nchunk = kpad / kKC;
  unsigned char* stage = sp;
  unsigned char* adig = sp + stage_bytes<ST>(rs);
  unsigned char* bdig = adig + 2 * kABuf;
  __shared__ int fexp[kNJ];
  // per-row exponent and new column j0 (compaction) of a tile, by tile parity: a worker warp
  // may start the next tile while others still read this tile's rows in their epilogue
  __shared__ int erow_[2][kTM];
  __shared__ float jh_[2][kTM], jl_[2][kTM];
  __shared__ float sh_s[kMaxK], sl_s[kMaxK];   // its coefficients s (compaction)
  __shared__ __align__(8) uint64_t bar_tma, bar_mma[2], bar_full[2], bar_drain;
  __shared__ volatile int abort_s;
  __shared__ uint32_t tmem_slot;
  const bool with_e = append != 0;
  dd inv = dd{0.f, 0.f};
  if (with_e) {
    // the new column's coefficients s and 1/rho0: of the update in flight (compaction) or
    // of the update that left the column pending (rollout)
    const float2* sco = COMPACT ? ws.sm.red : st.ps;
    if constexpr (COMPACT)
      inv = dd_from_double(1.0 / ctl->rho0);
    else
      inv = dd{st.hdr->pinv.x, st.hdr->pinv.y};
    for (int k = tid; k < kMaxK; k += kThreadsS) {
      const float2 v = k < r0 ? sco[k] : make_float2(0.f, 0.f);
      sh_s[k] = v.x;
      sl_s[k] = v.y;
    }
  }

  // ---- digits of the small operand: its column j is row j of the B operand (K-major)
  for (int j = warp; j < kNJ; j += kThreadsS / 32) {
    float mx = 0.f;
    if (j < J)
      for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(bsrc[(size_t)j * qld + k].x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) fexp[j] = grid_exp(mx);
  }
  __syncthreads();
  for (int o = tid; o < kNJ * kMaxK; o += kThreadsS) {
    const int j = o / kMaxK, k = o % kMaxK;
    float h = 0.f, l = 0.f;
    if (j < J && k < K) {
      const float2 q = bsrc[(size_t)j * qld + k];
      h = q.x;
      l = q.y;
    }
    const unsigned long long u = biased_fixed(h, l, fexp[j]);
    const int off = tc::kmajor_off(j, k, kMaxK / 8);
    uint16_t d[kSlices];
    d[0] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<1>(u)));
    d[1] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<2>(u)));
    d[2] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<3>(u)));
    d[3] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<4>(u)));
    d[4] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<5>(u)));
    d[5] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<6>(u)));
    d[6] = __bfloat16_as_ushort(__float2bfloat16_rn(digit_f<7>(u)));
#pragma unroll
    for (int s = 0; s < kSlices; ++s) *reinterpret_cast<uint16_t*>(bdig + s * kBSlice + off) = d[s];
  }
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    mbar_init(&bar_full[0], kWorkers);
    mbar_init(&bar_full[1], kWorkers);
    mbar_init(&bar_drain, 1);
    abort_s = 0;
    mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  const int64_t ntiles = (ws.n + kTM - 1) / kTM;
  const int G = cp.g;
  const int my_tiles = (int)((ntiles - cp.b + G - 1) / G);
  const uint32_t idesc = tc::instr_desc_bf16_f32(kTM, kNJ);
  // descriptors of digit slice 1 at chunk 0; every other operand differs only in its start
  // address, so its descriptor is this one plus (byte offset >> 4) in the start field (shared
  // memory addresses stay below 2^18, so the field never carries)
  const uint64_t adesc0 = tc::smem_desc(smem_addr(adig), tc::kCoreBytes, (kBufK / 8) * tc::kCoreBytes);
  static_assert((kABuf >> 4) < (1 << 13), "a buffer offset fits the descriptor's start field");
  const uint64_t bdesc0 = tc::smem_desc(smem_addr(bdig), tc::kCoreBytes, (kMaxK / 8) * tc::kCoreBytes);

  // Roles.  The last warp issues the copies and the products; the 16 workers form digits and
  // read the accumulators.  Handoffs by mbarriers: bar_tma (a tile is staged), bar_full[b]
  // (every worker has put its digits of a chunk in buffer b), bar_mma[b] (the products that
  // read buffer b are done: tcgen05.commit).  The workers never wait for the issuer to
  // finish issuing, so the digits of chunk c + 1 are formed while the products of chunk c
  // run.  Every wait is bounded: a timeout sets DEV_TIMEOUT and abort_s, and each role stops
  // at its next check (the other role's waits then run out as well).
  if (warp == kWorkerWarps) {
    if (lane == 0 && my_tiles > 0) {
      issue_tile<ST>(ws, stage, rs, cp.b, with_e, &bar_tma);
      int tma_issued = 1;
      uint32_t pf[2] = {0u, 0u};
      bool issued = false;
      for (int li = 0; li < my_tiles && !abort_s; ++li) {
        const int64_t tile = cp.b + (int64_t)li * G;
        for (int cc = 0; cc < nchunk; ++cc) {
          const int b = cc & 1;
          if (!mbar_wait(&bar_full[b], pf[b], &ctl->status)) {
            abort_s = 1;
            break;
          }
          pf[b] ^= 1u;
          tc::fence_after_sync();
          // the staging buffer is free once the tile's last digits are formed: next tile
          if (cc + 1 == nchunk && li + 1 < my_tiles) {
            issue_tile<ST>(ws, stage, rs, tile + G, with_e, &bar_tma);
            ++tma_issued;
          }
          const uint64_t ab = adesc0 + (uint64_t)((b * kABuf) >> 4);
          const uint64_t bb = bdesc0 + (uint64_t)((cc * 2 * tc::kCoreBytes) >> 4);
#pragma unroll
          for (int gs = 2; gs <= 8; ++gs)
#pragma unroll
            for (int s = 1; s < gs; ++s) {
              const int t = gs - s;  // s, t <= 7 since g <= 8
              const uint64_t ad = ab + (uint64_t)(((s - 1) * kASlice) >> 4);
              const uint64_t bd = bb + (uint64_t)(((t - 1) * kBSlice) >> 4);
              const uint32_t acc = (cc > 0 || s > 1) ? 1u : 0u;
              tc::mma_bf16(tmem + (uint32_t)((gs - 2) * kNJ), ad, bd, idesc, acc);
            }
          tc::mma_commit(&bar_mma[b]);
          issued = true;
        }
      }
      // before the shared and tensor memory are released: every product issued is done and
      // every copy issued has landed (bounded waits; normally already so)
      const uint64_t t0 = global_ns();
      if (issued) {
        tc::mma_commit(&bar_drain);
        while (!mbar_try_wait(&bar_drain, 0u) && global_ns() - t0 < 1000000000ull) {
        }
      }
      while (!mbar_try_wait(&bar_tma, (uint32_t)((tma_issued - 1) & 1)) && global_ns() - t0 < 1500000000ull) {
      }
    }
  } else {
    // digit phase: four threads per row, thread q of a row owning columns 4q .. 4q + 3 of a
    // chunk (half of a 16-byte core-matrix row per slice)
    const int row = tid >> 2, quad = tid & 3;
    const float* sh = reinterpret_cast<const float*>(stage) + (size_t)row * (rs / 4);
    // the lo plane (double-float storage; FP32 elements have a zero lo part)
    const float* sl = reinterpret_cast<const float*>(stage + (size_t)(kPlanes - 1) * kTM * rs) + (size_t)row * (rs / 4);
    auto lo_of = [&](int k) -> float { return kPlanes == 2 ? sl[k] : 0.f; };
    uint32_t par_tma = 0, par_mma[2] = {0u, 0u};
    bool ok = true;
    for (int li = 0; li < my_tiles; ++li) {
      const int64_t tile = cp.b + (int64_t)li * G;
      const int64_t row0 = tile * kTM;
      if (ok && !mbar_wait(&bar_tma, par_tma, &ctl->status)) {
        ok = false;
        abort_s = 1;
      }
      par_tma ^= 1u;
      int* erow = erow_[li & 1];
      float* jh = jh_[li & 1];
      float* jl = jl_[li & 1];
      const bool live = row0 + row < ws.n;
      if (with_e) {
        // j0 = (e - L0[:, :r0] s) / rho0 for this row, a quarter of the dot per thread
        Acc d = acc_zero();
        if (live)
          for (int k = quad; k < r0; k += 4) acc_fma(d, sh[k], lo_of(k), sh_s[k], sl_s[k]);
        acc_add(d, __shfl_xor_sync(0xffffffffu, d.h, 1), __shfl_xor_sync(0xffffffffu, d.l, 1));
        acc_add(d, __shfl_xor_sync(0xffffffffu, d.h, 2), __shfl_xor_sync(0xffffffffu, d.l, 2));
        if (quad == 0) {
          const float2 ev = reinterpret_cast<const float2*>(stage + (size_t)kPlanes * kTM * rs)[row];
          Acc e = Acc{ev.x, ev.y};
          acc_add(e, -d.h, -d.l);
          e = acc_norm(e);
          Acc j = acc_zero();
          acc_fma(j, e.h, e.l, inv.h, inv.l);
          j = acc_norm(j);
          // the column as stored (rounded to FP32 in that storage), and used as stored
          float h = j.h, l = j.l;
          if constexpr (kPlanes == 1) {
            h = h + l;
            l = 0.f;
          }
          jh[row] = live ? h : 0.f;
          jl[row] = live ? l : 0.f;
          if (!COMPACT && live) {  // the pending column, written back
            const size_t o = (size_t)(row0 + row) * ws.ldg + r0;
            reinterpret_cast<float*>(ws.Lh)[o] = h;
            if constexpr (kPlanes == 2) ws.Ll[o] = l;
          }
        }
        __syncwarp();
      }
      // the row's exponent: max |hi| over its K columns, a quarter of them per thread
      {
        float mx = 0.f;
        if (live)
          for (int k = quad; k < K; k += 4) mx = fmaxf(mx, fabsf(k < r0 ? sh[k] : jh[row]));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        if (quad == 0) erow[row] = grid_exp(mx);
      }
      __syncwarp();
      const int my_e = erow[row];
      for (int cc = 0; cc < nchunk; ++cc) {
        const int b = cc & 1;
        if (cc >= 2) {  // the products that read buffer b (chunk cc - 2) are done
          if (ok && !mbar_wait(&bar_mma[b], par_mma[b], &ctl->status)) {
            ok = false;
            abort_s = 1;
          }
          par_mma[b] ^= 1u;
          tc::fence_after_sync();
        }
        unsigned char* abuf = adig + b * kABuf;
        // digits of basis columns kb .. kb + 3 of this row; columns at or past K (the chunk's
        // zero padding) store zeros without arithmetic
        const int kb = cc * kKC + 4 * quad;
        const int off = tc::kmajor_off(row, 4 * quad, kBufK / 8);
        if (live && kb < K) {
          uint32_t w[kSlices][2];
#pragma unroll
          for (int kk = 0; kk < 4; kk += 2) {
            const int k = kb + kk;
            float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
            if (k < r0) {
              h0 = sh[k];
              l0 = lo_of(k);
            } else if (k < K) {  // the new column (compaction)
              h0 = jh[row];
              l0 = jl[row];
            }
            if (k + 1 < r0) {
              h1 = sh[k + 1];
              l1 = lo_of(k + 1);
            } else if (k + 1 < K) {
              h1 = jh[row];
              l1 = jl[row];
            }
            const unsigned long long u0 = biased_fixed(h0, l0, my_e), u1 = biased_fixed(h1, l1, my_e);
            w[0][kk >> 1] = digit_pair<1>(u0, u1);
            w[1][kk >> 1] = digit_pair<2>(u0, u1);
            w[2][kk >> 1] = digit_pair<3>(u0, u1);
            w[3][kk >> 1] = digit_pair<4>(u0, u1);
            w[4][kk >> 1] = digit_pair<5>(u0, u1);
            w[5][kk >> 1] = digit_pair<6>(u0, u1);
            w[6][kk >> 1] = digit_pair<7>(u0, u1);
          }
#pragma unroll
          for (int s = 0; s < kSlices; ++s) *reinterpret_cast<uint2*>(abuf + s * kASlice + off) = make_uint2(w[s][0], w[s][1]);
        } else {
#pragma unroll
          for (int s = 0; s < kSlices; ++s) *reinterpret_cast<uint2*>(abuf + s * kASlice + off) = make_uint2(0, 0);
        }
        tc::fence_proxy_async();
        mbar_arrive(&bar_full[b]);
      }
      // the accumulators are read only once every product of the tile is done: the commits
      // not yet waited for, the earlier one first
      for (int q = (nchunk >= 2 ? nchunk - 2 : 0); q < nchunk; ++q) {
        const int b = q & 1;
        if (ok && !mbar_wait(&bar_mma[b], par_mma[b], &ctl->status)) {
          ok = false;
          abort_s = 1;
        }
        par_mma[b] ^= 1u;
      }
      tc::fence_after_sync();
      // every worker's row exponents are in place (the epilogue reads other warps' rows), and
      // all workers agree whether to go on
      if (workers_sync_or(!ok || abort_s != 0)) break;
      // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and 16 columns
      // (quarter w / 4); X = 2^(e_i + f_j - 60) sum_g G_g 2^(8 (8 - g))
      {
        const int trow = 32 * (warp & 3) + lane;
        const int64_t orow = row0 + trow;
        const int er = erow[trow];
        const int jb = 16 * (warp >> 2);
        for (int c8 = 0; c8 < 16; c8 += 8) {
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
          if (orow >= ws.n || jb + c8 >= J) continue;
          float vh[8], vl[8];
          int sc[8];
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            // every term G_g 2^(8 (8 - g)) is an exact float (|G_g| < 2^24): a cascaded sum,
            // smallest term first, with the exact rounding error of each addition (two-sum)
            // gathered in a second float, then one renormalization; columns u and u + 1 share
            // each FP32x2 instruction
            f2x sh2 = f2x_pack(__uint_as_float(g[kGroups - 1][u]), __uint_as_float(g[kGroups - 1][u + 1]));
            f2x el2 = 0ull;
#pragma unroll
            for (int q = kGroups - 2; q >= 0; --q) {
              const f2x t = mul2(f2x_pack(__uint_as_float(g[q][u]), __uint_as_float(g[q][u + 1])),
                                 f2x_pack(group_scale(q), group_scale(q)));
              const f2x s2 = add2(sh2, t);
              const f2x bb = sub2(s2, sh2);
              el2 = add2(el2, add2(sub2(sh2, sub2(s2, bb)), sub2(t, bb)));
              sh2 = s2;
            }
            const f2x hs = add2(sh2, el2);  // fast two-sum: |sh| >= |el|
            const f2x ls = sub2(el2, sub2(hs, sh2));
            f2x_unpack(hs, vh[u], vh[u + 1]);
            f2x_unpack(ls, vl[u], vl[u + 1]);
            sc[u] = er + fexp[jb + c8 + u] - 60;  // the value is 2^sc (vh + vl)
            sc[u + 1] = er + fexp[jb + c8 + u + 1] - 60;
          }
          if constexpr (COMPACT) {
            // whole 8-column pieces of the row as two 16-byte stores per plane
            const size_t o = (size_t)orow * ws.ldg + jb + c8;
            float* Lh = reinterpret_cast<float*>(ws.Lh);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              // basis entries lie well inside the float range: an exact power-of-two product
              if (sc[u] >= -126 && sc[u] <= 127) {
                const float p2 = __int_as_float((sc[u] + 127) << 23);
                vh[u] = __fmul_rn(vh[u], p2);
                vl[u] = __fmul_rn(vl[u], p2);
              } else {
                vh[u] = ldexpf(vh[u], sc[u]);
                vl[u] = ldexpf(vl[u], sc[u]);
              }
            }
            if constexpr (kPlanes == 1) {  // FP32 storage: the pair rounded to one float
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                vh[u] = vh[u] + vl[u];
                vl[u] = 0.f;
              }
            }
            if (jb + c8 + 8 <= J) {
              *reinterpret_cast<float4*>(Lh + o) = make_float4(vh[0], vh[1], vh[2], vh[3]);
              *reinterpret_cast<float4*>(Lh + o + 4) = make_float4(vh[4], vh[5], vh[6], vh[7]);
              if constexpr (kPlanes == 2) {
                *reinterpret_cast<float4*>(ws.Ll + o) = make_float4(vl[0], vl[1], vl[2], vl[3]);
                *reinterpret_cast<float4*>(ws.Ll + o + 4) = make_float4(vl[4], vl[5], vl[6], vl[7]);
              }
            } else {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (jb + c8 + u < J) {
                  Lh[o + u] = vh[u];
                  if constexpr (kPlanes == 2) ws.Ll[o + u] = vl[u];
                }
            }
          } else if constexpr (kPlanes == 2) {
            // double-float storage predicts doubles: their bits from the pair by integer operations
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (jb + c8 + u < J) out[(size_t)(jb + c8 + u) * ld + orow] = pair_to_double_fast(vh[u], vl[u], sc[u]);
          } else {
            // FP32 storage predicts floats (its snapshot type): the pair rounded, then the exact
            // power-of-two scale
            float* outf = reinterpret_cast<float*>(out);
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (jb + c8 + u < J) {
                const float v = vh[u] + vl[u];
                outf[(size_t)(jb + c8 + u) * ld + orow] =
                    (sc[u] >= -126 && sc[u] <= 127) ? __fmul_rn(v, __int_as_float((sc[u] + 127) << 23)) : ldexpf(v, sc[u]);
              }
          }
        }
      }
      // the accumulators are read before the next tile's first products, which the issuer
      // starts after this worker's next arrival on bar_full
      tc::fence_before_sync();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (!COMPACT && with_e) {
    // the last CTA to finish (every CTA read the flag at its start) marks the column written
    __shared__ unsigned ticket;
    __threadfence();
    __syncthreads();
    if (tid == 0) ticket = atomicAdd(&ctl->ticket_b, 1u);
    __syncthreads();
    if (tid == 0 && ticket == (unsigned)(G - 1)) {
      st.hdr->pend = 0;
      ctl->ticket_b = 0u;
    }
  }
}

template <bool COMPACT, int ST>
__global__ void __launch_bounds__(kThreadsS, 1) k_split(const __grid_constant__ Ws ws, int kcols, double* out, int64_t ld) {
  split_body<COMPACT, ST>(ws, cta_single(), kcols, out, ld);
}
template <bool COMPACT, int ST>
__global__ void __launch_bounds__(kThreadsS, 1) k_split_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  split_body<COMPACT, ST>(*t.ws[i], batch_pos(t, i), 0, (double*)nullptr, (int64_t)0);
}

// the widest staged rows of each storage (its basis columns K padded: an odd chunk count)
template <int ST>
constexpr int widest_smem() {
  return smem_bytes<ST>(16 * ((Geo<ST>::kMaxK / 4) | 1));
}
static_assert(widest_smem<ST_DD>() <= 227 * 1024 && widest_smem<ST_F32>() <= 227 * 1024,
              "the widest staged tile and the digit buffers fit in shared memory");

}  // namespace split

// The tensor-core paths take double-float storage with at most 64 columns in the tall
// operand (r0 <= cap, plus the appended column of a compaction), and FP32 storage with at
// most 96: the small operand's digits for those K and one staged 128-row tile fit in shared
// memory.
static bool split_fits(const Ws& ws) {
  if (ws.prec == ST_DD) return split::smem_bytes<ST_DD>(ws.ldg * 4) <= 227 * 1024;
  if (ws.prec == ST_F32) return split::smem_bytes<ST_F32>(ws.ldg * 4) <= 227 * 1024;
  return false;
}
static int split_max_k(const Ws& ws) {
  return ws.prec == ST_DD ? split::Geo<ST_DD>::kMaxK : split::Geo<ST_F32>::kMaxK;
}
bool split_rollout_ok(const Ws& ws, int kcols) {
  return split_fits(ws) && kcols >= 8 && kcols <= split::kNJ && ws.cap <= split_max_k(ws);
}
bool split_compact_ok(const Ws& ws) {
  return split_fits(ws) && ws.cap + 1 <= split_max_k(ws) && ws.rmax <= split::kNJ;
}

// The shared-memory limit is a property of the kernel, shared by every handle in the process:
// set it for the widest rows each storage takes
cudaError_t prepare_split(const Ws& ws) {
  cudaError_t e = cudaSuccess;
  if (ws.prec == ST_DD) {
    const int sm = split::widest_smem<ST_DD>();
    e = cudaFuncSetAttribute(split::k_split<false, ST_DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(split::k_split<true, ST_DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  } else if (ws.prec == ST_F32) {
    const int sm = split::widest_smem<ST_F32>();
    e = cudaFuncSetAttribute(split::k_split<false, ST_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(split::k_split<true, ST_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  }
  return e;
}

static int split_grid(const Ws& ws, int sms) {
  const int64_t ntiles = (ws.n + split::kTM - 1) / split::kTM;
  return (int)(ntiles < sms ? ntiles : sms);
}

int split_grid_of(const Ws& ws, int sms) { return split_grid(ws, sms); }

cudaError_t prepare_split_batch() {
  cudaError_t e = cudaFuncSetAttribute(split::k_split_batch<true, ST_DD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       split::widest_smem<ST_DD>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(split::k_split_batch<true, ST_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             split::widest_smem<ST_F32>());
  return e;
}

// the compaction form over the instances of a batch (each instance's CTAs return at once
// unless its update compacts; every instance has the storage prec); the largest shared
// memory any instance can ask for
cudaError_t launch_split_compact_batch(const BatchTab& t, int prec, cudaStream_t s) {
  if (prec == ST_DD)
    return launch_dependent(split::k_split_batch<true, ST_DD>, t.first[t.ninst], split::kThreadsS,
                            (size_t)split::widest_smem<ST_DD>(), s, t);
  return launch_dependent(split::k_split_batch<true, ST_F32>, t.first[t.ninst], split::kThreadsS,
                          (size_t)split::widest_smem<ST_F32>(), s, t);
}

cudaError_t launch_split_rollout(const Ws& ws, int kcols, double* out, int64_t ld, int sms, cudaStream_t s) {
  if (ws.prec == ST_DD)
    split::k_split<false, ST_DD><<<split_grid(ws, sms), split::kThreadsS, split::smem_bytes<ST_DD>(ws.ldg * 4), s>>>(
        ws, kcols, out, ld);
  else
    split::k_split<false, ST_F32><<<split_grid(ws, sms), split::kThreadsS, split::smem_bytes<ST_F32>(ws.ldg * 4), s>>>(
        ws, kcols, out, ld);
  return cudaGetLastError();
}

// launched after the small solves of every update (in the update graph); it returns at once
// unless the update compacts
cudaError_t launch_split_compact(const Ws& ws, int sms, cudaStream_t s) {
  if (ws.prec == ST_DD)
    return launch_dependent(split::k_split<true, ST_DD>, split_grid(ws, sms), split::kThreadsS,
                            (size_t)split::smem_bytes<ST_DD>(ws.ldg * 4), s, ws, 0, (double*)nullptr, (int64_t)0);
  return launch_dependent(split::k_split<true, ST_F32>, split_grid(ws, sms), split::kThreadsS,
                          (size_t)split::smem_bytes<ST_F32>(ws.ldg * 4), s, ws, 0, (double*)nullptr, (int64_t)0);
}

}  // namespace odmd
