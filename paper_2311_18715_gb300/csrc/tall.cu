// Tall-skinny passes over the basis L0 (N x r0): the O(N r) part of every call.
//
//   pass A  (update, Sec. 2.3): e = c - L0 a, s = L0^T e, y = L0^T x, ||e||^2, e.x, ||x||^2
//   pass B  (update):           append j0 = (c - L0 a_c)/rho0, or compact L0 <- [L0 j0] QB
//   rollout (predict, Sec. 2.3): X = L0 C   (C = Q Re(V Lambda^t b), r0 x k)
//   check   (Sec. 2.2):          ||L0 c_t - x_fom||^2 and ||x_fom||^2, prediction never stored
//
// Each CTA is persistent over row tiles of kTile rows.  A tile of the basis (only the
// r0 active columns of each row) and the matching snapshot rows are brought into
// shared memory by TMA bulk copies (one per row and plane) completing on an mbarrier,
// several tiles in flight (pass A: as many as shared memory holds).  Shared rows are
// padded to an odd number of 16-byte chunks so that both the row-wise vector reads (dot
// products along a row) and the column-wise reads (sums down a column) are free of bank
// conflicts.
//
// Reductions are deterministic: per-CTA partials in a fixed order, then the last CTA to
// finish (atomic ticket) sums them in CTA order.
#include <type_traits>

#include "dd.cuh"
#include "odmd_internal.cuh"

namespace odmd {

template <int ST>
struct Traits;
// snap_t: the caller's snapshot element; stored_t: the workspace copy of a snapshot (a
// double is kept as a float pair so the tall passes need no FP64 instruction); vsz: bytes
// of stored_t.
template <>
struct Traits<ST_DD> {
  static constexpr int planes = 2, esz = 4, vsz = 8;
  using snap_t = double;
  using stored_t = float2;
};
template <>
struct Traits<ST_F32> {
  static constexpr int planes = 1, esz = 4, vsz = 4;
  using snap_t = float;
  using stored_t = float;
};
template <>
struct Traits<ST_BF16> {
  static constexpr int planes = 1, esz = 2, vsz = 4;
  using snap_t = float;
  using stored_t = float;
};

__device__ __forceinline__ int rows_in(int64_t n, int64_t row0) {
  const int64_t d = n - row0;
  return d < kTile ? (int)d : kTile;
}


// each stage: the basis rows (per plane, widest box) and three per-row slots of 8 bytes;
// every part starts on a 512-byte boundary (TMA tile destinations need 128).
template <int ST>
__host__ __device__ inline int stage_bytes(int cap) {
  using T = Traits<ST>;
  const int rs_max = 16 * box_chunks(cap, T::esz);
  return kTile * rs_max * T::planes + 3 * kTile * 8;
}

// Stored snapshot element -> float-float
__device__ __forceinline__ void load_snap(const float2* p, int i, float& h, float& l) {
  h = p[i].x;
  l = p[i].y;
}
__device__ __forceinline__ void load_snap(const float* p, int i, float& h, float& l) {
  h = p[i];
  l = 0.f;
}

// 8 basis elements of chunk q (16 bytes per plane) of smem row `row` -> hi/lo floats.
// For 4-byte elements a chunk holds 4 elements and only [0,4) are written.
template <int ST>
__device__ __forceinline__ int load_chunk(const unsigned char* plane_h, const unsigned char* plane_l,
                                          int rs, int row, int q, float* h, float* l) {
  if constexpr (ST == ST_BF16) {
    const uint4 v = *reinterpret_cast<const uint4*>(plane_h + row * rs + q * 16);
    const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(b[i]);
      h[2 * i] = f.x;
      h[2 * i + 1] = f.y;
      l[2 * i] = 0.f;
      l[2 * i + 1] = 0.f;
    }
    return 8;
  } else {
    const float4 vh = *reinterpret_cast<const float4*>(plane_h + row * rs + q * 16);
    h[0] = vh.x;
    h[1] = vh.y;
    h[2] = vh.z;
    h[3] = vh.w;
    if constexpr (ST == ST_DD) {
      const float4 vl = *reinterpret_cast<const float4*>(plane_l + row * rs + q * 16);
      l[0] = vl.x;
      l[1] = vl.y;
      l[2] = vl.z;
      l[3] = vl.w;
    } else {
      l[0] = l[1] = l[2] = l[3] = 0.f;
    }
    return 4;
  }
}

template <int ST>
__device__ __forceinline__ void load_elem(const unsigned char* plane_h, const unsigned char* plane_l, int rs,
                                          int row, int k, float& h, float& l) {
  if constexpr (ST == ST_BF16) {
    h = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(plane_h + row * rs)[k]);
    l = 0.f;
  } else {
    h = reinterpret_cast<const float*>(plane_h + row * rs)[k];
    l = (ST == ST_DD) ? reinterpret_cast<const float*>(plane_l + row * rs)[k] : 0.f;
  }
}

// Shared-memory pipeline over the row tiles owned by this CTA.  Each tile is one 2-D
// TMA load per basis plane (box: the active chunks of kTile rows) plus 1-D bulk copies
// of up to three per-row slots (8 bytes per row each), all completing on the stage's
// mbarrier.
template <int ST>
struct TilePipe {
  using T = Traits<ST>;
  static constexpr int kSlots = 3;
  unsigned char* base;
  uint64_t* bars;
  int stages, stage_sz, rs, nch, plane_off;
  int64_t n;
  const CUtensorMap* mh;    // map of the hi (or only) plane for the current box, or nullptr
  const CUtensorMap* ml;    // map of the lo plane (FP64 mode)
  const unsigned char* g[kSlots];  // per-row slots (or nullptr)
  int vb[kSlots];                  // bytes per row of each slot

  __device__ void setup(const Ws& ws, int r0, int nstages) {
    stages = nstages;
    stage_sz = stage_bytes<ST>(ws.cap);
    plane_off = kTile * 16 * box_chunks(ws.cap, T::esz);
    n = ws.n;
    if (r0 > 0) {
      const int c = box_chunks(r0, T::esz);
      rs = 16 * c;
      nch = c;
      mh = ws.maps + (c - 1) / 2;
      ml = (T::planes == 2) ? ws.maps + kMaxMaps + (c - 1) / 2 : nullptr;
    } else {
      rs = 16;
      nch = 0;
      mh = ml = nullptr;
    }
    for (int i = 0; i < kSlots; ++i) {
      g[i] = nullptr;
      vb[i] = 0;
    }
  }
  __device__ unsigned char* plane_h(int s) const { return base + (size_t)s * stage_sz; }
  __device__ unsigned char* plane_l(int s) const { return plane_h(s) + plane_off; }
  __device__ unsigned char* slot(int s, int i) const { return plane_h(s) + plane_off * T::planes + i * kTile * 8; }

  // Issue the copies of tile `tile` into stage `s` (called by one thread).
  __device__ void issue(int tile, int s) const {
    const int row0 = tile * kTile;
    uint32_t bytes = mh ? (uint32_t)(kTile * rs * T::planes) : 0u;
    for (int i = 0; i < kSlots; ++i)
      if (g[i]) bytes += kTile * vb[i];
    mbar_arrive_expect_tx(&bars[s], bytes);
    if (mh) {
      tma_load_2d(plane_h(s), mh, 0, row0, &bars[s]);
      if (T::planes == 2) tma_load_2d(plane_l(s), ml, 0, row0, &bars[s]);
    }
    for (int i = 0; i < kSlots; ++i)
      if (g[i]) bulk_g2s(slot(s, i), g[i] + (size_t)row0 * vb[i], kTile * vb[i], &bars[s]);
  }
};

// A basis element as stored (rounded to the storage format), as a float pair.
template <int ST>
__device__ __forceinline__ void round_to_storage(float& h, float& l) {
  if constexpr (ST == ST_BF16) {
    h = __bfloat162float(__float2bfloat16_rn(h));
    l = 0.f;
  } else if constexpr (ST == ST_F32) {
    h = h + l;
    l = 0.f;
  }
}

template <int ST>
__device__ __forceinline__ void store_elem_global(const Ws& ws, size_t o, float h, float l) {
  if constexpr (ST == ST_BF16) {
    reinterpret_cast<__nv_bfloat16*>(ws.Lh)[o] = __float2bfloat16_rn(h);
  } else {
    reinterpret_cast<float*>(ws.Lh)[o] = h;
    if constexpr (ST == ST_DD) ws.Ll[o] = l;
  }
}

template <int ST>
__device__ __forceinline__ void store_elem_smem(unsigned char* ph, unsigned char* pl, int rs, int row, int k, float h,
                                                float l) {
  if constexpr (ST == ST_BF16) {
    reinterpret_cast<__nv_bfloat16*>(ph + row * rs)[k] = __float2bfloat16_rn(h);
  } else {
    reinterpret_cast<float*>(ph + row * rs)[k] = h;
    if constexpr (ST == ST_DD) reinterpret_cast<float*>(pl + row * rs)[k] = l;
  }
}

// Partial row dot over chunks sub, sub + NSUB, ... of smem row t with a float-float
// coefficient vector (zero beyond its length).
template <int ST, int NSUB>
__device__ __forceinline__ Acc row_dot_partial(const TilePipe<ST>& P, int s, int t, int sub, const float* coh,
                                               const float* col) {
  constexpr int E = (ST == ST_BF16) ? 8 : 4;  // elements per 16-byte chunk
  Acc acc = acc_zero();
  const unsigned char* ph = P.plane_h(s);
  const unsigned char* pl = P.plane_l(s);
  for (int q = sub; q < P.nch; q += NSUB) {
    float h[8], l[8], ch[8], cl[8];
    load_chunk<ST>(ph, pl, P.rs, t, q, h, l);
#pragma unroll
    for (int i = 0; i < E; i += 4) {
      const float4 a = *reinterpret_cast<const float4*>(coh + q * E + i);
      const float4 b = *reinterpret_cast<const float4*>(col + q * E + i);
      ch[i] = a.x;
      ch[i + 1] = a.y;
      ch[i + 2] = a.z;
      ch[i + 3] = a.w;
      cl[i] = b.x;
      cl[i + 1] = b.y;
      cl[i + 2] = b.z;
      cl[i + 3] = b.w;
    }
#pragma unroll
    for (int i = 0; i < E; ++i) acc_fma(acc, h[i], l[i], ch[i], cl[i]);
  }
  return acc;
}

// Sum over the 8 adjacent lanes of a row group (every lane gets the sum).
__device__ __forceinline__ Acc group8_sum(Acc a) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, a.h, o);
    const float l = __shfl_xor_sync(0xffffffffu, a.l, o);
    acc_add(a, h, l);
  }
  return a;
}

// The elements of chunk q of smem row `row` as packed pairs (2 pairs for 4-byte elements,
// 4 for bf16); lo pairs are zero unless the basis is double-float.
template <int ST>
__device__ __forceinline__ void load_chunk2(const unsigned char* plane_h, const unsigned char* plane_l, int rs,
                                            int row, int q, f2x* H, f2x* L) {
  if constexpr (ST == ST_BF16) {
    const uint4 v = *reinterpret_cast<const uint4*>(plane_h + row * rs + q * 16);
    const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(b[i]);
      H[i] = f2x_pack(f.x, f.y);
      L[i] = 0ull;
    }
  } else {
    const ulonglong2 vh = *reinterpret_cast<const ulonglong2*>(plane_h + row * rs + q * 16);
    H[0] = vh.x;
    H[1] = vh.y;
    if constexpr (ST == ST_DD) {
      const ulonglong2 vl = *reinterpret_cast<const ulonglong2*>(plane_l + row * rs + q * 16);
      L[0] = vl.x;
      L[1] = vl.y;
    } else {
      L[0] = L[1] = 0ull;
    }
  }
}

// acc2_fma without the xl*yh term when the basis has no lo part
template <int ST>
__device__ __forceinline__ void acc2_fma_basis(Acc2& A, f2x xh, f2x xl, f2x yh, f2x nyh, f2x yl) {
  if constexpr (ST == ST_DD) {
    acc2_fma(A, xh, xl, yh, nyh, yl);
  } else {
    const f2x np = mul2(xh, nyh);
    f2x pe = fma2(xh, yh, np);
    pe = fma2(xh, yl, pe);
    const f2x s = sub2(A.h, np);
    const f2x bb = sub2(s, A.h);
    const f2x e = sub2(sub2(A.h, sub2(s, bb)), add2(np, bb));
    A.h = s;
    A.l = add2(A.l, add2(e, pe));
  }
}

// acc[r][c] += sum_k L0[t0 + 32 r][k] B[k][j0 + 2c .. j0 + 2c + 1]  (r < R, c < 4) over the
// nch chunks of the stage's rows, double-float.  B is in shared memory as three planes
// (hi, lo, -hi) with row stride ldb floats (a multiple of 4) and j0 a multiple of 8, so a
// column pair loads as a ready FP32x2 operand; a row element is broadcast to both lanes.
// A warp's lanes take consecutive rows, which keeps the row reads free of bank conflicts.
template <int ST, int R>
__device__ __forceinline__ void tile_dot8(const unsigned char* ph, const unsigned char* pl, int rs, int t0, int nch,
                                          const float* bh, const float* bl, const float* bn, int ldb, int j0,
                                          Acc2 (&A)[R][4]) {
  constexpr int E = (ST == ST_BF16) ? 8 : 4;
#pragma unroll 1
  for (int q = 0; q < nch; ++q) {
    float h[R][8], l[R][8];
#pragma unroll
    for (int r = 0; r < R; ++r) load_chunk<ST>(ph, pl, rs, t0 + 32 * r, q, h[r], l[r]);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int o = (q * E + i) * ldb + j0;
      const float4 h0 = *reinterpret_cast<const float4*>(bh + o), h1 = *reinterpret_cast<const float4*>(bh + o + 4);
      const float4 l0 = *reinterpret_cast<const float4*>(bl + o), l1 = *reinterpret_cast<const float4*>(bl + o + 4);
      const float4 n0 = *reinterpret_cast<const float4*>(bn + o), n1 = *reinterpret_cast<const float4*>(bn + o + 4);
      const f2x yh[4] = {f2x_pack(h0.x, h0.y), f2x_pack(h0.z, h0.w), f2x_pack(h1.x, h1.y), f2x_pack(h1.z, h1.w)};
      const f2x yl[4] = {f2x_pack(l0.x, l0.y), f2x_pack(l0.z, l0.w), f2x_pack(l1.x, l1.y), f2x_pack(l1.z, l1.w)};
      const f2x yn[4] = {f2x_pack(n0.x, n0.y), f2x_pack(n0.z, n0.w), f2x_pack(n1.x, n1.y), f2x_pack(n1.z, n1.w)};
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const f2x xb = f2x_pack(h[r][i], h[r][i]);
        const f2x xl = f2x_pack(l[r][i], l[r][i]);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2_fma_basis<ST>(A[r][c], xb, xl, yh[c], yn[c], yl[c]);
      }
    }
  }
}

// one extra term: acc[r][c] += x[r] B[k][j0 + 2c ..] (the appended column of a compaction)
template <int ST, int R>
__device__ __forceinline__ void tile_dot8_term(const float (&xh)[R], const float (&xl)[R], const float* bh,
                                               const float* bl, const float* bn, int o, Acc2 (&A)[R][4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const f2x yh = f2x_pack(bh[o + 2 * c], bh[o + 2 * c + 1]);
    const f2x yl = f2x_pack(bl[o + 2 * c], bl[o + 2 * c + 1]);
    const f2x yn = f2x_pack(bn[o + 2 * c], bn[o + 2 * c + 1]);
#pragma unroll
    for (int r = 0; r < R; ++r)
      acc2_fma(A[r][c], f2x_pack(xh[r], xh[r]), f2x_pack(xl[r], xl[r]), yh, yn, yl);
  }
}

// ---------------------------------------------------------------------------------------
// pass A: the pending column of the previous update (if any) is formed row by row from
// its stored residual, written to L0 and used at once; then
//   e = c - L0 a, s = L0^T e, y = L0^T x, ||e||^2, e.x, ||x||^2.
// Each CTA streams its 32-row tiles (whole rows of both basis planes, one bulk copy per
// plane) through a ring of shared stages; the warp that finishes with a stage refills it
// with the tile ns places ahead.  A warp takes whole tiles: lane i owns row i for the row
// dots, the pending column and the residual (no exchange between lanes; c, x and the
// stored residual of the row come in by plain loads issued before the tile's wait), then
// the lanes switch to owning 16-byte column chunks, 16 lanes per row and two rows at a
// time, and add the tile into column sums that stay in registers for the whole launch.
// Column sums meet across lanes, warps and CTAs once, at the end.  The double-float
// arithmetic runs on packed FP32x2 instructions; the row dots are unrolled for the
// tile's chunk count.
// ---------------------------------------------------------------------------------------
constexpr int kRowsA = kPassARows;              // rows per tile (one warp)
static_assert(kRowsA == 32, "a pass-A tile is one row per lane");
constexpr int kWarpsA = 8;                      // compute warps per CTA
constexpr int kThreadsA = 32 * kWarpsA;
#ifndef ODMD_PASS_A_MAX_STAGES
#define ODMD_PASS_A_MAX_STAGES 16
#endif
constexpr int kMaxStagesA = ODMD_PASS_A_MAX_STAGES;
constexpr int kBarBytesA = (8 * kMaxStagesA + 15) / 16 * 16;  // one barrier per stage
static_assert((kMaxCap + 8) * 4 % 16 == 0, "pass A coefficient arrays must stay 16-byte aligned");
constexpr int kSmemBudget = 227 * 1024 - 2048;  // dynamic shared memory per CTA, less the static part
// pass A's budget: enough stages to cover DRAM latency (~45 KB in flight per SM at the HBM
// rate) while leaving room on the SM for a CTA of the previous update's k_apply, which runs
// beside it in a pipelined update
constexpr int kSmemBudgetA = 168 * 1024;
constexpr int kCo = 128;  // length of a coefficient array: zero past r0, so chunk groups may overrun

// one stage: 32 whole rows (the full row pitch) of each basis plane
template <int ST>
__host__ __device__ inline int stage_bytes_a(int cap) {
  using T = Traits<ST>;
  return kRowsA * 16 * box_chunks(cap, T::esz) * T::planes;
}

// shared memory of pass A besides its stages: barriers, coefficients, per-warp e/x slots
__host__ __device__ inline int smem_a_fixed() { return kBarBytesA + 6 * kCo * 4 + kWarpsA * kRowsA * 3 * 16; }

// the column sums of every warp meet in the stage memory at the end
template <int ST>
__host__ __device__ inline size_t pass_a_region(int stage_sz, int nstages) {
  const size_t a = (size_t)nstages * stage_sz, b = (size_t)kWarpsA * 2 * kCo * sizeof(Acc);
  return a > b ? a : b;
}

// A tile is one 2-D tensor copy per plane of its 32 rows and only the chunks the row dots
// read (nch = the odd chunk count that covers r0, not the padded row pitch); in shared
// memory its rows are nch chunks apart (an odd number of 16-byte chunks, so the lanes of a
// warp reading one chunk of consecutive rows hit distinct banks).
template <int ST>
struct PipeA {
  using T = Traits<ST>;
  unsigned char* base;
  uint64_t* full;
  int stage_sz, rs, nch, plane_off;  // rs: shared-memory row pitch = 16 nch bytes
  const CUtensorMap* mh;             // hi (or only) plane's map of box (nch chunks, 32 rows)
  const CUtensorMap* ml;             // lo plane's (double-float)
  uint64_t policy;                   // L2 evict-first: the planes are streamed once per pass
  __device__ unsigned char* plane_h(int s) const { return base + (size_t)s * stage_sz; }
  __device__ unsigned char* plane_l(int s) const { return plane_h(s) + plane_off; }
  // the copies of tile `tile` into stage s (one thread)
  __device__ void issue(int tile, int s) const {
    mbar_arrive_expect_tx(&full[s], (uint32_t)(kRowsA * rs * T::planes));
    tma_load_2d_hint(plane_h(s), mh, 0, tile * kRowsA, &full[s], policy);
    if (T::planes == 2) tma_load_2d_hint(plane_l(s), ml, 0, tile * kRowsA, &full[s], policy);
  }
};

// Wait (at most 2 s) until the shared tile index *slot equals k.
__device__ __forceinline__ bool wait_issued(const int* slot, int k, int* status) {
  const volatile int* v = slot;
  if (*v == k) return true;
  const uint64_t t0 = global_ns();
  while (*v != k) {
    if (global_ns() - t0 > 2000000000ull) {
      atomicOr(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Row dots of one smem row (lane t) with the coefficient vectors a and s_prev over NCH
// chunks (a compile-time count).  The six coefficient arrays (a hi, -a hi, a lo, s hi, -s hi, s lo)
// are laid out back to back, kCo floats each.
template <int ST, int NCH>
__device__ __forceinline__ void row_dots(const unsigned char* ph, const unsigned char* pl, int rs, int t,
                                         const float* co, Acc2 (&DA)[2], Acc2 (&DS)[2]) {
  constexpr int kE = (ST == ST_BF16) ? 8 : 4, kP = kE / 2;
  // two chunks per loop body: fully unrolled row dots stall on instruction fetch
#pragma unroll 2
  for (int q = 0; q < NCH; ++q) {
    f2x H[kP], L[kP];
    load_chunk2<ST>(ph, pl, rs, t, q, H, L);
#pragma unroll
    for (int i = 0; i < kP; i += 2) {
      const int kk = q * kE + 2 * i;
      const ulonglong2 ah = *reinterpret_cast<const ulonglong2*>(co + kk);
      const ulonglong2 an = *reinterpret_cast<const ulonglong2*>(co + kCo + kk);
      const ulonglong2 al = *reinterpret_cast<const ulonglong2*>(co + 2 * kCo + kk);
      const ulonglong2 bh = *reinterpret_cast<const ulonglong2*>(co + 3 * kCo + kk);
      const ulonglong2 bn = *reinterpret_cast<const ulonglong2*>(co + 4 * kCo + kk);
      const ulonglong2 bl = *reinterpret_cast<const ulonglong2*>(co + 5 * kCo + kk);
      acc2_fma_basis<ST>(DA[q & 1], H[i], L[i], ah.x, an.x, al.x);
      acc2_fma_basis<ST>(DS[q & 1], H[i], L[i], bh.x, bn.x, bl.x);
      acc2_fma_basis<ST>(DA[q & 1], H[i + 1], L[i + 1], ah.y, an.y, al.y);
      acc2_fma_basis<ST>(DS[q & 1], H[i + 1], L[i + 1], bh.y, bn.y, bl.y);
    }
  }
}

// box widths are odd chunk counts: 1..25 for 4-byte elements, 1..13 for bf16
template <int ST>
__device__ __forceinline__ void row_dots_dispatch(int nch, const unsigned char* ph, const unsigned char* pl, int rs,
                                                  int t, const float* co, Acc2 (&DA)[2], Acc2 (&DS)[2]) {
#define ODMD_ROW_DOTS_CASE(n) \
  case n:                     \
    row_dots<ST, n>(ph, pl, rs, t, co, DA, DS); \
    break;
  switch (nch) {
    ODMD_ROW_DOTS_CASE(1)
    ODMD_ROW_DOTS_CASE(3)
    ODMD_ROW_DOTS_CASE(5)
    ODMD_ROW_DOTS_CASE(7)
    ODMD_ROW_DOTS_CASE(9)
    ODMD_ROW_DOTS_CASE(11)
    ODMD_ROW_DOTS_CASE(13)
    default:
      if constexpr (ST != ST_BF16) {
        switch (nch) {
          ODMD_ROW_DOTS_CASE(15)
          ODMD_ROW_DOTS_CASE(17)
          ODMD_ROW_DOTS_CASE(19)
          ODMD_ROW_DOTS_CASE(21)
          ODMD_ROW_DOTS_CASE(23)
          ODMD_ROW_DOTS_CASE(25)
          default:
            break;
        }
      }
  }
#undef ODMD_ROW_DOTS_CASE
}
static_assert(kMaxCap <= 96, "row_dots_dispatch covers box widths up to 25 chunks of 4-byte elements");

// ---------------------------------------------------------------------------------------
// Row blocks.  Every pass that ends in a reduction over rows (pass A, the check, the norm of
// the first snapshot) splits the rows the same way: ws.gridA blocks of whole 64-row tiles,
// block b holding tiles [b T / B, (b + 1) T / B) of the T = ceil(n / 64).  Logical CTA b of a
// pass works on block b alone and leaves its partial sums in slot b; the partials are then
// added in block order.  A run split over G row shards (each shard a contiguous range of
// blocks, as on G GPUs that each hold their rows) therefore computes bitwise the same
// partials, and folding them in the same order gives bitwise the unsharded result.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void block_tiles64(const Ws& ws, int b, int64_t& t0, int64_t& t1) {
  const int64_t T = (ws.n + kTile - 1) / kTile;
  t0 = (int64_t)b * T / ws.gridA;
  t1 = (int64_t)(b + 1) * T / ws.gridA;
}

// fold of pass A's per-block partials (one CTA of kThreadsA threads): 4 adjacent lanes per
// value, each summing every 4th block, then a fixed-order combine
__device__ void fold_pass_a(const Ws& ws, const StateBuf& st, int r0) {
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const int stride = 2 * ws.cap + 3;
  const int nv = 2 * r0 + 3;
  const int B = ws.gridA;
  for (int base = 0; base < 4 * nv; base += kThreadsA) {
    const int item = base + tid;
    const int v = item >> 2, q = item & 3;
    Acc sum = acc_zero();
    if (v < nv)
      for (int b = q; b < B; b += 4) {
        const float2 f = __ldcg(ws.part + (size_t)b * stride + v);
        acc_add(sum, f.x, f.y);
      }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, sum.h, o);
      const float l = __shfl_xor_sync(0xffffffffu, sum.l, o);
      acc_add(sum, h, l);
    }
    if (v < nv && q == 0) {
      sum = acc_norm(sum);
      if (!isfinite(sum.h) || !isfinite(sum.l)) atomicOr(&ctl->status, DEV_NONFINITE);
      ws.sm.red[v] = make_float2(sum.h, sum.l);
    }
  }
  if (tid == 0) {
    ctl->ticket_a = 0u;
    ctl->prof_r0_sum += (unsigned long long)r0;
    ctl->prof_a += 1ull;
    st.hdr->pend = 0;  // the pending column now exists in L0
  }
}

// sel < 0: the committed state and snapshot buffers (Ctl::cur, Ctl::cur_c).  sel >= 0 (the
// pipelined update, which runs this pass beside the previous update's SVD, before that
// update commits): state sel & 1, snapshot buffers (sel >> 1) & 1, and a gate sel >> 2: 0 run,
// 1 return at once if the previous update compacts (Ctl::pipe_flag; the pass then runs again
// after the compaction with gate 2), 2 run only if it compacts.
template <int ST>
__device__ __forceinline__ void pass_a_body(const Ws& ws, CtaPos cp, int cta0, int fold, int sel = -1) {
  pdl_wait();
  using T = Traits<ST>;
  using stored_t = typename T::stored_t;
  constexpr int kE = (ST == ST_BF16) ? 8 : 4;      // columns per 16-byte chunk
  constexpr int kP = kE / 2;                        // packed pairs per chunk
  constexpr int kCS = (ST == ST_BF16) ? 1 : 2;      // chunks a lane owns in the column sums
  extern __shared__ __align__(1024) unsigned char smem[];
  Ctl* ctl = ws.ctl;
  int cur, curc;
  if (sel < 0) {
    cur = ctl->cur;
    curc = ctl->cur_c;
  } else {
    const int gate = sel >> 2, compacts = ctl->pipe_flag;
    if ((gate == 1 && compacts) || (gate == 2 && !compacts)) return;  // uniform over the grid
    cur = sel & 1;
    curc = (sel >> 1) & 1;
  }
  const StateBuf st = ws.st[cur];
  const int r0 = st.hdr->r0;
  const int pend = st.hdr->pend;  // column p = r0 - 1 is formed here
  const int p = r0 - 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hrow = lane >> 4, cq = lane & 15;  // column phase: row parity and chunk of a lane
  const int ns = ws.stagesA;

  PipeA<ST> P;
  P.stage_sz = stage_bytes_a<ST>(ws.cap);
  P.nch = r0 > 0 ? box_chunks(r0, T::esz) : 0;
  {
    const int nb = P.nch > 0 ? P.nch : 1;  // with no columns yet, copy the first chunk anyway
    P.rs = 16 * nb;
    P.mh = ws.maps + 2 * kMaxMaps + (nb - 1) / 2;
    P.ml = ws.maps + 3 * kMaxMaps + (nb - 1) / 2;
  }
  P.plane_off = kRowsA * P.rs;
  // per-row vectors come in by plain loads, issued before the tile's wait: c, x, the stored
  // residual of the previous update
  const stored_t* cvec = reinterpret_cast<const stored_t*>(ws.cbuf[curc]);
  const stored_t* xvec = reinterpret_cast<const stored_t*>(ws.cbuf[curc ^ 1]);

  // shared layout: stages | one barrier per stage | coefficients a and s_prev (hi, -hi, lo
  // each) | per-warp e/x slots: 3 packed pairs per row (eh, eh, el, el), (-eh, -eh, xh, xh),
  // (xl, xl, -xh, -xh)
  P.base = smem;
  unsigned char* sp = smem + pass_a_region<ST>(P.stage_sz, ns);
  P.full = reinterpret_cast<uint64_t*>(sp);
  sp += kBarBytesA;
  float* coh = reinterpret_cast<float*>(sp);
  float* con = coh + kCo;
  float* col = con + kCo;
  float* csh = col + kCo;
  float* csn = csh + kCo;
  float* csl = csn + kCo;
  float4* ex4 = reinterpret_cast<float4*>(csl + kCo);
  __shared__ int abort_flag;
  __shared__ int last_issued[kMaxStagesA];  // tile last issued into each stage (for a drain)

  const int kpad = P.nch * kE;
  for (int k = tid; k < kCo; k += kThreadsA) {
    float h = 0.f, l = 0.f, sh = 0.f, sl = 0.f;
    if (k < r0 && !(pend && k == p)) {
      h = st.a[k].x;
      l = st.a[k].y;
    }
    if (pend && k < p) {
      sh = st.ps[k].x;
      sl = st.ps[k].y;
    }
    if (k >= kpad) h = l = sh = sl = 0.f;
    coh[k] = h;
    con[k] = -h;
    col[k] = l;
    csh[k] = sh;
    csn[k] = -sh;
    csl[k] = sl;
  }
  const float aph = pend ? st.a[p].x : 0.f, apl = pend ? st.a[p].y : 0.f;
  const float pih = st.hdr->pinv.x, pil = st.hdr->pinv.y;
  // this CTA's row block, in tiles of kRowsA = 32 rows
  static_assert(kTile == 2 * kRowsA, "a row block is whole 64-row tiles");
  const int blk = cta0 + cp.b;
  int64_t b0, b1;
  block_tiles64(ws, blk, b0, b1);
  const int64_t ntiles = (ws.n + kRowsA - 1) / kRowsA;
  const int64_t tbase = 2 * b0;
  const int my_tiles = (int)((2 * b1 < ntiles ? 2 * b1 : ntiles) - tbase);
  P.policy = l2_evict_first_policy();
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < ns; ++s) {
      mbar_init(&P.full[s], 1);
      last_issued[s] = -1;
    }
    mbar_fence_init();
    // the first ns tiles; afterwards the warp that releases a stage refills it
    for (int k = 0; k < ns && k < my_tiles; ++k) {
      last_issued[k] = k;
      P.issue((int)(tbase + k), k);
    }
  }
  __syncthreads();

  Acc2 Sacc[kCS][kP], Yacc[kCS][kP], Sacc2[kCS][kP], Yacc2[kCS][kP];
#pragma unroll
  for (int c = 0; c < kCS; ++c)
#pragma unroll
    for (int i = 0; i < kP; ++i) Sacc[c][i] = Yacc[c][i] = Sacc2[c][i] = Yacc2[c][i] = acc2_zero();
  Acc eta = acc_zero(), exa = acc_zero(), xi = acc_zero();

  {
    float4* ex = ex4 + warp * kRowsA * 3;
    for (int k = warp; k < my_tiles; k += kWarpsA) {
      const int s = k % ns;
      const int64_t row0 = (tbase + k) * kRowsA;
      const int rows = (int)((ws.n - row0) < kRowsA ? (ws.n - row0) : kRowsA);
      // rows past n (up to the padded length) read zeros
      const stored_t cv = cvec[row0 + lane], xv = xvec[row0 + lane];
      const float2 ep = pend ? ws.ebuf[row0 + lane] : make_float2(0.f, 0.f);
      // a stage's barrier is waited on by parity, which cannot tell tile k's phase from the
      // phase two refills earlier: first make sure tile k itself has been issued into it
      bool ok = !abort_flag;
      if (ok) ok = wait_issued(&last_issued[s], k, &ctl->status);
      if (ok) ok = mbar_wait(&P.full[s], (uint32_t)((k / ns) & 1), &ctl->status);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        abort_flag = 1;
        break;
      }
      const unsigned char* ph = P.plane_h(s);
      const unsigned char* pl = P.plane_l(s);
      // ---- row phase: lane = row
      {
        const int t = lane;
        // the chunk count is a compile-time constant in each branch, so the row dot is
        // straight-line code whose chains the compiler interleaves
        Acc2 DA[2] = {acc2_zero(), acc2_zero()}, DS[2] = {acc2_zero(), acc2_zero()};
        row_dots_dispatch<ST>(P.nch, ph, pl, P.rs, t, coh, DA, DS);
        Acc da, ds, u, v, w;
        acc2_split(DA[0], da, u);
        acc2_split(DA[1], v, w);
        acc_add(da, u.h, u.l);
        acc_add(da, v.h, v.l);
        acc_add(da, w.h, w.l);
        acc2_split(DS[0], ds, u);
        acc2_split(DS[1], v, w);
        acc_add(ds, u.h, u.l);
        acc_add(ds, v.h, v.l);
        acc_add(ds, w.h, w.l);
        float ch, cl, xh_, xl_;
        load_snap(&cv, 0, ch, cl);
        load_snap(&xv, 0, xh_, xl_);
        if (pend) {
          // j = (e_prev - L0[:, :p] s_prev) / rho0, as stored; a_p j joins the row dot
          Acc j = Acc{ep.x, ep.y};
          acc_add(j, -ds.h, -ds.l);
          j = acc_norm(j);
          Acc jj = acc_zero();
          acc_fma(jj, j.h, j.l, pih, pil);
          jj = acc_norm(jj);
          float jh = jj.h, jl = jj.l;
          round_to_storage<ST>(jh, jl);
          store_elem_smem<ST>(P.plane_h(s), P.plane_l(s), P.rs, t, p, jh, jl);
          if (t < rows) store_elem_global<ST>(ws, (size_t)(row0 + t) * ws.ldg + p, jh, jl);
          acc_fma(da, jh, jl, aph, apl);
        }
        Acc e = Acc{ch, cl};
        acc_add(e, -da.h, -da.l);
        e = acc_norm(e);
        if (t >= rows) {
          e = acc_zero();
          xh_ = xl_ = 0.f;
        } else {
          ws.ebuf[row0 + t] = make_float2(e.h, e.l);  // kept for the second Gram-Schmidt pass
        }
        ex[3 * t] = make_float4(e.h, e.h, e.l, e.l);
        ex[3 * t + 1] = make_float4(-e.h, -e.h, xh_, xh_);
        ex[3 * t + 2] = make_float4(xl_, xl_, -xh_, -xh_);
        acc_fma(eta, e.h, e.l, e.h, e.l);
        acc_fma(exa, e.h, e.l, xh_, xl_);
        acc_fma(xi, xh_, xl_, xh_, xl_);
      }
      __syncwarp();
      // ---- column phase: lanes 0-15 take row 2i, lanes 16-31 row 2i + 1; lane owns chunks cq, cq + 16
      {
        // all 32 rows, straight-line: rows past the end of the data are zero in the stage and
        // in the e/x slot, so they add exact zeros.  Lanes whose chunk is past nch read a valid
        // chunk; their sums land in columns that are never read.
        const ulonglong2* exv = reinterpret_cast<const ulonglong2*>(ex);
        auto rows16 = [&](int q, auto cc) {
          constexpr int c = decltype(cc)::value;
#pragma unroll 1
          for (int j0 = 0; j0 < kRowsA / 2; j0 += 4)
#pragma unroll
          for (int j1 = 0; j1 < 4; ++j1) {
            const int j = j0 + j1;
            const int tt = hrow + 2 * j;
            const ulonglong2 v0 = exv[3 * tt], v1 = exv[3 * tt + 1], v2 = exv[3 * tt + 2];
            f2x H[kP], L[kP];
            load_chunk2<ST>(ph, pl, P.rs, tt, q, H, L);
#pragma unroll
            for (int i = 0; i < kP; ++i) {
              if (j1 & 1) {
                acc2_fma_basis<ST>(Sacc2[c][i], H[i], L[i], v0.x, v1.x, v0.y);  // e
                acc2_fma_basis<ST>(Yacc2[c][i], H[i], L[i], v1.y, v2.y, v2.x);  // x
              } else {
                acc2_fma_basis<ST>(Sacc[c][i], H[i], L[i], v0.x, v1.x, v0.y);
                acc2_fma_basis<ST>(Yacc[c][i], H[i], L[i], v1.y, v2.y, v2.x);
              }
            }
          }
        };
        rows16(cq < P.nch ? cq : (P.nch > 0 ? P.nch - 1 : 0), std::integral_constant<int, 0>{});
        if constexpr (kCS > 1) {
          if (P.nch > 16) rows16(cq + 16 < P.nch ? cq + 16 : P.nch - 1, std::integral_constant<int, kCS - 1>{});
        }
      }
      // this warp is the stage's last reader: refill it with tile k + ns
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0 && k + ns < my_tiles && !abort_flag) {
        P.issue((int)(tbase + k + ns), s);
        *reinterpret_cast<volatile int*>(&last_issued[s]) = k + ns;
      }
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) {
    // give the copies still in flight (the last tile issued into each stage) up to 0.5 s
    const uint64_t t0 = global_ns();
    for (int st_ = 0; st_ < ns; ++st_) {
      const int k = last_issued[st_];
      if (k < 0) continue;
      while (!mbar_try_wait(&P.full[st_], (uint32_t)((k / ns) & 1)))
        if (global_ns() - t0 > 500000000ull) break;
    }
  }
  __syncthreads();

  // ---- per-CTA partials
  const int stride = 2 * ws.cap + 3;
  float2* mypart = ws.part + (size_t)blk * stride;
  // column sums: lanes cq and cq + 16 of a warp hold the same columns (even / odd rows)
  Acc* cacc = reinterpret_cast<Acc*>(smem);  // [warp][S | Y][kCo], in the idle stage memory
  {
#pragma unroll
    for (int c = 0; c < kCS; ++c)
#pragma unroll
      for (int i = 0; i < kP; ++i) {
        Acc s0, s1, y0, y1, u0, u1;
        acc2_split(Sacc[c][i], s0, s1);
        acc2_split(Sacc2[c][i], u0, u1);
        acc_add(s0, u0.h, u0.l);
        acc_add(s1, u1.h, u1.l);
        acc2_split(Yacc[c][i], y0, y1);
        acc2_split(Yacc2[c][i], u0, u1);
        acc_add(y0, u0.h, u0.l);
        acc_add(y1, u1.h, u1.l);
        acc_add(s0, __shfl_xor_sync(0xffffffffu, s0.h, 16), __shfl_xor_sync(0xffffffffu, s0.l, 16));
        acc_add(s1, __shfl_xor_sync(0xffffffffu, s1.h, 16), __shfl_xor_sync(0xffffffffu, s1.l, 16));
        acc_add(y0, __shfl_xor_sync(0xffffffffu, y0.h, 16), __shfl_xor_sync(0xffffffffu, y0.l, 16));
        acc_add(y1, __shfl_xor_sync(0xffffffffu, y1.h, 16), __shfl_xor_sync(0xffffffffu, y1.l, 16));
        const int c0 = (cq + 16 * c) * kE + 2 * i;
        if (hrow == 0 && c0 < kCo) {
          Acc* w = cacc + (size_t)warp * 2 * kCo;
          w[c0] = s0;
          w[c0 + 1] = s1;
          w[kCo + c0] = y0;
          w[kCo + c0 + 1] = y1;
        }
      }
  }
  // scalar sums live in the row lanes of every warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    acc_add(eta, __shfl_xor_sync(0xffffffffu, eta.h, o), __shfl_xor_sync(0xffffffffu, eta.l, o));
    acc_add(exa, __shfl_xor_sync(0xffffffffu, exa.h, o), __shfl_xor_sync(0xffffffffu, exa.l, o));
    acc_add(xi, __shfl_xor_sync(0xffffffffu, xi.h, o), __shfl_xor_sync(0xffffffffu, xi.l, o));
  }
  __shared__ Acc wsc[kThreadsA / 32][3];
  if (lane == 0) {
    wsc[warp][0] = eta;
    wsc[warp][1] = exa;
    wsc[warp][2] = xi;
  }
  __syncthreads();
  if (tid < r0) {
    Acc sS = acc_zero(), sY = acc_zero();
    for (int w = 0; w < kWarpsA; ++w) {
      const Acc a1 = cacc[(size_t)w * 2 * kCo + tid], a2 = cacc[(size_t)w * 2 * kCo + kCo + tid];
      acc_add(sS, a1.h, a1.l);
      acc_add(sY, a2.h, a2.l);
    }
    sS = acc_norm(sS);
    sY = acc_norm(sY);
    mypart[tid] = make_float2(sS.h, sS.l);
    mypart[r0 + tid] = make_float2(sY.h, sY.l);
  }
  if (tid < 3) {
    Acc a = acc_zero();
    for (int w = 0; w < kThreadsA / 32; ++w) acc_add(a, wsc[w][tid].h, wsc[w][tid].l);
    a = acc_norm(a);
    mypart[2 * r0 + tid] = make_float2(a.h, a.l);
  }

  // ---- the CTA that finishes last adds all partials in block order (a sharded run leaves
  // that to k_fold_a, after every shard's launch)
  __threadfence();
  if (!fold) return;
  __shared__ unsigned ticket;
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&ctl->ticket_a, 1u);
  __syncthreads();
  if (ticket != cp.g - 1) return;
  __threadfence();
  fold_pass_a(ws, st, r0);
}

template <int ST>
__global__ void __launch_bounds__(kThreadsA, 1) k_pass_a(const __grid_constant__ Ws ws, int cta0, int fold) {
  pass_a_body<ST>(ws, cta_single(), cta0, fold);
}
template <int ST>
__global__ void __launch_bounds__(kThreadsA, 1) k_pass_a_sel(const __grid_constant__ Ws ws, int sel) {
  pass_a_body<ST>(ws, cta_single(), 0, 1, sel);
}
template <int ST>
__global__ void __launch_bounds__(kThreadsA, 1) k_pass_a_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  pass_a_body<ST>(*t.ws[i], batch_pos(t, i), 0, 1);
}


// the fold of pass A after a sharded run (one CTA): the exchange of per-block partials of a
// row-sharded run, added in block order exactly as the unsharded pass adds them
__global__ void __launch_bounds__(kThreadsA) k_fold_a(Ws ws) {
  pdl_wait();
  const StateBuf st = ws.st[ws.ctl->cur];
  fold_pass_a(ws, st, st.hdr->r0);
}

// ---------------------------------------------------------------------------------------
// pass B: compaction L0 <- [L0, j0] QB (with the update's own new column j0 formed from
// its residual), or -- FLUSH -- writing a pending column before a predict or check.
// ---------------------------------------------------------------------------------------
constexpr int kStagesB = 2;
constexpr int kRowLanes = 8;
constexpr int kThreadsB = 512;

template <int ST, bool FLUSH>
__device__ __forceinline__ void pass_b_body(const Ws& ws, CtaPos cp) {
  pdl_wait();
  using T = Traits<ST>;
  constexpr int epcC = (ST == ST_BF16) ? 8 : 4;  // basis columns per 16-byte chunk
  extern __shared__ __align__(1024) unsigned char smem[];
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const StateBuf st = ws.st[ctl->cur];
  int r0, append, rnew;  // r0: columns of L0 that exist; append: form column r0 too
  float ih = 0.f, il = 0.f;
  const float2* sco;     // coefficients of the new column: (e - L0[:, :r0] s) / rho0
  bool work;
  if constexpr (FLUSH) {
    work = st.hdr->pend != 0;
    r0 = st.hdr->r0 - 1;
    append = 1;
    rnew = 0;
    ih = st.hdr->pinv.x;
    il = st.hdr->pinv.y;
    sco = st.ps;
  } else {
    work = ctl->mode == PB_COMPACT;
    append = ctl->append;
    r0 = ctl->r0e - append;
    rnew = ctl->rnew;
    if (append) {
      const dd inv = dd_from_double(1.0 / ctl->rho0);
      ih = inv.h;
      il = inv.l;
    }
    sco = ws.sm.red;
  }
  const int G = cp.g;
  if (work) {
    TilePipe<ST> P;
    P.setup(ws, r0, kStagesB);
    P.g[0] = (const unsigned char*)ws.ebuf;
    P.vb[0] = 8;
    P.base = smem;
    unsigned char* sp = smem + (size_t)kStagesB * P.stage_sz;
    P.bars = reinterpret_cast<uint64_t*>(sp);
    sp += 8 * kStagesB;
    float* coh = reinterpret_cast<float*>(sp);
    float* col = coh + (kMaxCap + 8);
    float* jh = col + (kMaxCap + 8);
    float* jl = jh + kTile;
    float* qbh = jl + kTile;                  // [(box columns + 1)][rnew padded] hi
    float* qbl = qbh + (kMaxCap + 9) * kMaxR;  // lo
    float* qbn = qbl + (kMaxCap + 9) * kMaxR;  // -hi

    const int epc = (ST == ST_BF16) ? 8 : 4;
    const int kpad = P.nch * epc;
    for (int k = tid; k < kMaxCap + 8; k += kThreadsB) {
      float h = 0.f, l = 0.f;
      if (k < r0 && append && k < kpad) {
        h = sco[k].x;
        l = sco[k].y;
      }
      coh[k] = h;
      col[k] = l;
    }
    const int rnp = (rnew + 7) & ~7;  // output columns padded to whole groups of 8 (zeros)
    const int kch = P.nch * epc;      // basis columns covered by the box (zero rows of QB beyond r0)
    if (!FLUSH) {
      for (int idx = tid; idx < (kch + 1) * rnp; idx += kThreadsB) {
        const int k = idx / rnp, j = idx % rnp;
        // row kch holds the coefficients of the new column j0 (QB row r0)
        const int kk = k < kch ? k : r0;
        float2 q = make_float2(0.f, 0.f);
        if (j < rnew && ((k < kch && k < r0) || (k == kch && append)))
          q = ws.sm.QB[(size_t)j * (ws.cap + 1) + kk];
        qbh[k * rnp + j] = q.x;
        qbl[k * rnp + j] = q.y;
        qbn[k * rnp + j] = -q.x;
      }
    }
    if (tid == 0) {
      for (int s = 0; s < kStagesB; ++s) mbar_init(&P.bars[s], 1);
      mbar_fence_init();
    }
    __syncthreads();

    const int64_t ntiles = (ws.n + kTile - 1) / kTile;
    const int my_tiles = (int)((ntiles - cp.b + G - 1) / G);
    if (tid == 0) {
      for (int li = 0; li < min(my_tiles, kStagesB); ++li) P.issue(cp.b + li * G, li);
    }
    const int t = tid >> 3, sub = tid & (kRowLanes - 1);

    for (int li = 0; li < my_tiles; ++li) {
      const int s = li % kStagesB;
      const uint32_t par = (uint32_t)((li / kStagesB) & 1);
      const int tile = cp.b + li * G;
      const int64_t row0 = (int64_t)tile * kTile;
      const int rows = rows_in(ws.n, row0);
      const bool ok = mbar_wait(&P.bars[s], par, &ctl->status);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) mbar_drain(P.bars, kStagesB, li, my_tiles);
        __syncthreads();
        break;
      }
      if (append) {
        Acc d = row_dot_partial<ST, kRowLanes>(P, s, t, sub, coh, col);
        d = group8_sum(d);
        if (sub == 0) {
          // j0 = (e - L0 s) / rho0: the second Gram-Schmidt pass, applied to the stored e
          const float2 ev = reinterpret_cast<const float2*>(P.slot(s, 0))[t];
          Acc e = Acc{ev.x, ev.y};
          acc_add(e, -d.h, -d.l);
          e = acc_norm(e);
          Acc j = acc_zero();
          acc_fma(j, e.h, e.l, ih, il);
          j = acc_norm(j);
          float h = j.h, l = j.l;
          round_to_storage<ST>(h, l);
          jh[t] = h;
          jl[t] = l;
          if (FLUSH && t < rows) store_elem_global<ST>(ws, (size_t)(row0 + t) * ws.ldg + r0, h, l);
        }
        __syncthreads();
      }
      if (!FLUSH) {
        // out[t][j] = sum_k L0[t][k] QB[k][j] + j0_t QB[r0][j]; a thread takes one row and
        // 8 adjacent output columns, the lanes of a warp consecutive rows
        const unsigned char* ph = P.plane_h(s);
        const unsigned char* pl = P.plane_l(s);
        const int ngrp = rnp >> 3;
        // results go through shared memory so that whole rows of the new L0 are written at
        // once: the stage just read holds them, [t][rnew] hi then (double-float) lo, which
        // fits because a stage holds kTile rows of at least cap elements per plane
        float* oh = reinterpret_cast<float*>(P.plane_h(s));
        float* ol = oh + kTile * rnew;
        float2 res[4][2];
        const bool mine = tid < kTile * ngrp;
        const int tt = tid % kTile, j0c = (tid / kTile) * 8;
        if (mine) {
          Acc2 acc[1][4];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[0][c] = acc2_zero();
          tile_dot8<ST, 1>(ph, pl, P.rs, tt, P.nch, qbh, qbl, qbn, rnp, j0c, acc);
          if (append) {
            const float xh[1] = {jh[tt]}, xl[1] = {jl[tt]};
            tile_dot8_term<ST, 1>(xh, xl, qbh, qbl, qbn, kch * rnp + j0c, acc);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            Acc a[2];
            acc2_split(acc[0][c], a[0], a[1]);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const Acc v = acc_norm(a[e]);
              res[c][e] = make_float2(v.h, v.l);
            }
          }
        }
        if constexpr (ST == ST_BF16) {
          if (mine && tt < rows)
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int col = j0c + 2 * c + e;
                if (col < rnew) store_elem_global<ST>(ws, (size_t)(row0 + tt) * ws.ldg + col, res[c][e].x, 0.f);
              }
        } else {
          __syncthreads();  // every thread is done reading the stage
          if (mine)
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int col = j0c + 2 * c + e;
                if (col < rnew) {
                  oh[tt * rnew + col] = res[c][e].x;
                  if constexpr (ST == ST_DD) ol[tt * rnew + col] = res[c][e].y;
                }
              }
          __syncthreads();
          for (int idx = tid; idx < rows * rnew; idx += kThreadsB) {
            const int t = idx / rnew, col = idx - t * rnew;
            store_elem_global<ST>(ws, (size_t)(row0 + t) * ws.ldg + col, oh[idx], ST == ST_DD ? ol[idx] : 0.f);
          }
        }
      }
      // the stage is refilled by TMA (async proxy) after generic reads and writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0 && li + kStagesB < my_tiles) P.issue(cp.b + (li + kStagesB) * G, s);
    }
  }
  if constexpr (FLUSH) {
    __shared__ unsigned ticket;
    __threadfence();
    __syncthreads();
    if (tid == 0) ticket = atomicAdd(&ctl->ticket_b, 1u);
    __syncthreads();
    if (ticket != (unsigned)(G - 1)) return;
    if (tid == 0) {
      st.hdr->pend = 0;
      ctl->ticket_b = 0u;
    }
  }
}

template <int ST, bool FLUSH>
__global__ void __launch_bounds__(kThreadsB) k_pass_b(const __grid_constant__ Ws ws) {
  pass_b_body<ST, FLUSH>(ws, cta_single());
}
template <int ST, bool FLUSH>
__global__ void __launch_bounds__(kThreadsB) k_pass_b_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  pass_b_body<ST, FLUSH>(*t.ws[i], batch_pos(t, i));
}


// ---------------------------------------------------------------------------------------
// rollout: X[:, j] = L0 coef[:, j] (j < kcols), written in the snapshot type
// check:   same with kcols = 1 against x_fom, reducing instead of storing
// ---------------------------------------------------------------------------------------
constexpr int kStagesR = 2;

// fold of the check's per-block partials (one thread): ||L c - x||^2 and ||x||^2
__device__ void fold_check(const Ws& ws) {
  Ctl* ctl = ws.ctl;
  Acc a = acc_zero(), b = acc_zero();
  for (int blk = 0; blk < ws.gridA; ++blk) {
    const float2 f1 = __ldcg(ws.part + 2 * blk), f2 = __ldcg(ws.part + 2 * blk + 1);
    acc_add(a, f1.x, f1.y);
    acc_add(b, f2.x, f2.y);
  }
  a = acc_norm(a);
  b = acc_norm(b);
  ctl->check_num = make_float2(a.h, a.l);
  ctl->check_den = make_float2(b.h, b.l);
  ws.out2[0] = make_float2(a.h, a.l);
  ws.out2[1] = make_float2(b.h, b.l);
  ctl->ticket_r = 0u;
}

__global__ void __launch_bounds__(32) k_fold_check(Ws ws) {
  pdl_wait();
  if (threadIdx.x == 0) fold_check(ws);
}

// Rollout (CHECK = false): out[:, j] = L0 coef[:, j] for j < kcols.  Check (CHECK = true):
// the partial sums of ||L0 coef[:, 0] - x||^2 and ||x||^2 over this CTA's row block, added
// in block order by the CTA that finishes last when `fold` is set.  Logical CTA cta0 +
// blockIdx.x works on that row block.
template <int ST, bool CHECK>
__global__ void __launch_bounds__(kThreads) k_rollout(Ws ws, int kcols, void* out, int64_t ld, int cta0, int fold) {
  pdl_wait();
  using T = Traits<ST>;
  using snap_t = typename T::snap_t;
  extern __shared__ __align__(1024) unsigned char smem[];
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur];
  const int r0 = st.hdr->r0;

  TilePipe<ST> P;
  P.setup(ws, r0, kStagesR);
  if (CHECK) {
    P.g[0] = (const unsigned char*)ws.xbuf;
    P.vb[0] = T::vsz;
  }
  P.base = smem;
  unsigned char* p = smem + (size_t)kStagesR * P.stage_sz;
  P.bars = reinterpret_cast<uint64_t*>(p);
  p += 8 * kStagesR;
  // coefficients, float-float, layout [k][ldc] in three planes (hi, lo, -hi); rows padded to
  // whole chunks with zeros.  From 3 columns on, a thread computes 2 rows x 8 columns and
  // the rows are padded to groups of 8 columns (ldc); below that, ldc = kcols.
  const int epc = (ST == ST_BF16) ? 8 : 4;
  const int kpad = P.nch * epc;
  const bool tiled = !CHECK && kcols >= 3;
  const int ldc = tiled ? (kcols + 7) & ~7 : kcols;
  float* cfh = reinterpret_cast<float*>(p);
  float* cfl = cfh + (kMaxCap + 8) * kRollK;
  float* cfn = cfl + (kMaxCap + 8) * kRollK;
  Acc* part = reinterpret_cast<Acc*>(cfn + (kMaxCap + 8) * kRollK);  // [4][kTile]

  for (int idx = tid; idx < (kMaxCap + 8) * ldc; idx += kThreads) {
    const int k = idx / ldc, j = idx % ldc;
    float h = 0.f, l = 0.f;
    if (k < r0 && j < kcols) {
      const float2 q = ws.sm.coef[(size_t)j * (ws.cap + 1) + k];
      h = q.x;
      l = q.y;
    }
    if (k >= kpad) h = l = 0.f;
    cfh[idx] = h;
    cfl[idx] = l;
    cfn[idx] = -h;
  }
  if (tid == 0) {
    for (int s = 0; s < kStagesR; ++s) mbar_init(&P.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  const int blk = cta0 + blockIdx.x;
  int64_t tb0, tb1;
  block_tiles64(ws, blk, tb0, tb1);
  const int my_tiles = (int)(tb1 - tb0);
  if (tid == 0) {
    for (int li = 0; li < min(my_tiles, kStagesR); ++li) P.issue((int)(tb0 + li), li);
  }
  // work split: items (t, j); with fewer than 4 columns each dot is split in nsub parts
  const int nsub = kcols == 1 ? 4 : (kcols == 2 ? 2 : 1);  // nsub * kTile * kcols <= 4 * kTile when > 1
  Acc num = acc_zero(), den = acc_zero();

  for (int li = 0; li < my_tiles; ++li) {
    const int s = li % kStagesR;
    const uint32_t par = (uint32_t)((li / kStagesR) & 1);
    const int64_t row0 = (tb0 + li) * kTile;
    const int rows = rows_in(ws.n, row0);
    const bool ok = mbar_wait(&P.bars[s], par, &ctl->status);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) mbar_drain(P.bars, kStagesR, li, my_tiles);
      __syncthreads();
      break;
    }
    {
      const unsigned char* ph = P.plane_h(s);
      const unsigned char* pl = P.plane_l(s);
      if (tiled) {
        // lanes take rows lane and lane + 32 of the tile, a warp one group of 8 columns
        snap_t* o = reinterpret_cast<snap_t*>(out);
        for (int it = tid; it < 32 * (ldc >> 3); it += kThreads) {
          const int t0 = it & 31, j0 = (it >> 5) * 8;
          Acc2 acc[2][4];
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = acc2_zero();
          tile_dot8<ST, 2>(ph, pl, P.rs, t0, P.nch, cfh, cfl, cfn, ldc, j0, acc);
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int tt = t0 + 32 * r;
            if (tt >= rows) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              Acc a[2];
              acc2_split(acc[r][c], a[0], a[1]);
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int j = j0 + 2 * c + e;
                if (j >= kcols) continue;
                const Acc v = acc_norm(a[e]);
                if constexpr (ST == ST_DD)
                  o[(size_t)j * ld + row0 + tt] = join_double(v.h, v.l);
                else
                  o[(size_t)j * ld + row0 + tt] = v.h + v.l;
              }
            }
          }
        }
      }
      const int items = tiled ? 0 : kTile * kcols * nsub;
      for (int it = tid; it < items; it += kThreads) {
        const int tt = it % kTile;
        const int rest = it / kTile;
        const int j = rest % kcols, sb = rest / kcols;
        Acc acc = acc_zero();
        for (int q = sb; q < P.nch; q += nsub) {
          float h[8], l[8];
          const int e = load_chunk<ST>(ph, pl, P.rs, tt, q, h, l);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (i < e) acc_fma(acc, h[i], l[i], cfh[(q * e + i) * kcols + j], cfl[(q * e + i) * kcols + j]);
        }
        if (nsub == 1) {
          if (tt < rows) {
            acc = acc_norm(acc);
            if constexpr (CHECK) {
              float fh, fl;
              load_snap(reinterpret_cast<const typename T::stored_t*>(P.slot(s, 0)), tt, fh, fl);
              Acc d = acc;
              acc_add(d, -fh, -fl);
              d = acc_norm(d);
              acc_fma(num, d.h, d.l, d.h, d.l);
              acc_fma(den, fh, fl, fh, fl);
            } else {
              snap_t* o = reinterpret_cast<snap_t*>(out);
              if constexpr (ST == ST_DD)
                o[(size_t)j * ld + row0 + tt] = join_double(acc.h, acc.l);
              else
                o[(size_t)j * ld + row0 + tt] = acc.h + acc.l;
            }
          }
        } else {
          part[sb * kTile * kcols + (it % (kTile * kcols))] = acc;  // nsub*kTile*kcols == 256
        }
      }
      if (nsub > 1) {
        __syncthreads();
        for (int it = tid; it < kTile * kcols; it += kThreads) {
          const int tt = it % kTile, j = it / kTile;
          Acc acc = part[it];
          for (int sb = 1; sb < nsub; ++sb) acc_add(acc, part[sb * kTile * kcols + it].h, part[sb * kTile * kcols + it].l);
          acc = acc_norm(acc);
          if (tt < rows) {
            if constexpr (CHECK) {
              float fh, fl;
              load_snap(reinterpret_cast<const typename T::stored_t*>(P.slot(s, 0)), tt, fh, fl);
              Acc d = acc;
              acc_add(d, -fh, -fl);
              d = acc_norm(d);
              acc_fma(num, d.h, d.l, d.h, d.l);
              acc_fma(den, fh, fl, fh, fl);
            } else {
              snap_t* o = reinterpret_cast<snap_t*>(out);
              if constexpr (ST == ST_DD)
                o[(size_t)j * ld + row0 + tt] = join_double(acc.h, acc.l);
              else
                o[(size_t)j * ld + row0 + tt] = acc.h + acc.l;
            }
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && li + kStagesR < my_tiles) P.issue((int)(tb0 + li + kStagesR), s);
  }

  if constexpr (CHECK) {
    // block reduce (num, den) then last CTA sums in CTA order
    num = warp_sum_acc(num);
    den = warp_sum_acc(den);
    __shared__ Acc wred[2][kThreads / 32];
    if ((tid & 31) == 0) {
      wred[0][tid >> 5] = num;
      wred[1][tid >> 5] = den;
    }
    __syncthreads();
    if (tid == 0) {
      Acc a = acc_zero(), b = acc_zero();
      for (int w = 0; w < kThreads / 32; ++w) {
        acc_add(a, wred[0][w].h, wred[0][w].l);
        acc_add(b, wred[1][w].h, wred[1][w].l);
      }
      a = acc_norm(a);
      b = acc_norm(b);
      ws.part[2 * blk] = make_float2(a.h, a.l);
      ws.part[2 * blk + 1] = make_float2(b.h, b.l);
    }
    __threadfence();
    if (!fold) return;
    __shared__ unsigned ticket;
    __syncthreads();
    if (tid == 0) ticket = atomicAdd(&ctl->ticket_r, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    if (tid == 0) {
      __threadfence();
      fold_check(ws);
    }
  }
}

// ---------------------------------------------------------------------------------------
// first snapshot: ||u^0||^2 into the committed state
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double stored_to_double(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double stored_to_double(float v) { return (double)v; }

// fold of the first snapshot's per-block sums of squares (one thread)
__device__ void fold_first(const Ws& ws) {
  Ctl* ctl = ws.ctl;
  double tot = 0.0;
  for (int b = 0; b < ws.gridA; ++b) tot += __ldcg(reinterpret_cast<const double*>(ws.part) + b);
  if (!isfinite(tot)) atomicOr(&ctl->status, DEV_NONFINITE);
  ws.st[ctl->cur].hdr->cn2 = f2_of(dd_from_double(tot));
  ctl->ticket_a = 0u;
}

__global__ void __launch_bounds__(32) k_fold_first(Ws ws) {
  pdl_wait();
  if (threadIdx.x == 0) fold_first(ws);
}

// ||u^0||^2 over this CTA's row block (logical CTA cta0 + blockIdx.x), in FP64: N FMAs once
// per stream, negligible
template <typename stored_t>
__global__ void __launch_bounds__(kThreads) k_first(Ws ws, int cta0, int fold) {
  pdl_wait();
  Ctl* ctl = ws.ctl;
  const stored_t* c = reinterpret_cast<const stored_t*>(ws.cbuf[ctl->cur_c]);
  const int blk = cta0 + blockIdx.x;
  int64_t t0, t1;
  block_tiles64(ws, blk, t0, t1);
  const int64_t i1 = t1 * kTile < ws.n ? t1 * kTile : ws.n;
  double acc = 0.0;
  for (int64_t i = t0 * kTile + threadIdx.x; i < i1; i += kThreads) {
    const double v = stored_to_double(c[i]);
    acc = fma(v, v, acc);
  }
  acc = warp_sum_d(acc);
  __shared__ double wsum[kThreads / 32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) b += wsum[w];
    reinterpret_cast<double*>(ws.part)[blk] = b;
  }
  __threadfence();
  if (!fold) return;
  __shared__ unsigned ticket;
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket_a, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1 || threadIdx.x != 0) return;
  __threadfence();
  fold_first(ws);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
static int stage_of(int prec, int cap) {
  return prec == ST_DD ? stage_bytes<ST_DD>(cap) : prec == ST_F32 ? stage_bytes<ST_F32>(cap) : stage_bytes<ST_BF16>(cap);
}
static int stage_a_of(int prec, int cap) {
  return prec == ST_DD ? stage_bytes_a<ST_DD>(cap) : prec == ST_F32 ? stage_bytes_a<ST_F32>(cap) : stage_bytes_a<ST_BF16>(cap);
}
// as many stages as fit in the dynamic shared memory a CTA may have (a deeper ring keeps
// more HBM reads in flight; a stage is held until its compute warp is done with it)
int stages_a(int prec, int cap) {
  const int sz = stage_a_of(prec, cap);
  int n = (kSmemBudgetA - 2048 - smem_a_fixed()) / sz;
  if (n > kMaxStagesA) n = kMaxStagesA;
  return n < 2 ? 2 : n;
}
static int smem_a(int prec, int cap) {
  const int ns = stages_a(prec, cap), sz = stage_a_of(prec, cap);
  const size_t region = prec == ST_DD    ? pass_a_region<ST_DD>(sz, ns)
                        : prec == ST_F32 ? pass_a_region<ST_F32>(sz, ns)
                                         : pass_a_region<ST_BF16>(sz, ns);
  return (int)region + smem_a_fixed();
}
static int smem_b(int prec, int cap) {
  return kStagesB * stage_of(prec, cap) + 8 * kStagesB + 2 * (kMaxCap + 8) * 4 + 2 * kTile * 4 +
         3 * (kMaxCap + 9) * kMaxR * 4;
}
static int smem_r(int prec, int cap) {
  const int sb = prec == ST_DD ? stage_bytes<ST_DD>(cap) : prec == ST_F32 ? stage_bytes<ST_F32>(cap) : stage_bytes<ST_BF16>(cap);
  return kStagesR * sb + 8 * kStagesR + 3 * (kMaxCap + 8) * kRollK * 4 + 4 * kTile * 8;
}

int tall_smem_bytes(int prec) { return smem_a(prec, kMaxCap); }

template <typename K>
static cudaError_t prep_attr(K kern, int bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Largest dynamic shared memory a kernel of this precision needs over every cap a handle
// can have (pass A's ring depth varies with the row width, so the largest cap is not
// always the largest request)
template <typename F>
static int max_over_caps(F f) {
  int m = 0;
  for (int cap = 1; cap <= kMaxCap; ++cap) m = f(cap) > m ? f(cap) : m;
  return m;
}

// Raise the dynamic shared-memory limit of every tall kernel once (not inside launches,
// which may be captured into a graph).  The limit is a property of the kernel, shared by
// every handle in the process, so it is set for every cap a handle can have.
cudaError_t prepare_tall(const Ws& ws) {
  const int p = ws.prec;
  const int sa = max_over_caps([p](int c) { return smem_a(p, c); });
  const int sb = max_over_caps([p](int c) { return smem_b(p, c); });
  const int sr = max_over_caps([p](int c) { return smem_r(p, c); });
  cudaError_t e = cudaSuccess;
  switch (p) {
    case ST_DD:
      if ((e = prep_attr(k_pass_a<ST_DD>, sa))) return e;
      if ((e = prep_attr(k_pass_a_sel<ST_DD>, sa))) return e;
      if ((e = prep_attr(k_pass_b<ST_DD, false>, sb))) return e;
      if ((e = prep_attr(k_pass_b<ST_DD, true>, sb))) return e;
      if ((e = prep_attr(k_rollout<ST_DD, false>, sr))) return e;
      return prep_attr(k_rollout<ST_DD, true>, sr);
    case ST_F32:
      if ((e = prep_attr(k_pass_a<ST_F32>, sa))) return e;
      if ((e = prep_attr(k_pass_a_sel<ST_F32>, sa))) return e;
      if ((e = prep_attr(k_pass_b<ST_F32, false>, sb))) return e;
      if ((e = prep_attr(k_pass_b<ST_F32, true>, sb))) return e;
      if ((e = prep_attr(k_rollout<ST_F32, false>, sr))) return e;
      return prep_attr(k_rollout<ST_F32, true>, sr);
    default:
      if ((e = prep_attr(k_pass_a<ST_BF16>, sa))) return e;
      if ((e = prep_attr(k_pass_a_sel<ST_BF16>, sa))) return e;
      if ((e = prep_attr(k_pass_b<ST_BF16, false>, sb))) return e;
      if ((e = prep_attr(k_pass_b<ST_BF16, true>, sb))) return e;
      if ((e = prep_attr(k_rollout<ST_BF16, false>, sr))) return e;
      return prep_attr(k_rollout<ST_BF16, true>, sr);
  }
}

// shard g of a run split over ws.shards row shards: row blocks [first, first + count)
static void shard_blocks(const Ws& ws, int g, int& first, int& count) {
  first = (int)((int64_t)g * ws.gridA / ws.shards);
  count = (int)((int64_t)(g + 1) * ws.gridA / ws.shards) - first;
}

// One launch over every row block (its last CTA folds), or one launch per row shard and
// then the fold: the sharded run's exchange of per-block partials
template <typename K, typename F>
static cudaError_t launch_blocks(K kern, F fold_kern, int threads, int fold_threads, int smem, const Ws& ws,
                                 cudaStream_t s) {
  if (ws.shards <= 1) return launch_dependent(kern, ws.gridA, threads, smem, s, ws, 0, 1);
  for (int g = 0; g < ws.shards; ++g) {
    int first, count;
    shard_blocks(ws, g, first, count);
    const cudaError_t e = launch_dependent(kern, count, threads, smem, s, ws, first, 0);
    if (e != cudaSuccess) return e;
  }
  return launch_dependent(fold_kern, 1, fold_threads, 0, s, ws);
}

cudaError_t launch_pass_a(const Ws& ws, cudaStream_t s) {
  const int sm = smem_a(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      return launch_blocks(k_pass_a<ST_DD>, &k_fold_a, kThreadsA, kThreadsA, sm, ws, s);
    case ST_F32:
      return launch_blocks(k_pass_a<ST_F32>, &k_fold_a, kThreadsA, kThreadsA, sm, ws, s);
    default:
      return launch_blocks(k_pass_a<ST_BF16>, &k_fold_a, kThreadsA, kThreadsA, sm, ws, s);
  }
}

// pass A of a pipelined update (one launch, no row shards): see pass_a_body for sel
cudaError_t launch_pass_a_sel(const Ws& ws, int sel, cudaStream_t s) {
  const int sm = smem_a(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      return launch_dependent(k_pass_a_sel<ST_DD>, ws.gridA, kThreadsA, sm, s, ws, sel);
    case ST_F32:
      return launch_dependent(k_pass_a_sel<ST_F32>, ws.gridA, kThreadsA, sm, s, ws, sel);
    default:
      return launch_dependent(k_pass_a_sel<ST_BF16>, ws.gridA, kThreadsA, sm, s, ws, sel);
  }
}

int launches_per_reduction(const Ws& ws) { return ws.shards <= 1 ? 1 : ws.shards + 1; }

template <bool FLUSH>
static cudaError_t pass_b_launch(const Ws& ws, cudaStream_t s) {
  const int sm = smem_b(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      return launch_dependent(k_pass_b<ST_DD, FLUSH>, ws.gridA, kThreadsB, sm, s, ws);
    case ST_F32:
      return launch_dependent(k_pass_b<ST_F32, FLUSH>, ws.gridA, kThreadsB, sm, s, ws);
    default:
      return launch_dependent(k_pass_b<ST_BF16, FLUSH>, ws.gridA, kThreadsB, sm, s, ws);
  }
}

cudaError_t launch_pass_b(const Ws& ws, cudaStream_t s) { return pass_b_launch<false>(ws, s); }
cudaError_t launch_flush(const Ws& ws, cudaStream_t s) { return pass_b_launch<true>(ws, s); }

cudaError_t launch_first(const Ws& ws, cudaStream_t s) {
  if (ws.prec == ST_DD) return launch_blocks(k_first<float2>, &k_fold_first, kThreads, 32, 0, ws, s);
  return launch_blocks(k_first<float>, &k_fold_first, kThreads, 32, 0, ws, s);
}

// Copy a caller's double snapshot into the workspace as float pairs (all SMs; the only
// FP64 instructions a snapshot meets).
// one pair of elements per thread (16-byte loads and stores where the caller's array allows),
// one thread per pair over the whole array: the loads of a launch are all in flight at once
__global__ void __launch_bounds__(kThreads) k_ingest_dd(const double* __restrict__ src, float2* __restrict__ dst,
                                                        int64_t n) {
  pdl_wait();
  const int64_t i = 2 * ((int64_t)blockIdx.x * kThreads + threadIdx.x);
  if (i >= n) return;
  const bool vec = i + 1 < n && (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
  double v0, v1 = 0.0;
  if (vec) {
    const double2 v = *reinterpret_cast<const double2*>(src + i);
    v0 = v.x;
    v1 = v.y;
  } else {
    v0 = src[i];
    if (i + 1 < n) v1 = src[i + 1];
  }
  float h0, l0, h1, l1;
  split_double(v0, h0, l0);
  split_double(v1, h1, l1);
  // dst is a workspace slot (256-byte aligned) and i is even
  if (i + 1 < n)
    *reinterpret_cast<float4*>(dst + i) = make_float4(h0, l0, h1, l1);
  else
    dst[i] = make_float2(h0, l0);
}

__global__ void __launch_bounds__(kThreads) k_ingest_f32(const float* __restrict__ src, float* __restrict__ dst,
                                                         int64_t n) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    dst[i] = src[i];
}

// the ingest of a batch: instance i's snapshot (n[i] elements) into its slot, one element
// pair per thread as in k_ingest_dd, pairs of all instances in one grid
template <bool DD>
__global__ void __launch_bounds__(kThreads) k_ingest_batch(const __grid_constant__ IngestTab t) {
  const int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x;  // global pair index
  if (q >= t.first[t.ninst]) return;
  int lo = 0, hi = t.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.first[mid] <= q)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int64_t n = t.n[lo], i = 2 * (q - t.first[lo]);
  if constexpr (DD) {
    const double* src = static_cast<const double*>(t.src[lo]);
    float2* dst = static_cast<float2*>(t.dst[lo]);
    const double v0 = src[i], v1 = i + 1 < n ? src[i + 1] : 0.0;
    float h0, l0, h1, l1;
    split_double(v0, h0, l0);
    split_double(v1, h1, l1);
    dst[i] = make_float2(h0, l0);
    if (i + 1 < n) dst[i + 1] = make_float2(h1, l1);
  } else {
    const float* src = static_cast<const float*>(t.src[lo]);
    float* dst = static_cast<float*>(t.dst[lo]);
    dst[i] = src[i];
    if (i + 1 < n) dst[i + 1] = src[i + 1];
  }
}

cudaError_t launch_ingest_batch(const IngestTab& t, int prec, cudaStream_t s) {
  const int64_t blocks = (t.first[t.ninst] + kThreads - 1) / kThreads;
  if (blocks == 0) return cudaSuccess;
  if (prec == ST_DD)
    k_ingest_batch<true><<<(unsigned)blocks, kThreads, 0, s>>>(t);
  else
    k_ingest_batch<false><<<(unsigned)blocks, kThreads, 0, s>>>(t);
  return cudaGetLastError();
}

int pass_a_smem(int prec, int cap) { return smem_a(prec, cap); }
int pass_b_smem(int prec, int cap) { return smem_b(prec, cap); }

// one launch of pass A (or of the compaction's pass B) over the instances of a batch: the
// grid is every instance's row blocks, each CTA doing what it does in the instance's own
// launch (the last CTA of each instance folds its partials)
cudaError_t launch_pass_a_batch(const BatchTab& t, int prec, int smem, cudaStream_t s) {
  const int grid = t.first[t.ninst];
  switch (prec) {
    case ST_DD:
      return launch_dependent(k_pass_a_batch<ST_DD>, grid, kThreadsA, smem, s, t);
    case ST_F32:
      return launch_dependent(k_pass_a_batch<ST_F32>, grid, kThreadsA, smem, s, t);
    default:
      return launch_dependent(k_pass_a_batch<ST_BF16>, grid, kThreadsA, smem, s, t);
  }
}
cudaError_t launch_pass_b_batch(const BatchTab& t, int prec, int smem, cudaStream_t s) {
  const int grid = t.first[t.ninst];
  switch (prec) {
    case ST_DD:
      return launch_dependent(k_pass_b_batch<ST_DD, false>, grid, kThreadsB, smem, s, t);
    case ST_F32:
      return launch_dependent(k_pass_b_batch<ST_F32, false>, grid, kThreadsB, smem, s, t);
    default:
      return launch_dependent(k_pass_b_batch<ST_BF16, false>, grid, kThreadsB, smem, s, t);
  }
}

// the batch kernels take the largest shared memory any instance asks for
cudaError_t prepare_tall_batch() {
  const int big = kSmemBudget;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* k) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  };
  set((const void*)k_pass_a_batch<ST_DD>);
  set((const void*)k_pass_a_batch<ST_F32>);
  set((const void*)k_pass_a_batch<ST_BF16>);
  set((const void*)k_pass_b_batch<ST_DD, false>);
  set((const void*)k_pass_b_batch<ST_F32, false>);
  set((const void*)k_pass_b_batch<ST_BF16, false>);
  return e;
}

static int ingest_grid(const Ws& ws) {
  const int64_t blocks = (ws.n + kThreads - 1) / kThreads;
  return (int)(blocks < 4 * 152 ? blocks : 4 * 152);
}

cudaError_t launch_ingest(const Ws& ws, const void* src, void* dst, cudaStream_t s) {
  if (ws.prec == ST_DD)
    k_ingest_dd<<<(int)((ws.n + 2 * kThreads - 1) / (2 * kThreads)), kThreads, 0, s>>>(
        reinterpret_cast<const double*>(src), reinterpret_cast<float2*>(dst), ws.n);
  else
    k_ingest_f32<<<ingest_grid(ws), kThreads, 0, s>>>(reinterpret_cast<const float*>(src),
                                                      reinterpret_cast<float*>(dst), ws.n);
  return cudaGetLastError();
}

const void* ingest_kernel(int prec) {
  return prec == ST_DD ? reinterpret_cast<const void*>(&k_ingest_dd) : reinterpret_cast<const void*>(&k_ingest_f32);
}


// coef_mode unused here (coefficients are always read from ws.sm.coef)
cudaError_t launch_rollout(const Ws& ws, const double*, int kcols, void* out, int64_t ld, int, cudaStream_t s) {
  const int sm = smem_r(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      k_rollout<ST_DD, false><<<ws.gridA, kThreads, sm, s>>>(ws, kcols, out, ld, 0, 1);
      break;
    case ST_F32:
      k_rollout<ST_F32, false><<<ws.gridA, kThreads, sm, s>>>(ws, kcols, out, ld, 0, 1);
      break;
    default:
      k_rollout<ST_BF16, false><<<ws.gridA, kThreads, sm, s>>>(ws, kcols, out, ld, 0, 1);
  }
  return cudaGetLastError();
}

// the check: the kernel's grid, block and shared memory as the rollout's, with kcols = 1
template <int ST>
static cudaError_t check_blocks(const Ws& ws, int sm, cudaStream_t s) {
  if (ws.shards <= 1) {
    k_rollout<ST, true><<<ws.gridA, kThreads, sm, s>>>(ws, 1, nullptr, 0, 0, 1);
    return cudaGetLastError();
  }
  for (int g = 0; g < ws.shards; ++g) {
    int first, count;
    shard_blocks(ws, g, first, count);
    k_rollout<ST, true><<<count, kThreads, sm, s>>>(ws, 1, nullptr, 0, first, 0);
  }
  k_fold_check<<<1, 32, 0, s>>>(ws);
  return cudaGetLastError();
}

cudaError_t launch_check(const Ws& ws, cudaStream_t s) {
  const int sm = smem_r(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      return check_blocks<ST_DD>(ws, sm, s);
    case ST_F32:
      return check_blocks<ST_F32>(ws, sm, s);
    default:
      return check_blocks<ST_BF16>(ws, sm, s);
  }
}

}  // namespace odmd
