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
// kStages tiles in flight.  Shared rows are padded to an odd number of 16-byte chunks so
// that both the row-wise float4 reads (dot products along a row) and the column-wise
// reads (sums down a column) are free of bank conflicts.
//
// Reductions are deterministic: per-CTA partials in a fixed order, then the last CTA to
// finish (atomic ticket) sums them in CTA order.
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


// each stage: the basis rows (per plane, widest box) and two per-row slots of 8 bytes;
// every part starts on a 1024-byte boundary (TMA tile destinations need 128).
template <int ST>
__host__ __device__ inline int stage_bytes(int cap) {
  using T = Traits<ST>;
  const int rs_max = 16 * box_chunks(cap, T::esz);
  return kTile * rs_max * T::planes + 2 * kTile * 8;
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
// of the per-row slots, all completing on the stage's mbarrier.
template <int ST>
struct TilePipe {
  using T = Traits<ST>;
  unsigned char* base;
  uint64_t* bars;
  int stages, stage_sz, rs, nch, plane_off;
  int64_t n;
  const CUtensorMap* mh;    // map of the hi (or only) plane for the current box, or nullptr
  const CUtensorMap* ml;    // map of the lo plane (FP64 mode)
  const unsigned char* gc;  // first per-row slot (snapshot c, or the residual e), or nullptr
  const unsigned char* gx;  // second per-row slot (snapshot x), or nullptr
  int vc, vx;               // bytes per row of the two slots

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
    gc = gx = nullptr;
    vc = vx = 0;
  }
  __device__ unsigned char* plane_h(int s) const { return base + (size_t)s * stage_sz; }
  __device__ unsigned char* plane_l(int s) const { return plane_h(s) + plane_off; }
  __device__ unsigned char* snap_c(int s) const { return plane_h(s) + plane_off * T::planes; }
  __device__ unsigned char* snap_x(int s) const { return snap_c(s) + kTile * 8; }

  // Issue the copies of tile `tile` into stage `s` (called by one thread).
  __device__ void issue(int tile, int s) const {
    const int row0 = tile * kTile;
    const uint32_t bytes = (mh ? (uint32_t)(kTile * rs * T::planes) : 0u) + (gc ? kTile * vc : 0) +
                           (gx ? kTile * vx : 0);
    mbar_arrive_expect_tx(&bars[s], bytes);
    if (mh) {
      tma_load_2d(plane_h(s), mh, 0, row0, &bars[s]);
      if (T::planes == 2) tma_load_2d(plane_l(s), ml, 0, row0, &bars[s]);
    }
    if (gc) bulk_g2s(snap_c(s), gc + (size_t)row0 * vc, kTile * vc, &bars[s]);
    if (gx) bulk_g2s(snap_x(s), gx + (size_t)row0 * vx, kTile * vx, &bars[s]);
  }
};

// Phase 1: NSUB threads per row (thread = sub*64 + t) form partial row dots with the
// coefficient vector (float-float, zero-padded to whole chunks) held in shared memory.
template <int ST, int NSUB = 4>
__device__ __forceinline__ Acc row_dot_partial(const TilePipe<ST>& P, int s, int t, int sub, const float* coh,
                                               const float* col) {
  Acc acc = acc_zero();
  const unsigned char* ph = P.plane_h(s);
  const unsigned char* pl = P.plane_l(s);
  for (int q = sub; q < P.nch; q += NSUB) {
    float h[8], l[8];
    const int e = load_chunk<ST>(ph, pl, P.rs, t, q, h, l);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < e) acc_fma(acc, h[i], l[i], coh[q * e + i], col[q * e + i]);
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------------------
// pass A (512 threads: 8 per row in phase 1, 512 / r0 row groups in phase 2)
// ---------------------------------------------------------------------------------------
constexpr int kThreadsA = 512;
constexpr int kSubA = kThreadsA / kTile;
template <int ST>
__global__ void __launch_bounds__(kThreadsA) k_pass_a(Ws ws) {
  using T = Traits<ST>;
  using snap_t = typename T::snap_t;
  extern __shared__ __align__(1024) unsigned char smem[];
  Ctl* ctl = ws.ctl;
  const int cur = ctl->cur, curc = ctl->cur_c;
  const StateBuf st = ws.st[cur];
  const int r0 = st.hdr->r0;
  const int tid = threadIdx.x;

  TilePipe<ST> P;
  P.setup(ws, r0, kStages);
  P.gc = (const unsigned char*)ws.cbuf[curc];
  P.gx = (const unsigned char*)ws.cbuf[curc ^ 1];
  P.vc = T::vsz;
  P.vx = T::vsz;

  // shared layout: stages | bars | a (hi, lo: kMaxCap+8 each) | e,x (4 x kTile) | red (4 x kTile Acc)
  P.base = smem;
  unsigned char* p = smem + (size_t)kStages * P.stage_sz;
  P.bars = reinterpret_cast<uint64_t*>(p);
  p += 8 * kStages;
  float* coh = reinterpret_cast<float*>(p);
  float* col = coh + (kMaxCap + 8);
  float* eh = col + (kMaxCap + 8);
  float* el = eh + kTile;
  float* xh = el + kTile;
  float* xl = xh + kTile;
  Acc* part = reinterpret_cast<Acc*>(xl + kTile);       // [kSubA][kTile]
  Acc* colacc = part + kSubA * kTile;                    // [kThreadsA][2] group accumulators

  const int elems_per_chunk = (ST == ST_BF16) ? 8 : 4;
  for (int k = tid; k < kMaxCap + 8; k += kThreadsA) {
    float h = 0.f, l = 0.f;
    if (k < r0) {
      h = st.a[k].x;
      l = st.a[k].y;
    }
    if (k >= P.nch * elems_per_chunk) h = l = 0.f;
    coh[k] = h;
    col[k] = l;
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&P.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  const int64_t ntiles = (ws.n + kTile - 1) / kTile;
  const int G = gridDim.x;
  const int my_tiles = (int)((ntiles - blockIdx.x + G - 1) / G);
  if (tid == 0) {
    for (int li = 0; li < min(my_tiles, kStages); ++li) P.issue(blockIdx.x + li * G, li);
  }

  const int t = tid & 63, sub = tid >> 6;
  const int ncol = max(r0, 1);
  const int G2 = kThreadsA / ncol;
  const int kcol = tid % ncol, grp = tid / ncol;
  const bool col_active = (r0 > 0) && grp < G2;
  Acc S_acc = acc_zero(), Y_acc = acc_zero();
  Acc eta = acc_zero(), ex = acc_zero(), xi = acc_zero();

  for (int li = 0; li < my_tiles; ++li) {
    const int s = li % kStages;
    const uint32_t par = (uint32_t)((li / kStages) & 1);
    const int tile = blockIdx.x + li * G;
    const int64_t row0 = (int64_t)tile * kTile;
    const int rows = rows_in(ws.n, row0);
    const bool ok = mbar_wait(&P.bars[s], par, &ctl->status);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) mbar_drain(P.bars, kStages, li, my_tiles);
      __syncthreads();
      break;
    }
    {
      // phase 1: residual e_t = c_t - L0_t . a
      part[sub * kTile + t] = row_dot_partial<ST, kSubA>(P, s, t, sub, coh, col);
      __syncthreads();
      if (sub == 0) {
        float ch, cl, xh_, xl_;
        load_snap(reinterpret_cast<const typename T::stored_t*>(P.snap_c(s)), t, ch, cl);
        load_snap(reinterpret_cast<const typename T::stored_t*>(P.snap_x(s)), t, xh_, xl_);
        Acc d = part[t];
#pragma unroll
        for (int q = 1; q < kSubA; ++q) acc_add(d, part[q * kTile + t].h, part[q * kTile + t].l);
        Acc e = Acc{ch, cl};
        acc_add(e, -d.h, -d.l);
        e = acc_norm(e);
        if (t >= rows) {
          e = acc_zero();
          xh_ = xl_ = 0.f;
        } else {
          ws.ebuf[row0 + t] = make_float2(e.h, e.l);  // kept for the second Gram-Schmidt pass
        }
        eh[t] = e.h;
        el[t] = e.l;
        xh[t] = xh_;
        xl[t] = xl_;
        acc_fma(eta, e.h, e.l, e.h, e.l);
        acc_fma(ex, e.h, e.l, xh_, xl_);
        acc_fma(xi, xh_, xl_, xh_, xl_);
      }
      __syncthreads();
      // phase 2: column sums s_k += L_tk e_t, y_k += L_tk x_t
      if (col_active) {
        const unsigned char* ph = P.plane_h(s);
        const unsigned char* pl = P.plane_l(s);
        for (int tt = grp; tt < rows; tt += G2) {
          float h, l;
          load_elem<ST>(ph, pl, P.rs, tt, kcol, h, l);
          acc_fma(S_acc, h, l, eh[tt], el[tt]);
          acc_fma(Y_acc, h, l, xh[tt], xl[tt]);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && li + kStages < my_tiles) P.issue(blockIdx.x + (li + kStages) * G, s);
  }

  // ---- per-CTA partials
  const int stride = 2 * ws.cap + 3;
  float2* mypart = ws.part + (size_t)blockIdx.x * stride;
  colacc[2 * tid] = S_acc;
  colacc[2 * tid + 1] = Y_acc;
  __syncthreads();
  if (tid < r0) {
    Acc sS = acc_zero(), sY = acc_zero();
    for (int g = 0; g < G2; ++g) {
      const Acc a1 = colacc[2 * (g * ncol + tid)], a2 = colacc[2 * (g * ncol + tid) + 1];
      acc_add(sS, a1.h, a1.l);
      acc_add(sY, a2.h, a2.l);
    }
    sS = acc_norm(sS);
    sY = acc_norm(sY);
    mypart[tid] = make_float2(sS.h, sS.l);
    mypart[r0 + tid] = make_float2(sY.h, sY.l);
  }
  if (tid < 64) {  // threads with sub == 0 hold the scalar sums (warps 0 and 1)
    eta = warp_sum_acc(eta);
    ex = warp_sum_acc(ex);
    xi = warp_sum_acc(xi);
  }
  __syncthreads();
  if (tid == 32) {
    part[0] = eta;
    part[1] = ex;
    part[2] = xi;
  }
  __syncthreads();
  if (tid == 0) {
    acc_add(eta, part[0].h, part[0].l);
    acc_add(ex, part[1].h, part[1].l);
    acc_add(xi, part[2].h, part[2].l);
    eta = acc_norm(eta);
    ex = acc_norm(ex);
    xi = acc_norm(xi);
    mypart[2 * r0] = make_float2(eta.h, eta.l);
    mypart[2 * r0 + 1] = make_float2(ex.h, ex.l);
    mypart[2 * r0 + 2] = make_float2(xi.h, xi.l);
  }

  // ---- last CTA reduces all partials in CTA order
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&ctl->ticket_a, 1u);
  __syncthreads();
  if (ticket != (unsigned)(G - 1)) return;
  __threadfence();
  // 4 adjacent lanes per value, each summing every 4th CTA, then a fixed-order combine
  const int nv = 2 * r0 + 3;
  for (int base = 0; base < 4 * nv; base += kThreadsA) {
    const int item = base + tid;
    const int v = item >> 2, q = item & 3;
    Acc sum = acc_zero();
    if (v < nv)
      for (int b = q; b < G; b += 4) {
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
  }
}

// ---------------------------------------------------------------------------------------
// pass B: append the new column, or compact the basis (fused with the append)
// ---------------------------------------------------------------------------------------
constexpr int kStagesB = 2;

template <int ST>
__global__ void __launch_bounds__(kThreads) k_pass_b(Ws ws) {
  using T = Traits<ST>;
  using snap_t = typename T::snap_t;
  extern __shared__ __align__(1024) unsigned char smem[];
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const int mode = ctl->mode;
  const int cur = ctl->cur, curc = ctl->cur_c;
  const StateBuf st = ws.st[cur];
  const int r0 = st.hdr->r0;
  const int append = ctl->append;
  const int rnew = ctl->rnew;
  const int G = gridDim.x;

  if (mode != PB_NONE) {
    TilePipe<ST> P;
    P.setup(ws, r0, kStagesB);
    P.gc = (const unsigned char*)ws.ebuf;
    P.vc = 8;
    P.base = smem;
    unsigned char* p = smem + (size_t)kStagesB * P.stage_sz;
    P.bars = reinterpret_cast<uint64_t*>(p);
    p += 8 * kStagesB;
    float* coh = reinterpret_cast<float*>(p);
    float* col = coh + (kMaxCap + 8);
    float* jh = col + (kMaxCap + 8);
    float* jl = jh + kTile;
    Acc* part = reinterpret_cast<Acc*>(jl + kTile);          // [4][kTile]
    float* qbh = reinterpret_cast<float*>(part + 4 * kTile);  // [(r0+1)][rnew] hi
    float* qbl = qbh + (kMaxCap + 1) * kMaxR;

    const int elems_per_chunk = (ST == ST_BF16) ? 8 : 4;
    for (int k = tid; k < kMaxCap + 8; k += kThreads) {
      float h = 0.f, l = 0.f;
      if (k < r0 && append) {  // s = L0^T e
        h = ws.sm.red[k].x;
        l = ws.sm.red[k].y;
      }
      if (k >= P.nch * elems_per_chunk) h = l = 0.f;
      coh[k] = h;
      col[k] = l;
    }
    float ih = 0.f, il = 0.f;  // 1/rho0
    if (append) {
      const dd inv = dd_div(dd_of(1.f), dd_of(ctl->rho0));
      ih = inv.h;
      il = inv.l;
    }
    const int r0e = r0 + append;
    if (mode == PB_COMPACT) {
      for (int idx = tid; idx < r0e * rnew; idx += kThreads) {
        const int k = idx / rnew, j = idx % rnew;
        const float2 q = ws.sm.QB[(size_t)j * (ws.cap + 1) + k];
        qbh[k * rnew + j] = q.x;
        qbl[k * rnew + j] = q.y;
      }
    }
    if (tid == 0) {
      for (int s = 0; s < kStagesB; ++s) mbar_init(&P.bars[s], 1);
      mbar_fence_init();
    }
    __syncthreads();

    const int64_t ntiles = (ws.n + kTile - 1) / kTile;
    const int my_tiles = (int)((ntiles - blockIdx.x + G - 1) / G);
    if (tid == 0) {
      for (int li = 0; li < min(my_tiles, kStagesB); ++li) P.issue(blockIdx.x + li * G, li);
    }
    const int t = tid & 63, sub = tid >> 6;
    unsigned char* gh = (unsigned char*)ws.Lh;
    float* gl = ws.Ll;

    for (int li = 0; li < my_tiles; ++li) {
      const int s = li % kStagesB;
      const uint32_t par = (uint32_t)((li / kStagesB) & 1);
      const int tile = blockIdx.x + li * G;
      const int64_t row0 = (int64_t)tile * kTile;
      const int rows = rows_in(ws.n, row0);
      const bool ok = mbar_wait(&P.bars[s], par, &ctl->status);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) mbar_drain(P.bars, kStagesB, li, my_tiles);
        __syncthreads();
        break;
      }
      {
        if (append) {
          part[sub * kTile + t] = row_dot_partial<ST>(P, s, t, sub, coh, col);
          __syncthreads();
          if (sub == 0) {
            // j0 = (e - L0 s) / rho0: the second Gram-Schmidt pass, applied to the stored e
            const float2 ev = reinterpret_cast<const float2*>(P.snap_c(s))[t];
            const float ch = ev.x, cl = ev.y;
            Acc d = part[t];
            acc_add(d, part[kTile + t].h, part[kTile + t].l);
            acc_add(d, part[2 * kTile + t].h, part[2 * kTile + t].l);
            acc_add(d, part[3 * kTile + t].h, part[3 * kTile + t].l);
            Acc e = Acc{ch, cl};
            acc_add(e, -d.h, -d.l);
            e = acc_norm(e);
            Acc j = acc_zero();
            acc_fma(j, e.h, e.l, ih, il);
            j = acc_norm(j);
            jh[t] = j.h;
            jl[t] = j.l;
            if (mode == PB_APPEND && t < rows) {
              const size_t o = (size_t)(row0 + t) * ws.ldg + r0;
              if constexpr (ST == ST_BF16) {
                reinterpret_cast<__nv_bfloat16*>(gh)[o] = __float2bfloat16_rn(j.h);
              } else {
                reinterpret_cast<float*>(gh)[o] = j.h;
                if constexpr (ST == ST_DD) gl[o] = j.l;
              }
            }
          }
          __syncthreads();
        }
        if (mode == PB_COMPACT) {
          // out[t][j] = sum_k L0[t][k] QB[k][j] + j0_t QB[r0][j]
          const unsigned char* ph = P.plane_h(s);
          const unsigned char* pl = P.plane_l(s);
          for (int idx = tid; idx < rows * rnew; idx += kThreads) {
            const int tt = idx / rnew, j = idx % rnew;
            Acc acc = acc_zero();
            for (int k = 0; k < r0; ++k) {
              float h, l;
              load_elem<ST>(ph, pl, P.rs, tt, k, h, l);
              acc_fma(acc, h, l, qbh[k * rnew + j], qbl[k * rnew + j]);
            }
            if (append) acc_fma(acc, jh[tt], jl[tt], qbh[r0 * rnew + j], qbl[r0 * rnew + j]);
            acc = acc_norm(acc);
            const size_t o = (size_t)(row0 + tt) * ws.ldg + j;
            if constexpr (ST == ST_BF16) {
              reinterpret_cast<__nv_bfloat16*>(gh)[o] = __float2bfloat16_rn(acc.h);
            } else {
              reinterpret_cast<float*>(gh)[o] = acc.h;
              if constexpr (ST == ST_DD) gl[o] = acc.l;
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0 && li + kStagesB < my_tiles) P.issue(blockIdx.x + (li + kStagesB) * G, s);
    }
  }

  // ---- last CTA commits the new state
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&ctl->ticket_b, 1u);
  __syncthreads();
  if (ticket != (unsigned)(G - 1)) return;
  if (tid == 0) {
    __threadfence();
    ctl->cur = cur ^ 1;
    ctl->cur_c = curc ^ 1;
    ctl->eig_valid = 0;
    ctl->ticket_b = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// rollout: X[:, j] = L0 coef[:, j] (j < kcols), written in the snapshot type
// check:   same with kcols = 1 against x_fom, reducing instead of storing
// ---------------------------------------------------------------------------------------
constexpr int kStagesR = 2;

template <int ST, bool CHECK>
__global__ void __launch_bounds__(kThreads) k_rollout(Ws ws, int kcols, void* out, int64_t ld) {
  using T = Traits<ST>;
  using snap_t = typename T::snap_t;
  extern __shared__ __align__(1024) unsigned char smem[];
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur];
  const int r0 = st.hdr->r0;
  const int G = gridDim.x;

  TilePipe<ST> P;
  P.setup(ws, r0, kStagesR);
  P.gc = CHECK ? (const unsigned char*)ws.xbuf : nullptr;
  P.vc = T::vsz;
  P.base = smem;
  unsigned char* p = smem + (size_t)kStagesR * P.stage_sz;
  P.bars = reinterpret_cast<uint64_t*>(p);
  p += 8 * kStagesR;
  // coefficients, float-float, layout [k][kcols]; rows padded to whole chunks with zeros
  const int epc = (ST == ST_BF16) ? 8 : 4;
  const int kpad = P.nch * epc;
  float* cfh = reinterpret_cast<float*>(p);
  float* cfl = cfh + (kMaxCap + 8) * kRollK;
  Acc* part = reinterpret_cast<Acc*>(cfl + (kMaxCap + 8) * kRollK);  // [4][kTile]

  for (int idx = tid; idx < (kMaxCap + 8) * kcols; idx += kThreads) {
    const int k = idx / kcols, j = idx % kcols;
    float h = 0.f, l = 0.f;
    if (k < r0) {
      const float2 q = ws.sm.coef[(size_t)j * (ws.cap + 1) + k];
      h = q.x;
      l = q.y;
    }
    if (k >= kpad) h = l = 0.f;
    cfh[idx] = h;
    cfl[idx] = l;
  }
  if (tid == 0) {
    for (int s = 0; s < kStagesR; ++s) mbar_init(&P.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  const int64_t ntiles = (ws.n + kTile - 1) / kTile;
  const int my_tiles = (int)((ntiles - blockIdx.x + G - 1) / G);
  if (tid == 0) {
    for (int li = 0; li < min(my_tiles, kStagesR); ++li) P.issue(blockIdx.x + li * G, li);
  }
  // work split: items (t, j); with fewer than 4 columns each dot is split in nsub parts
  const int nsub = kcols == 1 ? 4 : (kcols == 2 ? 2 : 1);  // nsub * kTile * kcols <= 4 * kTile when > 1
  Acc num = acc_zero(), den = acc_zero();

  for (int li = 0; li < my_tiles; ++li) {
    const int s = li % kStagesR;
    const uint32_t par = (uint32_t)((li / kStagesR) & 1);
    const int tile = blockIdx.x + li * G;
    const int64_t row0 = (int64_t)tile * kTile;
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
      const int items = kTile * kcols * nsub;
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
              load_snap(reinterpret_cast<const typename T::stored_t*>(P.snap_c(s)), tt, fh, fl);
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
              load_snap(reinterpret_cast<const typename T::stored_t*>(P.snap_c(s)), tt, fh, fl);
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
    if (tid == 0 && li + kStagesR < my_tiles) P.issue(blockIdx.x + (li + kStagesR) * G, s);
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
      ws.part[2 * blockIdx.x] = make_float2(a.h, a.l);
      ws.part[2 * blockIdx.x + 1] = make_float2(b.h, b.l);
    }
    __shared__ unsigned ticket;
    __threadfence();
    __syncthreads();
    if (tid == 0) ticket = atomicAdd(&ctl->ticket_r, 1u);
    __syncthreads();
    if (ticket != (unsigned)(G - 1)) return;
    if (tid == 0) {
      __threadfence();
      Acc a = acc_zero(), b = acc_zero();
      for (int blk = 0; blk < G; ++blk) {
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
  }
}

// ---------------------------------------------------------------------------------------
// first snapshot: ||u^0||^2 into the committed state
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double stored_to_double(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double stored_to_double(float v) { return (double)v; }

template <typename stored_t>
__global__ void __launch_bounds__(kThreads) k_first(Ws ws) {
  Ctl* ctl = ws.ctl;
  const stored_t* c = reinterpret_cast<const stored_t*>(ws.cbuf[ctl->cur_c]);
  double acc = 0.0;  // N FP64 FMAs once per stream: negligible
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < ws.n; i += (int64_t)gridDim.x * kThreads) {
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
    ws.part[blockIdx.x] = make_float2(0.f, 0.f);
    reinterpret_cast<double*>(ws.part)[blockIdx.x] = b;
  }
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&ctl->ticket_a, 1u);
  __syncthreads();
  if (ticket != (unsigned)(gridDim.x - 1) || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) tot += __ldcg(reinterpret_cast<const double*>(ws.part) + b);
  if (!isfinite(tot)) atomicOr(&ctl->status, DEV_NONFINITE);
  ws.st[ctl->cur].hdr->cn2 = f2_of(dd_from_double(tot));
  ctl->ticket_a = 0u;
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
static int smem_a(int prec, int cap) {
  const int sb = prec == ST_DD ? stage_bytes<ST_DD>(cap) : prec == ST_F32 ? stage_bytes<ST_F32>(cap) : stage_bytes<ST_BF16>(cap);
  return kStages * sb + 8 * kStages + 2 * (kMaxCap + 8) * 4 + 4 * kTile * 4 + kSubA * kTile * 8 + 2 * kThreadsA * 8;
}
static int smem_b(int prec, int cap) {
  const int sb = prec == ST_DD ? stage_bytes<ST_DD>(cap) : prec == ST_F32 ? stage_bytes<ST_F32>(cap) : stage_bytes<ST_BF16>(cap);
  return kStagesB * sb + 8 * kStagesB + 2 * (kMaxCap + 8) * 4 + 2 * kTile * 4 + 4 * kTile * 8 +
         2 * (kMaxCap + 1) * kMaxR * 4;
}
static int smem_r(int prec, int cap) {
  const int sb = prec == ST_DD ? stage_bytes<ST_DD>(cap) : prec == ST_F32 ? stage_bytes<ST_F32>(cap) : stage_bytes<ST_BF16>(cap);
  return kStagesR * sb + 8 * kStagesR + 2 * (kMaxCap + 8) * kRollK * 4 + 4 * kTile * 8;
}

int tall_smem_bytes(int prec) { return smem_a(prec, kMaxCap); }

template <typename K>
static cudaError_t prep_attr(K kern, int bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Raise the dynamic shared-memory limit of every tall kernel once (not inside launches,
// which may be captured into a graph).
cudaError_t prepare_tall(const Ws& ws) {
  const int cap = ws.cap;
  cudaError_t e = cudaSuccess;
  switch (ws.prec) {
    case ST_DD:
      if ((e = prep_attr(k_pass_a<ST_DD>, smem_a(ST_DD, cap)))) return e;
      if ((e = prep_attr(k_pass_b<ST_DD>, smem_b(ST_DD, cap)))) return e;
      if ((e = prep_attr(k_rollout<ST_DD, false>, smem_r(ST_DD, cap)))) return e;
      return prep_attr(k_rollout<ST_DD, true>, smem_r(ST_DD, cap));
    case ST_F32:
      if ((e = prep_attr(k_pass_a<ST_F32>, smem_a(ST_F32, cap)))) return e;
      if ((e = prep_attr(k_pass_b<ST_F32>, smem_b(ST_F32, cap)))) return e;
      if ((e = prep_attr(k_rollout<ST_F32, false>, smem_r(ST_F32, cap)))) return e;
      return prep_attr(k_rollout<ST_F32, true>, smem_r(ST_F32, cap));
    default:
      if ((e = prep_attr(k_pass_a<ST_BF16>, smem_a(ST_BF16, cap)))) return e;
      if ((e = prep_attr(k_pass_b<ST_BF16>, smem_b(ST_BF16, cap)))) return e;
      if ((e = prep_attr(k_rollout<ST_BF16, false>, smem_r(ST_BF16, cap)))) return e;
      return prep_attr(k_rollout<ST_BF16, true>, smem_r(ST_BF16, cap));
  }
}

cudaError_t launch_pass_a(const Ws& ws, cudaStream_t s) {
  const int sm = smem_a(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      k_pass_a<ST_DD><<<ws.gridA, kThreadsA, sm, s>>>(ws);
      break;
    case ST_F32:
      k_pass_a<ST_F32><<<ws.gridA, kThreadsA, sm, s>>>(ws);
      break;
    default:
      k_pass_a<ST_BF16><<<ws.gridA, kThreadsA, sm, s>>>(ws);
  }
  return cudaGetLastError();
}

cudaError_t launch_pass_b(const Ws& ws, cudaStream_t s) {
  const int sm = smem_b(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      k_pass_b<ST_DD><<<ws.gridA, kThreads, sm, s>>>(ws);
      break;
    case ST_F32:
      k_pass_b<ST_F32><<<ws.gridA, kThreads, sm, s>>>(ws);
      break;
    default:
      k_pass_b<ST_BF16><<<ws.gridA, kThreads, sm, s>>>(ws);
  }
  return cudaGetLastError();
}

cudaError_t launch_first(const Ws& ws, cudaStream_t s) {
  const int grid = 64;  // the partial buffer always holds at least 64 rows
  if (ws.prec == ST_DD)
    k_first<float2><<<grid, kThreads, 0, s>>>(ws);
  else
    k_first<float><<<grid, kThreads, 0, s>>>(ws);
  return cudaGetLastError();
}

// Copy a caller's double snapshot into the workspace as float pairs (all SMs; the only
// FP64 instructions a snapshot meets).
__global__ void __launch_bounds__(kThreads) k_ingest_dd(const double* __restrict__ src, float2* __restrict__ dst,
                                                        int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    float h, l;
    split_double(src[i], h, l);
    dst[i] = make_float2(h, l);
  }
}

__global__ void __launch_bounds__(kThreads) k_ingest_f32(const float* __restrict__ src, float* __restrict__ dst,
                                                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    dst[i] = src[i];
}

static int ingest_grid(const Ws& ws) {
  const int64_t blocks = (ws.n + kThreads - 1) / kThreads;
  return (int)(blocks < 4 * 152 ? blocks : 4 * 152);
}

cudaError_t launch_ingest(const Ws& ws, const void* src, void* dst, cudaStream_t s) {
  if (ws.prec == ST_DD)
    k_ingest_dd<<<ingest_grid(ws), kThreads, 0, s>>>(reinterpret_cast<const double*>(src),
                                                     reinterpret_cast<float2*>(dst), ws.n);
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
      k_rollout<ST_DD, false><<<ws.gridA, kThreads, sm, s>>>(ws, kcols, out, ld);
      break;
    case ST_F32:
      k_rollout<ST_F32, false><<<ws.gridA, kThreads, sm, s>>>(ws, kcols, out, ld);
      break;
    default:
      k_rollout<ST_BF16, false><<<ws.gridA, kThreads, sm, s>>>(ws, kcols, out, ld);
  }
  return cudaGetLastError();
}

cudaError_t launch_check(const Ws& ws, cudaStream_t s) {
  const int sm = smem_r(ws.prec, ws.cap);
  switch (ws.prec) {
    case ST_DD:
      k_rollout<ST_DD, true><<<ws.gridA, kThreads, sm, s>>>(ws, 1, nullptr, 0);
      break;
    case ST_F32:
      k_rollout<ST_F32, true><<<ws.gridA, kThreads, sm, s>>>(ws, 1, nullptr, 0);
      break;
    default:
      k_rollout<ST_BF16, true><<<ws.gridA, kThreads, sm, s>>>(ws, 1, nullptr, 0);
  }
  return cudaGetLastError();
}

}  // namespace odmd
