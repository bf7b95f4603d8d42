// Orthogonality refinement of the basis L = L0 Q.  The paper has no such step; it keeps
// the invariant L^T L = I over long streams (rounding in every rank-1 update lets it drift,
// most of all with FP32 storage of L0).
//
//   C = L^T L = Q^T (L0^T L0) Q           (k_gram + k_gram_sum: the Gram matrix of L0, one
//                                          pass over N; k_refine_c: the two small products)
//   C = R^T R                              (Cholesky, R upper triangular)
//   R diag(S) = U_s Sigma V_s^T            (one-sided Jacobi SVD; R ~ I, so one sweep rotates
//                                          and a second confirms)
//
// and, since U^- ~ L S W^T = (L R^-1)(R S) W^T = (L R^-1 U_s) Sigma (W V_s)^T,
//
//   Q <- Q R^-1 U_s,  S <- Sigma,  r_first <- r_first V_s,  r_last <- r_last V_s,
//   M <- (R^-1 U_s)^T M V_s                (M = L^T U^+ W with the new L and W)
//
// L0 itself is not rewritten; the carried projection a = L0^T c and the coefficients of a
// pending column are in L0 coordinates and stay as they are.  All arithmetic is
// double-float.  The state moves to the other state buffer like an update does, so the
// host's mirror of the committed buffer flips once per call whatever happens: when the
// rank is still 0 or the Cholesky factorisation fails (a non-positive pivot sets
// DEV_NONFINITE), the state is copied unchanged.
#include "dd.cuh"
#include "odmd_internal.cuh"

namespace odmd {

// ---------------------------------------------------------------- Gram pass G = L0^T L0
// A CTA streams 32-row tiles of L0 through shared memory.  The upper triangle of G is cut
// into 4 x 4 column blocks; a thread owns one block (two when there are more blocks than
// threads) and, when there are few blocks, a residue class of the tile's rows, so every
// thread has work for any r0.  A block is 16 double-float accumulations per row, done two
// at a time by the FP32x2 instructions.
constexpr int kGramThreads = 256;
constexpr int kGramRows = 32;
constexpr int kGramLd = kMaxCap + 4;  // floats per shared row (rows stay 16-byte aligned)
constexpr int kGramItems = 2;         // blocks per thread at most: ceil(B(B+1)/2 / 256), B = 24
constexpr int kRefineThreads = 512;
constexpr int kRefineLd = kMaxR;      // leading dimension of the small matrices in shared memory
static_assert((kMaxCap / 4 + 1) * (kMaxCap / 4) / 2 <= kGramItems * kGramThreads, "Gram blocks per thread");
static_assert(kMaxCap <= 128 && kMaxR <= 64, "refinement kernels size their CTAs for these limits");

__device__ __forceinline__ int gram_pairs(int r0) { return r0 * (r0 + 1) / 2; }
// index of (i, k), i <= k, in the row-major upper triangle (0,0), (0,1), .., (0,r0-1), (1,1), ..
__device__ __forceinline__ int gram_index(int i, int k, int r0) { return i * r0 - i * (i - 1) / 2 + (k - i); }
__device__ __forceinline__ void gram_pair(int p, int r0, int& i, int& k) {
  i = 0;
  while (p >= r0 - i) {
    p -= r0 - i;
    ++i;
  }
  k = i + p;
}

struct GramTile {
  float h[kGramRows][kGramLd], l[kGramRows][kGramLd];
};
union GramSmem {
  GramTile t;
  float2 red[kGramThreads][16];
};

template <int ST>
__device__ __forceinline__ void gram_row(Acc2 (&A)[8], const GramTile& t, int row, int bi, int bk) {
  const float4 xh = *reinterpret_cast<const float4*>(&t.h[row][4 * bi]);
  const float4 yh = *reinterpret_cast<const float4*>(&t.h[row][4 * bk]);
  const f2x y0 = f2x_pack(yh.x, yh.y), y1 = f2x_pack(yh.z, yh.w);
  const f2x ny0 = sub2(0ull, y0), ny1 = sub2(0ull, y1);
  const float xs[4] = {xh.x, xh.y, xh.z, xh.w};
  if constexpr (ST == ST_DD) {
    const float4 xl = *reinterpret_cast<const float4*>(&t.l[row][4 * bi]);
    const float4 yl = *reinterpret_cast<const float4*>(&t.l[row][4 * bk]);
    const f2x l0 = f2x_pack(yl.x, yl.y), l1 = f2x_pack(yl.z, yl.w);
    const float xls[4] = {xl.x, xl.y, xl.z, xl.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const f2x xb = f2x_pack(xs[i], xs[i]), xlb = f2x_pack(xls[i], xls[i]);
      acc2_fma(A[2 * i], xb, xlb, y0, ny0, l0);
      acc2_fma(A[2 * i + 1], xb, xlb, y1, ny1, l1);
    }
  } else {
    // FP32 storage: the low parts are zero, so only the product's own rounding error
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const f2x xb = f2x_pack(xs[i], xs[i]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const f2x y = h ? y1 : y0, ny = h ? ny1 : ny0;
        Acc2& a = A[2 * i + h];
        const f2x np = mul2(xb, ny);
        const f2x pe = fma2(xb, y, np);
        const f2x s = sub2(a.h, np);
        const f2x bb = sub2(s, a.h);
        const f2x e = sub2(sub2(a.h, sub2(s, bb)), add2(np, bb));
        a.h = s;
        a.l = add2(a.l, add2(e, pe));
      }
    }
  }
}

__device__ __forceinline__ void acc2_renorm(Acc2& a) {
  const f2x s = add2(a.h, a.l);
  a.l = sub2(a.l, sub2(s, a.h));
  a.h = s;
}

// element e = 4 i + 2 h + lane of a block: row 4 bi + i, column 4 bk + 2 h + lane
__device__ __forceinline__ void block_values(const Acc2 (&A)[8], float2 (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    Acc a0, a1;
    acc2_split(A[q], a0, a1);
    a0 = acc_norm(a0);
    a1 = acc_norm(a1);
    v[2 * q] = make_float2(a0.h, a0.l);
    v[2 * q + 1] = make_float2(a1.h, a1.l);
  }
}

__device__ __forceinline__ void block_of(int b, int B, int& bi, int& bk) {
  bi = 0;
  while (b >= B - bi) {
    b -= B - bi;
    ++bi;
  }
  bk = bi + b;
}

template <int ST>
__global__ void __launch_bounds__(kGramThreads, 2) k_gram(Ws ws, int cur) {
  const int r0 = ws.st[cur].hdr->r0;
  if (r0 < 1) return;
  const int B = (r0 + 3) >> 2, nb = B * (B + 1) / 2;
  int nsub = kGramThreads / nb;
  nsub = nsub < 1 ? 1 : (nsub > kGramRows ? kGramRows : nsub);
  const int items = nb * nsub;
  const int tid = threadIdx.x;
  __shared__ __align__(16) GramSmem sm;
  int bi[kGramItems], bk[kGramItems], sb[kGramItems];
  Acc2 acc[kGramItems][8];
#pragma unroll
  for (int q = 0; q < kGramItems; ++q) {
    const int it = tid + kGramThreads * q;
    bi[q] = bk[q] = 0;
    sb[q] = kGramRows;  // no rows: inactive
    if (it < items) {
      block_of(it % nb, B, bi[q], bk[q]);
      sb[q] = it / nb;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[q][e] = acc2_zero();
  }
  const int w = 4 * B;
  const int64_t ntiles = (ws.n + kGramRows - 1) / kGramRows;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * kGramRows;
    __syncthreads();
    for (int idx = tid; idx < kGramRows * w; idx += kGramThreads) {
      const int t = idx / w, c = idx - t * w;
      float h = 0.f, l = 0.f;
      if (c < r0 && row0 + t < ws.n) {
        const size_t o = (size_t)(row0 + t) * ws.ldg + c;
        h = reinterpret_cast<const float*>(ws.Lh)[o];
        if constexpr (ST == ST_DD) l = ws.Ll[o];
      }
      sm.t.h[t][c] = h;
      if constexpr (ST == ST_DD) sm.t.l[t][c] = l;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGramItems; ++q) {
      for (int t = sb[q]; t < kGramRows; t += nsub) gram_row<ST>(acc[q], sm.t, t, bi[q], bk[q]);
      // fold the low word back once per tile: left to grow over the hundreds of rows a
      // thread adds, its own FP32 rounding dominates the error of the diagonal sums
#pragma unroll
      for (int e = 0; e < 8; ++e) acc2_renorm(acc[q][e]);
    }
  }
  const size_t stride = (size_t)ws.cap * (ws.cap + 1) / 2;
  float2* out = ws.gpart + (size_t)blockIdx.x * stride;
  if (nsub == 1) {
#pragma unroll
    for (int q = 0; q < kGramItems; ++q) {
      if (tid + kGramThreads * q >= items) continue;
      float2 v[16];
      block_values(acc[q], v);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int ci = 4 * bi[q] + (e >> 2), ck = 4 * bk[q] + (e & 3);
        if (ci <= ck && ck < r0) out[gram_index(ci, ck, r0)] = v[e];
      }
    }
    return;
  }
  // several row classes per block (then items <= kGramThreads): add them in class order
  __syncthreads();
  if (tid < items) {
    float2 v[16];
    block_values(acc[0], v);
#pragma unroll
    for (int e = 0; e < 16; ++e) sm.red[tid][e] = v[e];
  }
  __syncthreads();
  for (int o = tid; o < nb * 16; o += kGramThreads) {
    const int b = o >> 4, e = o & 15;
    int i0, k0;
    block_of(b, B, i0, k0);
    const int ci = 4 * i0 + (e >> 2), ck = 4 * k0 + (e & 3);
    if (!(ci <= ck && ck < r0)) continue;
    dd a = dd_of(0.f);
    for (int s = 0; s < nsub; ++s) a = a + dd_of(sm.red[s * nb + b][e]);
    out[gram_index(ci, ck, r0)] = f2_of(a);
  }
}

// Matrices of the refinement in the scratch region (double-float pairs, column-major):
//   G cap x cap (ld cap) | C, W, V: rmax x rmax (ld rmax) | sig: rmax | perm: rmax ints, flag
struct RefineScratch {
  float2 *G, *C, *W, *V, *sig;
  int *perm, *flag;
};

__device__ __forceinline__ RefineScratch refine_scratch(const Ws& ws) {
  RefineScratch s;
  const size_t cap = ws.cap, rm = ws.rmax;
  float2* p = ws.rscr;
  s.G = p;
  p += cap * cap;
  s.C = p;
  p += rm * rm;
  s.W = p;
  p += rm * rm;
  s.V = p;
  p += rm * rm;
  s.sig = p;
  p += rm;
  s.perm = reinterpret_cast<int*>(p);
  s.flag = s.perm + rm;
  return s;
}

__device__ __forceinline__ void st2(float2* a, size_t i, dd v) { a[i] = make_float2(v.h, v.l); }
// a += x y, folding the low word back every 8 terms (sums of up to cap terms)
__device__ __forceinline__ void acc_fma_k(Acc& a, float2 x, float2 y, int k) {
  acc_fma(a, x.x, x.y, y.x, y.y);
  if ((k & 7) == 7) a = acc_norm(a);
}
__device__ __forceinline__ dd acc_dd(Acc a) {
  a = acc_norm(a);
  return dd{a.h, a.l};
}

// G: a warp per pair; lane L adds partials L, L + 32, .. in order, then a butterfly over the
// lanes (double-float addition is symmetric, so every lane ends with the same value).  The
// tree keeps the rounding of the sum of a few hundred partials at a few units of 2^-48.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_gram_sum(Ws ws, int cur, int nblocks) {
  const int r0 = ws.st[cur].hdr->r0;
  const int p = blockIdx.x * (kSumThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (p >= gram_pairs(r0)) return;  // whole warps leave together
  const size_t stride = (size_t)ws.cap * (ws.cap + 1) / 2;
  dd a = dd_of(0.f);
  for (int b = lane; b < nblocks; b += 32) a = a + dd_of(__ldcg(ws.gpart + (size_t)b * stride + p));
  a = dd_warp_sum(a);
  if (lane == 0) {
    int i, k;
    gram_pair(p, r0, i, k);
    const RefineScratch S = refine_scratch(ws);
    S.G[(size_t)k * ws.cap + i] = f2_of(a);
    S.G[(size_t)i * ws.cap + k] = f2_of(a);
  }
}

// C = Q^T G Q, one column per CTA: t = G Q[:, j] in shared memory, then C[:, j] = Q^T t
__global__ void __launch_bounds__(128) k_refine_c(Ws ws, int cur) {
  const StateBuf st = ws.st[cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, j = blockIdx.x;
  if (r < 1 || r0 < r || j >= r) return;
  const int cap = ws.cap, qld = cap + 1, tid = threadIdx.x;
  const RefineScratch S = refine_scratch(ws);
  __shared__ float2 t[kMaxCap];
  for (int a = tid; a < r0; a += 128) {
    Acc s = acc_zero();
    for (int b = 0; b < r0; ++b) acc_fma_k(s, S.G[(size_t)b * cap + a], d2f2(st.Q[(size_t)j * qld + b]), b);
    s = acc_norm(s);
    t[a] = make_float2(s.h, s.l);
  }
  __syncthreads();
  for (int i = tid; i < r; i += 128) {
    Acc s = acc_zero();
    for (int a = 0; a < r0; ++a) acc_fma_k(s, d2f2(st.Q[(size_t)i * qld + a]), t[a], a);
    s = acc_norm(s);
    S.C[(size_t)j * ws.rmax + i] = make_float2(s.h, s.l);
  }
}

// ------------------------------------------------- Cholesky, Jacobi SVD, R^-1 U_s (one CTA)
struct RefineSmem {
  float2 R[kMaxR * kRefineLd], T[kMaxR * kRefineLd], V[kMaxR * kRefineLd];
  float2 sig[kMaxR], dinv[kMaxR];
  int perm[kMaxR];
  int rot[32];
  int bad;
};

__device__ __forceinline__ dd half_sum(dd a, unsigned mask) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) a = a + dd{__shfl_xor_sync(mask, a.h, o), __shfl_xor_sync(mask, a.l, o)};
  return a;
}

__global__ void __launch_bounds__(kRefineThreads) k_refine(Ws ws, int cur) {
  const StateBuf st = ws.st[cur];
  const int r = st.hdr->r, r0 = st.hdr->r0;
  const int tid = threadIdx.x;
  const RefineScratch S = refine_scratch(ws);
  if (r < 1 || r0 < r) {
    if (tid == 0) *S.flag = 2;  // no basis yet: the state is carried over as it is
    return;
  }
  extern __shared__ __align__(16) unsigned char refine_smem_raw[];
  RefineSmem& sm = *reinterpret_cast<RefineSmem*>(refine_smem_raw);
  constexpr int ld = kRefineLd;
  const int rm = ws.rmax;
  if (tid == 0) sm.bad = 0;
  if (tid < 32) sm.rot[tid] = 0;
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, k = o / r;
    sm.R[k * ld + i] = S.C[(size_t)k * rm + i];
  }
  __syncthreads();

  // Cholesky C = R^T R, right-looking on the upper triangle.  Step j subtracts
  // a_ji a_jk / a_jj from the trailing block; the rows are scaled by 1/sqrt(a_jj) at the end
  // (row j is not touched after step j), so a step needs one barrier.
  for (int j = 0; j < r; ++j) {
    const dd d = dd_of(sm.R[j * ld + j]);
    if (!(d.h > 0.f) || !dd_isfinite(d)) {
      if (tid == 0) sm.bad = 1;
      break;  // every thread reads the same pivot and leaves here
    }
    const dd dinv = dd_div(dd_of(1.f), d);
    const int w = r - j - 1;
    for (int o = tid; o < w * w; o += kRefineThreads) {
      const int i = j + 1 + o % w, k = j + 1 + o / w;
      if (i > k) continue;
      const dd f = dd_of(sm.R[i * ld + j]) * dinv;
      const dd v = dd_of(sm.R[k * ld + i]) - f * dd_of(sm.R[k * ld + j]);
      sm.R[k * ld + i] = f2_of(v);
    }
    __syncthreads();
  }
  __syncthreads();
  if (sm.bad) {
    if (tid == 0) *S.flag = 1;
    return;
  }
  // row scaling (a_jj -> sqrt(a_jj), a_jk -> a_jk / sqrt(a_jj)), zero below the diagonal;
  // T = R diag(S), V = I
  for (int j = tid; j < r; j += kRefineThreads) sm.dinv[j] = f2_of(dd_sqrt(dd_of(sm.R[j * ld + j])));
  __syncthreads();
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, k = o / r;
    dd v = dd_of(0.f);
    if (i == k)
      v = dd_of(sm.dinv[i]);
    else if (i < k)
      v = dd_div(dd_of(sm.R[k * ld + i]), dd_of(sm.dinv[i]));
    sm.R[k * ld + i] = f2_of(v);
  }
  __syncthreads();
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, k = o / r;
    sm.T[k * ld + i] = f2_of(dd_of(sm.R[k * ld + i]) * dd_from_double(st.S[k]));
    sm.V[k * ld + i] = make_float2(i == k ? 1.f : 0.f, 0.f);
  }
  __syncthreads();

  // One-sided Jacobi on the columns of T, round-robin order: each round rotates m/2
  // disjoint column pairs at once, a half-warp per pair with the rows split over its
  // 16 lanes.  A sweep is m - 1 rounds; the sweeps stop when one rotates nothing.
  {
    const int m = r + (r & 1);
    const int hw = tid >> 4, hl = tid & 15;
    const unsigned mask = (tid & 16) ? 0xffff0000u : 0x0000ffffu;
    const float tol = 4.f * 7.105427357601002e-15f;
    for (int sweep = 0; sweep < 16; ++sweep) {
      int rotated = 0;
      for (int k = 0; k < m - 1; ++k) {
        for (int pi = hw; pi < m / 2; pi += kRefineThreads / 16) {
          int a = k, b = m - 1;
          if (pi > 0) {
            a = (k + pi) % (m - 1);
            b = (k - pi + m - 1) % (m - 1);
          }
          const int p = a < b ? a : b, q = a < b ? b : a;
          if (q >= r) continue;  // the dummy column of an odd r
          Acc al = acc_zero(), be = acc_zero(), ga = acc_zero();
          for (int i = hl; i < r; i += 16) {
            const float2 tp = sm.T[p * ld + i], tq = sm.T[q * ld + i];
            acc_fma(al, tp.x, tp.y, tp.x, tp.y);
            acc_fma(be, tq.x, tq.y, tq.x, tq.y);
            acc_fma(ga, tp.x, tp.y, tq.x, tq.y);
          }
          const dd A = half_sum(acc_dd(al), mask), Bv = half_sum(acc_dd(be), mask), G = half_sum(acc_dd(ga), mask);
          if (!(fabsf(G.h) > tol * sqrtf(A.h) * sqrtf(Bv.h))) continue;
          ++rotated;
          // rotation zeroing the (p, q) inner product: zeta = (be - al) / (2 ga),
          // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t.
          // For |zeta| >= 2^26, t = ga / (be - al) and c = 1 to double-float accuracy.
          const dd diff = Bv - A;
          dd c, s;
          if (fabsf(diff.h) >= 134217728.f * fabsf(G.h)) {
            c = dd_of(1.f);
            s = dd_div(G, diff);
          } else {
            const dd one = dd_of(1.f);
            const dd zeta = dd_div(diff, G * 2.f);
            const dd t = dd_div(zeta.h >= 0.f ? one : -one, dd_abs(zeta) + dd_sqrt(one + zeta * zeta));
            c = dd_div(one, dd_sqrt(one + t * t));
            s = c * t;
          }
          for (int i = hl; i < r; i += 16) {
            const dd tp = dd_of(sm.T[p * ld + i]), tq = dd_of(sm.T[q * ld + i]);
            sm.T[p * ld + i] = f2_of(c * tp - s * tq);
            sm.T[q * ld + i] = f2_of(s * tp + c * tq);
            const dd vp = dd_of(sm.V[p * ld + i]), vq = dd_of(sm.V[q * ld + i]);
            sm.V[p * ld + i] = f2_of(c * vp - s * vq);
            sm.V[q * ld + i] = f2_of(s * vp + c * vq);
          }
        }
        __syncthreads();
      }
      if (rotated && hl == 0) atomicAdd(&sm.rot[sweep], 1);
      __syncthreads();
      if (sm.rot[sweep] == 0) break;
    }
  }

  // singular values (column norms, a half-warp per column), descending order by rank count
  {
    const int hw = tid >> 4, hl = tid & 15;
    const unsigned mask = (tid & 16) ? 0xffff0000u : 0x0000ffffu;
    for (int j = hw; j < r; j += kRefineThreads / 16) {
      Acc s = acc_zero();
      for (int i = hl; i < r; i += 16) {
        const float2 t = sm.T[j * ld + i];
        acc_fma(s, t.x, t.y, t.x, t.y);
      }
      const dd n = dd_sqrt(half_sum(acc_dd(s), mask));
      if (hl == 0) {
        sm.sig[j] = f2_of(n);
        if (!(n.h > 0.f) || !dd_isfinite(n)) sm.bad = 1;
      }
    }
  }
  __syncthreads();
  if (sm.bad) {
    if (tid == 0) *S.flag = 1;
    return;
  }
  for (int j = tid; j < r; j += kRefineThreads) {
    const dd sj = dd_of(sm.sig[j]);
    int rank = 0;
    for (int k = 0; k < r; ++k) {
      const dd sk = dd_of(sm.sig[k]);
      rank += dd_gt(sk, sj) || (!dd_lt(sk, sj) && k < j);
    }
    sm.perm[rank] = j;
  }
  // U_s = T Sigma^-1 in place; 1 / R_ii
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, k = o / r;
    sm.T[k * ld + i] = f2_of(dd_div(dd_of(sm.T[k * ld + i]), dd_of(sm.sig[k])));
  }
  for (int i = tid; i < r; i += kRefineThreads) sm.dinv[i] = f2_of(dd_div(dd_of(1.f), dd_of(sm.R[i * ld + i])));
  __syncthreads();
  // W = R^-1 U_s in place, column-oriented back substitution: step i removes the final
  // row i (its unscaled value times 1/R_ii) from the rows above; rows are scaled at the end
  for (int i = r - 1; i > 0; --i) {
    const dd di = dd_of(sm.dinv[i]);
    for (int o = tid; o < i * r; o += kRefineThreads) {
      const int k = o % i, j = o / i;
      const dd u = dd_of(sm.T[j * ld + i]) * di;
      sm.T[j * ld + k] = f2_of(dd_of(sm.T[j * ld + k]) - dd_of(sm.R[i * ld + k]) * u);
    }
    __syncthreads();
  }
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, j = o / r;
    st2(S.W, (size_t)j * rm + i, dd_of(sm.T[j * ld + i]) * dd_of(sm.dinv[i]));
    S.V[(size_t)j * rm + i] = sm.V[j * ld + i];
  }
  for (int j = tid; j < r; j += kRefineThreads) {
    S.sig[j] = sm.sig[j];
    S.perm[j] = sm.perm[j];
  }
  if (tid == 0) *S.flag = 0;
}

// --------------------------------------------------- the new state, one column per CTA
// Column j takes Sigma's j-th largest value: pj = perm[j].
//   M'[:, j] = W[:, perm]^T (M V[:, pj]),  Q'[:, j] = Q W[:, pj]
// CTA 0 also writes S, r_first, r_last, copies a, ps and the header, and commits.
__global__ void __launch_bounds__(128) k_refine_out(Ws ws, int cur) {
  const StateBuf st = ws.st[cur], nx = ws.st[cur ^ 1];
  const int r = st.hdr->r, r0 = st.hdr->r0, rm = ws.rmax, qld = ws.cap + 1;
  const int j = blockIdx.x, tid = threadIdx.x;
  const RefineScratch S = refine_scratch(ws);
  const int flag = *S.flag;
  if (flag != 0) {
    // carried over unchanged (flag 2) or refused (flag 1: a non-positive pivot)
    if (j < r) {
      for (int i = tid; i < r; i += 128) nx.M[(size_t)j * rm + i] = st.M[(size_t)j * rm + i];
      for (int a = tid; a < r0; a += 128) nx.Q[(size_t)j * qld + a] = st.Q[(size_t)j * qld + a];
    }
    if (j == 0) {
      for (int i = tid; i < r; i += 128) {
        nx.S[i] = st.S[i];
        nx.rf[i] = st.rf[i];
        nx.rl[i] = st.rl[i];
      }
    }
  } else if (j < r) {
    // M and the rows of R are FP64 state: the rotation is applied in FP64
    __shared__ double m2[kMaxR];
    const int pj = S.perm[j];
    for (int i = tid; i < r; i += 128) {
      double s = 0.0;
      for (int k = 0; k < r; ++k) s = fma(st.M[(size_t)k * rm + i], dd2d(S.V[(size_t)pj * rm + k]), s);
      m2[i] = s;
    }
    __syncthreads();
    for (int i = tid; i < r; i += 128) {
      const int pi = S.perm[i];
      double s = 0.0;
      for (int k = 0; k < r; ++k) s = fma(dd2d(S.W[(size_t)pi * rm + k]), m2[k], s);
      nx.M[(size_t)j * rm + i] = s;
    }
    for (int a = tid; a < r0; a += 128) {
      Acc s = acc_zero();
      for (int k = 0; k < r; ++k) acc_fma_k(s, d2f2(st.Q[(size_t)k * qld + a]), S.W[(size_t)pj * rm + k], k);
      s = acc_norm(s);
      nx.Q[(size_t)j * qld + a] = (double)s.h + (double)s.l;
    }
    if (j == 0) {
      for (int jj = tid; jj < r; jj += 128) {
        const int pjj = S.perm[jj];
        double f = 0.0, l = 0.0;
        for (int k = 0; k < r; ++k) {
          const double v = dd2d(S.V[(size_t)pjj * rm + k]);
          f = fma(st.rf[k], v, f);
          l = fma(st.rl[k], v, l);
        }
        nx.rf[jj] = f;
        nx.rl[jj] = l;
        nx.S[jj] = dd2d(S.sig[pjj]);
      }
    }
  }
  if (j == 0) {
    for (int i = tid; i < qld; i += 128) {
      nx.a[i] = st.a[i];
      nx.ps[i] = st.ps[i];
    }
    if (tid == 0) {
      *nx.hdr = *st.hdr;
      // the kernels of this call take the committed buffer from their argument, so the
      // switch can be made before the other CTAs finish
      ws.ctl->cur = cur ^ 1;
      ws.ctl->eig_valid = 0;
      ws.ctl->model_ver += 1ull;
      if (flag == 1) atomicOr(&ws.ctl->status, DEV_NONFINITE);
    }
  }
}

int refine_smem_bytes() { return (int)sizeof(RefineSmem); }

cudaError_t prepare_refine() {
  return cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, refine_smem_bytes());
}

cudaError_t launch_refine(const Ws& ws, int cur, cudaStream_t s) {
  switch (ws.prec) {
    case ST_DD:
      k_gram<ST_DD><<<ws.gridG, kGramThreads, 0, s>>>(ws, cur);
      break;
    case ST_F32:
      k_gram<ST_F32><<<ws.gridG, kGramThreads, 0, s>>>(ws, cur);
      break;
    default:
      return cudaErrorInvalidValue;  // BF16 storage is refused when a handle is created
  }
  const int np = ws.cap * (ws.cap + 1) / 2, per = kSumThreads / 32;
  k_gram_sum<<<(np + per - 1) / per, kSumThreads, 0, s>>>(ws, cur, ws.gridG);
  k_refine_c<<<ws.rmax, 128, 0, s>>>(ws, cur);
  k_refine<<<1, kRefineThreads, refine_smem_bytes(), s>>>(ws, cur);
  k_refine_out<<<ws.rmax, 128, 0, s>>>(ws, cur);
  return cudaGetLastError();
}

}  // namespace odmd
