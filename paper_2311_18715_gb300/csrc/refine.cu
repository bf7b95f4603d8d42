// Orthogonality refinement of the basis L = L0 Q.  The paper has no such step; it keeps
// the invariant L^T L = I over long streams (rounding in every rank-1 update lets it drift,
// most of all with FP32 storage of L0).
//
//   C = L^T L = Q^T (L0^T L0) Q           (k_gram: the Gram matrix of L0, one pass over N)
//   C = R^T R                              (Cholesky, R upper triangular)
//   R diag(S) = U_s Sigma V_s^T            (one-sided Jacobi SVD; R ~ I so one or two sweeps)
//
// and, since U^- ~ L S W^T = (L R^-1)(R S) W^T = (L R^-1 U_s) Sigma (W V_s)^T,
//
//   Q <- Q R^-1 U_s,  S <- Sigma,  r_first <- r_first V_s,  r_last <- r_last V_s,
//   M <- (R^-1 U_s)^T M V_s                (M = L^T U^+ W with the new L and W)
//
// L0 itself is not rewritten; the carried projection a = L0^T c and the coefficients of a
// pending column are in L0 coordinates and stay as they are.  Both kernels work in
// double-float arithmetic.
#include "dd.cuh"
#include "odmd_internal.cuh"

namespace odmd {

constexpr int kGramThreads = 256;
constexpr int kGramRows = 32;
constexpr int kGramMaxPairs = (kMaxCap * (kMaxCap + 1) / 2 + kGramThreads - 1) / kGramThreads;
constexpr int kRefineThreads = 256;

__device__ __forceinline__ int gram_pairs(int r0) { return r0 * (r0 + 1) / 2; }

// pair p of the upper triangle (row-major: (0,0), (0,1), .., (0,r0-1), (1,1), ..) -> (i, k)
__device__ __forceinline__ void gram_pair(int p, int r0, int& i, int& k) {
  i = 0;
  while (p >= r0 - i) {
    p -= r0 - i;
    ++i;
  }
  k = i + p;
}

template <int ST>
__device__ __forceinline__ void load_basis(const Ws& ws, size_t o, float& h, float& l) {
  if constexpr (ST == ST_BF16) {
    h = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(ws.Lh)[o]);
    l = 0.f;
  } else {
    h = reinterpret_cast<const float*>(ws.Lh)[o];
    l = (ST == ST_DD) ? ws.Ll[o] : 0.f;
  }
}

// G = L0^T L0 (upper triangle), per-CTA partial sums in fixed order, written to ws.gpart
template <int ST>
__global__ void __launch_bounds__(kGramThreads) k_gram(Ws ws) {
  const int r0 = ws.st[ws.ctl->cur].hdr->r0;
  const int np = gram_pairs(r0);
  const int tid = threadIdx.x;
  __shared__ float th[kGramRows][kMaxCap + 1], tl[kGramRows][kMaxCap + 1];
  int pi[kGramMaxPairs], pk[kGramMaxPairs];
  Acc acc[kGramMaxPairs];
#pragma unroll
  for (int q = 0; q < kGramMaxPairs; ++q) {
    const int p = tid + kGramThreads * q;
    pi[q] = pk[q] = 0;
    if (p < np) gram_pair(p, r0, pi[q], pk[q]);
    acc[q] = acc_zero();
  }
  const int64_t ntiles = (ws.n + kGramRows - 1) / kGramRows;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * kGramRows;
    __syncthreads();
    for (int idx = tid; idx < kGramRows * r0; idx += kGramThreads) {
      const int t = idx / r0, c = idx % r0;
      float h = 0.f, l = 0.f;
      if (row0 + t < ws.n) load_basis<ST>(ws, (size_t)(row0 + t) * ws.ldg + c, h, l);
      th[t][c] = h;
      tl[t][c] = l;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGramMaxPairs; ++q) {
      if (tid + kGramThreads * q < np) {
        const int i = pi[q], k = pk[q];
        for (int t = 0; t < kGramRows; ++t) acc_fma(acc[q], th[t][i], tl[t][i], th[t][k], tl[t][k]);
      }
    }
  }
  const size_t stride = (size_t)ws.cap * (ws.cap + 1) / 2;
#pragma unroll
  for (int q = 0; q < kGramMaxPairs; ++q) {
    const int p = tid + kGramThreads * q;
    if (p < np) {
      const Acc a = acc_norm(acc[q]);
      ws.gpart[(size_t)blockIdx.x * stride + p] = make_float2(a.h, a.l);
    }
  }
}

// Matrices of the refinement in the scratch region (double-float pairs, column-major):
//   G cap x cap | T1 cap x rmax | C, R, T, V, W, M2: rmax x rmax | sig: rmax | perm: rmax ints
struct RefineScratch {
  float2 *G, *T1, *C, *R, *T, *V, *W, *M2, *sig;
  int* perm;
};

__device__ RefineScratch refine_scratch(const Ws& ws) {
  RefineScratch s;
  const size_t cap = ws.cap, rm = ws.rmax;
  float2* p = ws.rscr;
  s.G = p;
  p += cap * cap;
  s.T1 = p;
  p += cap * rm;
  s.C = p;
  p += rm * rm;
  s.R = p;
  p += rm * rm;
  s.T = p;
  p += rm * rm;
  s.V = p;
  p += rm * rm;
  s.W = p;
  p += rm * rm;
  s.M2 = p;
  p += rm * rm;
  s.sig = p;
  p += rm;
  s.perm = reinterpret_cast<int*>(p);
  return s;
}

__device__ __forceinline__ dd ld2(const float2* a, size_t i) { return dd{a[i].x, a[i].y}; }
__device__ __forceinline__ dd dzero() { return dd{0.f, 0.f}; }
__device__ __forceinline__ void st2(float2* a, size_t i, dd v) { a[i] = make_float2(v.h, v.l); }

__global__ void __launch_bounds__(kRefineThreads) k_refine(Ws ws, int nblocks) {
  Ctl* ctl = ws.ctl;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur], nx = ws.st[cur ^ 1];
  const int r = st.hdr->r, r0 = st.hdr->r0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (r < 1 || r0 < r) return;
  const int cap = ws.cap, rm = ws.rmax, qld = cap + 1;
  const RefineScratch S = refine_scratch(ws);
  __shared__ int bad;
  if (tid == 0) bad = 0;

  // G: sum the per-CTA partials in CTA order, mirror the upper triangle
  const int np = gram_pairs(r0);
  const size_t stride = (size_t)cap * (cap + 1) / 2;
  for (int p = tid; p < np; p += kRefineThreads) {
    dd s = dzero();
    for (int b = 0; b < nblocks; ++b) s = s + ld2(ws.gpart, (size_t)b * stride + p);
    int i, k;
    gram_pair(p, r0, i, k);
    st2(S.G, (size_t)k * cap + i, s);
    st2(S.G, (size_t)i * cap + k, s);
  }
  __syncthreads();
  // T1 = G Q  (r0 x r),  C = Q^T T1  (r x r)
  for (int o = tid; o < r0 * r; o += kRefineThreads) {
    const int a = o % r0, j = o / r0;
    dd s = dzero();
    for (int b = 0; b < r0; ++b) s = dd_fma(ld2(S.G, (size_t)b * cap + a), ld2(st.Q, (size_t)j * qld + b), s);
    st2(S.T1, (size_t)j * cap + a, s);
  }
  __syncthreads();
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, j = o / r;
    dd s = dzero();
    for (int a = 0; a < r0; ++a) s = dd_fma(ld2(st.Q, (size_t)i * qld + a), ld2(S.T1, (size_t)j * cap + a), s);
    st2(S.C, (size_t)j * rm + i, s);
  }
  __syncthreads();
  // Cholesky C = R^T R, column by column (R upper triangular, column-major)
  for (int o = tid; o < r * r; o += kRefineThreads) st2(S.R, (size_t)(o / r) * rm + (o % r), dzero());
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      dd d = ld2(S.C, (size_t)j * rm + j);
      for (int k = 0; k < j; ++k) {
        const dd rk = ld2(S.R, (size_t)j * rm + k);
        d = d - rk * rk;
      }
      if (!(d.h > 0.f) || !dd_isfinite(d)) {
        bad = 1;
        d = dd_of(1.f);
      }
      st2(S.R, (size_t)j * rm + j, dd_sqrt(d));
    }
    __syncthreads();
    const dd rjj = ld2(S.R, (size_t)j * rm + j);
    for (int i = j + 1 + tid; i < r; i += kRefineThreads) {
      dd s = ld2(S.C, (size_t)i * rm + j);
      for (int k = 0; k < j; ++k) s = s - ld2(S.R, (size_t)j * rm + k) * ld2(S.R, (size_t)i * rm + k);
      st2(S.R, (size_t)i * rm + j, dd_div(s, rjj));
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicOr(&ctl->status, DEV_NONFINITE);
    return;
  }
  // T = R diag(S), V = I
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, j = o / r;
    st2(S.T, (size_t)j * rm + i, ld2(S.R, (size_t)j * rm + i) * ld2(st.S, j));
    st2(S.V, (size_t)j * rm + i, dd_of(i == j ? 1.f : 0.f));
  }
  __syncthreads();
  // one-sided Jacobi on the columns of T (warp 0; rows split over the lanes)
  if (warp == 0) {
    const float tol = 4.f * 7.105427357601002e-15f;
    for (int sweep = 0; sweep < 12; ++sweep) {
      int rotated = 0;
      for (int p = 0; p < r - 1; ++p)
        for (int q = p + 1; q < r; ++q) {
          dd al = dzero(), be = dzero(), ga = dzero();
          for (int i = lane; i < r; i += 32) {
            const dd tp = ld2(S.T, (size_t)p * rm + i), tq = ld2(S.T, (size_t)q * rm + i);
            al = dd_fma(tp, tp, al);
            be = dd_fma(tq, tq, be);
            ga = dd_fma(tp, tq, ga);
          }
          al = dd_warp_sum(al);
          be = dd_warp_sum(be);
          ga = dd_warp_sum(ga);
          if (!(fabsf(ga.h) > tol * sqrtf(al.h) * sqrtf(be.h))) continue;
          ++rotated;
          // rotation zeroing the (p, q) inner product: zeta = (be - al) / (2 ga)
          const dd zeta = dd_div(be - al, ga * 2.f);
          const dd one = dd_of(1.f);
          const dd tt = dd_div(zeta.h >= 0.f ? one : -one, dd_abs(zeta) + dd_sqrt(one + zeta * zeta));
          const dd c = dd_div(one, dd_sqrt(one + tt * tt)), sn = c * tt;
          for (int i = lane; i < r; i += 32) {
            const dd tp = ld2(S.T, (size_t)p * rm + i), tq = ld2(S.T, (size_t)q * rm + i);
            st2(S.T, (size_t)p * rm + i, c * tp - sn * tq);
            st2(S.T, (size_t)q * rm + i, sn * tp + c * tq);
            const dd vp = ld2(S.V, (size_t)p * rm + i), vq = ld2(S.V, (size_t)q * rm + i);
            st2(S.V, (size_t)p * rm + i, c * vp - sn * vq);
            st2(S.V, (size_t)q * rm + i, sn * vp + c * vq);
          }
          __syncwarp();
        }
      if (rotated == 0) break;
    }
    // singular values (column norms) and their descending order
    for (int j = 0; j < r; ++j) {
      dd s = dzero();
      for (int i = lane; i < r; i += 32) {
        const dd t = ld2(S.T, (size_t)j * rm + i);
        s = dd_fma(t, t, s);
      }
      s = dd_warp_sum(s);
      if (lane == 0) st2(S.sig, j, dd_sqrt(s));
    }
    __syncwarp();
    if (lane == 0) {
      for (int j = 0; j < r; ++j) S.perm[j] = j;
      for (int j = 0; j < r; ++j) {
        int best = j;
        for (int k = j + 1; k < r; ++k)
          if (dd_gt(ld2(S.sig, S.perm[k]), ld2(S.sig, S.perm[best]))) best = k;
        const int t = S.perm[j];
        S.perm[j] = S.perm[best];
        S.perm[best] = t;
      }
    }
  }
  __syncthreads();
  // U_s = T Sigma^-1 (in place), then W = R^-1 U_s by back substitution (a thread per column)
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, j = o / r;
    st2(S.T, (size_t)j * rm + i, dd_div(ld2(S.T, (size_t)j * rm + i), ld2(S.sig, j)));
  }
  __syncthreads();
  for (int j = tid; j < r; j += kRefineThreads)
    for (int i = r - 1; i >= 0; --i) {
      dd s = ld2(S.T, (size_t)j * rm + i);
      for (int k = i + 1; k < r; ++k) s = s - ld2(S.R, (size_t)k * rm + i) * ld2(S.W, (size_t)j * rm + k);
      st2(S.W, (size_t)j * rm + i, dd_div(s, ld2(S.R, (size_t)i * rm + i)));
    }
  __syncthreads();
  // M2 = M V
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, j = o / r;
    dd s = dzero();
    for (int k = 0; k < r; ++k) s = dd_fma(ld2(st.M, (size_t)k * rm + i), ld2(S.V, (size_t)j * rm + k), s);
    st2(S.M2, (size_t)j * rm + i, s);
  }
  __syncthreads();
  // the new state, columns in descending order of Sigma
  for (int o = tid; o < r * r; o += kRefineThreads) {
    const int i = o % r, j = o / r;
    const int pi_ = S.perm[i], pj = S.perm[j];
    dd s = dzero();
    for (int k = 0; k < r; ++k) s = dd_fma(ld2(S.W, (size_t)pi_ * rm + k), ld2(S.M2, (size_t)pj * rm + k), s);
    st2(nx.M, (size_t)j * rm + i, s);
  }
  for (int o = tid; o < r0 * r; o += kRefineThreads) {
    const int a = o % r0, j = o / r0, pj = S.perm[j];
    dd s = dzero();
    for (int k = 0; k < r; ++k) s = dd_fma(ld2(st.Q, (size_t)k * qld + a), ld2(S.W, (size_t)pj * rm + k), s);
    st2(nx.Q, (size_t)j * qld + a, s);
  }
  for (int j = tid; j < r; j += kRefineThreads) {
    const int pj = S.perm[j];
    dd f = dzero(), l = dzero();
    for (int k = 0; k < r; ++k) {
      const dd v = ld2(S.V, (size_t)pj * rm + k);
      f = dd_fma(ld2(st.rf, k), v, f);
      l = dd_fma(ld2(st.rl, k), v, l);
    }
    st2(nx.rf, j, f);
    st2(nx.rl, j, l);
    nx.S[j] = S.sig[pj];
  }
  for (int i = tid; i < qld; i += kRefineThreads) {
    nx.a[i] = st.a[i];
    nx.ps[i] = st.ps[i];
  }
  if (tid == 0) *nx.hdr = *st.hdr;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    ctl->cur = cur ^ 1;
    ctl->eig_valid = 0;
  }
}

cudaError_t launch_refine(const Ws& ws, cudaStream_t s) {
  switch (ws.prec) {
    case ST_DD:
      k_gram<ST_DD><<<kGramCtas, kGramThreads, 0, s>>>(ws);
      break;
    case ST_F32:
      k_gram<ST_F32><<<kGramCtas, kGramThreads, 0, s>>>(ws);
      break;
    default:
      k_gram<ST_BF16><<<kGramCtas, kGramThreads, 0, s>>>(ws);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_refine<<<1, kRefineThreads, 0, s>>>(ws, kGramCtas);
  return cudaGetLastError();
}

}  // namespace odmd
