// Online DMD fed (x, y) snapshot pairs: the update of Sec. 2.3 for the hybrid loop of
// Sec. 2 (Fig. 1) in the reading where only FOM steps update the model.  Each FOM step
// gives a pair (x, y = FOM(x)); x is a DMD state whenever the step before it was accepted,
// so consecutive pairs need not share a snapshot, and the contiguous stream's shortcut
// j^T U^+ R = rho r_last^T does not hold.  The model keeps, in double-float rows of a
// workspace the caller owns:
//
//   L (N x r)  orthonormal basis of the kept part of X = [x_1 .. x_m] ~ L S R^T
//   P (N x r)  Y R, with Y = [y_1 .. y_m] paired column by column with X
//   S (r), M = L^T P (r x r), so that A~ = L^T Y R S^{-1} = M S^{-1}.
//
// An update is three passes over the rows and one small solve:
//
//   pass 1  p = L^T x, ||x||^2, x.y                                     (k_pr_proj)
//   pass 2  e = x - L p (stored), s = L^T e, q = P^T e, w = L^T y,
//           ||e||^2, e.y                                                (k_pr_resid)
//   small   rho = sqrt(||e||^2 - ||s||^2) (zero at or below tau max(sigma_1, ||x||));
//           K = [[diag S, p + s], [0, rho]] = U' S' V'^T by one-sided Jacobi, singular
//           values <= tau sigma'_1 dropped, at most r_max kept;
//           M' = U'^T [[M, w], [j^T P, j^T y]] V' with j = (e - L s) / rho, so that
//           j^T P = (q - M^T s) / rho and j^T y = (e.y - s.w) / rho        (k_pr_small)
//   pass 3  L <- [L, j] U',  P <- [P, y] V', row by row in place        (k_pr_rotate)
//
// The first pair with x != 0 starts L = x/||x||, S = ||x||, P = y, M = x.y/||x||.
// A prediction starts from a given state u: u(t) = L A~^t L^T u for integer t >= 0
// (k_pr_proj on u, k_pr_coef, k_pr_rollout).
//
// The passes give a warp one row at a time (lanes over columns), so the column sums stay in
// lane registers and only the row dot of pass 2 and pass 3 needs a warp reduction.  Sums are
// compensated (a float high word kept exact by two-sum, a float low word) and reduced in a
// fixed order: per CTA over its warps, then over CTAs by the last CTA to finish.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/odmd.h"
#include "dd.cuh"
#include "odmd_internal.cuh"

namespace odmd {
namespace pairs {

constexpr int kCols = kMaxR + 1;      // columns of [L, j] and [P, y]
constexpr int kThreads = 256;         // tall passes: 8 warps, a warp per row
constexpr int kWarps = kThreads / 32;
constexpr int kPart = 3 * kMaxR + 2;  // partial sums per CTA: three r-vectors, two scalars
constexpr int kS0 = 3 * kMaxR;        // offset of the scalars
constexpr int kMaxCtas = 512;
constexpr int kSmallThreads = 1024;   // small solve: 64 half-warps
constexpr int kLdT = kCols + 1;       // leading dimension of the small matrices in shared memory
constexpr int kPowThreads = 1024;
constexpr int kPowLd = kMaxR + 1;
constexpr int kRotThreads = 256;

enum : int { MODE_SKIP = 0, MODE_INIT = 1, MODE_ROTATE = 2 };
enum : int { PST_NONFINITE = 1, PST_JACOBI = 2, PST_NOMODEL = 4 };

struct Hdr {
  int r;          // committed rank
  int r_in;       // rank before the update in flight (columns pass 3 reads)
  int mode;       // what pass 3 does
  int status;     // PST_* bits, cleared by the host when read
  unsigned ticket;
  int pad[3];
};

struct PWs {
  int64_t n;
  int rmax, ld, grid;
  float tau_h, tau_l;
  Hdr* hdr;
  float2* L;      // n x ld, row-major
  float2* P;      // n x ld, row-major
  float2* xs;     // n: x (or u) as a float pair
  float2* ys;     // n: y as a float pair
  float2* e;      // n: residual e = x - L p of the update in flight
  float2* part;   // kMaxCtas x kPart
  float2* red1;   // kPart: pass 1 sums
  float2* red2;   // kPart: pass 2 sums
  float2* S;      // rmax
  float2* M;      // rmax x rmax, column-major (ld rmax)
  float2* U1;     // kCols x kCols, column-major (ld kCols): kept left singular vectors of K
  float2* V1;     // kCols x kCols: kept right singular vectors of K
  float2* sv;     // kCols: the second Gram-Schmidt coefficients s
  float2* aux;    // [0] 1/rho or 1/||x||
  float2* coef;   // kRollK x rmax: rollout coefficients, one column per horizon
};

__device__ __forceinline__ dd ld2(const float2* p, size_t i) { return dd_of(p[i]); }
__device__ __forceinline__ dd acc_to_dd(Acc a) {
  const Acc n = acc_norm(a);
  return dd{n.h, n.l};
}
__device__ __forceinline__ float2 acc_f2(Acc a) {
  const Acc n = acc_norm(a);
  return make_float2(n.h, n.l);
}
// warp sum of a compensated value, the same in every lane (lane 0's is broadcast)
__device__ __forceinline__ dd warp_sum_bcast(Acc a) {
  dd v = acc_to_dd(a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + dd{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
  return dd{__shfl_sync(0xffffffffu, v.h, 0), __shfl_sync(0xffffffffu, v.l, 0)};
}

// Per-CTA sums of kPart values (lanes hold up to three columns of each of three vectors,
// lane 0 the two scalars), then the last CTA adds the CTA partials in CTA order into out.
__device__ void reduce_parts(const PWs& w, Acc (&vec)[3][3], Acc (&scal)[2], int r, int nvec, float2* out) {
  __shared__ Acc sh[kWarps][kPart];
  __shared__ unsigned ticket;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int c = lane + 32 * i;
      if (c < kMaxR) sh[warp][v * kMaxR + c] = (v < nvec && c < r) ? vec[v][i] : acc_zero();
    }
  if (lane == 0) {
    sh[warp][kS0] = scal[0];
    sh[warp][kS0 + 1] = scal[1];
  }
  __syncthreads();
  float2* mine = w.part + (size_t)blockIdx.x * kPart;
  for (int v = tid; v < kPart; v += kThreads) {
    Acc a = acc_zero();
    for (int k = 0; k < kWarps; ++k) acc_add(a, sh[k][v].h, sh[k][v].l);
    mine[v] = acc_f2(a);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&w.hdr->ticket, 1u);
  __syncthreads();
  if (ticket != (unsigned)(gridDim.x - 1)) return;
  __threadfence();
  for (int v = tid; v < kPart; v += kThreads) {
    Acc a = acc_zero();
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const float2 f = __ldcg(w.part + (size_t)b * kPart + v);
      acc_add(a, f.x, f.y);
      if ((b & 31) == 31) a = acc_norm(a);
    }
    const float2 f = acc_f2(a);
    if (!isfinite(f.x) || !isfinite(f.y)) atomicOr(&w.hdr->status, PST_NONFINITE);
    out[v] = f;
  }
  if (tid == 0) w.hdr->ticket = 0u;
}

// Snapshots into the workspace as float pairs (y may be null).
__global__ void k_pr_ingest(PWs w, const double* x, const double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = x[i];
    const float ah = __double2float_rn(a);
    w.xs[i] = make_float2(ah, __double2float_rn(a - (double)ah));
    if (y) {
      const double b = y[i];
      const float bh = __double2float_rn(b);
      w.ys[i] = make_float2(bh, __double2float_rn(b - (double)bh));
    }
  }
}

// pass 1: p = L^T x (vector 0), ||x||^2 and x.y (scalars; x.y only when with_y)
__global__ void __launch_bounds__(kThreads) k_pr_proj(PWs w, int with_y) {
  const int lane = threadIdx.x & 31;
  const int r = w.hdr->r;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5), tw = (int64_t)gridDim.x * kWarps;
  Acc vec[3][3], scal[2] = {acc_zero(), acc_zero()};
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i) vec[v][i] = acc_zero();
  int cnt = 0;
  for (int64_t t = gw; t < w.n; t += tw) {
    const float2 x = w.xs[t];
    const float2* row = w.L + (size_t)t * w.ld;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int c = lane + 32 * i;
      if (c < r) {
        const float2 l = row[c];
        acc_fma(vec[0][i], l.x, l.y, x.x, x.y);
      }
    }
    if (lane == 0) {
      acc_fma(scal[0], x.x, x.y, x.x, x.y);
      if (with_y) {
        const float2 y = w.ys[t];
        acc_fma(scal[1], x.x, x.y, y.x, y.y);
      }
    }
    if ((++cnt & 31) == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) vec[0][i] = acc_norm(vec[0][i]);
      scal[0] = acc_norm(scal[0]);
      scal[1] = acc_norm(scal[1]);
    }
  }
  reduce_parts(w, vec, scal, r, 1, w.red1);
}

// pass 2: e = x - L p (stored); s = L^T e, q = P^T e, w = L^T y; ||e||^2, e.y
__global__ void __launch_bounds__(kThreads) k_pr_resid(PWs w) {
  const int lane = threadIdx.x & 31;
  const int r = w.hdr->r;
  if (r == 0) return;  // the first pair needs no residual
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5), tw = (int64_t)gridDim.x * kWarps;
  dd p[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int c = lane + 32 * i;
    p[i] = c < r ? ld2(w.red1, c) : dd{0.f, 0.f};
  }
  Acc vec[3][3], scal[2] = {acc_zero(), acc_zero()};
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i) vec[v][i] = acc_zero();
  int cnt = 0;
  for (int64_t t = gw; t < w.n; t += tw) {
    const float2* lrow = w.L + (size_t)t * w.ld;
    const float2* prow = w.P + (size_t)t * w.ld;
    float2 lv[3], pv[3];
    Acc d = acc_zero();
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int c = lane + 32 * i;
      lv[i] = c < r ? lrow[c] : make_float2(0.f, 0.f);
      pv[i] = c < r ? prow[c] : make_float2(0.f, 0.f);
      acc_fma(d, lv[i].x, lv[i].y, p[i].h, p[i].l);
    }
    const dd dot = warp_sum_bcast(d);
    const float2 x = w.xs[t], y = w.ys[t];
    Acc ea = Acc{x.x, x.y};
    acc_add(ea, -dot.h, -dot.l);
    const Acc e = acc_norm(ea);
    if (lane == 0) w.e[t] = make_float2(e.h, e.l);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      acc_fma(vec[0][i], lv[i].x, lv[i].y, e.h, e.l);
      acc_fma(vec[1][i], pv[i].x, pv[i].y, e.h, e.l);
      acc_fma(vec[2][i], lv[i].x, lv[i].y, y.x, y.y);
    }
    if (lane == 0) {
      acc_fma(scal[0], e.h, e.l, e.h, e.l);
      acc_fma(scal[1], e.h, e.l, y.x, y.y);
    }
    if ((++cnt & 31) == 0) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int i = 0; i < 3; ++i) vec[v][i] = acc_norm(vec[v][i]);
      scal[0] = acc_norm(scal[0]);
      scal[1] = acc_norm(scal[1]);
    }
  }
  reduce_parts(w, vec, scal, r, 3, w.red2);
}

// ------------------------------------------------------------------ small solve (one CTA)
struct SmallSmem {
  float2 T[kCols * kLdT];   // K, then K V (column j = sigma_j u_j); column-major
  float2 V[kCols * kLdT];   // right rotations
  float2 BV[kCols * kLdT];  // [[M, w], [j^T P, j^T y]] V'
  float2 sig[kCols], s[kCols], jp[kCols];
  int perm[kCols];
  int rot[32];
  int keep;
  int bad;
};

__device__ __forceinline__ dd half_sum16(dd a, unsigned mask) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) a = a + dd{__shfl_xor_sync(mask, a.h, o), __shfl_xor_sync(mask, a.l, o)};
  return a;
}

__global__ void __launch_bounds__(kSmallThreads) k_pr_small(PWs w) {
  extern __shared__ __align__(16) unsigned char pr_small_raw[];
  SmallSmem& sm = *reinterpret_cast<SmallSmem*>(pr_small_raw);
  const int tid = threadIdx.x;
  Hdr* hdr = w.hdr;
  const int r = hdr->r, rm = w.rmax;
  const dd tau = dd{w.tau_h, w.tau_l};
  if (r == 0) {
    // first pair with a nonzero x starts the model; a zero x adds nothing
    if (tid == 0) {
      const dd xx = ld2(w.red1, kS0), xy = ld2(w.red1, kS0 + 1);
      hdr->r_in = 0;
      if (!(xx.h > 0.f)) {
        hdr->mode = MODE_SKIP;
      } else {
        const dd nx = dd_sqrt(xx);
        w.S[0] = f2_of(nx);
        w.M[0] = f2_of(dd_div(xy, nx));
        w.aux[0] = f2_of(dd_div(dd_of(1.f), nx));
        hdr->r = 1;
        hdr->mode = MODE_INIT;
        if (!dd_isfinite(nx) || !dd_isfinite(xy)) atomicOr(&hdr->status, PST_NONFINITE);
      }
    }
    return;
  }
  const int n = r + 1;
  if (tid == 0) {
    sm.bad = 0;
    sm.keep = 0;
  }
  if (tid < 32) sm.rot[tid] = 0;
  for (int i = tid; i < r; i += kSmallThreads) sm.s[i] = w.red2[i];
  // ||s||^2 by one warp (r <= 64)
  __shared__ float2 rho_sh;
  if (tid < 32) {
    Acc a = acc_zero();
    for (int i = tid; i < r; i += 32) {
      const float2 si = w.red2[i];
      acc_fma(a, si.x, si.y, si.x, si.y);
    }
    const dd ss = warp_sum_bcast(a);
    if (tid == 0) {
      const dd ee = ld2(w.red2, kS0), xx = ld2(w.red1, kS0);
      dd rho2 = ee - ss;
      if (!(rho2.h > 0.f)) rho2 = dd{0.f, 0.f};
      dd rho = dd_sqrt(rho2);
      const dd thr = tau * dd_max(ld2(w.S, 0), dd_sqrt(xx));
      if (!dd_gt(rho, thr)) rho = dd{0.f, 0.f};
      rho_sh = f2_of(rho);
    }
  }
  __syncthreads();
  const dd rho = dd_of(rho_sh);
  // T = K = [[diag S, p + s], [0, rho]], V = I
  for (int o = tid; o < n * n; o += kSmallThreads) {
    const int i = o % n, c = o / n;
    dd v = dd{0.f, 0.f};
    if (c < r) {
      if (i == c) v = ld2(w.S, c);
    } else {
      v = i < r ? ld2(w.red1, i) + ld2(w.red2, i) : rho;
    }
    sm.T[c * kLdT + i] = f2_of(v);
    sm.V[c * kLdT + i] = make_float2(i == c ? 1.f : 0.f, 0.f);
  }
  // ||K||_F^2 (invariant under the rotations below), for the test of negligible columns
  __shared__ float fro2_sh;
  if (tid < 32) {
    float f = 0.f;
    for (int o = tid; o < n * n; o += 32) {
      const float t = sm.T[(o / n) * kLdT + o % n].x;
      f = fmaf(t, t, f);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
    if (tid == 0) fro2_sh = f;
  }
  __syncthreads();

  // One-sided Jacobi on the columns of T, round-robin: each round rotates m/2 disjoint column
  // pairs at once, a half-warp per pair; a sweep is m - 1 rounds; stop after a sweep that
  // rotates nothing (at most 24 sweeps, else the update is refused).  A pair is left alone
  // when its columns are orthogonal to working accuracy, or when one of them has shrunk to
  // the rounding level of ||K||_F: a pair that adds no new direction (rho = 0) makes K
  // singular, one column then tends to zero, and the relative test alone would keep
  // rotating its rounding noise (its singular value is truncated in any case).
  const int m = n + (n & 1);
  const int hw = tid >> 4, hl = tid & 15;
  const unsigned mask = (tid & 16) ? 0xffff0000u : 0x0000ffffu;
  const float tol = 4.f * 7.105427357601002e-15f;
  const float negl = fro2_sh * (16.f * 7.105427357601002e-15f) * (16.f * 7.105427357601002e-15f);
  for (int sweep = 0; sweep < 24; ++sweep) {
    for (int k = 0; k < m - 1; ++k) {
      for (int pi = hw; pi < m / 2; pi += kSmallThreads / 16) {
        int a = k, b = m - 1;
        if (pi > 0) {
          a = (k + pi) % (m - 1);
          b = (k - pi + m - 1) % (m - 1);
        }
        const int pc = a < b ? a : b, qc = a < b ? b : a;
        if (qc >= n) continue;  // the dummy column of an odd n
        Acc al = acc_zero(), be = acc_zero(), ga = acc_zero();
        for (int i = hl; i < n; i += 16) {
          const float2 tp = sm.T[pc * kLdT + i], tq = sm.T[qc * kLdT + i];
          acc_fma(al, tp.x, tp.y, tp.x, tp.y);
          acc_fma(be, tq.x, tq.y, tq.x, tq.y);
          acc_fma(ga, tp.x, tp.y, tq.x, tq.y);
        }
        const dd A = half_sum16(acc_to_dd(al), mask), B = half_sum16(acc_to_dd(be), mask),
                 G = half_sum16(acc_to_dd(ga), mask);
        if (!(fabsf(G.h) > tol * sqrtf(A.h) * sqrtf(B.h)) || A.h <= negl || B.h <= negl) continue;
        if (hl == 0) atomicAdd(&sm.rot[sweep & 31], 1);
        const dd diff = B - A;
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
        for (int i = hl; i < n; i += 16) {
          const dd tp = dd_of(sm.T[pc * kLdT + i]), tq = dd_of(sm.T[qc * kLdT + i]);
          sm.T[pc * kLdT + i] = f2_of(c * tp - s * tq);
          sm.T[qc * kLdT + i] = f2_of(s * tp + c * tq);
          const dd vp = dd_of(sm.V[pc * kLdT + i]), vq = dd_of(sm.V[qc * kLdT + i]);
          sm.V[pc * kLdT + i] = f2_of(c * vp - s * vq);
          sm.V[qc * kLdT + i] = f2_of(s * vp + c * vq);
        }
      }
      __syncthreads();
    }
    const int rotated = sm.rot[sweep & 31];
    __syncthreads();
    if (rotated == 0) break;
    if (tid == 0) sm.rot[(sweep + 1) & 31] = 0;
    __syncthreads();
    if (sweep == 23) {
      if (tid == 0) sm.bad = 1;
    }
  }
  // singular values: column norms, a half-warp per column
  for (int j = hw; j < n; j += kSmallThreads / 16) {
    Acc a = acc_zero();
    for (int i = hl; i < n; i += 16) {
      const float2 t = sm.T[j * kLdT + i];
      acc_fma(a, t.x, t.y, t.x, t.y);
    }
    const dd nrm = dd_sqrt(half_sum16(acc_to_dd(a), mask));
    if (hl == 0) {
      sm.sig[j] = f2_of(nrm);
      if (!dd_isfinite(nrm)) sm.bad = 1;
    }
  }
  __syncthreads();
  // descending order by rank count; keep sigma > tau sigma_1, at most r_max, at least one
  for (int j = tid; j < n; j += kSmallThreads) {
    const dd sj = dd_of(sm.sig[j]);
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const dd sk = dd_of(sm.sig[k]);
      rank += dd_gt(sk, sj) || (!dd_lt(sk, sj) && k < j);
    }
    sm.perm[rank] = j;
  }
  __syncthreads();
  if (tid == 0) {
    const dd s1 = dd_of(sm.sig[sm.perm[0]]);
    const dd lim = tau * s1;
    int keep = 0;
    for (int j = 0; j < n; ++j)
      if (dd_gt(dd_of(sm.sig[sm.perm[j]]), lim)) ++keep;
    if (keep > rm) keep = rm;
    if (keep < 1) keep = 1;
    if (!(s1.h > 0.f)) sm.bad = 1;
    sm.keep = keep;
  }
  __syncthreads();
  if (sm.bad) {
    if (tid == 0) {
      atomicOr(&hdr->status, PST_JACOBI);
      hdr->mode = MODE_SKIP;  // the committed model stays as it was
      hdr->r_in = r;
    }
    return;
  }
  const int keep = sm.keep;
  // U' = T[:, perm] / sigma, V' = V[:, perm] (kept columns) into global memory
  for (int o = tid; o < n * keep; o += kSmallThreads) {
    const int i = o % n, j = o / n, pj = sm.perm[j];
    w.U1[(size_t)j * kCols + i] = f2_of(dd_div(dd_of(sm.T[pj * kLdT + i]), dd_of(sm.sig[pj])));
    w.V1[(size_t)j * kCols + i] = sm.V[pj * kLdT + i];
  }
  // j^T P = (q - M^T s) / rho (k < r), j^T y = (e.y - s.w) / rho (zero when rho = 0)
  const dd inv_rho = rho.h > 0.f ? dd_div(dd_of(1.f), rho) : dd{0.f, 0.f};
  for (int k = tid; k < n; k += kSmallThreads) {
    Acc a = acc_zero();
    if (k < r) {
      const float2 q = w.red2[kMaxR + k];
      a = Acc{q.x, q.y};
      for (int mm = 0; mm < r; ++mm) {
        const float2 s = sm.s[mm], mk = w.M[(size_t)k * rm + mm];
        acc_fma(a, -s.x, -s.y, mk.x, mk.y);
      }
    } else {
      const float2 ey = w.red2[kS0 + 1];
      a = Acc{ey.x, ey.y};
      for (int mm = 0; mm < r; ++mm) {
        const float2 s = sm.s[mm], wv = w.red2[2 * kMaxR + mm];
        acc_fma(a, -s.x, -s.y, wv.x, wv.y);
      }
    }
    sm.jp[k] = f2_of(acc_to_dd(a) * inv_rho);
  }
  __syncthreads();
  // BV = B V' with B = [[M, w], [j^T P, j^T y]] (n x keep)
  for (int o = tid; o < n * keep; o += kSmallThreads) {
    const int i = o % n, j = o / n;
    Acc a = acc_zero();
    for (int k = 0; k < n; ++k) {
      float2 b;
      if (i < r)
        b = k < r ? w.M[(size_t)k * rm + i] : w.red2[2 * kMaxR + i];
      else
        b = sm.jp[k];
      const float2 v = w.V1[(size_t)j * kCols + k];
      acc_fma(a, b.x, b.y, v.x, v.y);
    }
    sm.BV[j * kLdT + i] = acc_f2(a);
  }
  __syncthreads();
  // M' = U'^T BV (keep x keep); all reads of the old M are done
  for (int o = tid; o < keep * keep; o += kSmallThreads) {
    const int a_ = o % keep, j = o / keep;
    Acc a = acc_zero();
    for (int i = 0; i < n; ++i) {
      const float2 u = w.U1[(size_t)a_ * kCols + i], b = sm.BV[j * kLdT + i];
      acc_fma(a, u.x, u.y, b.x, b.y);
    }
    const float2 f = acc_f2(a);
    if (!isfinite(f.x)) atomicOr(&hdr->status, PST_NONFINITE);
    w.M[(size_t)j * rm + a_] = f;
  }
  for (int j = tid; j < keep; j += kSmallThreads) w.S[j] = sm.sig[sm.perm[j]];
  for (int i = tid; i < r; i += kSmallThreads) w.sv[i] = sm.s[i];
  if (tid == 0) {
    w.aux[0] = f2_of(inv_rho);
    hdr->r_in = r;
    hdr->r = keep;
    hdr->mode = MODE_ROTATE;
  }
}

// pass 3: L <- [L, j] U', P <- [P, y] V' (or the first pair's L = x/||x||, P = y)
__global__ void __launch_bounds__(kRotThreads) k_pr_rotate(PWs w) {
  const int mode = w.hdr->mode;
  if (mode == MODE_SKIP) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kRW = kRotThreads / 32;
  if (mode == MODE_INIT) {
    const dd inv = dd_of(w.aux[0]);
    for (int64_t t = (int64_t)blockIdx.x * kRotThreads + tid; t < w.n; t += (int64_t)gridDim.x * kRotThreads) {
      w.L[(size_t)t * w.ld] = f2_of(dd_of(w.xs[t]) * inv);
      w.P[(size_t)t * w.ld] = w.ys[t];
    }
    return;
  }
  const int r_in = w.hdr->r_in, keep = w.hdr->r, n = r_in + 1;
  extern __shared__ __align__(16) unsigned char pr_rot_raw[];
  float2* U = reinterpret_cast<float2*>(pr_rot_raw);  // n x keep, column-major ld kCols
  float2* V = U + kCols * kMaxR;
  float2* rows = V + kCols * kMaxR;                    // per warp: [L row | j], [P row | y]
  __shared__ float2 s_sh[kCols];
  for (int o = tid; o < n * keep; o += kRotThreads) {
    const int i = o % n, j = o / n;
    U[j * kCols + i] = w.U1[(size_t)j * kCols + i];
    V[j * kCols + i] = w.V1[(size_t)j * kCols + i];
  }
  for (int i = tid; i < r_in; i += kRotThreads) s_sh[i] = w.sv[i];
  __syncthreads();
  const dd inv_rho = dd_of(w.aux[0]);
  float2* lr = rows + (size_t)warp * 2 * kCols;
  float2* pr = lr + kCols;
  const int64_t gw = (int64_t)blockIdx.x * kRW + warp, tw = (int64_t)gridDim.x * kRW;
  for (int64_t t = gw; t < w.n; t += tw) {
    float2* lrow = w.L + (size_t)t * w.ld;
    float2* prow = w.P + (size_t)t * w.ld;
    Acc d = acc_zero();
    for (int c = lane; c < r_in; c += 32) {
      const float2 l = lrow[c], s = s_sh[c];
      lr[c] = l;
      pr[c] = prow[c];
      acc_fma(d, l.x, l.y, s.x, s.y);
    }
    const dd dot = warp_sum_bcast(d);
    if (lane == 0) {
      Acc j = Acc{w.e[t].x, w.e[t].y};
      acc_add(j, -dot.h, -dot.l);
      lr[r_in] = f2_of(acc_to_dd(j) * inv_rho);
      pr[r_in] = w.ys[t];
    }
    __syncwarp();
    for (int c = lane; c < keep; c += 32) {
      Acc a = acc_zero(), b = acc_zero();
      for (int k = 0; k < n; ++k) {
        const float2 l = lr[k], u = U[c * kCols + k], p = pr[k], v = V[c * kCols + k];
        acc_fma(a, l.x, l.y, u.x, u.y);
        acc_fma(b, p.x, p.y, v.x, v.y);
      }
      lrow[c] = acc_f2(a);
      prow[c] = acc_f2(b);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ prediction
struct PowSmem {
  float2 A[kMaxR * kPowLd];  // A~ = M S^{-1}, row-major
  float2 Pw[kMaxR * kPowLd];
  float2 Tm[kMaxR * kPowLd];
  float2 v[2][kMaxR];
};

struct Horizons {
  double t[kRollK];
  int order[kRollK];  // ascending
};

__device__ void pow_mv(const float2* A, const float2* x, float2* y, int r) {
  for (int i = threadIdx.x; i < r; i += kPowThreads) {
    Acc a = acc_zero();
    for (int k = 0; k < r; ++k) {
      const float2 m = A[i * kPowLd + k], xv = x[k];
      acc_fma(a, m.x, m.y, xv.x, xv.y);
    }
    y[i] = acc_f2(a);
  }
}

// coef[:, j] = A~^{t_j} L^T u (L^T u from pass 1 in red1), horizons taken in ascending order
__global__ void __launch_bounds__(kPowThreads) k_pr_coef(PWs w, Horizons hz, int k) {
  extern __shared__ __align__(16) unsigned char pr_pow_raw[];
  PowSmem& S = *reinterpret_cast<PowSmem*>(pr_pow_raw);
  const int r = w.hdr->r, rm = w.rmax, tid = threadIdx.x;
  if (r == 0) {
    if (tid == 0) atomicOr(&w.hdr->status, PST_NOMODEL);
    return;
  }
  for (int o = tid; o < r * r; o += kPowThreads) {
    const int i = o / r, c = o % r;
    S.A[i * kPowLd + c] = f2_of(dd_div(ld2(w.M, (size_t)c * rm + i), ld2(w.S, c)));
  }
  for (int i = tid; i < r; i += kPowThreads) S.v[0][i] = w.red1[i];
  __syncthreads();
  int cur = 0;
  long long tcur = 0;
  for (int q = 0; q < k; ++q) {
    const int j = hz.order[q];
    long long d = (long long)hz.t[j] - tcur;
    tcur += d;
    if (d <= 8) {
      for (; d > 0; --d) {
        pow_mv(S.A, S.v[cur], S.v[cur ^ 1], r);
        cur ^= 1;
        __syncthreads();
      }
    } else {
      for (int o = tid; o < r * r; o += kPowThreads) S.Pw[(o / r) * kPowLd + o % r] = S.A[(o / r) * kPowLd + o % r];
      __syncthreads();
      while (d > 0) {
        if (d & 1) {
          pow_mv(S.Pw, S.v[cur], S.v[cur ^ 1], r);
          cur ^= 1;
          __syncthreads();
        }
        d >>= 1;
        if (d) {
          for (int o = tid; o < r * r; o += kPowThreads) {
            const int i = o / r, c = o % r;
            Acc a = acc_zero();
            for (int l = 0; l < r; ++l) {
              const float2 x = S.Pw[i * kPowLd + l], y = S.Pw[l * kPowLd + c];
              acc_fma(a, x.x, x.y, y.x, y.y);
            }
            S.Tm[i * kPowLd + c] = acc_f2(a);
          }
          __syncthreads();
          for (int o = tid; o < r * r; o += kPowThreads) S.Pw[(o / r) * kPowLd + o % r] = S.Tm[(o / r) * kPowLd + o % r];
          __syncthreads();
        }
      }
    }
    for (int i = tid; i < r; i += kPowThreads) w.coef[(size_t)j * rm + i] = S.v[cur][i];
    __syncthreads();
  }
}

// out[:, j] = L coef[:, j] for j < k, a thread per row
__global__ void k_pr_rollout(PWs w, int k, double* out, int64_t ld) {
  __shared__ float2 c[kRollK * kMaxR];
  const int r = w.hdr->r, rm = w.rmax;
  for (int o = threadIdx.x; o < k * r; o += blockDim.x) {
    const int i = o % r, j = o / r;
    c[j * kMaxR + i] = w.coef[(size_t)j * rm + i];
  }
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < w.n; t += (int64_t)gridDim.x * blockDim.x) {
    const float2* row = w.L + (size_t)t * w.ld;
    for (int j = 0; j < k; ++j) {
      Acc a = acc_zero();
      for (int i = 0; i < r; ++i) {
        const float2 l = row[i], cv = c[j * kMaxR + i];
        acc_fma(a, l.x, l.y, cv.x, cv.y);
      }
      const Acc f = acc_norm(a);
      out[(size_t)j * ld + t] = (double)f.h + (double)f.l;
    }
  }
}

// ||r||^2 and ||b||^2 in double (the relative residual of the hybrid step), per-CTA partials
// in part, then the last CTA sums them in CTA order into aux (as doubles, bytes 32..47)
__global__ void __launch_bounds__(kThreads) k_pr_norms(PWs w, const double* r, const double* b) {
  __shared__ double sh[2][kWarps];
  __shared__ unsigned ticket;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double sr = 0.0, sb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + tid; i < w.n; i += (int64_t)gridDim.x * kThreads) {
    sr = fma(r[i], r[i], sr);
    sb = fma(b[i], b[i], sb);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if (lane == 0) {
    sh[0][warp] = sr;
    sh[1][warp] = sb;
  }
  __syncthreads();
  double* mine = reinterpret_cast<double*>(w.part + (size_t)blockIdx.x * kPart);
  if (tid == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < kWarps; ++k) {
      a += sh[0][k];
      c += sh[1][k];
    }
    mine[0] = a;
    mine[1] = c;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&w.hdr->ticket, 1u);
  __syncthreads();
  if (ticket != (unsigned)(gridDim.x - 1)) return;
  __threadfence();
  if (tid == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) {
      const double* pk = reinterpret_cast<const double*>(w.part + (size_t)k * kPart);
      a += __ldcg(pk);
      c += __ldcg(pk + 1);
    }
    double* out = reinterpret_cast<double*>(w.aux + 4);
    out[0] = a;
    out[1] = c;
    w.hdr->ticket = 0u;
  }
}

}  // namespace pairs
}  // namespace odmd

// ------------------------------------------------------------------ host side
using namespace odmd::pairs;
using odmd::kMaxR;
using odmd::kRollK;

struct odmd_pairs_instance {
  PWs w;
  cudaStream_t stream;
  int sms;
  int64_t pairs;
  std::string err;
};

namespace {

thread_local std::string g_pairs_err;

odmd_status pfail(odmd_pairs_t h, odmd_status s, const std::string& m) {
  if (h)
    h->err = m;
  else
    g_pairs_err = m;
  return s;
}

#define PCK(h, call, where)                                                                 \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return pfail(h, ODMD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct PLayout {
  size_t hdr, part, red1, red2, S, M, U1, V1, sv, aux, coef, xs, ys, e, L, P, total;
};

PLayout playout(int64_t n, int rmax) {
  PLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = up256(o + b);
    return at;
  };
  const size_t f2 = sizeof(float2);
  const size_t ld = (size_t)rmax + 1;
  L.hdr = take(sizeof(Hdr));
  L.part = take((size_t)kMaxCtas * kPart * f2);
  L.red1 = take((size_t)kPart * f2);
  L.red2 = take((size_t)kPart * f2);
  L.S = take((size_t)rmax * f2);
  L.M = take((size_t)rmax * rmax * f2);
  L.U1 = take((size_t)kCols * kCols * f2);
  L.V1 = take((size_t)kCols * kCols * f2);
  L.sv = take((size_t)kCols * f2);
  L.aux = take(8 * f2);
  L.coef = take((size_t)kRollK * rmax * f2);
  L.xs = take((size_t)n * f2);
  L.ys = take((size_t)n * f2);
  L.e = take((size_t)n * f2);
  L.L = take((size_t)n * ld * f2);
  L.P = take((size_t)n * ld * f2);
  L.total = o;
  return L;
}

odmd_status check_args(int64_t n, int32_t r_max, std::string& why) {
  if (n < 1 || n > 2147483647LL) {
    why = "n must be in [1, 2^31 - 1]";
    return ODMD_ERR_ARG;
  }
  if (r_max < 1 || r_max > kMaxR) {
    why = "r_max must be in [1, 64]";
    return ODMD_ERR_ARG;
  }
  return ODMD_OK;
}

odmd_status read_status(odmd_pairs_t h) {
  Hdr hd;
  PCK(h, cudaMemcpyAsync(&hd, h->w.hdr, sizeof hd, cudaMemcpyDeviceToHost, h->stream), "read status");
  PCK(h, cudaStreamSynchronize(h->stream), "sync");
  if (hd.status) {
    const int zero = 0;
    PCK(h, cudaMemcpy(&h->w.hdr->status, &zero, sizeof zero, cudaMemcpyHostToDevice), "clear status");
    if (hd.status & PST_NOMODEL) return pfail(h, ODMD_ERR_STATE, "no model yet: every x so far was zero");
    if (hd.status & PST_JACOBI) return pfail(h, ODMD_ERR_NUMERIC, "core SVD did not converge; the update was not applied");
    return pfail(h, ODMD_ERR_NUMERIC, "non-finite value in an update or prediction");
  }
  return ODMD_OK;
}

}  // namespace

extern "C" {

odmd_status odmd_pairs_footprint(int64_t n, int32_t r_max, size_t* device_bytes) {
  std::string why;
  if (odmd_status s = check_args(n, r_max, why)) return pfail(nullptr, s, why);
  if (!device_bytes) return pfail(nullptr, ODMD_ERR_ARG, "device_bytes is NULL");
  *device_bytes = playout(n, r_max).total;
  return ODMD_OK;
}

odmd_status odmd_pairs_create(int64_t n, int32_t r_max, double trunc_tol, void* workspace_dev, size_t bytes,
                              void* stream, odmd_pairs_t* out) {
  std::string why;
  if (odmd_status s = check_args(n, r_max, why)) return pfail(nullptr, s, why);
  if (!out) return pfail(nullptr, ODMD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!(trunc_tol >= 1e-13 && trunc_tol < 1.0)) return pfail(nullptr, ODMD_ERR_ARG, "trunc_tol must be in [1e-13, 1)");
  if (!workspace_dev) return pfail(nullptr, ODMD_ERR_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0)
    return pfail(nullptr, ODMD_ERR_ARG, "workspace must be 256-byte aligned");
  const PLayout L = playout(n, r_max);
  if (bytes < L.total) return pfail(nullptr, ODMD_ERR_NOMEM, "workspace smaller than odmd_pairs_footprint()");
  odmd_pairs_instance* h = new (std::nothrow) odmd_pairs_instance();
  if (!h) return pfail(nullptr, ODMD_ERR_NOMEM, "host allocation failed");
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->pairs = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pr_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallSmem));
  const int rot_smem = (int)((2 * (size_t)kCols * kMaxR + (size_t)(kRotThreads / 32) * 2 * kCols) * sizeof(float2));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pr_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, rot_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pr_coef, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PowSmem));
  unsigned char* base = static_cast<unsigned char*>(workspace_dev);
  if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, L.total, h->stream);
  if (e != cudaSuccess) {
    std::string m = std::string("create: ") + cudaGetErrorString(e);
    delete h;
    return pfail(nullptr, ODMD_ERR_CUDA, m);
  }
  PWs& w = h->w;
  w.n = n;
  w.rmax = r_max;
  w.ld = r_max + 1;
  const int64_t warps_needed = (n + 7) / 8;
  int grid = h->sms > 0 ? 2 * h->sms : 1;
  if (grid > kMaxCtas) grid = kMaxCtas;
  if ((int64_t)grid > warps_needed) grid = (int)warps_needed;
  w.grid = grid < 1 ? 1 : grid;
  const float th = (float)trunc_tol;
  w.tau_h = th;
  w.tau_l = (float)(trunc_tol - (double)th);
  w.hdr = reinterpret_cast<Hdr*>(base + L.hdr);
  w.part = reinterpret_cast<float2*>(base + L.part);
  w.red1 = reinterpret_cast<float2*>(base + L.red1);
  w.red2 = reinterpret_cast<float2*>(base + L.red2);
  w.S = reinterpret_cast<float2*>(base + L.S);
  w.M = reinterpret_cast<float2*>(base + L.M);
  w.U1 = reinterpret_cast<float2*>(base + L.U1);
  w.V1 = reinterpret_cast<float2*>(base + L.V1);
  w.sv = reinterpret_cast<float2*>(base + L.sv);
  w.aux = reinterpret_cast<float2*>(base + L.aux);
  w.coef = reinterpret_cast<float2*>(base + L.coef);
  w.xs = reinterpret_cast<float2*>(base + L.xs);
  w.ys = reinterpret_cast<float2*>(base + L.ys);
  w.e = reinterpret_cast<float2*>(base + L.e);
  w.L = reinterpret_cast<float2*>(base + L.L);
  w.P = reinterpret_cast<float2*>(base + L.P);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::string m = std::string("create: ") + cudaGetErrorString(e);
    delete h;
    return pfail(nullptr, ODMD_ERR_CUDA, m);
  }
  *out = h;
  return ODMD_OK;
}

odmd_status odmd_pairs_update(odmd_pairs_t h, const double* x_dev, const double* y_dev) {
  if (!h) return pfail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (!x_dev || !y_dev) return pfail(h, ODMD_ERR_ARG, "x and y must not be NULL");
  const PWs& w = h->w;
  const int ig = (int)((w.n + 255) / 256 < 4 * (int64_t)h->sms ? (w.n + 255) / 256 : 4 * (int64_t)h->sms);
  k_pr_ingest<<<ig < 1 ? 1 : ig, 256, 0, h->stream>>>(w, x_dev, y_dev);
  k_pr_proj<<<w.grid, kThreads, 0, h->stream>>>(w, 1);
  k_pr_resid<<<w.grid, kThreads, 0, h->stream>>>(w);
  k_pr_small<<<1, kSmallThreads, sizeof(SmallSmem), h->stream>>>(w);
  const int rot_smem = (int)((2 * (size_t)kCols * kMaxR + (size_t)(kRotThreads / 32) * 2 * kCols) * sizeof(float2));
  k_pr_rotate<<<w.grid, kRotThreads, rot_smem, h->stream>>>(w);
  PCK(h, cudaGetLastError(), "update launch");
  h->pairs += 1;
  return ODMD_OK;
}

odmd_status odmd_pairs_predict(odmd_pairs_t h, const double* u_dev, const double* t_host, int32_t k, double* out_dev,
                               int64_t ld) {
  if (!h) return pfail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (k < 0 || k > kRollK) return pfail(h, ODMD_ERR_ARG, "k must be in [0, 64]");
  if (k == 0) return ODMD_OK;
  if (!u_dev || !t_host || !out_dev) return pfail(h, ODMD_ERR_ARG, "u, t and out must not be NULL");
  if (ld < h->w.n) return pfail(h, ODMD_ERR_ARG, "ld < n");
  Horizons hz{};
  for (int i = 0; i < k; ++i) {
    const double t = t_host[i];
    if (!(t >= 0.0) || !(t <= 1e12) || t != std::floor(t))
      return pfail(h, ODMD_ERR_ARG, "t must be an integer in [0, 1e12]");
    hz.t[i] = t;
    hz.order[i] = i;
  }
  for (int i = 1; i < k; ++i) {  // insertion sort of the horizon order
    const int v = hz.order[i];
    int b = i - 1;
    while (b >= 0 && hz.t[hz.order[b]] > hz.t[v]) {
      hz.order[b + 1] = hz.order[b];
      --b;
    }
    hz.order[b + 1] = v;
  }
  const PWs& w = h->w;
  const int ig = (int)((w.n + 255) / 256 < 4 * (int64_t)h->sms ? (w.n + 255) / 256 : 4 * (int64_t)h->sms);
  k_pr_ingest<<<ig < 1 ? 1 : ig, 256, 0, h->stream>>>(w, u_dev, nullptr);
  k_pr_proj<<<w.grid, kThreads, 0, h->stream>>>(w, 0);
  k_pr_coef<<<1, kPowThreads, sizeof(PowSmem), h->stream>>>(w, hz, k);
  k_pr_rollout<<<ig < 1 ? 1 : ig, 256, 0, h->stream>>>(w, k, out_dev, ld);
  PCK(h, cudaGetLastError(), "predict launch");
  return read_status(h);
}

odmd_status odmd_pairs_get_singular_values(odmd_pairs_t h, double* s_host, int32_t cap, int32_t* r) {
  if (!h) return pfail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (!r || (cap > 0 && !s_host)) return pfail(h, ODMD_ERR_ARG, "r (and s when cap > 0) must not be NULL");
  if (odmd_status s = read_status(h)) return s;
  Hdr hd;
  PCK(h, cudaMemcpy(&hd, h->w.hdr, sizeof hd, cudaMemcpyDeviceToHost), "read rank");
  *r = hd.r;
  const int m = hd.r < cap ? hd.r : cap;
  if (m > 0) {
    float2 buf[kMaxR];
    PCK(h, cudaMemcpy(buf, h->w.S, (size_t)m * sizeof(float2), cudaMemcpyDeviceToHost), "read S");
    for (int i = 0; i < m; ++i) s_host[i] = (double)buf[i].x + (double)buf[i].y;
  }
  return ODMD_OK;
}

odmd_status odmd_pairs_get_count(odmd_pairs_t h, int64_t* pairs) {
  if (!h || !pairs) return pfail(h, ODMD_ERR_ARG, "handle and pairs must not be NULL");
  *pairs = h->pairs;
  return ODMD_OK;
}

odmd_status odmd_pairs_hybrid_step_residual(odmd_pairs_t h, odmd_residual_fn residual, odmd_fom_fn fom, void* user,
                                            double tol, int64_t step, double* state_dev, double* next_dev,
                                            double* r_dev, double* b_dev, int32_t* accepted, double* rel_res) {
  if (!h) return pfail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (!residual || !fom) return pfail(h, ODMD_ERR_ARG, "the residual and FOM callbacks must not be NULL");
  if (!state_dev || !next_dev || !r_dev || !b_dev) return pfail(h, ODMD_ERR_ARG, "state, next, r and b must not be NULL");
  const double* bufs[4] = {state_dev, next_dev, r_dev, b_dev};
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (bufs[i] == bufs[j]) return pfail(h, ODMD_ERR_ARG, "state, next, r and b must be four different buffers");
  if (!(tol > 0.0)) tol = 1e-5;  // Sec. 3's tolerance
  const size_t bytes = (size_t)h->w.n * sizeof(double);
  Hdr hd;
  PCK(h, cudaStreamSynchronize(h->stream), "sync");
  PCK(h, cudaMemcpy(&hd, h->w.hdr, sizeof hd, cudaMemcpyDeviceToHost), "read rank");
  int32_t acc = 0;
  double rel = INFINITY;
  if (hd.r > 0) {
    const double one = 1.0;
    if (odmd_status s = odmd_pairs_predict(h, state_dev, &one, 1, next_dev, h->w.n)) return s;
    if (residual(user, step, next_dev, r_dev, b_dev, h->stream) != 0)
      return pfail(h, ODMD_ERR_STATE, "residual callback reported a failure");
    k_pr_norms<<<h->w.grid, kThreads, 0, h->stream>>>(h->w, r_dev, b_dev);
    PCK(h, cudaGetLastError(), "residual norm launch");
    double nd[2];
    PCK(h, cudaMemcpyAsync(nd, reinterpret_cast<double*>(h->w.aux + 4), sizeof nd, cudaMemcpyDeviceToHost, h->stream),
        "read back");
    PCK(h, cudaStreamSynchronize(h->stream), "sync");
    if (!std::isfinite(nd[0]) || !std::isfinite(nd[1])) return pfail(h, ODMD_ERR_NUMERIC, "non-finite residual");
    rel = nd[1] > 0.0 ? std::sqrt(nd[0] / nd[1]) : (nd[0] == 0.0 ? 0.0 : INFINITY);
    acc = rel <= tol ? 1 : 0;
  }
  if (acc) {
    PCK(h, cudaMemcpyAsync(state_dev, next_dev, bytes, cudaMemcpyDeviceToDevice, h->stream), "take the prediction");
  } else {
    // the FOM's step starts from u^{k-1}; the pair (u^{k-1}, u^k) updates the model
    PCK(h, cudaMemcpyAsync(next_dev, state_dev, bytes, cudaMemcpyDeviceToDevice, h->stream), "FOM input");
    if (fom(user, step, next_dev, h->stream) != 0) return pfail(h, ODMD_ERR_STATE, "FOM callback reported a failure");
    if (odmd_status s = odmd_pairs_update(h, state_dev, next_dev)) return s;
    PCK(h, cudaMemcpyAsync(state_dev, next_dev, bytes, cudaMemcpyDeviceToDevice, h->stream), "take the FOM state");
  }
  if (accepted) *accepted = acc;
  if (rel_res) *rel_res = rel;
  return ODMD_OK;
}

const char* odmd_pairs_last_error(odmd_pairs_t h) { return h ? h->err.c_str() : g_pairs_err.c_str(); }

odmd_status odmd_pairs_destroy(odmd_pairs_t h) {
  if (!h) return pfail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  cudaStreamSynchronize(h->stream);
  delete h;
  return ODMD_OK;
}

}  // extern "C"
