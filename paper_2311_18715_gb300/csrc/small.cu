// Small dense solves of the online DMD update and of the eigen-cache, in double-float
// arithmetic (dd.cuh) on the FP32 pipes.
//
// Update (Sec. 2.3, Brand's rank-1 append in product form L = L0 Q):
//   k_prep     reduced tall sums -> projection p = L^T c, new direction, core matrix
//              K = [[diag(S), p], [0, rho]] and the deflated secular problem
//   k_roots    one CTA per singular value of K: root of the secular equation
//   k_zhat     one CTA per pole: Loewner weights; one extra CTA orders the values
//   k_vectors  one CTA per kept singular pair: left/right singular vectors of K
//   k_apply    one CTA per kept column: M' = U'^T B V', Q' = [Q 0; 0 q] U', rows of R
//
// Core SVD.  K K^T = D^2 + z z^T with D = diag(S, 0) and z = [p; rho], so sigma'^2 are
// the roots of the secular equation 1 + sum_i z_i^2 / (d_i^2 - lambda) = 0 and, with
// z-hat from Loewner's formula, u ~ (D^2 - lambda)^{-1} z-hat and v ~ (d_i z-hat_i /
// (d_i^2 - lambda), -1): the broken-arrow SVD of Gu and Eisenstat (SIAM J. Matrix Anal.
// Appl. 16, 1995).  Every difference d_i^2 - lambda is formed as (d_i - d_o)(d_i + d_o)
// - mu with lambda = d_o^2 + mu and d_o the nearer pole, which keeps the singular vectors
// orthogonal to working accuracy.  Negligible z_i and nearly equal d_i are deflated first
// (a Givens rotation merges the weights of two equal poles).  K is scaled by a power of
// two so that its largest entry lies in [1/2, 1).
//
// Eigensolve (lazy, Sec. 2.3: A~ = V Lambda V^{-1}, b = Phi^+ u^0): balancing by powers of
// two, Householder reduction to Hessenberg form, Francis double-shift QR with Schur
// vectors (Golub and Van Loan, Matrix Computations, Ch. 7), eigenvectors of the
// quasi-triangular factor by back substitution, then b from a complex LU solve.
#include "dd.cuh"
#include "odmd_internal.cuh"

namespace odmd {

constexpr float kEpsDD = 7.105427357601002e-15f;  // 2^-47, a safe bound on the unit roundoff

__device__ __forceinline__ dd LD(const float2* p, size_t i) { return dd_of(p[i]); }
__device__ __forceinline__ void STd(float2* p, size_t i, dd v) { p[i] = f2_of(v); }
__device__ __forceinline__ dd dzero() { return dd{0.f, 0.f}; }

// sum over the 4 adjacent lanes of a group (every lane of the warp must call it)
__device__ __forceinline__ dd group4_sum(dd a) {
  a = a + dd_shfl_xor(a, 1);
  return a + dd_shfl_xor(a, 2);
}

// sum_{t < cnt} A[a0 + t as] B[b0 + t bs] in double-float.  The sums are short and their
// operands sit in L2 or shared memory, so the loads are issued 8 at a time ahead of the
// arithmetic, and even and odd terms go to two accumulators (added at the end).
__device__ __forceinline__ dd dot_dd(const float2* A, size_t a0, size_t as, const float2* B, size_t b0, size_t bs,
                                     int cnt) {
  dd acc0 = dzero(), acc1 = dzero();
  for (int t0 = 0; t0 < cnt; t0 += 8) {
    float2 a[8], b[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const bool ok = t0 + t < cnt;
      a[t] = ok ? A[a0 + (size_t)(t0 + t) * as] : make_float2(0.f, 0.f);
      b[t] = ok ? B[b0 + (size_t)(t0 + t) * bs] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      acc0 = dd_fma(dd_of(a[t]), dd_of(b[t]), acc0);
      acc1 = dd_fma(dd_of(a[t + 1]), dd_of(b[t + 1]), acc1);
    }
  }
  return acc0 + acc1;
}

// terms t = sub, sub + 4, .. below n: how many
__device__ __forceinline__ int count4(int sub, int n) { return n > sub ? (n - sub + 3) >> 2 : 0; }

// out[j] = sum_{i < nrows} A[j*lda + i] v[i] for j < ncols (4 threads per output).
// Called by every thread of a 256-thread block; A, v, out in shared memory.
__device__ void colsum(float2* out, const float2* A, int lda, const float2* v, int nrows, int ncols) {
  const int tid = threadIdx.x;
  for (int base = 0; base < 4 * ncols; base += 256) {
    const int item = base + tid;
    const int j = item >> 2, sub = item & 3;
    dd acc = dzero();
    if (j < ncols)
      for (int i = sub; i < nrows; i += 4) acc = dd_fma(LD(A, (size_t)j * lda + i), LD(v, i), acc);
    acc = group4_sum(acc);
    if (j < ncols && sub == 0) out[j] = f2_of(acc);
  }
}

// out[i] = sum_{j < ncols} A[j*lda + i] v[j] for i < nrows (4 threads per output)
__device__ void rowsum(float2* out, const float2* A, int lda, const float2* v, int ncols, int nrows) {
  const int tid = threadIdx.x;
  for (int base = 0; base < 4 * nrows; base += 256) {
    const int item = base + tid;
    const int i = item >> 2, sub = item & 3;
    dd acc = dzero();
    if (i < nrows)
      for (int j = sub; j < ncols; j += 4) acc = dd_fma(LD(A, (size_t)j * lda + i), LD(v, j), acc);
    acc = group4_sum(acc);
    if (i < nrows && sub == 0) out[i] = f2_of(acc);
  }
}

// block-wide sum for 256 threads; every thread gets the result
__device__ dd block_sum256(dd a, float2* scratch8) {
  a = dd_warp_sum(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch8[warp] = f2_of(a);
  __syncthreads();
  dd t = dzero();
  for (int w = 0; w < 8; ++w) t = t + LD(scratch8, w);
  return t;
}

// ---------------------------------------------------------------------------------------
// k_prep
// ---------------------------------------------------------------------------------------
constexpr int kPrepThreads = 256;

__global__ void __launch_bounds__(kPrepThreads) k_prep(Ws ws) {
  pdl_wait();
  extern __shared__ __align__(16) float2 psm[];
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, qld = ws.cap + 1;
  float2* sQ = psm;  // r columns of Q, ld qld
  float2* ac = sQ + (size_t)qld * kMaxR;
  float2* yx = ac + qld;
  float2* z = yx + qld;
  float2* t1 = z + qld;
  float2* p = t1 + qld;
  float2* p2 = p + kMaxN;
  __shared__ float2 red8[16];
  __shared__ float2 sc[4];
  __shared__ int isc[4];
  __shared__ float2 dsc[kMaxN], zsc[kMaxN];
  __shared__ int defl[kMaxN];
  const float2* red = ws.sm.red;

  for (int idx = tid; idx < r * qld; idx += kPrepThreads) sQ[idx] = st.Q[idx];
  for (int i = tid; i < r0; i += kPrepThreads) {
    ac[i] = f2_of(LD(st.a, i) + LD(red, i));
    yx[i] = red[r0 + i];
  }
  __syncthreads();
  // p = Q^T ac and w = Q^T y in one pass (4 threads per column j < r; Q has r0 rows, the
  // appended coordinate lies outside span(L)); one warp with no column work meanwhile
  // decides whether the residual is appended (rho0 against the truncation threshold)
  {
    const int j = tid >> 2, sub = tid & 3;
    dd ap = dzero(), aw = dzero();
    if (j < r)
      for (int i = sub; i < r0; i += 4) {
        const dd q = LD(sQ, (size_t)j * qld + i);
        ap = dd_fma(q, LD(ac, i), ap);
        aw = dd_fma(q, LD(yx, i), aw);
      }
    ap = group4_sum(ap);
    aw = group4_sum(aw);
    if (j < r && sub == 0) {
      p[j] = f2_of(ap);
      ws.sm.w[j] = f2_of(aw);
    }
  }
  const int dwarp = 4 * r <= kPrepThreads - 32 ? 7 : 0;  // a warp without columns when there is one
  if (warp == dwarp) {
    dd ssq = dzero(), sy = dzero();
    for (int i = lane; i < r0; i += 32) {
      const dd si = LD(red, i);
      ssq = dd_fma(si, si, ssq);
      sy = dd_fma(si, LD(red, r0 + i), sy);
    }
    ssq = dd_warp_sum(ssq);
    sy = dd_warp_sum(sy);
    if (lane == 0) {
      const dd eta = LD(red, 2 * r0), ex = LD(red, 2 * r0 + 1);
      dd rho0sq = eta - ssq;
      if (rho0sq.h < 0.f) rho0sq = dzero();
      const dd rho0 = dd_sqrt(rho0sq);
      const dd cn = dd_sqrt(dd_of(st.hdr->cn2));
      const dd sig1 = r > 0 ? LD(st.S, 0) : dzero();
      const dd thr = dd{ws.tau_h, ws.tau_l} * dd_max(sig1, cn);
      const int append = dd_gt(rho0, thr) ? 1 : 0;
      ctl->thr = f2_of(thr);
      ctl->rho0 = f2_of(rho0);
      ctl->append = append;
      ctl->r0e = r0 + append;
      if (append) {
        ac[r0] = f2_of(rho0);
        yx[r0] = f2_of(dd_div(ex - sy, rho0));
      }
      isc[0] = append;
      sc[0] = f2_of(thr);
    }
  }
  __syncthreads();
  const int append = isc[0];
  const int r0e = r0 + append;
  const dd thr = dd_of(sc[0]);
  // z = ac - Q p (rows < r0; the appended coordinate is ac itself)
  for (int base = 0; base < 4 * r0e; base += kPrepThreads) {
    const int i = (base + tid) >> 2, sub = tid & 3;
    dd acc = dzero();
    if (i < r0)
      for (int j = sub; j < r; j += 4) acc = dd_fma(LD(sQ, (size_t)j * qld + i), LD(p, j), acc);
    acc = group4_sum(acc);
    if (i < r0e && sub == 0) z[i] = i < r0 ? f2_of(LD(ac, i) - acc) : ac[i];
  }
  __syncthreads();
  // second Gram-Schmidt pass in the small space: p2 = Q^T z, z -= Q p2, p += p2
  colsum(p2, sQ, qld, z, r0, r);
  __syncthreads();
  for (int base = 0; base < 4 * r0; base += kPrepThreads) {
    const int i = (base + tid) >> 2, sub = tid & 3;
    dd acc = dzero();
    if (i < r0)
      for (int j = sub; j < r; j += 4) acc = dd_fma(LD(sQ, (size_t)j * qld + i), LD(p2, j), acc);
    acc = group4_sum(acc);
    if (i < r0 && sub == 0) z[i] = f2_of(LD(z, i) - acc);
  }
  for (int j = tid; j < r; j += kPrepThreads) {
    p[j] = f2_of(LD(p, j) + LD(p2, j));
    ws.sm.p[j] = p[j];
  }
  __syncthreads();
  // ||z||^2 and z . y in one block reduction; rho = ||z||, gamma = q_n . y = (z . y) / rho
  dd zz = dzero(), zy = dzero();
  for (int i = tid; i < r0e; i += kPrepThreads) {
    const dd zi = LD(z, i);
    zz = dd_fma(zi, zi, zz);
    zy = dd_fma(zi, LD(yx, i), zy);
  }
  zz = dd_warp_sum(zz);
  zy = dd_warp_sum(zy);
  if (lane == 0) {
    red8[warp] = f2_of(zz);
    red8[8 + warp] = f2_of(zy);
  }
  __syncthreads();
  zz = dzero();
  zy = dzero();
  for (int w8 = 0; w8 < 8; ++w8) {
    zz = zz + LD(red8, w8);
    zy = zy + LD(red8, 8 + w8);
  }
  dd rho = dd_sqrt(zz);
  if (!dd_gt(rho, thr)) rho = dzero();
  const dd inv_rho = rho.h > 0.f ? dd_div(dd_of(1.f), rho) : dzero();
  const dd g = zy * inv_rho;
  for (int i = tid; i < r0e; i += kPrepThreads) {
    STd(ws.sm.qn, i, LD(z, i) * inv_rho);
    ws.sm.yext[i] = yx[i];
    if (i < r0) ws.sm.ac[i] = ac[i];
  }
  if (tid == 0) {
    ctl->rho = f2_of(rho);
    ctl->gamma = f2_of(g);
  }
  // ---- secular problem of K = [[diag(S), p], [0, rho]], n = r + 1, scaled to max 1
  if (warp == 0) {
    const int n = r + 1;
    dd mx = dzero();
    for (int i = lane; i < n; i += 32) {
      const dd zi = i < r ? LD(p, i) : rho;
      mx = dd_max(mx, dd_abs(zi));
      if (i == 0 && r > 0) mx = dd_max(mx, LD(st.S, 0));
    }
    mx = dd_warp_max(mx);
    int e = 0;
    if (mx.h > 0.f) frexpf(mx.h, &e);
    const float tol = 8.f * kEpsDD;  // in scaled units
    for (int i = lane; i < n; i += 32) {
      const dd di = i < r ? dd_ldexp(LD(st.S, i), -e) : dzero();
      const dd zi = dd_ldexp(i < r ? LD(p, i) : rho, -e);
      dsc[i] = f2_of(di);
      const bool small = !(fabsf(zi.h) > tol);
      zsc[i] = small ? make_float2(0.f, 0.f) : f2_of(zi);
      defl[i] = small ? 1 : 0;
      STd(ws.sm.dc, i, di);
    }
    __syncwarp();
    if (lane == 0) {
      // merge nearly equal poles (the pole at 0, coordinate r, is never merged)
      int nrot = 0, last = -1;
      for (int i = 0; i < r; ++i) {
        if (defl[i]) continue;
        if (last >= 0 && (dd_of(dsc[last]) - dd_of(dsc[i])).h <= tol) {
          const dd zl = dd_of(zsc[last]), zi = dd_of(zsc[i]);
          const dd h = dd_sqrt(zl * zl + zi * zi);
          ws.sm.rot_i[nrot] = last;
          ws.sm.rot_j[nrot] = i;
          STd(ws.sm.rot_c, nrot, dd_div(zl, h));
          STd(ws.sm.rot_s, nrot, dd_div(zi, h));
          ++nrot;
          zsc[last] = f2_of(h);
          zsc[i] = make_float2(0.f, 0.f);
          defl[i] = 1;
        } else {
          last = i;
        }
      }
      int m = 0, nd = 0;
      for (int i = n - 1; i >= 0; --i) {  // ascending poles
        if (defl[i]) {
          ws.sm.defl[nd++] = i;
        } else {
          ws.sm.pole[m] = i;
          ws.sm.d[m] = dsc[i];
          ws.sm.z[m] = zsc[i];
          ++m;
        }
      }
      ctl->n = n;
      ctl->m = m;
      ctl->ndefl = nd;
      ctl->nrot = nrot;
      ctl->scale_exp = e;
      if (!dd_isfinite(rho) || !dd_isfinite(mx)) atomicOr(&ctl->status, DEV_NONFINITE);
    }
  }
}

// ---------------------------------------------------------------------------------------
// k_roots: root j of 1 + sum_i z_i^2/(d_i^2 - lambda) = 0 in (d_j^2, d_{j+1}^2)
// ---------------------------------------------------------------------------------------
struct SecSums {
  dd psi, dpsi, phi, dphi;
};

// sums over poles i <= j (psi) and i > j (phi) at lambda = d_o^2 + mu
__device__ SecSums sec_eval(const float2* d, const float2* z, int m, int j, int o, dd mu) {
  SecSums s{dzero(), dzero(), dzero(), dzero()};
  const int lane = threadIdx.x & 31;
  const dd dob = LD(d, o);
  #pragma unroll
  for (int q_ = 0; q_ < (kMaxN + 31) / 32; ++q_) {
    const int i = lane + 32 * q_;
    if (i >= m) break;
    const dd di = LD(d, i);
    const dd del = (di - dob) * (di + dob) - mu;  // d_i^2 - lambda
    const dd zi = LD(z, i);
    const dd t = dd_div(zi, del);
    const dd term = zi * t, dterm = t * t;
    if (i <= j) {
      s.psi = s.psi + term;
      s.dpsi = s.dpsi + dterm;
    } else {
      s.phi = s.phi + term;
      s.dphi = s.dphi + dterm;
    }
  }
  s.psi = dd_warp_sum(s.psi);
  s.dpsi = dd_warp_sum(s.dpsi);
  s.phi = dd_warp_sum(s.phi);
  s.dphi = dd_warp_sum(s.dphi);
  return s;
}

__global__ void __launch_bounds__(32) k_roots(Ws ws) {
  pdl_wait();
  Ctl* ctl = ws.ctl;
  const int m = ctl->m;
  const int j = blockIdx.x;
  if (j >= m) return;
  const float2* d = ws.sm.d;
  const float2* z = ws.sm.z;
  const int lane = threadIdx.x;
  dd zsq = dzero();
  for (int i = lane; i < m; i += 32) zsq = dd_fma(LD(z, i), LD(z, i), zsq);
  zsq = dd_warp_sum(zsq);
  if (m == 1) {
    if (lane == 0) {
      ws.sm.org[0] = 0;
      STd(ws.sm.mu, 0, zsq);
      STd(ws.sm.sig, 0, dd_sqrt(LD(d, 0) * LD(d, 0) + zsq));
    }
    return;
  }
  int o;
  dd lo, hi, A, B;  // bracket of mu and the neighbouring poles, relative to d_o^2
  const bool last = (j == m - 1);
  if (!last) {
    const dd dj = LD(d, j), dj1 = LD(d, j + 1);
    const dd gap = (dj1 - dj) * (dj1 + dj);
    const dd mid = gap * 0.5f;
    const SecSums s = sec_eval(d, z, m, j, j, mid);
    if ((dd_of(1.f) + s.psi + s.phi).h >= 0.f) {
      o = j;
      lo = dzero();
      hi = mid;
      A = dzero();
      B = gap;
    } else {
      o = j + 1;
      lo = -mid;
      hi = dzero();
      A = -gap;
      B = dzero();
    }
  } else {
    o = j;
    lo = dzero();
    hi = zsq;
    A = dzero();
    B = dzero();
  }
  // ---- stage 1, FP32: locate the root to ~1e-7 relative (cheap), keeping the bracket
  dd mu = (lo + hi) * 0.5f;
  {
    const float dof = LD(d, o).h;
    const float Af = A.h, Bf = B.h;
    float lof = lo.h, hif = hi.h, muf = mu.h;
    for (int it = 0; it < 40; ++it) {
      float psi = 0.f, dpsi = 0.f, phi = 0.f, dphi = 0.f;
      #pragma unroll
  for (int q_ = 0; q_ < (kMaxN + 31) / 32; ++q_) {
    const int i = lane + 32 * q_;
    if (i >= m) break;
        const float di = d[i].x, zi = z[i].x;
        const float del = (di - dof) * (di + dof) - muf;
        const float t = zi / del;
        if (i <= j) {
          psi = fmaf(zi, t, psi);
          dpsi = fmaf(t, t, dpsi);
        } else {
          phi = fmaf(zi, t, phi);
          dphi = fmaf(t, t, dphi);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        psi += __shfl_xor_sync(0xffffffffu, psi, off);
        dpsi += __shfl_xor_sync(0xffffffffu, dpsi, off);
        phi += __shfl_xor_sync(0xffffffffu, phi, off);
        dphi += __shfl_xor_sync(0xffffffffu, dphi, off);
      }
      const float f = 1.f + psi + phi;
      if (f < 0.f)
        lof = muf;
      else
        hif = muf;
      if (fabsf(f) <= 16.f * 6e-8f * (1.f + fabsf(psi) + fabsf(phi))) break;
      const float Am = Af - muf, c1 = dpsi * Am * Am, a1 = psi - dpsi * Am;
      float x;
      if (!last) {
        const float Bm = Bf - muf, c2 = dphi * Bm * Bm, a2 = phi - dphi * Bm;
        const float C = 1.f + a1 + a2;
        const float qb = -(C * (Af + Bf) + c1 + c2), qc = C * Af * Bf + c1 * Bf + c2 * Af;
        if (fabsf(C) <= 1e-7f * (fabsf(qb) + fabsf(qc))) {
          x = -qc / qb;
        } else {
          const float sq = sqrtf(fmaxf(qb * qb - 4.f * C * qc, 0.f));
          const float q = -0.5f * (qb >= 0.f ? qb + sq : qb - sq);
          const float x1 = q / C, x2 = qc / q;
          const bool in1 = x1 > lof && x1 < hif, in2 = x2 > lof && x2 < hif;
          x = in1 && !in2 ? x1 : (in2 && !in1 ? x2 : (fabsf(x1 - muf) < fabsf(x2 - muf) ? x1 : x2));
        }
      } else {
        const float C = 1.f + a1 + phi;
        x = C > 0.f ? Af + c1 / C : 0.5f * (lof + hif);
      }
      if (!(x > lof && x < hif)) x = 0.5f * (lof + hif);
      const float step = fabsf(x - muf);
      muf = x;
      if (step <= 4e-7f * fabsf(muf) || hif - lof <= 4e-7f * fmaxf(fabsf(lof), fabsf(hif))) break;
    }
    // FP32 cannot resolve poles closer than ~1e-7 relative: keep its root only when it is
    // finite and strictly inside the double-float bracket
    const dd cand = dd_of(muf);
    if (isfinite(muf) && dd_gt(cand, lo) && dd_lt(cand, hi)) mu = cand;
  }
  // ---- stage 2: f in double-float, derivatives and the model step in FP32.  The model is
  // solved for the correction delta = x - mu (shifted poles A - mu, B - mu), so an FP32
  // step applied to a double-float mu converges like Newton to double-float accuracy.
  bool conv = false;
  for (int it = 0; it < 100; ++it) {
    dd psi = dzero(), phi = dzero();
    float dpsi = 0.f, dphi = 0.f;
    {
      const dd dob = LD(d, o);
      #pragma unroll
  for (int q_ = 0; q_ < (kMaxN + 31) / 32; ++q_) {
    const int i = lane + 32 * q_;
    if (i >= m) break;
        const dd di = LD(d, i);
        const dd del = (di - dob) * (di + dob) - mu;  // d_i^2 - lambda
        const dd zi = LD(z, i);
        // t = z / del: FP32 reciprocal, then one correction of the quotient
        const float rc = __frcp_rn(del.h);
        const float t0 = __fmul_rn(zi.h, rc);
        const dd rem = zi - del * t0;
        const dd t = fast_two_sum(t0, __fmul_rn(rem.h, rc));
        const dd term = zi * t;
        const float dterm = t.h * t.h;
        if (i <= j) {
          psi = psi + term;
          dpsi += dterm;
        } else {
          phi = phi + term;
          dphi += dterm;
        }
      }
      psi = dd_warp_sum(psi);
      phi = dd_warp_sum(phi);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        dpsi += __shfl_xor_sync(0xffffffffu, dpsi, off);
        dphi += __shfl_xor_sync(0xffffffffu, dphi, off);
      }
    }
    const dd f = dd_of(1.f) + psi + phi;
    if (f.h < 0.f)
      lo = mu;
    else
      hi = mu;
    const float ftol = 8.f * kEpsDD * (float)m * (1.f + fabsf(psi.h) + fabsf(phi.h));
    if (fabsf(f.h) <= ftol) {
      conv = true;
      break;
    }
    // Two-pole model written around mu with f explicit, so that FP32 coefficients give a
    // step accurate relative to itself:  f + psi' a d/(a - d) + phi' b d/(b - d) = 0,
    // with the neighbouring poles at a = A - mu and b = B - mu and the unknown d = x - mu.
    const float fh = f.h;
    const float a = (A - mu).h;
    const float b = last ? 0.f : (B - mu).h;
    // the unknown is scaled by a power of two so that the model's coefficients stay inside
    // the FP32 exponent range: offsets between clustered tiny singular values square to
    // 1e-23 and their products to 1e-46, below the smallest float
    int ex = 0;
    frexpf(fmaxf(fabsf(a), fabsf(b)), &ex);
    const float sc = ldexpf(1.f, ex), as = ldexpf(a, -ex), bs = ldexpf(b, -ex);
    const float ps = dpsi * sc, hs = dphi * sc;
    float delta;
    if (!last) {
      const float Qa = fh - ps * as - hs * bs;
      const float Qb = as * bs * (ps + hs) - fh * (as + bs);
      const float Qc = fh * as * bs;
      const float disc = fmaxf(Qb * Qb - 4.f * Qa * Qc, 0.f);
      const float q = -0.5f * (Qb >= 0.f ? Qb + sqrtf(disc) : Qb - sqrtf(disc));
      const float d2 = q != 0.f ? Qc / q : 0.f;  // the root that tends to -f / f'
      const float d1 = Qa != 0.f ? q / Qa : d2;
      const float lo_s = ldexpf((lo - mu).h, -ex), hi_s = ldexpf((hi - mu).h, -ex);
      const bool in2 = d2 > lo_s && d2 < hi_s, in1 = d1 > lo_s && d1 < hi_s;
      delta = ldexpf(in2 ? d2 : (in1 ? d1 : d2), ex);
    } else {
      const float den = fh - ps * as;
      delta = den != 0.f ? ldexpf(fh * as / den, ex) : 0.f;
    }
    dd x = mu + dd_of(delta);
    if (!isfinite(delta) || !(dd_gt(x, lo) && dd_lt(x, hi))) x = (lo + hi) * 0.5f;
    const dd step = dd_abs(x - mu);
    mu = x;
    if (step.h <= 4.f * kEpsDD * fabsf(mu.h) ||
        (hi - lo).h <= 4.f * kEpsDD * fmaxf(fabsf(lo.h), fabsf(hi.h))) {
      conv = true;
      break;
    }
  }
  if (lane == 0) {
    if (!conv) atomicOr(&ctl->status, DEV_SECULAR);
    ws.sm.org[j] = o;
    STd(ws.sm.mu, j, mu);
    const dd dob = LD(d, o);
    dd lam = dob * dob + mu;
    if (lam.h < 0.f) lam = dzero();
    STd(ws.sm.sig, j, dd_sqrt(lam));
  }
}

// ---------------------------------------------------------------------------------------
// k_zhat: Loewner weights z^_i^2 = prod_k (lambda_k - d_i^2) / prod_{k != i} (d_k^2 - d_i^2),
// paired so every factor is O(1).  Block kMaxN orders all singular values of K.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_zhat(Ws ws) {
  pdl_wait();
  Ctl* ctl = ws.ctl;
  const int m = ctl->m;
  const int lane = threadIdx.x;
  if (blockIdx.x == kMaxN) {
    // order roots (sig[0..m)) and deflated values (scaled diagonal at defl[k]), descending
    const int nd = ctl->ndefl;
    __shared__ float2 val[kMaxN];
    __shared__ int code[kMaxN];
    const int tot = m + nd;
    for (int e = lane; e < tot; e += 32) {
      if (e < m) {
        val[e] = ws.sm.sig[e];
        code[e] = e;
      } else {
        const int c = ws.sm.defl[e - m];
        val[e] = ws.sm.dc[c];
        code[e] = -c - 1;
      }
    }
    __syncwarp();
    dd vmax = dzero();
    for (int e = 0; e < tot; ++e) vmax = dd_max(vmax, LD(val, e));
    const dd cut = dd{ws.tau_h, ws.tau_l} * vmax;
    for (int e = lane; e < tot; e += 32) {
      int pos = 0;
      const dd ve = LD(val, e);
      for (int f = 0; f < tot; ++f) {
        const dd vf = LD(val, f);
        pos += dd_gt(vf, ve) || (vf.h == ve.h && vf.l == ve.l && f < e);
      }
      ws.sm.src[pos] = code[e];
      ws.sm.sig[kMaxN + pos] = val[e];
    }
    if (lane == 0) {
      int keep = 0;
      if (vmax.h > 0.f)
        for (int e = 0; e < tot; ++e) keep += dd_gt(LD(val, e), cut);
      ctl->rnew = min(keep, ws.rmax);
    }
    return;
  }
  const int i = blockIdx.x;
  if (i >= m) return;
  const float2* d = ws.sm.d;
  const dd di = LD(d, i);
  dd prod = dd_of(1.f);
  #pragma unroll
  for (int q_ = 0; q_ < (kMaxN + 31) / 32; ++q_) {
    const int k = lane + 32 * q_;
    if (k >= m) break;
    const dd dko = LD(d, ws.sm.org[k]);
    const dd lam_m_di = LD(ws.sm.mu, k) - (di - dko) * (di + dko);  // lambda_k - d_i^2
    dd f;
    if (k == m - 1) {
      f = lam_m_di;
    } else {
      const dd dk = LD(d, k < i ? k : k + 1);
      f = dd_div(lam_m_di, (dk - di) * (dk + di));
    }
    prod = prod * f;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) prod = prod * dd_shfl_xor(prod, off);
  if (lane == 0) {
    dd zh = dd_sqrt(prod.h > 0.f ? prod : dzero());
    if (ws.sm.z[i].x < 0.f) zh = -zh;
    STd(ws.sm.zhat, i, zh);
  }
}

// ---------------------------------------------------------------------------------------
// k_vectors: kept column j -> u_j, v_j (core coordinates 0..r; r is the p/rho column)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_vectors(Ws ws) {
  pdl_wait();
  Ctl* ctl = ws.ctl;
  const int j = blockIdx.x;
  if (j >= ctl->rnew) return;
  const int n = ctl->n, m = ctl->m, r = n - 1;
  const int tid = threadIdx.x;
  __shared__ float2 u[kMaxN], v[kMaxN], red[4];
  for (int i = tid; i < n; i += 64) {
    u[i] = make_float2(0.f, 0.f);
    v[i] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int code = ws.sm.src[j];
  if (code >= 0) {
    const float2* d = ws.sm.d;
    const dd dob = LD(d, ws.sm.org[code]);
    const dd mu = LD(ws.sm.mu, code);
    for (int i = tid; i < m; i += 64) {
      const dd di = LD(d, i);
      const dd del = (di - dob) * (di + dob) - mu;  // d_i^2 - lambda
      const dd ui = dd_div(LD(ws.sm.zhat, i), del);
      const int c = ws.sm.pole[i];
      u[c] = f2_of(ui);
      if (c < r) v[c] = f2_of(di * ui);
    }
    __syncthreads();
    if (tid == 0) v[r] = make_float2(-1.f, 0.f);
    __syncthreads();
    dd su = dzero(), sv = dzero();
    for (int i = tid; i < n; i += 64) {
      su = dd_fma(LD(u, i), LD(u, i), su);
      sv = dd_fma(LD(v, i), LD(v, i), sv);
    }
    su = dd_warp_sum(su);
    sv = dd_warp_sum(sv);
    if ((tid & 31) == 0) {
      red[(tid >> 5) * 2] = f2_of(su);
      red[(tid >> 5) * 2 + 1] = f2_of(sv);
    }
    __syncthreads();
    const dd iu = dd_div(dd_of(1.f), dd_sqrt(LD(red, 0) + LD(red, 2)));
    const dd iv = dd_div(dd_of(1.f), dd_sqrt(LD(red, 1) + LD(red, 3)));
    for (int i = tid; i < n; i += 64) {
      u[i] = f2_of(LD(u, i) * iu);
      v[i] = f2_of(LD(v, i) * iv);
    }
  } else if (tid == 0) {
    const int c = -code - 1;
    u[c] = make_float2(1.f, 0.f);
    v[c] = make_float2(1.f, 0.f);
  }
  __syncthreads();
  if (tid == 0) {
    for (int t = ctl->nrot - 1; t >= 0; --t) {
      const int a = ws.sm.rot_i[t], b = ws.sm.rot_j[t];
      const dd c = LD(ws.sm.rot_c, t), s = LD(ws.sm.rot_s, t);
      const dd ua = LD(u, a), ub = LD(u, b), va = LD(v, a), vb = LD(v, b);
      u[a] = f2_of(c * ua - s * ub);
      u[b] = f2_of(s * ua + c * ub);
      v[a] = f2_of(c * va - s * vb);
      v[b] = f2_of(s * va + c * vb);
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += 64) {
    ws.sm.U[(size_t)j * kMaxN + i] = u[i];
    ws.sm.V[(size_t)j * kMaxN + i] = v[i];
  }
}

// ---------------------------------------------------------------------------------------
// k_apply: column j of the new small state (written to the other state buffer)
//   M'    = U'^T [[M, w], [rho r_last^T, gamma]] V'
//   Q'    = [[Q, q_n(0:r0)], [0, q_n(r0)]] U'     (rows: L0 coordinates incl. the append)
//   r_first' = [r_first, 0] V'  (= last row of V' when c is u^0),  r_last' = V'[r, :]
//   S' = sigma'[0:rnew] (unscaled);  a' = L0'^T x
// ---------------------------------------------------------------------------------------
constexpr int kApplyThreads = 256;

__device__ void apply_column(const Ws& ws, int j, const StateBuf& st, const StateBuf& nx, int r, int r0, int r0e,
                             bool compact);

__global__ void __launch_bounds__(kApplyThreads) k_apply(Ws ws) {
  pdl_wait();
  Ctl* ctl = ws.ctl;
  const int j = blockIdx.x;
  const int rnew = ctl->rnew;
  const int tid = threadIdx.x;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur], nx = ws.st[cur ^ 1];
  const int r = st.hdr->r, r0 = st.hdr->r0, n = r + 1;
  const int r0e = ctl->r0e;
  const int cap = ws.cap, qld = cap + 1, rm = ws.rmax;
  const bool compact = r0e > cap;
  const int append = ctl->append;
  if (j == 0 && tid == 0) {
    nx.hdr->r = rnew;
    nx.hdr->r0 = compact ? rnew : r0e;
    nx.hdr->pairs = st.hdr->pairs + 1;
    nx.hdr->compactions = st.hdr->compactions + (compact ? 1 : 0);
    nx.hdr->cn2 = ws.sm.red[2 * r0 + 2];
    // an appended column is formed by the next tall pass (compaction forms it at once)
    nx.hdr->pend = (append && !compact) ? 1 : 0;
    nx.hdr->pinv = append ? f2_of(dd_div(dd_of(1.f), dd_of(ctl->rho0))) : make_float2(0.f, 0.f);
    ctl->mode = compact ? PB_COMPACT : (append ? PB_APPEND : PB_NONE);
  }
  if (j == 0) {
    if (!compact)
      for (int i = tid; i < r0e; i += kApplyThreads) nx.a[i] = ws.sm.yext[i];
    if (append && !compact)
      for (int i = tid; i < r0; i += kApplyThreads) nx.ps[i] = ws.sm.red[i];
  }
  if (j < rnew) apply_column(ws, j, st, nx, r, r0, r0e, compact);
  // the last CTA commits the new state and snapshot buffers
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&ctl->ticket_b, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  if (tid == 0) {
    __threadfence();
    ctl->cur = cur ^ 1;
    ctl->cur_c = ctl->cur_c ^ 1;
    ctl->eig_valid = 0;
    ctl->model_ver += 1ull;
    ctl->ticket_b = 0u;
  }
}

__device__ void apply_column(const Ws& ws, int j, const StateBuf& st, const StateBuf& nx, int r, int r0, int r0e,
                             bool compact) {
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const int n = r + 1, rnew = ctl->rnew;
  const int qld = ws.cap + 1, rm = ws.rmax;
  const dd rho = dd_of(ctl->rho), gamma = dd_of(ctl->gamma);
  __shared__ float2 v[kMaxN], u[kMaxN], bv[kMaxN], qcol[kMaxCap + 1], rlv[2];
  for (int i = tid; i < n; i += kApplyThreads) {
    v[i] = ws.sm.V[(size_t)j * kMaxN + i];
    u[i] = ws.sm.U[(size_t)j * kMaxN + i];
  }
  __syncthreads();
  // B v, rows 0..r-1: M v[0:r] + w v_r  (4 threads per row; r <= 64 rows)
  {
    const int i = tid >> 2, sub = tid & 3;
    dd acc = dzero();
    if (i < r) acc = dot_dd(st.M, (size_t)sub * rm + i, (size_t)4 * rm, v, sub, 4, count4(sub, r));
    acc = group4_sum(acc);
    if (i < r && sub == 0) bv[i] = f2_of(dd_fma(LD(ws.sm.w, i), LD(v, r), acc));
  }
  // row r: rho (r_last . v[0:r]) + gamma v_r   (warp 7)
  if ((tid >> 5) == 7) {
    const int lane = tid & 31;
    dd t = dzero();
    if (lane < r) t = dot_dd(st.rl, lane, 32, v, lane, 32, (r - lane + 31) >> 5);
    t = dd_warp_sum(t);
    if (lane == 0) rlv[0] = f2_of(t);
  }
  // Q' column j (rows 0..r0e-1): Q u[0:r] + qn u_r
  for (int base = 0; base < 4 * r0e; base += kApplyThreads) {
    const int item = base + tid;
    const int i = item >> 2, sub = item & 3;
    dd acc = dzero();
    if (i < r0) acc = dot_dd(st.Q, (size_t)sub * qld + i, (size_t)4 * qld, u, sub, 4, count4(sub, r));
    acc = group4_sum(acc);
    if (i < r0e && sub == 0) qcol[i] = f2_of(dd_fma(LD(ws.sm.qn, i), LD(u, r), acc));
  }
  __syncthreads();
  if (tid == 0) bv[r] = f2_of(dd_fma(rho, LD(rlv, 0), gamma * LD(v, r)));
  __syncthreads();
  // M' column j: U'^T (B v)   (4 threads per output row i < rnew)
  {
    const int i = tid >> 2, sub = tid & 3;
    dd acc = dzero();
    if (i < rnew) acc = dot_dd(ws.sm.U, (size_t)i * kMaxN + sub, 4, bv, sub, 4, count4(sub, n));
    acc = group4_sum(acc);
    if (i < rnew && sub == 0) nx.M[(size_t)j * rm + i] = f2_of(acc);
  }
  if (compact) {
    for (int i = tid; i < r0e; i += kApplyThreads) ws.sm.QB[(size_t)j * qld + i] = qcol[i];
    for (int i = tid; i < rnew; i += kApplyThreads)
      nx.Q[(size_t)j * qld + i] = make_float2(i == j ? 1.f : 0.f, 0.f);
  } else {
    for (int i = tid; i < r0e; i += kApplyThreads) nx.Q[(size_t)j * qld + i] = qcol[i];
  }
  // r_first', r_last', S', a' (compaction)  -- warp 0
  if (tid < 32) {
    const int lane = tid;
    dd rf = dzero();
    if (st.hdr->pairs != 0)
      for (int k = lane; k < r; k += 32) rf = dd_fma(LD(st.rf, k), LD(v, k), rf);
    rf = dd_warp_sum(rf);
    dd a = dzero();
    if (compact)
      for (int i = lane; i < r0e; i += 32) a = dd_fma(LD(qcol, i), LD(ws.sm.yext, i), a);
    a = dd_warp_sum(a);
    if (lane == 0) {
      nx.rf[j] = st.hdr->pairs == 0 ? v[r] : f2_of(rf);
      nx.rl[j] = v[r];
      STd(nx.S, j, dd_ldexp(LD(ws.sm.sig, kMaxN + j), ctl->scale_exp));
      if (compact) STd(nx.a, j, a);
    }
  }
}

// ---------------------------------------------------------------------------------------
// eigensolver (one CTA of 128 threads).  Scalars are computed identically by every
// thread from shared data; row/column updates are split across the threads.
// ---------------------------------------------------------------------------------------
constexpr int kLD = kMaxR + 1;
constexpr int kEigThreads = 128;

struct EigSmem {
  float2 H[kMaxR * kLD];   // Hessenberg / quasi-triangular Schur factor T, row-major
  float2 Z[kMaxR * kLD];   // Schur vectors, row-major
  float2 Xr[kMaxR * kLD];  // eigenvectors of T, X[i][j] = component i of vector j
  float2 Xi[kMaxR * kLD];
  float scale[kMaxR];      // balancing (powers of two)
  float2 wr[kMaxR], wi[kMaxR];
  float2 v[kMaxR];         // reflector / scratch
  float2 tmp[kMaxR];
};

__device__ __forceinline__ dd HH(const float2* A, int i, int k) { return dd_of(A[i * kLD + k]); }

// rows i0..i0+len-1 of A, columns c0..cn-1: A <- A - beta v (v^T A)
__device__ void refl_left(float2* A, int i0, int len, int c0, int cn, const dd* v, dd beta) {
  for (int c = c0 + (int)threadIdx.x; c < cn; c += kEigThreads) {
    dd s = dzero();
    for (int i = 0; i < len; ++i) s = dd_fma(v[i], HH(A, i0 + i, c), s);
    s = s * beta;
    for (int i = 0; i < len; ++i) A[(i0 + i) * kLD + c] = f2_of(HH(A, i0 + i, c) - s * v[i]);
  }
}

// rows rs..rn-1 (split over nth threads), columns j0..j0+len-1: A <- A - (A v) beta v^T
__device__ void refl_right(float2* A, int rs, int rn, int j0, int len, const dd* v, dd beta, int tid, int nth) {
  for (int row = rs + tid; row < rn; row += nth) {
    dd s = dzero();
    for (int i = 0; i < len; ++i) s = dd_fma(HH(A, row, j0 + i), v[i], s);
    s = s * beta;
    for (int i = 0; i < len; ++i) A[row * kLD + j0 + i] = f2_of(HH(A, row, j0 + i) - s * v[i]);
  }
}

// Power of two that brings the largest |a_i| into [1/2, 1) (0 for a zero vector).  The
// double-float format has the exponent range of FP32, so reflector inputs are scaled
// before squaring; a reflector is unchanged when its vector is scaled.
__device__ __forceinline__ int scale_exp_of(const dd* a, int len) {
  float mx = 0.f;
  for (int i = 0; i < len; ++i) mx = fmaxf(mx, fabsf(a[i].h));
  int e = 0;
  if (mx > 0.f) frexpf(mx, &e);
  return e;
}

// Reflector (I - beta v v^T) a = -sign(a0) ||a|| e1 for len 2 or 3, unnormalised v
// (of the scaled input).
__device__ __forceinline__ dd house3(const dd* a_in, int len, dd* v) {
  const int e = scale_exp_of(a_in, len);
  dd a[3];
  for (int i = 0; i < len; ++i) a[i] = dd_ldexp(a_in[i], -e);
  dd sig = dzero();
  for (int i = 1; i < len; ++i) sig = dd_fma(a[i], a[i], sig);
  for (int i = 0; i < len; ++i) v[i] = a[i];
  if (sig.h == 0.f) return dzero();
  const dd mu = dd_sqrt(dd_fma(a[0], a[0], sig));
  const dd ax = dd_abs(a[0]);
  v[0] = a[0].h >= 0.f ? a[0] + mu : a[0] - mu;  // a0 + sign(a0) mu
  return dd_div(dd_of(1.f), mu * (mu + ax));      // 2 / (v^T v)
}

__global__ void __launch_bounds__(kEigThreads) k_eig(Ws ws) {
  extern __shared__ __align__(16) unsigned char esm[];
  EigSmem& E = *reinterpret_cast<EigSmem*>(esm);
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const StateBuf st = ws.st[ctl->cur];
  const int r = st.hdr->r, rm = ws.rmax;
  __shared__ float2 nrm_s[1];
  __shared__ int piv_s;
  if (r == 0) {
    if (tid == 0) {
      atomicOr(&ctl->status, DEV_NOMODEL);
      ctl->eig_r = 0;
      ctl->eig_valid = 1;
    }
    return;
  }
  float2* H = E.H;
  float2* Z = E.Z;
  // A~ = M diag(S)^-1
  for (int idx = tid; idx < r * r; idx += kEigThreads) {
    const int i = idx / r, k = idx % r;
    H[i * kLD + k] = f2_of(dd_div(LD(st.M, (size_t)k * rm + i), LD(st.S, k)));
    Z[i * kLD + k] = make_float2(i == k ? 1.f : 0.f, 0.f);
  }
  for (int i = tid; i < r; i += kEigThreads) E.scale[i] = 1.f;
  __syncthreads();

  // ---- balancing by powers of two (row/column 1-norms from the hi parts), warp 0
  if (tid < 32) {
    const int lane = tid;
    for (int sweep = 0; sweep < 40; ++sweep) {
      bool changed = false;
      for (int i = 0; i < r; ++i) {
        float c = 0.f, rr = 0.f;
        for (int k = lane; k < r; k += 32)
          if (k != i) {
            c += fabsf(H[k * kLD + i].x);
            rr += fabsf(H[i * kLD + k].x);
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          c += __shfl_xor_sync(0xffffffffu, c, o);
          rr += __shfl_xor_sync(0xffffffffu, rr, o);
        }
        if (c == 0.f || rr == 0.f) continue;
        const float s = c + rr;
        float f = 1.f, g = rr * 0.5f;
        while (c < g && f < 1e18f) {
          f *= 2.f;
          c *= 4.f;
        }
        g = rr * 2.f;
        while (c >= g && f > 1e-18f) {
          f *= 0.5f;
          c *= 0.25f;
        }
        if ((c + rr) / f < 0.95f * s) {
          changed = true;
          const float inv = 1.f / f;  // exact: f is a power of two
          for (int k = lane; k < r; k += 32) {
            const float2 a = H[i * kLD + k];
            H[i * kLD + k] = make_float2(a.x * inv, a.y * inv);
          }
          __syncwarp();
          for (int k = lane; k < r; k += 32) {
            const float2 a = H[k * kLD + i];
            H[k * kLD + i] = make_float2(a.x * f, a.y * f);
          }
          if (lane == 0) E.scale[i] *= f;
          __syncwarp();
        }
      }
      if (!changed) break;
    }
  }
  __syncthreads();

  // ---- Householder reduction to upper Hessenberg form, Z accumulates the reflectors
  __shared__ int col_exp;
  for (int k = 0; k + 2 < r; ++k) {
    const int len = r - k - 1;
    if (tid < 32) {
      float mx = 0.f;
      for (int i = tid; i < len; i += 32) mx = fmaxf(mx, fabsf(H[(k + 1 + i) * kLD + k].x));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int e = 0;
      if (mx > 0.f) frexpf(mx, &e);
      dd sg = dzero();
      for (int i = 1 + tid; i < len; i += 32) {
        const dd hs = dd_ldexp(HH(H, k + 1 + i, k), -e);
        sg = dd_fma(hs, hs, sg);
      }
      sg = dd_warp_sum(sg);
      if (tid == 0) {
        E.tmp[0] = f2_of(sg);
        col_exp = e;
      }
    }
    __syncthreads();
    const dd sigma = dd_of(E.tmp[0]);
    const int ce = col_exp;
    if (sigma.h == 0.f) {
      __syncthreads();
      continue;
    }
    // reflector of the column scaled by 2^-ce (v scaled alike; the reflector is the same)
    const dd x0 = dd_ldexp(HH(H, k + 1, k), -ce);
    const dd mu = dd_sqrt(dd_fma(x0, x0, sigma));
    const dd v0 = x0.h >= 0.f ? x0 + mu : x0 - mu;
    const dd beta = dd_div(dd_of(1.f), mu * (mu + dd_abs(x0)));
    for (int i = tid; i < len; i += kEigThreads)
      E.v[i] = i == 0 ? f2_of(v0) : f2_of(dd_ldexp(HH(H, k + 1 + i, k), -ce));
    __syncthreads();
    // left: rows k+1.., columns k..r-1
    for (int c = k + tid; c < r; c += kEigThreads) {
      dd s = dzero();
      for (int i = 0; i < len; ++i) s = dd_fma(LD(E.v, i), HH(H, k + 1 + i, c), s);
      s = s * beta;
      for (int i = 0; i < len; ++i) H[(k + 1 + i) * kLD + c] = f2_of(HH(H, k + 1 + i, c) - s * LD(E.v, i));
    }
    __syncthreads();
    // right on H and Z (rows 0..r-1): threads 0..63 -> H, 64..127 -> Z
    {
      float2* A = tid < 64 ? H : Z;
      for (int row = tid & 63; row < r; row += 64) {
        dd s = dzero();
        for (int i = 0; i < len; ++i) s = dd_fma(HH(A, row, k + 1 + i), LD(E.v, i), s);
        s = s * beta;
        for (int i = 0; i < len; ++i) A[row * kLD + k + 1 + i] = f2_of(HH(A, row, k + 1 + i) - s * LD(E.v, i));
      }
    }
    __syncthreads();
    if (tid == 0) {
      H[(k + 1) * kLD + k] = f2_of(dd_ldexp(x0.h >= 0.f ? -mu : mu, ce));
      for (int i = k + 2; i < r; ++i) H[i * kLD + k] = make_float2(0.f, 0.f);
    }
    __syncthreads();
  }

  // ---- Francis double-shift QR (Golub & Van Loan, Alg. 7.5.1 with deflation)
  // Deflation: a subdiagonal entry is negligible next to its diagonal neighbours, or
  // next to ||H||_F (double-float rounding leaves absolute noise of order eps ||H||,
  // which a purely local test could wait on forever; both are within backward error).
  float fro = 0.f;
  for (int idx = 0; idx < r * r; ++idx) {
    const float hv = H[(idx / r) * kLD + idx % r].x;
    fro = fmaf(hv, hv, fro);
  }
  const float gtol = 2.f * kEpsDD * sqrtf(fro);
  int hi = r - 1, iter = 0, total = 0;
  bool failed = false;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      const float s = fabsf(H[(l - 1) * kLD + l - 1].x) + fabsf(H[l * kLD + l].x);
      const float sub = fabsf(H[l * kLD + l - 1].x);
      if (sub <= kEpsDD * s || sub <= gtol) break;
      --l;
    }
    __syncthreads();
    if (l > 0 && tid == 0) H[l * kLD + l - 1] = make_float2(0.f, 0.f);
    __syncthreads();
    if (l == hi) {
      if (tid == 0) {
        E.wr[hi] = H[hi * kLD + hi];
        E.wi[hi] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {
      const dd a = HH(H, hi - 1, hi - 1), b = HH(H, hi - 1, hi);
      const dd c = HH(H, hi, hi - 1), d = HH(H, hi, hi);
      const dd p = (a - d) * 0.5f;
      const dd disc = dd_fma(p, p, b * c);
      __syncthreads();
      if (disc.h >= 0.f) {
        // real pair: rotate the block to upper triangular form
        const dd sq = dd_sqrt(disc);
        const dd l1 = (a + d) * 0.5f + (p.h >= 0.f ? sq : -sq);
        dd ur = b, vr = l1 - a;
        const dd ur2 = l1 - d, vr2 = c;
        if (fabsf(ur2.h) + fabsf(vr2.h) > fabsf(ur.h) + fabsf(vr.h)) {
          ur = ur2;
          vr = vr2;
        }
        {
          const dd uv[2] = {ur, vr};
          const int e2 = scale_exp_of(uv, 2);
          ur = dd_ldexp(ur, -e2);
          vr = dd_ldexp(vr, -e2);
        }
        const dd nn = dd_sqrt(ur * ur + vr * vr);
        dd cs = dd_of(1.f), sn = dzero();
        if (nn.h > 0.f) {
          cs = dd_div(ur, nn);
          sn = dd_div(vr, nn);
        }
        for (int col = hi - 1 + tid; col < r; col += kEigThreads) {
          const dd x1 = HH(H, hi - 1, col), x2 = HH(H, hi, col);
          H[(hi - 1) * kLD + col] = f2_of(cs * x1 + sn * x2);
          H[hi * kLD + col] = f2_of(cs * x2 - sn * x1);
        }
        __syncthreads();
        {
          float2* A = tid < 64 ? H : Z;
          const int rn = tid < 64 ? hi + 1 : r;
          for (int row = tid & 63; row < rn; row += 64) {
            const dd x1 = HH(A, row, hi - 1), x2 = HH(A, row, hi);
            A[row * kLD + hi - 1] = f2_of(cs * x1 + sn * x2);
            A[row * kLD + hi] = f2_of(cs * x2 - sn * x1);
          }
        }
        __syncthreads();
        if (tid == 0) {
          H[hi * kLD + hi - 1] = make_float2(0.f, 0.f);
          E.wr[hi - 1] = H[(hi - 1) * kLD + hi - 1];
          E.wr[hi] = H[hi * kLD + hi];
          E.wi[hi - 1] = make_float2(0.f, 0.f);
          E.wi[hi] = make_float2(0.f, 0.f);
        }
      } else if (tid == 0) {
        const dd re = (a + d) * 0.5f, im = dd_sqrt(-disc);
        E.wr[hi - 1] = f2_of(re);
        E.wr[hi] = f2_of(re);
        E.wi[hi - 1] = f2_of(im);
        E.wi[hi] = f2_of(-im);
      }
      __syncthreads();
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++total > 60 * r) {
      failed = true;
      break;
    }
    ++iter;
    dd ssum, tprod;
    if (iter % 11 == 10) {  // exceptional shift
      const dd s = dd_abs(HH(H, hi, hi - 1)) + dd_abs(HH(H, hi - 1, hi - 2));
      const dd h = s * 0.75f + HH(H, hi, hi);
      ssum = h * 2.f;
      tprod = dd_fma(h, h, s * s * 0.4375f);
    } else {
      ssum = HH(H, hi - 1, hi - 1) + HH(H, hi, hi);
      tprod = HH(H, hi - 1, hi - 1) * HH(H, hi, hi) - HH(H, hi - 1, hi) * HH(H, hi, hi - 1);
    }
    const dd hll = HH(H, l, l), hl1l = HH(H, l + 1, l);
    dd x = hll * hll + HH(H, l, l + 1) * hl1l - ssum * hll + tprod;
    dd y = hl1l * (hll + HH(H, l + 1, l + 1) - ssum);
    dd zz = hl1l * HH(H, l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      const dd a3[3] = {x, y, zz};
      dd v[3];
      const dd beta = house3(a3, 3, v);
      __syncthreads();
      if (beta.h != 0.f) {
        refl_left(H, k, 3, max(l, k - 1), r, v, beta);
        __syncthreads();
        {
          float2* A = tid < 64 ? H : Z;
          const int rn = tid < 64 ? min(k + 4, hi + 1) : r;
          refl_right(A, 0, rn, k, 3, v, beta, tid & 63, 64);
        }
        __syncthreads();
        if (k > l && tid == 0) {
          H[(k + 1) * kLD + k - 1] = make_float2(0.f, 0.f);
          H[(k + 2) * kLD + k - 1] = make_float2(0.f, 0.f);
        }
        __syncthreads();
      }
      x = HH(H, k + 1, k);
      y = HH(H, k + 2, k);
      if (k < hi - 2) zz = HH(H, k + 3, k);
    }
    {
      const dd a2[2] = {x, y};
      dd v[3];
      const dd beta = house3(a2, 2, v);
      __syncthreads();
      if (beta.h != 0.f) {
        refl_left(H, hi - 1, 2, max(l, hi - 2), r, v, beta);
        __syncthreads();
        {
          float2* A = tid < 64 ? H : Z;
          const int rn = tid < 64 ? hi + 1 : r;
          refl_right(A, 0, rn, hi - 1, 2, v, beta, tid & 63, 64);
        }
        __syncthreads();
        if (hi - 2 >= l && tid == 0) H[hi * kLD + hi - 2] = make_float2(0.f, 0.f);
        __syncthreads();
      }
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(&ctl->status, DEV_EIG_NOCONV);
      ctl->eig_r = r;
      ctl->eig_valid = 1;
    }
    return;
  }
  __syncthreads();

  // ---- eigenvectors of T by back substitution (one thread per eigenvector); column j
  // solves (T - lambda_j) x = 0: x_j = 1 for a real eigenvalue; for a complex pair
  // (j, j+1) with wi[j] > 0 the block's eigenvector starts the substitution and column
  // j+1 receives the conjugate afterwards.
  float tnorm = 0.f;
  for (int idx = 0; idx < r * r; ++idx) tnorm = fmaxf(tnorm, fabsf(H[(idx / r) * kLD + idx % r].x));
  const float smin = fmaxf(kEpsDD * tnorm, 1e-30f);
  for (int j = tid; j < r; j += kEigThreads) {
    const cdd lam{dd_of(E.wr[j]), dd_of(E.wi[j])};
    if (lam.im.h < 0.f) continue;
    for (int i = 0; i < r; ++i) {
      E.Xr[i * kLD + j] = make_float2(0.f, 0.f);
      E.Xi[i * kLD + j] = make_float2(0.f, 0.f);
    }
    if (lam.im.h == 0.f) {
      E.Xr[j * kLD + j] = make_float2(1.f, 0.f);
    } else {
      const dd a = HH(H, j, j), b = HH(H, j, j + 1), c = HH(H, j + 1, j), d = HH(H, j + 1, j + 1);
      if (fabsf(b.h) >= fabsf(c.h)) {
        E.Xr[j * kLD + j] = f2_of(b);
        E.Xr[(j + 1) * kLD + j] = f2_of(lam.re - a);
        E.Xi[(j + 1) * kLD + j] = f2_of(lam.im);
      } else {
        E.Xr[j * kLD + j] = f2_of(lam.re - d);
        E.Xi[j * kLD + j] = f2_of(lam.im);
        E.Xr[(j + 1) * kLD + j] = f2_of(c);
      }
    }
    int i = j - 1;
    while (i >= 0) {
      const bool pair = (i > 0) && H[i * kLD + i - 1].x != 0.f;
      const int i0 = pair ? i - 1 : i;
      cdd r1{dzero(), dzero()}, r0v{dzero(), dzero()};
      for (int k = i + 1; k < r; ++k) {
        const cdd xk{HH(E.Xr, k, j), HH(E.Xi, k, j)};
        const dd h1 = HH(H, i, k);
        r1 = r1 - cdd{h1 * xk.re, h1 * xk.im};
        if (pair) {
          const dd h0 = HH(H, i0, k);
          r0v = r0v - cdd{h0 * xk.re, h0 * xk.im};
        }
      }
      if (!pair) {
        cdd den{HH(H, i, i) - lam.re, -lam.im};
        if (fabsf(den.re.h) + fabsf(den.im.h) < smin) den.re = dd_of(smin);
        const cdd xi = cdd_div(r1, den);
        E.Xr[i * kLD + j] = f2_of(xi.re);
        E.Xi[i * kLD + j] = f2_of(xi.im);
        i -= 1;
      } else {
        // [[a - lam, b], [c, d - lam]] [x0; x1] = [r0; r1]
        const cdd am{HH(H, i0, i0) - lam.re, -lam.im};
        const cdd dm{HH(H, i, i) - lam.re, -lam.im};
        const dd bb = HH(H, i0, i), cc = HH(H, i, i0);
        cdd det = am * dm - cdd{bb * cc, dzero()};
        if (fabsf(det.re.h) + fabsf(det.im.h) < smin * tnorm) det.re = dd_of(smin * tnorm);
        const cdd n0 = r0v * dm - cdd{bb * r1.re, bb * r1.im};
        const cdd n1 = am * r1 - cdd{cc * r0v.re, cc * r0v.im};
        const cdd x0 = cdd_div(n0, det), x1 = cdd_div(n1, det);
        E.Xr[i0 * kLD + j] = f2_of(x0.re);
        E.Xi[i0 * kLD + j] = f2_of(x0.im);
        E.Xr[i * kLD + j] = f2_of(x1.re);
        E.Xi[i * kLD + j] = f2_of(x1.im);
        i -= 2;
      }
      float mx = 0.f;
      for (int k = 0; k < r; ++k) mx = fmaxf(mx, fabsf(E.Xr[k * kLD + j].x) + fabsf(E.Xi[k * kLD + j].x));
      if (mx > 1e8f) {
        int e = 0;
        frexpf(mx, &e);
        for (int k = 0; k < r; ++k) {
          E.Xr[k * kLD + j] = f2_of(dd_ldexp(HH(E.Xr, k, j), -e));
          E.Xi[k * kLD + j] = f2_of(dd_ldexp(HH(E.Xi, k, j), -e));
        }
      }
    }
  }
  __syncthreads();
  // ---- V = D Z X, unit 2-norm columns; conjugate partners
  float2* Vre = ws.eig.Vre;
  float2* Vim = ws.eig.Vim;
  for (int j = 0; j < r; ++j) {
    if (E.wi[j].x < 0.f) continue;
    for (int row = tid; row < r; row += kEigThreads) {
      dd sr = dzero(), si = dzero();
      for (int k = 0; k < r; ++k) {
        sr = dd_fma(HH(Z, row, k), HH(E.Xr, k, j), sr);
        si = dd_fma(HH(Z, row, k), HH(E.Xi, k, j), si);
      }
      E.tmp[row] = f2_of(sr * E.scale[row]);
      E.v[row] = f2_of(si * E.scale[row]);
    }
    __syncthreads();
    if (tid < 32) {
      dd nrm = dzero();
      for (int row = tid; row < r; row += 32)
        nrm = dd_fma(LD(E.tmp, row), LD(E.tmp, row), dd_fma(LD(E.v, row), LD(E.v, row), nrm));
      nrm = dd_warp_sum(nrm);
      if (tid == 0) nrm_s[0] = f2_of(nrm.h > 0.f ? dd_div(dd_of(1.f), dd_sqrt(nrm)) : dzero());
    }
    __syncthreads();
    const dd inv = dd_of(nrm_s[0]);
    for (int row = tid; row < r; row += kEigThreads) {
      const dd re = LD(E.tmp, row) * inv, im = LD(E.v, row) * inv;
      Vre[(size_t)j * rm + row] = f2_of(re);
      Vim[(size_t)j * rm + row] = f2_of(im);
      if (E.wi[j].x > 0.f) {
        Vre[(size_t)(j + 1) * rm + row] = f2_of(re);
        Vim[(size_t)(j + 1) * rm + row] = f2_of(-im);
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < r; j += kEigThreads) {
    ws.eig.lre[j] = E.wr[j];
    ws.eig.lim[j] = E.wi[j];
  }
  __syncthreads();

  // ---- b = V^{-1} (S * r_first): complex Gaussian elimination with partial pivoting
  float2* Ar = E.H;
  float2* Ai = E.Z;
  float2* br = E.tmp;
  float2* bi = E.v;
  for (int idx = tid; idx < r * r; idx += kEigThreads) {
    const int i = idx / r, k = idx % r;
    Ar[i * kLD + k] = Vre[(size_t)k * rm + i];
    Ai[i * kLD + k] = Vim[(size_t)k * rm + i];
  }
  for (int i = tid; i < r; i += kEigThreads) {
    br[i] = f2_of(LD(st.S, i) * LD(st.rf, i));
    bi[i] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  float amax = 0.f;
  for (int idx = 0; idx < r * r; ++idx)
    amax = fmaxf(amax, fabsf(Ar[(idx / r) * kLD + idx % r].x) + fabsf(Ai[(idx / r) * kLD + idx % r].x));
  bool singular = false;
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      int piv = k;
      float pv = 0.f;
      for (int i = k; i < r; ++i) {
        const float a = fabsf(Ar[i * kLD + k].x) + fabsf(Ai[i * kLD + k].x);
        if (a > pv) {
          pv = a;
          piv = i;
        }
      }
      piv_s = pv > 0.f ? piv : -1;
      if (pv <= 1e-13f * amax) singular = true;
    }
    __syncthreads();
    const int piv = piv_s;
    if (piv < 0) break;
    if (piv != k) {
      for (int c = tid; c < r; c += kEigThreads) {
        float2 t = Ar[k * kLD + c];
        Ar[k * kLD + c] = Ar[piv * kLD + c];
        Ar[piv * kLD + c] = t;
        t = Ai[k * kLD + c];
        Ai[k * kLD + c] = Ai[piv * kLD + c];
        Ai[piv * kLD + c] = t;
      }
      if (tid == 0) {
        float2 t = br[k];
        br[k] = br[piv];
        br[piv] = t;
        t = bi[k];
        bi[k] = bi[piv];
        bi[piv] = t;
      }
    }
    __syncthreads();
    const cdd pk{HH(Ar, k, k), HH(Ai, k, k)};
    // multipliers of rows k+1.. (one thread per row), then the updates split by column
    for (int i = k + 1 + tid; i < r; i += kEigThreads) {
      const cdd f = cdd_div(cdd{HH(Ar, i, k), HH(Ai, i, k)}, pk);
      Ar[i * kLD + k] = f2_of(f.re);
      Ai[i * kLD + k] = f2_of(f.im);
    }
    __syncthreads();
    const int rows = r - k - 1, cols = r - k;  // columns k+1..r-1 plus the right-hand side
    for (int idx = tid; idx < rows * cols; idx += kEigThreads) {
      const int i = k + 1 + idx / cols, cc = idx % cols;
      const cdd f{HH(Ar, i, k), HH(Ai, i, k)};
      if (cc < cols - 1) {
        const int c = k + 1 + cc;
        const cdd x{HH(Ar, k, c), HH(Ai, k, c)};
        const cdd y = cdd{HH(Ar, i, c), HH(Ai, i, c)} - f * x;
        Ar[i * kLD + c] = f2_of(y.re);
        Ai[i * kLD + c] = f2_of(y.im);
      } else {
        const cdd x{LD(br, k), LD(bi, k)};
        const cdd y = cdd{LD(br, i), LD(bi, i)} - f * x;
        br[i] = f2_of(y.re);
        bi[i] = f2_of(y.im);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int i = r - 1; i >= 0; --i) {
      cdd s{LD(br, i), LD(bi, i)};
      for (int c = i + 1; c < r; ++c) s = s - cdd{HH(Ar, i, c), HH(Ai, i, c)} * cdd{LD(br, c), LD(bi, c)};
      const cdd pv{HH(Ar, i, i), HH(Ai, i, i)};
      const cdd x = (pv.re.h != 0.f || pv.im.h != 0.f) ? cdd_div(s, pv) : cdd{dzero(), dzero()};
      br[i] = f2_of(x.re);
      bi[i] = f2_of(x.im);
    }
    for (int i = 0; i < r; ++i) {
      ws.eig.bre[i] = br[i];
      ws.eig.bim[i] = bi[i];
      if (!isfinite(br[i].x) || !isfinite(bi[i].x)) singular = true;
    }
    if (singular) atomicOr(&ctl->status, DEV_EIG_COND);
    ctl->eig_r = r;
    ctl->eig_valid = 1;
  }
}

// ---------------------------------------------------------------------------------------
// rollout coefficients: coef[:, j] = Q Re(V Lambda^{t_j} b)  (r0 values, L0 coordinates)
// Lambda^t: for integer t by binary powering in complex double-float; otherwise from
// |lambda|^t and t arg(lambda) in FP64 (principal branch).
// ---------------------------------------------------------------------------------------
struct TArr {
  double t[kRollK];
};
struct TOrd {
  int i[kRollK];
};

__device__ cdd cpow_int(cdd base, long long e) {
  cdd res{dd_of(1.f), dzero()};
  while (e > 0) {
    if (e & 1) res = res * base;
    e >>= 1;
    if (e) base = base * base;
  }
  return res;
}

__global__ void __launch_bounds__(64) k_coef(Ws ws, TArr ts, int k) {
  Ctl* ctl = ws.ctl;
  const int j = blockIdx.x;
  if (j >= k) return;
  const StateBuf st = ws.st[ctl->cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, rm = ws.rmax, qld = ws.cap + 1;
  const int tid = threadIdx.x;
  __shared__ float2 gr[kMaxR], gi[kMaxR], c[kMaxR];
  const double t = ts.t[j];
  const bool integral = (t == floor(t)) && t < 9.0e15;
  for (int l = tid; l < r; l += 64) {
    const cdd lam{LD(ws.eig.lre, l), LD(ws.eig.lim, l)};
    const cdd b{LD(ws.eig.bre, l), LD(ws.eig.bim, l)};
    cdd pw;
    if (t == 0.0) {
      pw = cdd{dd_of(1.f), dzero()};
    } else if (lam.re.h == 0.f && lam.im.h == 0.f) {
      pw = cdd{dzero(), dzero()};
    } else if (integral) {
      pw = cpow_int(lam, (long long)t);
    } else {
      const double lr = dd_to_double(lam.re), li = dd_to_double(lam.im);
      const double mag = pow(hypot(lr, li), t);
      double sn, cs;
      sincos(t * atan2(li, lr), &sn, &cs);
      pw = cdd{dd_from_double(mag * cs), dd_from_double(mag * sn)};
    }
    const cdd g = pw * b;
    gr[l] = f2_of(g.re);
    gi[l] = f2_of(g.im);
  }
  __syncthreads();
  for (int i = tid; i < r; i += 64) {
    dd acc = dzero();
    for (int l = 0; l < r; ++l) {
      acc = dd_fma(LD(ws.eig.Vre, (size_t)l * rm + i), LD(gr, l), acc);
      acc = acc - LD(ws.eig.Vim, (size_t)l * rm + i) * LD(gi, l);
    }
    c[i] = f2_of(acc);
  }
  __syncthreads();
  for (int i = tid; i < r0; i += 64) {
    dd acc = dzero();
    for (int l = 0; l < r; ++l) acc = dd_fma(LD(st.Q, (size_t)l * qld + i), LD(c, l), acc);
    ws.sm.coef[(size_t)j * qld + i] = f2_of(acc);
  }
}

// Rollout coefficients for integer horizons without the eigensolve: with A~ = V Lambda V^-1
// and b = V^-1 y, y = S * r_first = L^T u^0,  V Lambda^t b = A~^t y  exactly, so
// coef[:, j] = Q A~^{t_j} y.  The horizons are taken in ascending order (ord): the vector
// advances by single products with A~ over short gaps and by binary powering (repeated
// squaring of A~, applied to the vector on set bits) over long ones.  Double-float
// throughout; one CTA.
constexpr int kPowThreads = 1024;  // eight warps per scheduler hide the latency of the dependent double-float sums
constexpr int kPowDirect = 8;  // gaps up to this many steps: repeated products
// row stride of the r x r matrices: one element more than kMaxR, so that the rows a warp
// reads at the same column fall in different shared-memory banks
constexpr int kPowLd = kMaxR + 1;

struct PowSmem {
  float2 A[kMaxR * kPowLd];  // A~, row-major
  float2 P[kMaxR * kPowLd];  // current power of A~
  float2 T[kMaxR * kPowLd];  // scratch of a squaring
  float2 v[2][kMaxR];        // the vector, ping-pong
  float2 C[kRollK * kMaxR];  // A~^{t_j} y for every horizon j (row j)
};

// out = B v (B row-major r x r in shared memory), 4 threads per row
__device__ __forceinline__ void pow_matvec(const float2* B, const float2* v, float2* out, int r) {
  const int tid = threadIdx.x;
  for (int base = 0; base < 4 * r; base += kPowThreads) {
    const int i = (base + tid) >> 2, sub = tid & 3;
    dd acc = dzero();
    if (i < r)
      for (int l = sub; l < r; l += 4) acc = dd_fma(LD(B, (size_t)i * kPowLd + l), LD(v, l), acc);
    acc = group4_sum(acc);
    if (i < r && sub == 0) out[i] = f2_of(acc);
  }
}

__global__ void __launch_bounds__(kPowThreads) k_coef_pow(Ws ws, TArr ts, TOrd ord, int k) {
  extern __shared__ __align__(16) unsigned char pow_raw[];
  PowSmem& S = *reinterpret_cast<PowSmem*>(pow_raw);
  Ctl* ctl = ws.ctl;
  const StateBuf st = ws.st[ctl->cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, rm = ws.rmax, qld = ws.cap + 1;
  const int tid = threadIdx.x;
  if (r == 0) {
    if (tid == 0) atomicOr(&ctl->status, DEV_NOMODEL);
    return;
  }
  for (int idx = tid; idx < r * r; idx += kPowThreads) {
    const int i = idx / r, l = idx % r;
    S.A[i * kPowLd + l] = f2_of(dd_div(LD(st.M, (size_t)l * rm + i), LD(st.S, l)));
  }
  // start from a vector of the previous call when it belongs to this model: the latest of
  // its first and last horizons that is not after the first one asked for (a check of the
  // first or of the next state after a predict needs no powering)
  const unsigned long long ver = ctl->model_ver;
  int slot = -1;
  if (k > 0 && ctl->pc_ver == ver + 1ull) {
    const double t0 = ts.t[ord.i[0]];
    for (int q = 0; q < 2; ++q)
      if (ctl->pc_t[q] <= t0 && (slot < 0 || ctl->pc_t[q] > ctl->pc_t[slot])) slot = q;
  }
  long long tcur = slot >= 0 ? (long long)ctl->pc_t[slot] : 0;
  for (int l = tid; l < r; l += kPowThreads)
    S.v[0][l] = slot >= 0 ? ws.sm.pc[slot * kMaxN + l] : f2_of(LD(st.S, l) * LD(st.rf, l));
  __syncthreads();
  int cur = 0;  // S.v[cur] holds the vector
  for (int q = 0; q < k; ++q) {
    const int j = ord.i[q];
    long long d = (long long)ts.t[j] - tcur;
    tcur += d;
    if (d <= kPowDirect) {
      for (; d > 0; --d) {
        pow_matvec(S.A, S.v[cur], S.v[cur ^ 1], r);
        cur ^= 1;
        __syncthreads();
      }
    } else {
      for (int idx = tid; idx < r * r; idx += kPowThreads) S.P[(idx / r) * kPowLd + idx % r] = S.A[(idx / r) * kPowLd + idx % r];
      __syncthreads();
      while (d > 0) {
        if (d & 1) {
          pow_matvec(S.P, S.v[cur], S.v[cur ^ 1], r);
          cur ^= 1;
          __syncthreads();
        }
        d >>= 1;
        if (d) {  // P <- P P
          for (int base = 0; base < 4 * r * r; base += kPowThreads) {
            const int e = (base + tid) >> 2, sub = tid & 3;
            const int i = e / r, jj = e % r;
            dd acc = dzero();
            if (e < r * r)
              for (int l = sub; l < r; l += 4) acc = dd_fma(LD(S.P, (size_t)i * kPowLd + l), LD(S.P, (size_t)l * kPowLd + jj), acc);
            acc = group4_sum(acc);
            if (e < r * r && sub == 0) S.T[i * kPowLd + jj] = f2_of(acc);
          }
          __syncthreads();
          for (int idx = tid; idx < r * r; idx += kPowThreads) S.P[(idx / r) * kPowLd + idx % r] = S.T[(idx / r) * kPowLd + idx % r];
          __syncthreads();
        }
      }
    }
    for (int l = tid; l < r; l += kPowThreads) S.C[j * kMaxR + l] = S.v[cur][l];
    if (q == 0) {
      const long long tf = tcur;
      __syncthreads();  // slot 0 may be the vector this call started from
      for (int l = tid; l < r; l += kPowThreads) ws.sm.pc[l] = S.v[cur][l];
      if (tid == 0) ctl->pc_t[0] = (double)tf;
    }
    // (read only after the barrier that ends the next step, or the final one)
  }
  __syncthreads();
  // coef[:, j] = Q C[j] for every horizon at once (4 threads per output)
  for (int base = 0; base < 4 * r0 * k; base += kPowThreads) {
    const int e = (base + tid) >> 2, sub = tid & 3;
    const int i = e % r0, j = e / r0;
    dd acc = dzero();
    if (e < r0 * k)
      for (int l = sub; l < r; l += 4) acc = dd_fma(LD(st.Q, (size_t)l * qld + i), LD(S.C, (size_t)j * kMaxR + l), acc);
    acc = group4_sum(acc);
    if (e < r0 * k && sub == 0) ws.sm.coef[(size_t)j * qld + i] = f2_of(acc);
  }
  if (k > 0) {
    for (int l = tid; l < r; l += kPowThreads) ws.sm.pc[kMaxN + l] = S.v[cur][l];
    if (tid == 0) {
      ctl->pc_t[1] = (double)tcur;
      ctl->pc_ver = ver + 1ull;
    }
  }
  if (tid == 0) {
    bool bad = false;
    for (int l = 0; l < r; ++l) bad |= !dd_isfinite(LD(S.v[cur], l));
    if (bad) atomicOr(&ctl->status, DEV_NONFINITE);
  }
}

// basis export coefficients: coef[:, j] = Q[:, j]
__global__ void __launch_bounds__(64) k_basis_coef(Ws ws) {
  Ctl* ctl = ws.ctl;
  const StateBuf st = ws.st[ctl->cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, qld = ws.cap + 1;
  const int j = blockIdx.x;
  if (j >= r) return;
  for (int i = threadIdx.x; i < r0; i += 64) ws.sm.coef[(size_t)j * qld + i] = st.Q[(size_t)j * qld + i];
}

// ---------------------------------------------------------------------------------------
static int prep_smem_cap(int cap) {
  const int qld = cap + 1;
  return (int)sizeof(float2) * (qld * kMaxR + 4 * qld + 2 * kMaxN);
}
static int prep_smem(const Ws& ws) { return prep_smem_cap(ws.cap); }

// The shared-memory limit is a property of the kernel, shared by every handle in the
// process: set it for the largest cap any handle can have.
cudaError_t prepare_small(const Ws&) {
  cudaError_t e = cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, prep_smem_cap(kMaxCap));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EigSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_coef_pow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PowSmem));
}

cudaError_t launch_small(const Ws& ws, cudaStream_t s) {
  const int ps = prep_smem(ws);
  cudaError_t e = launch_dependent(k_prep, 1, kPrepThreads, ps, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_roots, kMaxN, 32, 0, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_zhat, kMaxN + 1, 32, 0, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_vectors, kMaxN, 64, 0, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_apply, kMaxN, kApplyThreads, 0, s, ws);
  return e;
}

cudaError_t launch_eig(const Ws& ws, cudaStream_t s) {
  const int bytes = (int)sizeof(EigSmem);
  k_eig<<<1, kEigThreads, bytes, s>>>(ws);
  return cudaGetLastError();
}

cudaError_t launch_coef(const Ws& ws, const double* t_host, int k, cudaStream_t s) {
  TArr ta;
  for (int i = 0; i < kRollK; ++i) ta.t[i] = i < k ? t_host[i] : 0.0;
  k_coef<<<k, 64, 0, s>>>(ws, ta, k);
  return cudaGetLastError();
}

// integer horizons only (the caller checks): coefficients by powers of A~, no eigensolve
cudaError_t launch_coef_pow(const Ws& ws, const double* t_host, int k, cudaStream_t s) {
  TArr ta;
  TOrd ord;
  for (int i = 0; i < kRollK; ++i) {
    ta.t[i] = i < k ? t_host[i] : 0.0;
    ord.i[i] = i;
  }
  // ascending order of the horizons (insertion sort of at most kRollK indices, stable)
  for (int a = 1; a < k; ++a) {
    const int v = ord.i[a];
    int b = a - 1;
    while (b >= 0 && ta.t[ord.i[b]] > ta.t[v]) {
      ord.i[b + 1] = ord.i[b];
      --b;
    }
    ord.i[b + 1] = v;
  }
  k_coef_pow<<<1, kPowThreads, sizeof(PowSmem), s>>>(ws, ta, ord, k);
  return cudaGetLastError();
}

cudaError_t launch_basis_coef(const Ws& ws, cudaStream_t s) {
  k_basis_coef<<<kMaxR, 64, 0, s>>>(ws);
  return cudaGetLastError();
}

cudaError_t launch_init(const Ws&, cudaStream_t) { return cudaSuccess; }

}  // namespace odmd
