// Small dense solves in double-float arithmetic (dd.cuh) on the FP32 pipes: the
// eigen-cache and the modal coefficients of predictions and checks.  (The small solves of
// the update itself, which feed back into every later model, run in FP64: core.cu.)
//
// Eigensolve (lazy, Sec. 2.3: A~ = V Lambda V^{-1}, b = Phi^+ u^0): balancing by powers of
// two, Householder reduction to Hessenberg form, Francis double-shift QR with Schur
// vectors (Golub and Van Loan, Matrix Computations, Ch. 7), eigenvectors of the
// quasi-triangular factor by back substitution, then b from a complex LU solve.  The
// inputs M, S and r_first are read from their FP64 state and rounded to double-float.
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
    H[i * kLD + k] = f2_of(dd_from_double(st.M[(size_t)k * rm + i] / st.S[k]));
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
    br[i] = f2_of(dd_from_double(st.S[i] * st.rf[i]));
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
    for (int l = 0; l < r; ++l) acc = dd_fma(dd_from_double(st.Q[(size_t)l * qld + i]), LD(c, l), acc);
    ws.sm.coef[(size_t)j * qld + i] = f2_of(acc);
  }
}

// Rollout coefficients for integer horizons without the eigensolve: with A~ = V Lambda V^-1
// and b = V^-1 y, y = S * r_first = L^T u^0,  V Lambda^t b = A~^t y  exactly, so
// coef[:, j] = Q A~^{t_j} y.  The horizons are taken in ascending order (ord).  The vector
// reaches the first horizon t_1 by single products with A~ over a short gap and by binary
// powering (repeated squaring of A~, applied to the vector on set bits) over a long one.
// When every other horizon lies within 63 steps of t_1 (a rollout of consecutive states),
// the vectors of all offsets 0 .. span-1 come from doubling rounds: round k multiplies the
// 2^k vectors of offsets 0 .. 2^k - 1 by A~^(2^k) at once (a small matrix product), so 50
// horizons take six products instead of 49 dependent ones.  Otherwise the horizons are
// reached one after another as before.  Then coef = Q C for all horizons in one product.
// Double-float throughout (the products accumulate two columns per FP32x2 instruction);
// one CTA.  Q and A~ = M diag(S)^-1 are rounded from their FP64 state to double-float once,
// into shared memory.
constexpr int kPowThreads = 1024;
constexpr int kPowDirect = 8;   // a gap up to this many steps: repeated products
constexpr int kPowLd = kMaxR + 2;  // even row stride: column pairs are 8-byte aligned
constexpr int kPowSpan = 64;    // offsets from the first horizon formed by doubling
constexpr int kPowQRows = kMaxCap + 1;

struct PowSmem {
  float Ah[kMaxR * kPowLd], Al[kMaxR * kPowLd];  // A~ (row-major planes: hi, lo)
  float Ph[kMaxR * kPowLd], Pl[kMaxR * kPowLd];  // a power of A~
  float Th[kMaxR * kPowLd], Tl[kMaxR * kPowLd];  // the next power (squaring output)
  float Vh[kMaxR * kPowLd], Vl[kMaxR * kPowLd];  // vectors as columns (an offset or a horizon each)
  float Qh[kPowQRows * kPowLd], Ql[kPowQRows * kPowLd];  // Q (r0 x r, row-major)
  float wh[2][kMaxR * 2], wl[2][kMaxR * 2];  // the advancing vector, ping-pong (column 0 of ld 2)
  int col_of[kRollK];                         // the column of Vh/Vl that holds horizon j
};

// Out[i][oc0 + c] = sum_{l < kdim} X[i][l] Y[l][c0 + c] for i < rows, c < ncol (planes
// row-major with the given row strides; c0, yld even).  A thread forms two adjacent output
// columns with packed double-float accumulation (acc2_fma); an odd last column pairs with
// zero instead of reading past the range.  `store(i, c, acc)` writes output column c.
template <class Store>
__device__ __forceinline__ void mm_dd(const float* Xh, const float* Xl, int xld, const float* Yh, const float* Yl,
                                      int yld, int c0, int rows, int kdim, int ncol, Store store) {
  const int npairs = (ncol + 1) >> 1;
  for (int it = threadIdx.x; it < rows * npairs; it += kPowThreads) {
    const int i = it / npairs, c = 2 * (it - i * npairs);
    const bool pair = c + 1 < ncol;
    Acc2 acc = acc2_zero();
    for (int l = 0; l < kdim; ++l) {
      const float xh = Xh[i * xld + l], xl = Xl[i * xld + l];
      const float* yh = Yh + l * yld + c0 + c;
      const float* yl = Yl + l * yld + c0 + c;
      const f2x ph = pair ? *reinterpret_cast<const f2x*>(yh) : f2x_pack(yh[0], 0.f);
      const f2x pl = pair ? *reinterpret_cast<const f2x*>(yl) : f2x_pack(yl[0], 0.f);
      acc2_fma(acc, ph, pl, f2x_pack(xh, xh), f2x_pack(-xh, -xh), f2x_pack(xl, xl));
    }
    Acc a0, a1;
    acc2_split(acc, a0, a1);
    store(i, c, acc_norm(a0));
    if (pair) store(i, c + 1, acc_norm(a1));
  }
}

// a store into a row-major plane pair at column offset oc0
struct PlaneStore {
  float* h;
  float* l;
  int ld, oc0;
  __device__ void operator()(int i, int c, Acc a) const {
    h[i * ld + oc0 + c] = a.h;
    l[i * ld + oc0 + c] = a.l;
  }
};

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
  if (k <= 0) return;
  // A~ = M diag(S)^-1 (one FP64 reciprocal per column) and Q, rounded to double-float once
  __shared__ double sinv[kMaxR];
  __shared__ int bad;
  for (int l = tid; l < r; l += kPowThreads) sinv[l] = 1.0 / st.S[l];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int idx = tid; idx < r * r; idx += kPowThreads) {
    const int i = idx / r, l = idx - i * r;
    const dd a = dd_from_double(st.M[(size_t)l * rm + i] * sinv[l]);
    S.Ah[i * kPowLd + l] = a.h;
    S.Al[i * kPowLd + l] = a.l;
  }
  for (int idx = tid; idx < r0 * r; idx += kPowThreads) {
    const int i = idx / r, l = idx - i * r;
    const dd q = dd_from_double(st.Q[(size_t)l * qld + i]);
    S.Qh[i * kPowLd + l] = q.h;
    S.Ql[i * kPowLd + l] = q.l;
  }
  // start from a vector of the previous call when it belongs to this model: the latest of
  // its first and last horizons that is not after the first one asked for (a check of the
  // first or of the next state after a predict needs no powering)
  const unsigned long long ver = ctl->model_ver;
  int slot = -1;
  const double t0 = ts.t[ord.i[0]];
  if (ctl->pc_ver == ver + 1ull)
    for (int q = 0; q < 2; ++q)
      if (ctl->pc_t[q] <= t0 && (slot < 0 || ctl->pc_t[q] > ctl->pc_t[slot])) slot = q;
  long long tcur = slot >= 0 ? (long long)ctl->pc_t[slot] : 0;
  for (int l = tid; l < r; l += kPowThreads) {
    const dd y = slot >= 0 ? dd_of(ws.sm.pc[slot * kMaxN + l]) : dd_from_double(st.S[l] * st.rf[l]);
    S.wh[0][2 * l] = y.h;
    S.wl[0][2 * l] = y.l;
  }
  __syncthreads();
  int cur = 0;  // S.wh[cur] holds the vector
  // vector <- A~^d vector: d single products, or binary powering (A~^(2^i) in P and T in turn)
  auto advance = [&](long long d) {
    if (d <= kPowDirect) {
      for (; d > 0; --d) {
        mm_dd(S.Ah, S.Al, kPowLd, S.wh[cur], S.wl[cur], 2, 0, r, r, 1, PlaneStore{S.wh[cur ^ 1], S.wl[cur ^ 1], 2, 0});
        cur ^= 1;
        __syncthreads();
      }
      return;
    }
    const float *bh = S.Ah, *bl = S.Al;
    float *nh = S.Ph, *nl = S.Pl;
    while (d > 0) {
      // the product with the vector and the next squaring read the same power and write
      // different buffers: one barrier for both
      if (d & 1) {
        mm_dd(bh, bl, kPowLd, S.wh[cur], S.wl[cur], 2, 0, r, r, 1, PlaneStore{S.wh[cur ^ 1], S.wl[cur ^ 1], 2, 0});
        cur ^= 1;
      }
      d >>= 1;
      if (d) mm_dd(bh, bl, kPowLd, bh, bl, kPowLd, 0, r, r, r, PlaneStore{nh, nl, kPowLd, 0});
      __syncthreads();
      if (d) {
        bh = nh;
        bl = nl;
        nh = (nh == S.Ph) ? S.Th : S.Ph;
        nl = (nl == S.Pl) ? S.Tl : S.Pl;
      }
    }
  };
  // column c of V <- the current vector
  auto keep = [&](int c) {
    for (int l = tid; l < r; l += kPowThreads) {
      S.Vh[l * kPowLd + c] = S.wh[cur][2 * l];
      S.Vl[l * kPowLd + c] = S.wl[cur][2 * l];
    }
  };
  advance((long long)t0 - tcur);
  tcur = (long long)t0;
  // the first horizon's vector is kept for later calls
  for (int l = tid; l < r; l += kPowThreads) ws.sm.pc[l] = make_float2(S.wh[cur][2 * l], S.wl[cur][2 * l]);
  if (tid == 0) ctl->pc_t[0] = t0;
  const double tlast = ts.t[ord.i[k - 1]];
  const long long span = (long long)tlast - (long long)t0 + 1;
  int last_col;
  if (span <= kPowSpan) {
    // doubling: offsets h .. 2h - 1 are A~^h times offsets 0 .. h - 1
    keep(0);
    __syncthreads();
    if (span > 1) {
      mm_dd(S.Ah, S.Al, kPowLd, S.Vh, S.Vl, kPowLd, 0, r, r, 1, PlaneStore{S.Vh, S.Vl, kPowLd, 1});
      __syncthreads();
    }
    const float *bh = S.Ah, *bl = S.Al;
    float *nh = S.Ph, *nl = S.Pl;
    for (int h = 2; h < span; h *= 2) {
      mm_dd(bh, bl, kPowLd, bh, bl, kPowLd, 0, r, r, r, PlaneStore{nh, nl, kPowLd, 0});  // A~^h
      __syncthreads();
      bh = nh;
      bl = nl;
      nh = (nh == S.Ph) ? S.Th : S.Ph;
      nl = (nl == S.Pl) ? S.Tl : S.Pl;
      const int ncols = (int)(span - h < h ? span - h : h);
      mm_dd(bh, bl, kPowLd, S.Vh, S.Vl, kPowLd, 0, r, r, ncols, PlaneStore{S.Vh, S.Vl, kPowLd, h});
      __syncthreads();
    }
    for (int j = tid; j < k; j += kPowThreads) S.col_of[j] = (int)((long long)ts.t[j] - (long long)t0);
    last_col = (int)(span - 1);
  } else {
    // spread horizons: one after another
    for (int q = 0; q < k; ++q) {
      const int j = ord.i[q];
      advance((long long)ts.t[j] - tcur);
      tcur = (long long)ts.t[j];
      keep(q);
      if (tid == 0) S.col_of[j] = q;
    }
    last_col = k - 1;
  }
  __syncthreads();
  // coef[:, j] = Q C[:, j], C[:, j] = V[:, col_of[j]] gathered into T first
  for (int idx = tid; idx < r * k; idx += kPowThreads) {
    const int l = idx / k, j = idx - l * k;
    S.Th[l * kPowLd + j] = S.Vh[l * kPowLd + S.col_of[j]];
    S.Tl[l * kPowLd + j] = S.Vl[l * kPowLd + S.col_of[j]];
  }
  for (int l = tid; l < r; l += kPowThreads)
    ws.sm.pc[kMaxN + l] = make_float2(S.Vh[l * kPowLd + last_col], S.Vl[l * kPowLd + last_col]);
  __syncthreads();
  float2* coef = ws.sm.coef;
  int* badp = &bad;
  mm_dd(S.Qh, S.Ql, kPowLd, S.Th, S.Tl, kPowLd, 0, r0, r, k, [=](int i, int j, Acc a) {
    coef[(size_t)j * qld + i] = make_float2(a.h, a.l);
    if (!isfinite(a.h) || !isfinite(a.l)) *badp = 1;
  });
  __syncthreads();
  if (tid == 0) {
    ctl->pc_t[1] = tlast;
    ctl->pc_ver = ver + 1ull;
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
  for (int i = threadIdx.x; i < r0; i += 64) ws.sm.coef[(size_t)j * qld + i] = d2f2(st.Q[(size_t)j * qld + i]);
}

// ---------------------------------------------------------------------------------------
// The shared-memory limit is a property of the kernel, shared by every handle in the
// process: set it for the largest cap any handle can have.
cudaError_t prepare_small(const Ws&) {
  cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EigSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_coef_pow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PowSmem));
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
