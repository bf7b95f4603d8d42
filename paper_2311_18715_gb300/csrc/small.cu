// Small dense solves of the online DMD update and of the eigen-cache, FP64.
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
// (a Givens rotation merges the weights of two equal poles).
//
// Eigensolve (lazy, Sec. 2.3: A~ = V Lambda V^{-1}, b = Phi^+ u^0): balancing by powers of
// two, Householder reduction to Hessenberg form, Francis double-shift QR with Schur
// vectors (Golub and Van Loan, Matrix Computations, Ch. 7), eigenvectors of the
// quasi-triangular factor by back substitution, then b from a complex LU solve.
#include "odmd_internal.cuh"

namespace odmd {

constexpr double kEps = 1.1102230246251565e-16;  // 2^-53

// ---------------------------------------------------------------------------------------
// k_prep
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_prep(Ws ws) {
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, qld = ws.cap + 1;
  const double* red = ws.sm.red;
  __shared__ double ac[kMaxCap + 1], yext[kMaxCap + 1], z[kMaxCap + 1], p[kMaxN], p2[kMaxN];
  __shared__ double sc[8];
  __shared__ double dd[kMaxN], zc[kMaxN];

  for (int i = tid; i < r0; i += 128) {
    ac[i] = st.a[i] + red[i];
    yext[i] = red[r0 + i];
  }
  __syncthreads();
  if (tid == 0) {
    double ssq = 0.0, sy = 0.0;
    for (int i = 0; i < r0; ++i) {
      ssq = fma(red[i], red[i], ssq);
      sy = fma(red[i], red[r0 + i], sy);
    }
    const double eta = red[2 * r0], ex = red[2 * r0 + 1];
    const double rho0 = sqrt(fmax(eta - ssq, 0.0));
    const double cn = sqrt(fmax(st.hdr->cn2, 0.0));
    const double sig1 = r > 0 ? st.S[0] : 0.0;
    const double thr = ws.tau * fmax(sig1, cn);
    const int append = rho0 > thr ? 1 : 0;
    ctl->thr = thr;
    ctl->rho0 = rho0;
    ctl->append = append;
    ctl->r0e = r0 + append;
    if (append) {
      ac[r0] = rho0;
      yext[r0] = (ex - sy) / rho0;
    }
    sc[0] = append;
  }
  __syncthreads();
  const int append = (int)sc[0];
  const int r0e = r0 + append;
  // p = Q^T ac (Q has r0 rows; the appended coordinate is outside span(L))
  for (int j = tid; j < r; j += 128) {
    double acc = 0.0;
    for (int i = 0; i < r0; ++i) acc = fma(st.Q[(size_t)j * qld + i], ac[i], acc);
    p[j] = acc;
  }
  __syncthreads();
  for (int i = tid; i < r0e; i += 128) {
    double acc = ac[i];
    if (i < r0)
      for (int j = 0; j < r; ++j) acc = fma(-st.Q[(size_t)j * qld + i], p[j], acc);
    z[i] = acc;
  }
  __syncthreads();
  // second Gram-Schmidt pass in the small space
  for (int j = tid; j < r; j += 128) {
    double acc = 0.0;
    for (int i = 0; i < r0; ++i) acc = fma(st.Q[(size_t)j * qld + i], z[i], acc);
    p2[j] = acc;
  }
  __syncthreads();
  for (int i = tid; i < r0; i += 128) {
    double acc = z[i];
    for (int j = 0; j < r; ++j) acc = fma(-st.Q[(size_t)j * qld + i], p2[j], acc);
    z[i] = acc;
  }
  for (int j = tid; j < r; j += 128) p[j] += p2[j];
  __syncthreads();
  if (tid == 0) {
    double zz = 0.0;
    for (int i = 0; i < r0e; ++i) zz = fma(z[i], z[i], zz);
    double rho = sqrt(zz);
    if (!(rho > ctl->thr)) rho = 0.0;
    sc[1] = rho;
    ctl->rho = rho;
  }
  __syncthreads();
  const double rho = sc[1];
  for (int i = tid; i < r0e; i += 128) {
    ws.sm.qn[i] = rho > 0.0 ? z[i] / rho : 0.0;
    ws.sm.yext[i] = yext[i];
    if (i < r0) ws.sm.ac[i] = ac[i];
  }
  // w = L^T x = Q^T y
  for (int j = tid; j < r; j += 128) {
    double acc = 0.0;
    for (int i = 0; i < r0; ++i) acc = fma(st.Q[(size_t)j * qld + i], yext[i], acc);
    ws.sm.w[j] = acc;
    ws.sm.p[j] = p[j];
  }
  __syncthreads();
  if (tid == 0) {
    double g = 0.0;
    if (rho > 0.0)
      for (int i = 0; i < r0e; ++i) g = fma(z[i] / rho, yext[i], g);
    ctl->gamma = g;
    // ---- secular problem of K = [[diag(S), p], [0, rho]], n = r + 1
    const int n = r + 1;
    double zmax = 0.0;
    for (int i = 0; i < n; ++i) {
      dd[i] = i < r ? st.S[i] : 0.0;
      zc[i] = i < r ? p[i] : rho;
      zmax = fmax(zmax, fabs(zc[i]));
    }
    const double tol = 8.0 * kEps * fmax(r > 0 ? dd[0] : 0.0, zmax);
    int* defl = ws.sm.defl;
    int ndefl = 0, nrot = 0;
    bool isdefl[kMaxN];
    for (int i = 0; i < n; ++i) {
      isdefl[i] = !(fabs(zc[i]) > tol);
      if (isdefl[i]) zc[i] = 0.0;
    }
    // merge nearly equal poles (coordinate r, the pole at 0, is never merged)
    int last = -1;
    for (int i = 0; i < r; ++i) {
      if (isdefl[i]) continue;
      if (last >= 0 && dd[last] - dd[i] <= tol) {
        const double h = hypot(zc[last], zc[i]);
        const double c = zc[last] / h, s = zc[i] / h;
        zc[last] = h;
        zc[i] = 0.0;
        isdefl[i] = true;
        ws.sm.rot_i[nrot] = last;
        ws.sm.rot_j[nrot] = i;
        ws.sm.rot_c[nrot] = c;
        ws.sm.rot_s[nrot] = s;
        ++nrot;
      } else {
        last = i;
      }
    }
    int m = 0;
    for (int i = n - 1; i >= 0; --i) {  // ascending poles
      if (isdefl[i]) {
        defl[ndefl++] = i;
      } else {
        ws.sm.pole[m] = i;
        ws.sm.d[m] = dd[i];
        ws.sm.z[m] = zc[i];
        ++m;
      }
    }
    for (int i = 0; i < n; ++i) ws.sm.zrot[i] = zc[i];
    ctl->n = n;
    ctl->m = m;
    ctl->ndefl = ndefl;
    ctl->nrot = nrot;
    if (!isfinite(tol) || !isfinite(rho)) atomicOr(&ctl->status, DEV_NONFINITE);
  }
}

// ---------------------------------------------------------------------------------------
// k_roots: root j of 1 + sum_i z_i^2/(d_i^2 - lambda) = 0 in (d_j^2, d_{j+1}^2)
// ---------------------------------------------------------------------------------------
struct SecSums {
  double psi, dpsi, phi, dphi;
};

// sums over poles i <= j (psi) and i > j (phi) at lambda = d_o^2 + mu
__device__ SecSums sec_eval(const double* d, const double* z, int m, int j, int o, double mu) {
  SecSums s{0.0, 0.0, 0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const double dob = d[o];
  for (int i = lane; i < m; i += 32) {
    const double del = (d[i] - dob) * (d[i] + dob) - mu;  // d_i^2 - lambda
    const double zi = z[i];
    const double t = zi / del;
    const double term = zi * t, dterm = t * t;
    if (i <= j) {
      s.psi += term;
      s.dpsi += dterm;
    } else {
      s.phi += term;
      s.dphi += dterm;
    }
  }
  s.psi = warp_sum_d(s.psi);
  s.dpsi = warp_sum_d(s.dpsi);
  s.phi = warp_sum_d(s.phi);
  s.dphi = warp_sum_d(s.dphi);
  return s;
}

__global__ void __launch_bounds__(32) k_roots(Ws ws) {
  Ctl* ctl = ws.ctl;
  const int m = ctl->m;
  const int j = blockIdx.x;
  if (j >= m) return;
  const double* d = ws.sm.d;
  const double* z = ws.sm.z;
  const int lane = threadIdx.x;
  double zsq = 0.0;
  for (int i = lane; i < m; i += 32) zsq = fma(z[i], z[i], zsq);
  zsq = warp_sum_d(zsq);
  if (m == 1) {
    if (lane == 0) {
      ws.sm.org[0] = 0;
      ws.sm.mu[0] = zsq;
      ws.sm.sig[0] = sqrt(d[0] * d[0] + zsq);
    }
    return;
  }
  int o;
  double lo, hi;  // bracket of mu, relative to d_o^2
  double A, B;    // left and right pole relative to d_o^2 (B unused for the last root)
  const bool last = (j == m - 1);
  if (!last) {
    const double gap = (d[j + 1] - d[j]) * (d[j + 1] + d[j]);
    const double mid = 0.5 * gap;
    SecSums s = sec_eval(d, z, m, j, j, mid);
    if (1.0 + s.psi + s.phi >= 0.0) {
      o = j;
      lo = 0.0;
      hi = mid;
      A = 0.0;
      B = gap;
    } else {
      o = j + 1;
      lo = -mid;
      hi = 0.0;
      A = -gap;
      B = 0.0;
    }
  } else {
    o = j;
    lo = 0.0;
    hi = zsq;
    A = 0.0;
    B = 0.0;
  }
  double mu = 0.5 * (lo + hi);
  bool conv = false;
  for (int it = 0; it < 64; ++it) {
    const SecSums s = sec_eval(d, z, m, j, o, mu);
    const double f = 1.0 + s.psi + s.phi;
    if (f < 0.0)
      lo = mu;
    else
      hi = mu;
    const double ftol = 8.0 * kEps * (double)m * (1.0 + fabs(s.psi) + fabs(s.phi));
    if (fabs(f) <= ftol) {
      conv = true;
      break;
    }
    // two-pole rational model of f matching value and slope at mu
    const double c1 = s.dpsi * (A - mu) * (A - mu);
    const double a1 = s.psi - s.dpsi * (A - mu);
    double x;
    if (!last) {
      const double c2 = s.dphi * (B - mu) * (B - mu);
      const double a2 = s.phi - s.dphi * (B - mu);
      const double C = 1.0 + a1 + a2;
      // C (A-x)(B-x) + c1 (B-x) + c2 (A-x) = 0
      const double qa = C;
      const double qb = -(C * (A + B) + c1 + c2);
      const double qc = C * A * B + c1 * B + c2 * A;
      if (fabs(qa) <= kEps * (fabs(qb) + fabs(qc))) {
        x = -qc / qb;
      } else {
        const double disc = fmax(qb * qb - 4.0 * qa * qc, 0.0);
        const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
        const double x1 = q / qa, x2 = qc / q;
        const bool in1 = x1 > lo && x1 < hi, in2 = x2 > lo && x2 < hi;
        x = in1 && !in2 ? x1 : (in2 && !in1 ? x2 : (fabs(x1 - mu) < fabs(x2 - mu) ? x1 : x2));
      }
    } else {
      const double C = 1.0 + a1 + s.phi;
      x = C > 0.0 ? A + c1 / C : 0.5 * (lo + hi);
    }
    if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
    const double step = fabs(x - mu);
    mu = x;
    if (step <= 4.0 * kEps * fabs(mu) || hi - lo <= 4.0 * kEps * fmax(fabs(lo), fabs(hi))) {
      conv = true;
      break;
    }
  }
  if (lane == 0) {
    if (!conv) atomicOr(&ctl->status, DEV_SECULAR);
    ws.sm.org[j] = o;
    ws.sm.mu[j] = mu;
    ws.sm.sig[j] = sqrt(fmax(d[o] * d[o] + mu, 0.0));
  }
}

// ---------------------------------------------------------------------------------------
// k_zhat: Loewner weights z^_i^2 = prod_k (lambda_k - d_i^2) / prod_{k != i} (d_k^2 - d_i^2),
// paired so every factor is O(1).  Block kMaxN orders all singular values of K.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_zhat(Ws ws) {
  Ctl* ctl = ws.ctl;
  const int m = ctl->m, n = ctl->n;
  const int lane = threadIdx.x;
  if (blockIdx.x == kMaxN) {
    // order: roots (sig[0..m)) and deflated values (d at coordinate defl[k]); descending
    const StateBuf st = ws.st[ctl->cur];
    const int r = st.hdr->r;
    const int ndefl = ctl->ndefl;
    __shared__ double val[kMaxN];
    __shared__ int code[kMaxN];
    const int tot = m + ndefl;  // == n
    for (int e = lane; e < tot; e += 32) {
      if (e < m) {
        val[e] = ws.sm.sig[e];
        code[e] = e;
      } else {
        const int c = ws.sm.defl[e - m];
        val[e] = c < r ? st.S[c] : 0.0;
        code[e] = -c - 1;
      }
    }
    __syncwarp();
    double vmax = 0.0;
    for (int e = 0; e < tot; ++e) vmax = fmax(vmax, val[e]);
    const double cut = ws.tau * vmax;
    for (int e = lane; e < tot; e += 32) {
      int pos = 0;
      for (int f = 0; f < tot; ++f) pos += (val[f] > val[e]) || (val[f] == val[e] && f < e);
      ws.sm.src[pos] = code[e];
      ws.sm.sig[kMaxN + pos] = val[e];  // sorted copy after the root slots
    }
    if (lane == 0) {
      int keep = 0;
      if (vmax > 0.0)
        for (int e = 0; e < tot; ++e) keep += val[e] > cut;
      ctl->rnew = min(keep, ws.rmax);
      (void)n;
    }
    return;
  }
  const int i = blockIdx.x;
  if (i >= m) return;
  const double* d = ws.sm.d;
  const double di = d[i];
  double prod = 1.0;
  for (int k = lane; k < m; k += 32) {
    const int o = ws.sm.org[k];
    const double lam_m_di = ws.sm.mu[k] - (di - d[o]) * (di + d[o]);  // lambda_k - d_i^2
    double f;
    if (k == m - 1)
      f = lam_m_di;
    else if (k < i)
      f = lam_m_di / ((d[k] - di) * (d[k] + di));
    else
      f = lam_m_di / ((d[k + 1] - di) * (d[k + 1] + di));
    prod *= f;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) prod *= __shfl_xor_sync(0xffffffffu, prod, off);
  if (lane == 0) ws.sm.zhat[i] = copysign(sqrt(fmax(prod, 0.0)), ws.sm.z[i]);
}

// ---------------------------------------------------------------------------------------
// k_vectors: kept column j -> u_j, v_j (core coordinates 0..r; r is the p/rho column)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_vectors(Ws ws) {
  Ctl* ctl = ws.ctl;
  const int j = blockIdx.x;
  if (j >= ctl->rnew) return;
  const int n = ctl->n, m = ctl->m, r = n - 1;
  const int tid = threadIdx.x;
  __shared__ double u[kMaxN], v[kMaxN], red[4];
  for (int i = tid; i < n; i += 64) {
    u[i] = 0.0;
    v[i] = 0.0;
  }
  __syncthreads();
  const int code = ws.sm.src[j];
  if (code >= 0) {
    const double* d = ws.sm.d;
    const int o = ws.sm.org[code];
    const double mu = ws.sm.mu[code];
    for (int i = tid; i < m; i += 64) {
      const double del = (d[i] - d[o]) * (d[i] + d[o]) - mu;  // d_i^2 - lambda
      const double ui = ws.sm.zhat[i] / del;
      const int c = ws.sm.pole[i];
      u[c] = ui;
      if (c < r) v[c] = d[i] * ui;
    }
    __syncthreads();
    if (tid == 0) v[r] = -1.0;
    __syncthreads();
    double su = 0.0, sv = 0.0;
    for (int i = tid; i < n; i += 64) {
      su = fma(u[i], u[i], su);
      sv = fma(v[i], v[i], sv);
    }
    su = warp_sum_d(su);
    sv = warp_sum_d(sv);
    if ((tid & 31) == 0) {
      red[(tid >> 5) * 2] = su;
      red[(tid >> 5) * 2 + 1] = sv;
    }
    __syncthreads();
    const double iu = 1.0 / sqrt(red[0] + red[2]), iv = 1.0 / sqrt(red[1] + red[3]);
    for (int i = tid; i < n; i += 64) {
      u[i] *= iu;
      v[i] *= iv;
    }
  } else if (tid == 0) {
    const int c = -code - 1;
    u[c] = 1.0;
    v[c] = 1.0;
  }
  __syncthreads();
  if (tid == 0) {
    for (int t = ctl->nrot - 1; t >= 0; --t) {
      const int a = ws.sm.rot_i[t], b = ws.sm.rot_j[t];
      const double c = ws.sm.rot_c[t], s = ws.sm.rot_s[t];
      const double ua = u[a], ub = u[b], va = v[a], vb = v[b];
      u[a] = c * ua - s * ub;
      u[b] = s * ua + c * ub;
      v[a] = c * va - s * vb;
      v[b] = s * va + c * vb;
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
//   S' = sigma'[0:rnew];  a' = L0'^T x
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_apply(Ws ws) {
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
  const double rho = ctl->rho, gamma = ctl->gamma;
  if (j == 0 && tid == 0) {
    nx.hdr->r = rnew;
    nx.hdr->r0 = compact ? rnew : r0e;
    nx.hdr->pairs = st.hdr->pairs + 1;
    nx.hdr->compactions = st.hdr->compactions + (compact ? 1 : 0);
    nx.hdr->cn2 = ws.sm.red[2 * r0 + 2];
    ctl->mode = compact ? PB_COMPACT : (ctl->append ? PB_APPEND : PB_NONE);
  }
  if (!compact && j == 0)
    for (int i = tid; i < r0e; i += 128) nx.a[i] = ws.sm.yext[i];
  if (j >= rnew) return;
  __shared__ double v[kMaxN], u[kMaxN], bv[kMaxN], qcol[kMaxCap + 1];
  for (int i = tid; i < n; i += 128) {
    v[i] = ws.sm.V[(size_t)j * kMaxN + i];
    u[i] = ws.sm.U[(size_t)j * kMaxN + i];
  }
  __syncthreads();
  // B v
  for (int i = tid; i < n; i += 128) {
    double acc;
    if (i < r) {
      acc = ws.sm.w[i] * v[r];
      for (int k = 0; k < r; ++k) acc = fma(st.M[(size_t)k * rm + i], v[k], acc);
    } else {
      acc = gamma * v[r];
      double t = 0.0;
      for (int k = 0; k < r; ++k) t = fma(st.rl[k], v[k], t);
      acc = fma(rho, t, acc);
    }
    bv[i] = acc;
  }
  // Q' column j (rows 0..r0e-1)
  for (int i = tid; i < r0e; i += 128) {
    double acc = ws.sm.qn[i] * u[r];
    if (i < r0)
      for (int k = 0; k < r; ++k) acc = fma(st.Q[(size_t)k * qld + i], u[k], acc);
    qcol[i] = acc;
  }
  __syncthreads();
  // M' column j
  for (int i = tid; i < rnew; i += 128) {
    double acc = 0.0;
    for (int l = 0; l < n; ++l) acc = fma(ws.sm.U[(size_t)i * kMaxN + l], bv[l], acc);
    nx.M[(size_t)j * rm + i] = acc;
  }
  if (compact) {
    for (int i = tid; i < r0e; i += 128) ws.sm.QB[(size_t)j * qld + i] = qcol[i];
    for (int i = tid; i < rnew; i += 128) nx.Q[(size_t)j * qld + i] = (i == j) ? 1.0 : 0.0;
  } else {
    for (int i = tid; i < r0e; i += 128) nx.Q[(size_t)j * qld + i] = qcol[i];
  }
  if (tid == 0) {
    double rf = 0.0;
    if (st.hdr->pairs == 0) {
      rf = v[r];
    } else {
      for (int k = 0; k < r; ++k) rf = fma(st.rf[k], v[k], rf);
    }
    nx.rf[j] = rf;
    nx.rl[j] = v[r];
    nx.S[j] = ws.sm.sig[kMaxN + j];
    if (compact) {
      double a = 0.0;
      for (int i = 0; i < r0e; ++i) a = fma(qcol[i], ws.sm.yext[i], a);
      nx.a[j] = a;
    }
  }
}

// ---------------------------------------------------------------------------------------
// eigensolver (one warp; scalar decisions are computed identically by every lane)
// ---------------------------------------------------------------------------------------
constexpr int kLD = kMaxR + 1;

struct EigSmem {
  double H[kMaxR * kLD];   // Hessenberg / quasi-triangular Schur factor T, row-major
  double Z[kMaxR * kLD];   // Schur vectors, row-major
  double Xr[kMaxR * kLD];  // eigenvectors of T, X[i][j] = component i of vector j
  double Xi[kMaxR * kLD];
  double scale[kMaxR];
  double wr[kMaxR], wi[kMaxR];
};

__device__ __forceinline__ void warp_sync() { __syncwarp(0xffffffffu); }

// Householder reflector (I - beta v v^T) a = alpha e1 with v[0] = 1 (len 2 or 3).
__device__ __forceinline__ double house_small(const double* a, int len, double* v) {
  double sigma = 0.0;
  for (int i = 1; i < len; ++i) sigma = fma(a[i], a[i], sigma);
  v[0] = 1.0;
  for (int i = 1; i < len; ++i) v[i] = 0.0;
  if (sigma == 0.0) return 0.0;
  const double x0 = a[0];
  const double mu = sqrt(x0 * x0 + sigma);
  const double v0 = x0 <= 0.0 ? x0 - mu : -sigma / (x0 + mu);
  const double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int i = 1; i < len; ++i) v[i] = a[i] / v0;
  return beta;
}

// rows i0..i0+len-1, columns c0..cn-1 of row-major A: A <- (I - beta v v^T) A
__device__ __forceinline__ void refl_left(double* A, int i0, int len, int c0, int cn, const double* v, double beta) {
  for (int c = c0 + (int)threadIdx.x; c < cn; c += 32) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s = fma(v[i], A[(i0 + i) * kLD + c], s);
    s *= beta;
    for (int i = 0; i < len; ++i) A[(i0 + i) * kLD + c] = fma(-s, v[i], A[(i0 + i) * kLD + c]);
  }
}

// rows 0..rn-1, columns j0..j0+len-1: A <- A (I - beta v v^T)
__device__ __forceinline__ void refl_right(double* A, int rn, int j0, int len, const double* v, double beta) {
  for (int row = (int)threadIdx.x; row < rn; row += 32) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s = fma(A[row * kLD + j0 + i], v[i], s);
    s *= beta;
    for (int i = 0; i < len; ++i) A[row * kLD + j0 + i] = fma(-s, v[i], A[row * kLD + j0 + i]);
  }
}

__global__ void __launch_bounds__(32) k_eig(Ws ws) {
  extern __shared__ __align__(16) unsigned char esm[];
  EigSmem& E = *reinterpret_cast<EigSmem*>(esm);
  Ctl* ctl = ws.ctl;
  const int lane = threadIdx.x;
  const StateBuf st = ws.st[ctl->cur];
  const int r = st.hdr->r, rm = ws.rmax;
  if (r == 0) {
    if (lane == 0) {
      atomicOr(&ctl->status, DEV_NOMODEL);
      ctl->eig_r = 0;
      ctl->eig_valid = 1;
    }
    return;
  }
  double* H = E.H;
  double* Z = E.Z;
  // A~ = M diag(S)^-1
  for (int idx = lane; idx < r * r; idx += 32) {
    const int i = idx / r, k = idx % r;
    H[i * kLD + k] = st.M[(size_t)k * rm + i] / st.S[k];
    Z[i * kLD + k] = (i == k) ? 1.0 : 0.0;
  }
  for (int i = lane; i < r; i += 32) E.scale[i] = 1.0;
  warp_sync();

  // ---- balancing: D^-1 A D with D a diagonal of powers of two (row/column 1-norms)
  for (int sweep = 0; sweep < 64; ++sweep) {
    bool changed = false;
    for (int i = 0; i < r; ++i) {
      double c = 0.0, rr = 0.0;
      for (int k = lane; k < r; k += 32)
        if (k != i) {
          c += fabs(H[k * kLD + i]);
          rr += fabs(H[i * kLD + k]);
        }
      c = warp_sum_d(c);
      rr = warp_sum_d(rr);
      if (c == 0.0 || rr == 0.0) continue;
      const double s = c + rr;
      double f = 1.0, g = rr / 2.0;
      while (c < g && f < 1e18) {
        f *= 2.0;
        c *= 4.0;
      }
      g = rr * 2.0;
      while (c >= g && f > 1e-18) {
        f /= 2.0;
        c /= 4.0;
      }
      if ((c + rr) / f < 0.95 * s) {
        changed = true;
        for (int k = lane; k < r; k += 32) H[i * kLD + k] /= f;
        warp_sync();
        for (int k = lane; k < r; k += 32) H[k * kLD + i] *= f;
        if (lane == 0) E.scale[i] *= f;
        warp_sync();
      }
    }
    if (!changed) break;
  }
  warp_sync();

  // ---- Householder reduction to upper Hessenberg form, Z accumulates the reflectors
  {
    double* v = E.wr;  // scratch (length r)
    for (int k = 0; k + 2 < r; ++k) {
      const int len = r - k - 1;
      double sigma = 0.0;
      for (int i = 1; i < len; ++i) sigma = fma(H[(k + 1 + i) * kLD + k], H[(k + 1 + i) * kLD + k], sigma);
      if (sigma == 0.0) continue;
      const double x0 = H[(k + 1) * kLD + k];
      const double mu = sqrt(x0 * x0 + sigma);
      const double v0 = x0 <= 0.0 ? x0 - mu : -sigma / (x0 + mu);
      const double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
      warp_sync();
      for (int i = lane; i < len; i += 32) v[i] = i == 0 ? 1.0 : H[(k + 1 + i) * kLD + k] / v0;
      warp_sync();
      refl_left(H, k + 1, len, k, r, v, beta);
      warp_sync();
      refl_right(H, r, k + 1, len, v, beta);
      refl_right(Z, r, k + 1, len, v, beta);
      warp_sync();
      if (lane == 0) {
        H[(k + 1) * kLD + k] = mu;
        for (int i = k + 2; i < r; ++i) H[i * kLD + k] = 0.0;
      }
      warp_sync();
    }
  }

  // ---- Francis double-shift QR (Golub & Van Loan, Alg. 7.5.1 with deflation)
  double norm = 0.0;
  for (int idx = lane; idx < r * r; idx += 32) norm += fabs(H[(idx / r) * kLD + idx % r]);
  norm = warp_sum_d(norm);
  int hi = r - 1, iter = 0, total = 0;
  bool failed = false;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      double s = fabs(H[(l - 1) * kLD + l - 1]) + fabs(H[l * kLD + l]);
      if (s == 0.0) s = norm;
      if (fabs(H[l * kLD + l - 1]) <= kEps * s) break;
      --l;
    }
    warp_sync();
    if (l > 0 && lane == 0) H[l * kLD + l - 1] = 0.0;
    warp_sync();
    if (l == hi) {
      if (lane == 0) {
        E.wr[hi] = H[hi * kLD + hi];
        E.wi[hi] = 0.0;
      }
      warp_sync();
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {
      const double a = H[(hi - 1) * kLD + hi - 1], b = H[(hi - 1) * kLD + hi];
      const double c = H[hi * kLD + hi - 1], d = H[hi * kLD + hi];
      const double p = 0.5 * (a - d);
      const double disc = p * p + b * c;
      warp_sync();
      if (disc >= 0.0) {
        // real pair: rotate the block to upper triangular form
        const double sq = sqrt(disc);
        const double l1 = 0.5 * (a + d) + copysign(sq, p);
        double ur = b, vr = l1 - a;
        const double ur2 = l1 - d, vr2 = c;
        if (fabs(ur2) + fabs(vr2) > fabs(ur) + fabs(vr)) {
          ur = ur2;
          vr = vr2;
        }
        const double nn = hypot(ur, vr);
        double cs = 1.0, sn = 0.0;
        if (nn > 0.0) {
          cs = ur / nn;
          sn = vr / nn;
        }
        for (int col = hi - 1 + lane; col < r; col += 32) {
          const double x1 = H[(hi - 1) * kLD + col], x2 = H[hi * kLD + col];
          H[(hi - 1) * kLD + col] = cs * x1 + sn * x2;
          H[hi * kLD + col] = -sn * x1 + cs * x2;
        }
        warp_sync();
        for (int row = lane; row <= hi; row += 32) {
          const double x1 = H[row * kLD + hi - 1], x2 = H[row * kLD + hi];
          H[row * kLD + hi - 1] = cs * x1 + sn * x2;
          H[row * kLD + hi] = -sn * x1 + cs * x2;
        }
        for (int row = lane; row < r; row += 32) {
          const double x1 = Z[row * kLD + hi - 1], x2 = Z[row * kLD + hi];
          Z[row * kLD + hi - 1] = cs * x1 + sn * x2;
          Z[row * kLD + hi] = -sn * x1 + cs * x2;
        }
        warp_sync();
        if (lane == 0) {
          H[hi * kLD + hi - 1] = 0.0;
          E.wr[hi - 1] = H[(hi - 1) * kLD + hi - 1];
          E.wr[hi] = H[hi * kLD + hi];
          E.wi[hi - 1] = 0.0;
          E.wi[hi] = 0.0;
        }
      } else if (lane == 0) {
        E.wr[hi - 1] = E.wr[hi] = 0.5 * (a + d);
        E.wi[hi - 1] = sqrt(-disc);
        E.wi[hi] = -sqrt(-disc);
      }
      warp_sync();
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++total > 60 * r) {
      failed = true;
      break;
    }
    ++iter;
    double ssum, tprod;
    if (iter % 11 == 10) {  // exceptional shift
      const double s = fabs(H[hi * kLD + hi - 1]) + fabs(H[(hi - 1) * kLD + hi - 2]);
      const double h = 0.75 * s + H[hi * kLD + hi];
      ssum = 2.0 * h;
      tprod = h * h + 0.4375 * s * s;
    } else {
      ssum = H[(hi - 1) * kLD + hi - 1] + H[hi * kLD + hi];
      tprod = H[(hi - 1) * kLD + hi - 1] * H[hi * kLD + hi] - H[(hi - 1) * kLD + hi] * H[hi * kLD + hi - 1];
    }
    double x = H[l * kLD + l] * H[l * kLD + l] + H[l * kLD + l + 1] * H[(l + 1) * kLD + l] -
               ssum * H[l * kLD + l] + tprod;
    double y = H[(l + 1) * kLD + l] * (H[l * kLD + l] + H[(l + 1) * kLD + l + 1] - ssum);
    double zz = H[(l + 1) * kLD + l] * H[(l + 2) * kLD + l + 1];
    for (int k = l; k <= hi - 2; ++k) {
      double a3[3] = {x, y, zz}, v[3];
      const double beta = house_small(a3, 3, v);
      warp_sync();
      if (beta != 0.0) {
        refl_left(H, k, 3, max(l, k - 1), r, v, beta);
        warp_sync();
        refl_right(H, min(k + 4, hi + 1), k, 3, v, beta);
        refl_right(Z, r, k, 3, v, beta);
        warp_sync();
        if (k > l && lane == 0) {
          H[(k + 1) * kLD + k - 1] = 0.0;
          H[(k + 2) * kLD + k - 1] = 0.0;
        }
        warp_sync();
      }
      x = H[(k + 1) * kLD + k];
      y = H[(k + 2) * kLD + k];
      if (k < hi - 2) zz = H[(k + 3) * kLD + k];
    }
    {
      double a2[2] = {x, y}, v[3];
      const double beta = house_small(a2, 2, v);
      warp_sync();
      if (beta != 0.0) {
        refl_left(H, hi - 1, 2, max(l, hi - 2), r, v, beta);
        warp_sync();
        refl_right(H, hi + 1, hi - 1, 2, v, beta);
        refl_right(Z, r, hi - 1, 2, v, beta);
        warp_sync();
        if (hi - 2 >= l && lane == 0) H[hi * kLD + hi - 2] = 0.0;
        warp_sync();
      }
    }
  }
  if (failed) {
    if (lane == 0) {
      atomicOr(&ctl->status, DEV_EIG_NOCONV);
      ctl->eig_r = r;
      ctl->eig_valid = 1;
    }
    return;
  }
  warp_sync();

  // ---- eigenvectors of T by back substitution: column j of X solves (T - lambda_j) x = 0
  // (x_j = 1 for a real eigenvalue; for a complex pair (j, j+1) with wi[j] > 0 the block's
  // own eigenvector [b; lambda - a] starts the substitution; column j+1 is its conjugate).
  double tnorm = 0.0;
  for (int idx = lane; idx < r * r; idx += 32) tnorm = fmax(tnorm, fabs(H[(idx / r) * kLD + idx % r]));
  for (int o = 16; o > 0; o >>= 1) tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  const double smin = fmax(kEps * tnorm, 1e-290);
  for (int j = lane; j < r; j += 32) {  // each lane owns whole eigenvectors
    const double lr = E.wr[j], li = E.wi[j];
    if (li < 0.0) continue;
    double* xr = E.Xr + j;
    double* xi = E.Xi + j;
    for (int i = 0; i < r; ++i) {
      xr[i * kLD] = 0.0;
      xi[i * kLD] = 0.0;
    }
    if (li == 0.0) {
      xr[j * kLD] = 1.0;
    } else {
      const double a = H[j * kLD + j], b = H[j * kLD + j + 1];
      const double c = H[(j + 1) * kLD + j], d = H[(j + 1) * kLD + j + 1];
      if (fabs(b) >= fabs(c)) {
        xr[j * kLD] = b;
        xr[(j + 1) * kLD] = lr - a;
        xi[(j + 1) * kLD] = li;
      } else {
        xr[j * kLD] = lr - d;
        xi[j * kLD] = li;
        xr[(j + 1) * kLD] = c;
      }
    }
    int i = j - 1;
    while (i >= 0) {
      const bool pair = (i > 0) && H[i * kLD + i - 1] != 0.0;
      const int i0 = pair ? i - 1 : i;
      double rr0 = 0.0, ri0 = 0.0, rr1 = 0.0, ri1 = 0.0;
      for (int k = i + 1; k < r; ++k) {
        rr1 -= H[i * kLD + k] * xr[k * kLD];
        ri1 -= H[i * kLD + k] * xi[k * kLD];
        if (pair) {
          rr0 -= H[i0 * kLD + k] * xr[k * kLD];
          ri0 -= H[i0 * kLD + k] * xi[k * kLD];
        }
      }
      if (!pair) {
        double dr = H[i * kLD + i] - lr, di = -li;
        if (fabs(dr) + fabs(di) < smin) dr = smin;
        const double den = dr * dr + di * di;
        xr[i * kLD] = (rr1 * dr + ri1 * di) / den;
        xi[i * kLD] = (ri1 * dr - rr1 * di) / den;
        i -= 1;
      } else {
        const double ar = H[i0 * kLD + i0] - lr, ai = -li;
        const double br = H[i0 * kLD + i], cr = H[i * kLD + i0];
        const double dr = H[i * kLD + i] - lr, di = -li;
        double detr = ar * dr - ai * di - br * cr;
        const double deti = ar * di + ai * dr;
        if (fabs(detr) + fabs(deti) < smin * tnorm) detr = smin * tnorm;
        const double dn = detr * detr + deti * deti;
        const double n0r = rr0 * dr - ri0 * di - br * rr1;
        const double n0i = rr0 * di + ri0 * dr - br * ri1;
        const double n1r = ar * rr1 - ai * ri1 - cr * rr0;
        const double n1i = ar * ri1 + ai * rr1 - cr * ri0;
        xr[i0 * kLD] = (n0r * detr + n0i * deti) / dn;
        xi[i0 * kLD] = (n0i * detr - n0r * deti) / dn;
        xr[i * kLD] = (n1r * detr + n1i * deti) / dn;
        xi[i * kLD] = (n1i * detr - n1r * deti) / dn;
        i -= 2;
      }
      double mx = 0.0;
      for (int k = 0; k < r; ++k) mx = fmax(mx, fabs(xr[k * kLD]) + fabs(xi[k * kLD]));
      if (mx > 1e100) {
        for (int k = 0; k < r; ++k) {
          xr[k * kLD] /= mx;
          xi[k * kLD] /= mx;
        }
      }
    }
  }
  warp_sync();
  // ---- V = D Z X, unit 2-norm columns; conjugate partners
  double* Vre = ws.eig.Vre;
  double* Vim = ws.eig.Vim;
  for (int j = 0; j < r; ++j) {
    const double li = E.wi[j];
    if (li < 0.0) continue;
    double nrm = 0.0;
    for (int row = lane; row < r; row += 32) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < r; ++k) {
        sr = fma(Z[row * kLD + k], E.Xr[k * kLD + j], sr);
        si = fma(Z[row * kLD + k], E.Xi[k * kLD + j], si);
      }
      sr *= E.scale[row];
      si *= E.scale[row];
      Vre[(size_t)j * rm + row] = sr;
      Vim[(size_t)j * rm + row] = si;
      nrm += sr * sr + si * si;
    }
    nrm = warp_sum_d(nrm);
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int row = lane; row < r; row += 32) {
      Vre[(size_t)j * rm + row] *= inv;
      Vim[(size_t)j * rm + row] *= inv;
      if (li > 0.0) {
        Vre[(size_t)(j + 1) * rm + row] = Vre[(size_t)j * rm + row];
        Vim[(size_t)(j + 1) * rm + row] = -Vim[(size_t)j * rm + row];
      }
    }
  }
  for (int j = lane; j < r; j += 32) {
    ws.eig.lre[j] = E.wr[j];
    ws.eig.lim[j] = E.wi[j];
  }
  __threadfence_block();
  warp_sync();

  // ---- b = V^{-1} (S * r_first): complex Gaussian elimination with partial pivoting
  double* Ar = E.H;
  double* Ai = E.Z;
  double* br = E.Xr;
  double* bi = E.Xi;
  for (int idx = lane; idx < r * r; idx += 32) {
    const int i = idx / r, k = idx % r;
    Ar[i * kLD + k] = Vre[(size_t)k * rm + i];
    Ai[i * kLD + k] = Vim[(size_t)k * rm + i];
  }
  for (int i = lane; i < r; i += 32) {
    br[i] = st.S[i] * st.rf[i];
    bi[i] = 0.0;
  }
  warp_sync();
  double amax = 0.0;
  for (int idx = lane; idx < r * r; idx += 32)
    amax = fmax(amax, hypot(Ar[(idx / r) * kLD + idx % r], Ai[(idx / r) * kLD + idx % r]));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  bool singular = false;
  for (int k = 0; k < r; ++k) {
    int piv = k;
    double pv = 0.0;
    for (int i = k; i < r; ++i) {
      const double a = hypot(Ar[i * kLD + k], Ai[i * kLD + k]);
      if (a > pv) {
        pv = a;
        piv = i;
      }
    }
    if (pv <= 1e-14 * amax) singular = true;
    if (pv == 0.0) break;
    warp_sync();
    if (piv != k) {
      for (int c = lane; c < r; c += 32) {
        double t = Ar[k * kLD + c];
        Ar[k * kLD + c] = Ar[piv * kLD + c];
        Ar[piv * kLD + c] = t;
        t = Ai[k * kLD + c];
        Ai[k * kLD + c] = Ai[piv * kLD + c];
        Ai[piv * kLD + c] = t;
      }
      if (lane == 0) {
        double t = br[k];
        br[k] = br[piv];
        br[piv] = t;
        t = bi[k];
        bi[k] = bi[piv];
        bi[piv] = t;
      }
    }
    warp_sync();
    const double pr = Ar[k * kLD + k], pi = Ai[k * kLD + k];
    const double pd = pr * pr + pi * pi;
    for (int i = k + 1 + lane; i < r; i += 32) {
      const double ar = Ar[i * kLD + k], ai = Ai[i * kLD + k];
      const double fr = (ar * pr + ai * pi) / pd, fi = (ai * pr - ar * pi) / pd;
      for (int c = k; c < r; ++c) {
        const double xr = Ar[k * kLD + c], xi = Ai[k * kLD + c];
        Ar[i * kLD + c] -= fr * xr - fi * xi;
        Ai[i * kLD + c] -= fr * xi + fi * xr;
      }
      const double yr = br[k], yi = bi[k];
      br[i] -= fr * yr - fi * yi;
      bi[i] -= fr * yi + fi * yr;
    }
    warp_sync();
  }
  if (lane == 0) {
    for (int i = r - 1; i >= 0; --i) {
      double sr = br[i], si = bi[i];
      for (int c = i + 1; c < r; ++c) {
        sr -= Ar[i * kLD + c] * br[c] - Ai[i * kLD + c] * bi[c];
        si -= Ar[i * kLD + c] * bi[c] + Ai[i * kLD + c] * br[c];
      }
      const double pr = Ar[i * kLD + i], pi = Ai[i * kLD + i];
      const double pd = pr * pr + pi * pi;
      br[i] = pd > 0.0 ? (sr * pr + si * pi) / pd : 0.0;
      bi[i] = pd > 0.0 ? (si * pr - sr * pi) / pd : 0.0;
    }
    for (int i = 0; i < r; ++i) {
      ws.eig.bre[i] = br[i];
      ws.eig.bim[i] = bi[i];
      if (!isfinite(br[i]) || !isfinite(bi[i])) singular = true;
    }
    if (singular) atomicOr(&ctl->status, DEV_EIG_COND);
    ctl->eig_r = r;
    ctl->eig_valid = 1;
  }
}

// ---------------------------------------------------------------------------------------
// rollout coefficients: coef[:, j] = Q Re(V Lambda^{t_j} b)  (r0 values, L0 coordinates)
// ---------------------------------------------------------------------------------------
struct TArr {
  double t[kRollK];
};

__global__ void __launch_bounds__(64) k_coef(Ws ws, TArr ts, int k) {
  Ctl* ctl = ws.ctl;
  const int j = blockIdx.x;
  if (j >= k) return;
  const StateBuf st = ws.st[ctl->cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, rm = ws.rmax, qld = ws.cap + 1;
  const int tid = threadIdx.x;
  __shared__ double gr[kMaxR], gi[kMaxR], c[kMaxR];
  const double t = ts.t[j];
  for (int l = tid; l < r; l += 64) {
    const double lr = ws.eig.lre[l], li = ws.eig.lim[l];
    const double b_r = ws.eig.bre[l], b_i = ws.eig.bim[l];
    double pr, pi;  // lambda^t on the principal branch
    if (t == 0.0) {
      pr = 1.0;
      pi = 0.0;
    } else if (lr == 0.0 && li == 0.0) {
      pr = 0.0;
      pi = 0.0;
    } else {
      const double mag = pow(hypot(lr, li), t);
      double sn, cs;
      sincos(t * atan2(li, lr), &sn, &cs);
      pr = mag * cs;
      pi = mag * sn;
    }
    gr[l] = pr * b_r - pi * b_i;
    gi[l] = pr * b_i + pi * b_r;
  }
  __syncthreads();
  for (int i = tid; i < r; i += 64) {
    double acc = 0.0;
    for (int l = 0; l < r; ++l) {
      acc = fma(ws.eig.Vre[(size_t)l * rm + i], gr[l], acc);
      acc = fma(-ws.eig.Vim[(size_t)l * rm + i], gi[l], acc);
    }
    c[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < r0; i += 64) {
    double acc = 0.0;
    for (int l = 0; l < r; ++l) acc = fma(st.Q[(size_t)l * qld + i], c[l], acc);
    ws.sm.coef[(size_t)j * qld + i] = acc;
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
cudaError_t launch_small(const Ws& ws, cudaStream_t s) {
  k_prep<<<1, 128, 0, s>>>(ws);
  k_roots<<<kMaxN, 32, 0, s>>>(ws);
  k_zhat<<<kMaxN + 1, 32, 0, s>>>(ws);
  k_vectors<<<kMaxN, 64, 0, s>>>(ws);
  k_apply<<<kMaxN, 128, 0, s>>>(ws);
  return cudaGetLastError();
}

cudaError_t launch_eig(const Ws& ws, cudaStream_t s) {
  const int bytes = (int)sizeof(EigSmem);
  cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_eig<<<1, 32, bytes, s>>>(ws);
  return cudaGetLastError();
}

cudaError_t launch_coef(const Ws& ws, const double* t_host, int k, cudaStream_t s) {
  TArr ta;
  for (int i = 0; i < kRollK; ++i) ta.t[i] = i < k ? t_host[i] : 0.0;
  k_coef<<<k, 64, 0, s>>>(ws, ta, k);
  return cudaGetLastError();
}

cudaError_t launch_basis_coef(const Ws& ws, cudaStream_t s) {
  k_basis_coef<<<kMaxR, 64, 0, s>>>(ws);
  return cudaGetLastError();
}

cudaError_t launch_init(const Ws&, cudaStream_t) { return cudaSuccess; }

}  // namespace odmd
