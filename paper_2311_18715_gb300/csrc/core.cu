// Small solves of the online DMD update in FP64 (Sec. 2.3: Brand's rank-1 append, kept in
// product form L = L0 Q).  These steps decide which directions of the snapshot stream
// survive truncation, and the reduced operator they update is carried from one snapshot to
// the next, so rounding here feeds back into every later model; they run in IEEE double.
// The tall passes hand over their reductions as double-float pairs (exact in double).
//
//   k_prep     reduced tall sums -> projections p = L^T c, w = L^T x, the new direction,
//              the core matrix K = [[diag(S), p], [0, rho]] and its deflated secular problem
//              (a pipelined update runs it in two launches: k_prep_a, the append decision
//              and the next state's inputs of the next pass A; k_prep_b, the rest, at the
//              head of the tail that runs beside that pass)
//   k_roots    one CTA per singular value of K: root of the secular equation
//   k_zhat     one CTA per pole: Loewner weights; one extra CTA orders the values
//   k_vectors  one CTA per kept singular pair: left/right singular vectors of K
//   k_apply    one CTA per kept column: M' = U'^T B V', Q' = [Q 0; 0 q] U', rows of R
//
// Core SVD.  K K^T = D^2 + z z^T with D = diag(S, 0) and z = [p; rho], so sigma'^2 are the
// roots of 1 + sum_i z_i^2 / (d_i^2 - lambda) = 0 and, with z-hat from Loewner's formula,
// u ~ (D^2 - lambda)^{-1} z-hat and v ~ (d_i z-hat_i / (d_i^2 - lambda), -1): the
// broken-arrow SVD of Gu and Eisenstat (SIAM J. Matrix Anal. Appl. 16, 1995).  Every
// difference d_i^2 - lambda is formed as (d_i - d_o)(d_i + d_o) - mu with lambda = d_o^2 +
// mu and d_o the nearer pole.  Negligible z_i and nearly equal d_i are deflated first (a
// Givens rotation merges the weights of two equal poles).  K is scaled by a power of two so
// that its largest entry lies in [1/2, 1).
//
// GB300 issues FP64 arithmetic at 1/64 of its FP32 rate, so each root is first located by
// FP32 iterations (to ~1e-7) and then refined with the secular function in FP64 and an
// FP32 two-pole model step for the correction (Newton-like convergence to FP64 accuracy);
// the sums over poles are spread over the threads of the CTA.
#include "dd.cuh"
#include "odmd_internal.cuh"

namespace odmd {

constexpr double kEps64 = 2.220446049250313e-16;  // 2^-52, a safe bound on the unit roundoff

__device__ __forceinline__ double group4_sum_d(double a) {
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  return a + __shfl_xor_sync(0xffffffffu, a, 2);
}
// the binary exponent of |v| from its bits (zero and subnormals give -1023)
__device__ __forceinline__ int dexp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF) - 1023;
}
// nonnegative doubles order like their bit patterns read as integers
__device__ __forceinline__ long long ord_key(double v) { return __double_as_longlong(v); }

// Asynchronous copies of doubles from global into shared memory (cp.async, 8 bytes each):
// every thread issues all of its copies before anyone waits, so staging an array costs one
// L2 round trip instead of one per loop iteration.  Complete with cp_async_wait_all() and a
// barrier.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void stage_doubles(double* dst, const double* src, int n, int tid, int nthreads) {
  for (int i = tid; i < n; i += nthreads) cp_async8(dst + i, src + i);
}

// Staging of the larger arrays by the bulk copy engine: one thread issues one copy per
// array, completing on an mbarrier, instead of every thread issuing 8-byte copies.  A bulk
// copy moves whole 16-byte units between 16-byte aligned addresses, so an array's shared
// copy starts at the same address modulo 16 as its source (bulk_dst: a 16-byte aligned
// region one double longer than the array), and a first or last double outside the
// aligned body is copied by a plain load (bulk_ends).
struct BulkSpan {
  int head, body;  // doubles: the unaligned first one (0 or 1), then an even count
};
__device__ __forceinline__ BulkSpan bulk_span(const double* src, int n) {
  const int h = (n > 0 && (reinterpret_cast<uintptr_t>(src) & 8u)) ? 1 : 0;
  return BulkSpan{h, (n - h) & ~1};
}
__device__ __forceinline__ double* bulk_dst(double* region, const double* src) {
  return region + ((reinterpret_cast<uintptr_t>(src) & 8u) ? 1 : 0);
}
__device__ __forceinline__ void bulk_issue(double* dst, const double* src, BulkSpan sp, uint64_t* bar) {
  if (sp.body > 0) bulk_g2s(dst + sp.head, src + sp.head, 8u * (uint32_t)sp.body, bar);
}
__device__ __forceinline__ void bulk_ends(double* dst, const double* src, int n) {
  const BulkSpan sp = bulk_span(src, n);
  if (sp.head) dst[0] = src[0];
  if (n - sp.head - sp.body == 1) dst[n - 1] = src[n - 1];
}
// every thread: the copies on bar have landed (bounded; on a timeout the status is set, and
// the copies still in flight get a last bounded wait before the block may go on and exit)
__device__ __forceinline__ void bulk_wait(uint64_t* bar, int* status) {
  if (!mbar_wait(bar, 0u, status)) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, 0u) && global_ns() - t0 < 1000000000ull) {
    }
  }
}

// ---------------------------------------------------------------------------------------
// k_prep
// ---------------------------------------------------------------------------------------
constexpr int kPrepThreads = 256;

__device__ __forceinline__ void prep_rest(const Ws& ws, const StateBuf& st, int r, int r0, int r0e, double thr,
                                          const double* sQ, const double* sS, const double* ac, const double* yx,
                                          double* z, double* p, double* p2);

// PART 1: the append decision and the next state's inputs of the next tall pass (all a
// pipelined next pass A waits for); ac = a + L0^T e and y (with the appended coordinate)
// are left in ws.sm.ac / ws.sm.yext, since the next pass A overwrites the reduced sums.
// PART 2: the rest, from those (the head of a pipelined update's tail).  PART 3: both.
template <int PART>
__device__ __forceinline__ void prep_body(const Ws& ws, CtaPos cp) {
  constexpr bool kA = (PART & 1) != 0, kB = (PART & 2) != 0;
  extern __shared__ __align__(16) double psm[];
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur];
  const int r = st.hdr->r, r0 = st.hdr->r0, qld = ws.cap + 1;
  double* sQ = bulk_dst(psm, st.Q);  // r columns of Q, ld qld (bulk-copied, region qld kMaxR + 2)
  double* ac = psm + (size_t)qld * kMaxR + 2;
  double* yx = ac + qld;
  double* z = yx + qld;
  double* p = z + qld;
  double* p2 = p + kMaxN;
  __shared__ double thr_s, rho0_s, cn2_s;
  __shared__ int append_s, pairs_s, comp_s;
  __shared__ double sS[kMaxN];
  __shared__ __align__(8) uint64_t sbar;
  const float2* red = ws.sm.red;

  if constexpr (kB) {
    if (tid == 0) {
      mbar_init(&sbar, 1);
      mbar_fence_init();
      const BulkSpan sp = bulk_span(st.Q, r * qld);
      mbar_arrive_expect_tx(&sbar, 8u * (uint32_t)sp.body);
      bulk_issue(sQ, st.Q, sp, &sbar);
    }
    if (tid == 32) bulk_ends(sQ, st.Q, r * qld);
    stage_doubles(sS, st.S, r, tid, kPrepThreads);
  } else {
    if (tid == 0) sS[0] = r > 0 ? st.S[0] : 0.0;
  }
  if constexpr (kA) {
    // the committed state's part of ac = a + L0^T e, and the header fields the next state
    // continues from
    for (int i = tid; i < r0; i += kPrepThreads) ac[i] = dd2d(st.a[i]);
    if (tid == 0) {
      pairs_s = st.hdr->pairs;
      comp_s = st.hdr->compactions;
      cn2_s = dd2d(st.hdr->cn2);
    }
  }
  // Until here only the committed state is read (written by the last kernel of the previous
  // update, which completed before pass A started), so its copies run during the wait for
  // pass A; the reduced sums of pass A (or the first part's results) are read after it
  pdl_wait();
  pdl_trigger();  // the next kernel's CTAs are placed now and wait in their pdl_wait for this grid
  if constexpr (kA) {
    for (int i = tid; i < r0; i += kPrepThreads) {  // the same thread's entry as above
      ac[i] += dd2d(red[i]);
      yx[i] = dd2d(red[r0 + i]);
    }
  } else {
    const int n_e = ctl->r0e;  // r0 + the first part's append decision
    stage_doubles(ac, ws.sm.ac, n_e, tid, kPrepThreads);
    stage_doubles(yx, ws.sm.yext, n_e, tid, kPrepThreads);
  }
  cp_async_wait_all();
  __syncthreads();
  if constexpr (kB) bulk_wait(&sbar, &ctl->status);
  // p = Q^T ac and w = Q^T y (4 threads per column j < r; Q has r0 rows, the appended
  // coordinate lies outside span(L)); a warp without column work meanwhile decides whether
  // the residual is appended (rho0 against the truncation threshold)
  // (FP64 instructions cost the SM's FP64 pipe whether or not a lane has work, so warps
  // with no column or row skip each phase as a whole)
  if (kB && 8 * warp < r) {
    const int j = tid >> 2, sub = tid & 3;
    double ap = 0.0, aw = 0.0;
    if (j < r)
      #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
      for (int i = sub; i < r0; i += 4) {
        const double q = sQ[(size_t)j * qld + i];
        ap = fma(q, ac[i], ap);
        aw = fma(q, yx[i], aw);
      }
    ap = group4_sum_d(ap);
    aw = group4_sum_d(aw);
    if (j < r && sub == 0) {
      p[j] = ap;
      ws.sm.w[j] = aw;
    }
  }
  const int dwarp = 4 * r <= kPrepThreads - 32 ? 7 : 0;
  if (kA && warp == dwarp) {
    double ssq = 0.0, sy = 0.0;
    #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
    for (int i = lane; i < r0; i += 32) {
      const double si = dd2d(red[i]);
      ssq = fma(si, si, ssq);
      sy = fma(si, dd2d(red[r0 + i]), sy);
    }
    ssq = warp_sum_d(ssq);
    sy = warp_sum_d(sy);
    if (lane == 0) {
      const double eta = dd2d(red[2 * r0]), ex = dd2d(red[2 * r0 + 1]);
      // rho0 and 1 / rho0 from one reciprocal square root: every dependent FP64 operation of
      // this one thread costs ~100 cycles, and a square root followed by a division is a
      // chain about twice as long
      const double e2 = fmax(eta - ssq, 0.0);
      const double irho0 = e2 > 0.0 ? rsqrt(e2) : 0.0;
      const double rho0 = e2 * irho0;
      const double cn = sqrt(cn2_s);
      const double sig1 = r > 0 ? sS[0] : 0.0;
      const double thr = ws.tau * fmax(sig1, cn);
      const int append = rho0 > thr ? 1 : 0;
      ctl->thr = thr;
      ctl->rho0 = rho0;
      ctl->append = append;
      ctl->r0e = r0 + append;
      if (append) {
        ac[r0] = rho0;
        yx[r0] = (ex - sy) * irho0;
      }
      append_s = append;
      thr_s = thr;
      rho0_s = rho0;
    }
  }
  __syncthreads();
  const int append = kA ? append_s : ctl->append;
  const int r0e = r0 + append;
  const double thr = kA ? thr_s : ctl->thr;
  // The next state's inputs of the next tall pass, published here rather than by k_apply so
  // that a pipelined next pass A may run beside this update's SVD: its header (all but the
  // rank; r0 too unless the update compacts, when k_apply writes it with the new rank), its
  // projection a = L0'^T x and the pending column's s.  A compacting update also sets
  // pipe_flag, on which a pipelined next pass A waits for the compaction.
  if constexpr (kA) {
    const bool compact = r0e > ws.cap;
    const StateBuf nx = ws.st[cur ^ 1];
    if (tid == 0) {
      nx.hdr->pairs = pairs_s + 1;
      nx.hdr->compactions = comp_s + (compact ? 1 : 0);
      nx.hdr->cn2 = red[2 * r0 + 2];
      nx.hdr->pend = (append && !compact) ? 1 : 0;
      nx.hdr->pinv = append ? d2f2(1.0 / rho0_s) : make_float2(0.f, 0.f);
      if (!compact) nx.hdr->r0 = r0e;
      ctl->pipe_flag = compact ? 1 : 0;
    }
    if (!compact) {
      for (int i = tid; i < r0e; i += kPrepThreads) nx.a[i] = d2f2(yx[i]);
      if (append)
        for (int i = tid; i < r0; i += kPrepThreads) nx.ps[i] = red[i];
    }
    for (int i = tid; i < r0e; i += kPrepThreads) {
      ws.sm.ac[i] = ac[i];
      ws.sm.yext[i] = yx[i];
    }
  }
  if constexpr (kB) prep_rest(ws, st, r, r0, r0e, thr, sQ, sS, ac, yx, z, p, p2);
}

// the second part of k_prep from the appended basis: z, the second Gram-Schmidt pass, rho
// and gamma, and the secular problem
__device__ __forceinline__ void prep_rest(const Ws& ws, const StateBuf& st, int r, int r0, int r0e, double thr,
                                          const double* sQ, const double* sS, const double* ac, const double* yx,
                                          double* z, double* p, double* p2) {
  Ctl* ctl = ws.ctl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, qld = ws.cap + 1;
  __shared__ double red8[16];
  __shared__ double dsc[kMaxN], zsc[kMaxN];
  __shared__ int defl[kMaxN];
  // z = ac - Q p (rows < r0; the appended coordinate is ac itself)
  for (int base = 0; base < 4 * r0e; base += kPrepThreads) {
    if (base + 32 * warp >= 4 * r0e) continue;
    const int i = (base + tid) >> 2, sub = tid & 3;
    double acc = 0.0;
    if (i < r0)
      #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
      for (int j = sub; j < r; j += 4) acc = fma(sQ[(size_t)j * qld + i], p[j], acc);
    acc = group4_sum_d(acc);
    if (i < r0e && sub == 0) z[i] = i < r0 ? ac[i] - acc : ac[i];
  }
  __syncthreads();
  // second Gram-Schmidt pass in the small space: p2 = Q^T z, z -= Q p2, p += p2
  if (8 * warp < r) {
    const int j = tid >> 2, sub = tid & 3;
    double acc = 0.0;
    if (j < r)
      #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
      for (int i = sub; i < r0; i += 4) acc = fma(sQ[(size_t)j * qld + i], z[i], acc);
    acc = group4_sum_d(acc);
    if (j < r && sub == 0) p2[j] = acc;
  }
  __syncthreads();
  for (int base = 0; base < 4 * r0; base += kPrepThreads) {
    if (base + 32 * warp >= 4 * r0) continue;
    const int i = (base + tid) >> 2, sub = tid & 3;
    double acc = 0.0;
    if (i < r0)
      #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
      for (int j = sub; j < r; j += 4) acc = fma(sQ[(size_t)j * qld + i], p2[j], acc);
    acc = group4_sum_d(acc);
    if (i < r0 && sub == 0) z[i] -= acc;
  }
  for (int j = tid; j < r; j += kPrepThreads) {
    p[j] += p2[j];
    ws.sm.p[j] = p[j];
  }
  __syncthreads();
  // ||z||^2 and z . y in one block reduction; rho = ||z||, gamma = q_n . y = (z . y) / rho
  double zz = 0.0, zy = 0.0;
  const int zw = (r0e + 31) >> 5;  // warps holding entries of z (r0e <= cap + 1 <= 256)
  if (warp < zw) {
    for (int i = tid; i < r0e; i += kPrepThreads) {
      zz = fma(z[i], z[i], zz);
      zy = fma(z[i], yx[i], zy);
    }
    zz = warp_sum_d(zz);
    zy = warp_sum_d(zy);
  }
  if (lane == 0) {
    red8[warp] = zz;  // zero for the warps without entries
    red8[8 + warp] = zy;
  }
  __syncthreads();
  // rho, 1/rho and gamma once (FP64 square roots and divisions run at the FP64 rate); the
  // eight warp partials are added by shuffles in warp 0 (three dependent additions, not seven)
  __shared__ double rho_s, inv_s;
  if (warp == 0) {
    zz = lane < 8 ? red8[lane] : 0.0;
    zy = lane < 8 ? red8[8 + lane] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      zz += __shfl_xor_sync(0xffffffffu, zz, o);
      zy += __shfl_xor_sync(0xffffffffu, zy, o);
    }
  }
  if (tid == 0) {
    const double irh = zz > 0.0 ? rsqrt(zz) : 0.0;  // rho and 1 / rho from one reciprocal root
    double rh = zz * irh, iv = irh;
    if (!(rh > thr)) rh = iv = 0.0;
    rho_s = rh;
    inv_s = iv;
    ctl->rho = rh;
    ctl->gamma = zy * iv;
  }
  __syncthreads();
  const double rho = rho_s, inv_rho = inv_s;
  for (int i = tid; i < r0e; i += kPrepThreads) {
    ws.sm.qn[i] = z[i] * inv_rho;
  }
  // ---- secular problem of K = [[diag(S), p], [0, rho]], n = r + 1, scaled to max < 1
  if (warp == 0) {
    const int n = r + 1;
    // the largest magnitude by integer maxima of the bit patterns with the sign cleared
    // (nonnegative doubles order like their bits; an infinity or NaN orders above every
    // finite value and is caught below), and its exponent from the bits
    long long mb = 0;
    for (int i = lane; i < n; i += 32) {
      mb = max(mb, __double_as_longlong(i < r ? p[i] : rho) & 0x7FFFFFFFFFFFFFFFll);
      if (i == 0 && r > 0) mb = max(mb, __double_as_longlong(sS[0]) & 0x7FFFFFFFFFFFFFFFll);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const double mx = __longlong_as_double(mb);
    const int bexp = (int)(mb >> 52);
    int e = 0;  // mx = f 2^e with f in [1/2, 1)
    if (bexp > 0 && bexp < 2047)
      e = bexp - 1022;
    else if (mb > 0 && bexp == 0)
      frexp(mx, &e);  // subnormal
    const double tol = 8.0 * kEps64;  // in scaled units
    // 2^-e built from its bits (|e| stays far inside the exponent range of doubles), so each
    // scaling is one exact product
    const double pw = __longlong_as_double((long long)(1023 - e) << 52);
    for (int i = lane; i < n; i += 32) {
      const double di = i < r ? sS[i] * pw : 0.0;
      const double zi = (i < r ? p[i] : rho) * pw;
      dsc[i] = di;
      const bool small = !(fabs(zi) > tol);
      zsc[i] = small ? 0.0 : zi;
      defl[i] = small ? 1 : 0;
      ws.sm.dc[i] = di;
    }
    __syncwarp();
    // merge nearly equal poles (the pole at 0, coordinate r, is never merged).  A pole merges
    // into the last kept one above it; S is sorted in descending order, so a merge needs two
    // neighbouring values within tol.  All lanes look for such neighbours (or an unsorted
    // pair); the sequential merge runs only if they find one.
    bool near = false;
    for (int i = lane + 1; i < r; i += 32) near = near || !(dsc[i - 1] - dsc[i] > tol);
    if (!__any_sync(0xffffffffu, near)) {
      if (lane == 0) ctl->nrot = 0;
    } else if (lane == 0) {
      int nrot = 0, last = -1;
      for (int i = 0; i < r; ++i) {
        if (defl[i]) continue;
        if (last >= 0 && dsc[last] - dsc[i] <= tol) {
          const double zl = zsc[last], zi = zsc[i];
          const double h = sqrt(zl * zl + zi * zi);
          ws.sm.rot_i[nrot] = last;
          ws.sm.rot_j[nrot] = i;
          ws.sm.rot_c[nrot] = zl / h;
          ws.sm.rot_s[nrot] = zi / h;
          ++nrot;
          zsc[last] = h;
          zsc[i] = 0.0;
          defl[i] = 1;
        } else {
          last = i;
        }
      }
      ctl->nrot = nrot;
    }
    __syncwarp();
    // the poles in ascending order (core coordinates n-1 .. 0) and the deflated coordinates,
    // positions by ballots over 32 coordinates at a time
    int m = 0, nd = 0;
    for (int base = 0; base < n; base += 32) {
      const int i = n - 1 - (base + lane);  // ascending poles: descending coordinates
      const bool in = base + lane < n;
      const bool dfl = in && defl[i];
      const unsigned bd = __ballot_sync(0xffffffffu, dfl), bp = __ballot_sync(0xffffffffu, in && !dfl);
      const unsigned below = (1u << lane) - 1u;
      if (dfl) ws.sm.defl[nd + __popc(bd & below)] = i;
      if (in && !dfl) {
        const int q = m + __popc(bp & below);
        ws.sm.pole[q] = i;
        ws.sm.d[q] = dsc[i];
        ws.sm.z[q] = zsc[i];
      }
      nd += __popc(bd);
      m += __popc(bp);
    }
    if (lane == 0) {
      ctl->n = n;
      ctl->m = m;
      ctl->ndefl = nd;
      ctl->scale_exp = e;
      if (!isfinite(rho) || !isfinite(mx)) atomicOr(&ctl->status, DEV_NONFINITE);
    }
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_prep(const __grid_constant__ Ws ws) {
  prep_body<3>(ws, cta_single());
}
__global__ void __launch_bounds__(kPrepThreads) k_prep_a(const __grid_constant__ Ws ws) {
  prep_body<1>(ws, cta_single());
}
__global__ void __launch_bounds__(kPrepThreads) k_prep_b(const __grid_constant__ Ws ws) {
  prep_body<2>(ws, cta_single());
}
__global__ void __launch_bounds__(kPrepThreads) k_prep_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  prep_body<3>(*t.ws[i], batch_pos(t, i));
}


// ---------------------------------------------------------------------------------------
// k_roots: root j of 1 + sum_i z_i^2/(d_i^2 - lambda) = 0 in (d_j^2, d_{j+1}^2)
// ---------------------------------------------------------------------------------------
constexpr int kRootThreads = 128;  // >= kMaxN: one pole per thread in the FP64 sums
static_assert(kRootThreads >= kMaxN, "one pole per thread");

// block sums (every thread gets the same results, in a fixed order): one double, or NF floats
__device__ __forceinline__ double block_sum_d(double v, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_d(v);
  if (lane == 0) part[warp] = v;
  __syncthreads();
  double s = part[0];
  for (int w = 1; w < kRootThreads / 32; ++w) s += part[w];
  return s;
}
template <int NF>
__device__ __forceinline__ void block_sum_f(float (&v)[NF], float* part) {  // part: warps x NF
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NF; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NF; ++k) part[warp * NF + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    float s = part[k];
    for (int w = 1; w < kRootThreads / 32; ++w) s += part[w * NF + k];
    v[k] = s;
  }
}

__device__ __forceinline__ void roots_body(const Ws& ws, CtaPos cp) {
  pdl_wait();
  // after the wait, so that a successor placed now may read what any kernel before this one
  // wrote; it waits in its own pdl_wait for this grid, on the SMs this grid leaves free
  pdl_trigger();
  Ctl* ctl = ws.ctl;
  const int m = ctl->m;
  const int j = cp.b;
  if (j >= m) return;
  const double* d = ws.sm.d;
  const double* z = ws.sm.z;
  const int tid = threadIdx.x, lane = tid & 31;
  __shared__ float zf[kMaxN];
  __shared__ float partf[2][kRootThreads / 32 * 3];
  __shared__ double part64[2][kRootThreads / 32];
  const bool mine = tid < m;
  const double di = mine ? d[tid] : 0.0, zi = mine ? z[tid] : 0.0;
  const float zif = __double2float_rn(zi);
  if (mine) {
    zf[tid] = zif;
  }
  if (m == 1) {
    if (tid == 0) {
      const double zsq = zi * zi;
      ws.sm.org[0] = 0;
      ws.sm.mu[0] = zsq;
      ws.sm.sig[0] = sqrt(di * di + zsq);
    }
    return;
  }
  int o;
  double lo, hi, A, B;  // bracket of mu and the neighbouring poles, relative to d_o^2
  const bool last = (j == m - 1);
  int it_total = 0;  // parity of the partial-sum buffers in use
  if (!last) {
    // the side of the interval's midpoint on which the root lies: the sign of f(mid), its
    // terms in FP64 (a pole per thread), summed in FP32 with an error bound; only when the
    // bound cannot decide the sign is the sum repeated in FP64
    const double dj = d[j], dj1 = d[j + 1];
    const double gap = (dj1 - dj) * (dj1 + dj);
    const double mid = gap * 0.5;
    // the terms in FP32 from d_i^2 - d_j^2 formed in FP64: every pole lies outside the
    // interval, so |d_i^2 - d_j^2 - mid| >= mid and each term carries at most ~8 units of
    // 2^-24 of relative error; with the summation's the bound below stays under
    // (m + 10) 2^-23 (1 + sum |t|)
    const double ddj = mine ? (di - dj) * (di + dj) : 0.0;
    const float tf = mine ? zif * (zif / (__double2float_rn(ddj) - __double2float_rn(mid))) : 0.f;
    float v[2] = {tf, fabsf(tf)};
    block_sum_f<2>(v, partf[it_total & 1]);
    const float fm = 1.f + v[0];
    bool right;  // f(mid) >= 0: the root lies left of the midpoint, next to d_j
    if (fabsf(fm) > (float)(m + 10) * 0x1p-23f * (1.f + v[1])) {
      right = fm >= 0.f;
    } else {
      const double t = mine ? zi * (zi / (ddj - mid)) : 0.0;
      right = 1.0 + block_sum_d(t, part64[it_total & 1]) >= 0.0;
    }
    ++it_total;
    if (right) {
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
    // the largest root lies below d_last^2 + |z|^2: |z|^2 in FP32 (values below 1 after
    // the scaling), widened past its rounding error, is the upper end of the bracket
    float v[1] = {zif * zif};
    block_sum_f<1>(v, partf[it_total & 1]);
    ++it_total;
    o = j;
    lo = 0.0;
    hi = (double)v[0] * (1.0 + 0x1p-10);
    A = 0.0;
    B = 0.0;
  }
  const double dob = d[o];
  // d_i^2 - d_o^2 in FP64 (the difference of two nearby squares would lose the leading bits
  // in FP32), rounded to FP32 for stage 1
  const double ddo = mine ? (di - dob) * (di + dob) : 0.0;
  __shared__ float ddf[kMaxN];
  if (mine) ddf[tid] = __double2float_rn(ddo);
  __syncthreads();
  // ---- stage 1, FP32: locate the root to ~1e-7 relative (every warp the same way)
  double mu = 0.5 * (lo + hi);
  {
    const float Af = (float)A, Bf = (float)B;
    float lof = (float)lo, hif = (float)hi, muf = (float)mu;
    for (int it = 0; it < 40; ++it) {
      float psi = 0.f, dpsi = 0.f, phi = 0.f, dphi = 0.f;
#pragma unroll
      for (int q_ = 0; q_ < (kMaxN + 31) / 32; ++q_) {
        const int i = lane + 32 * q_;
        if (i >= m) break;
        const float zv = zf[i];
        const float del = ddf[i] - muf;
        const float t = zv / del;
        if (i <= j) {
          psi = fmaf(zv, t, psi);
          dpsi = fmaf(t, t, dpsi);
        } else {
          phi = fmaf(zv, t, phi);
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
    // finite and strictly inside the FP64 bracket
    const double cand = (double)muf;
    if (isfinite(muf) && cand > lo && cand < hi) mu = cand;
  }
  // ---- stage 2: f in FP64 (one pole per thread, one block sum), then the step by thread 0
  // alone -- the bracket, the tests and the FP32 model step for the correction delta = x - mu
  // (shifted poles A - mu, B - mu) -- broadcast through shared memory.  FP64 operations run
  // at 1/64 of the FP32 rate, so scalar work is not repeated in every thread, and what only
  // steers the iteration is summed in FP32: the derivatives psi', phi' of the model step and
  // |psi| + |phi| = sum |z_i^2 / (d_i^2 - lambda)| of the stopping test (the terms of psi are
  // negative and those of phi positive inside the bracket)
  __shared__ double mu_s;
  __shared__ int done_s;
  bool conv = false;
  double prev_step = 0.0;  // thread 0: the previous FP64 step (none yet: the test below fails)
  for (int it = 0; it < 100; ++it) {
    double term = 0.0;
    float v[3] = {0.f, 0.f, 0.f};  // sum |term|, psi', phi'
    if (mine) {
      const double t = zi / (ddo - mu);
      term = zi * t;
      const float tf = __double2float_rn(t);
      v[0] = fabsf(zif * tf);
      v[tid <= j ? 1 : 2] = tf * tf;
    }
    // the FP64 sum and the FP32 sums share one barrier; the buffers alternate between
    // iterations so a fast thread cannot overwrite partials another is still reading
    const int pb = it_total & 1;
    ++it_total;
    if (32 * (tid >> 5) < m) {  // warps without poles hold zeros: no sums there
      term = warp_sum_d(term);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o2);
    }
    if (lane == 0) {
      part64[pb][tid >> 5] = term;
#pragma unroll
      for (int k = 0; k < 3; ++k) partf[pb][(tid >> 5) * 3 + k] = v[k];
    }
    __syncthreads();
    if (tid == 0) {
      double sum = part64[pb][0];
      float mag = partf[pb][0], dps = partf[pb][1], dph = partf[pb][2];
      for (int w = 1; w < kRootThreads / 32; ++w) {
        sum += part64[pb][w];
        mag += partf[pb][w * 3];
        dps += partf[pb][w * 3 + 1];
        dph += partf[pb][w * 3 + 2];
      }
      const double f = 1.0 + sum;
      if (f < 0.0)
        lo = mu;
      else
        hi = mu;
      int stop = 0;
      // f is formed from sums of terms of one sign each, so its rounding error is a few units
      // of 1 + |psi| + |phi|; stop there (the step and bracket tests below end the iteration
      // when the rounding of f alone moves it)
      if (fabs(f) <= 8.0 * kEps64 * (1.0 + (double)mag)) {
        stop = 1;
      } else {
        // two-pole model written around mu with f explicit:  f + psi' a d/(a - d) + phi' b
        // d/(b - d) = 0, neighbouring poles at a = A - mu and b = B - mu, unknown d = x - mu,
        // scaled by a power of two so that the FP32 coefficients stay inside the exponent range
        const float fh = (float)f;
        const float a = (float)(A - mu);
        const float b = last ? 0.f : (float)(B - mu);
        int ex = 0;
        frexpf(fmaxf(fabsf(a), fabsf(b)), &ex);
        const float sc = ldexpf(1.f, ex), as = ldexpf(a, -ex), bs = ldexpf(b, -ex);
        const float ps = (float)dps * sc, hs = (float)dph * sc;
        float delta;
        if (!last) {
          const float Qa = fh - ps * as - hs * bs;
          const float Qb = as * bs * (ps + hs) - fh * (as + bs);
          const float Qc = fh * as * bs;
          const float disc = fmaxf(Qb * Qb - 4.f * Qa * Qc, 0.f);
          const float q = -0.5f * (Qb >= 0.f ? Qb + sqrtf(disc) : Qb - sqrtf(disc));
          const float d2 = q != 0.f ? Qc / q : 0.f;  // the root that tends to -f / f'
          const float d1 = Qa != 0.f ? q / Qa : d2;
          const float lo_s = ldexpf((float)(lo - mu), -ex), hi_s = ldexpf((float)(hi - mu), -ex);
          const bool in2 = d2 > lo_s && d2 < hi_s, in1 = d1 > lo_s && d1 < hi_s;
          delta = ldexpf(in2 ? d2 : (in1 ? d1 : d2), ex);
        } else {
          const float den = fh - ps * as;
          delta = den != 0.f ? ldexpf(fh * as / den, ex) : 0.f;
        }
        double x = mu + (double)delta;
        if (!isfinite(delta) || !(x > lo && x < hi)) x = 0.5 * (lo + hi);
        const double step = fabs(x - mu);
        mu = x;
        if (step <= 4.0 * kEps64 * fabs(mu) || hi - lo <= 4.0 * kEps64 * fmax(fabs(lo), fabs(hi))) stop = 1;
        // the model step converges quadratically: with steps s1 then s2 the constant is about
        // s2 / s1^2, so the error left after s2 is about s2^3 / s1^2.  Once that lies below
        // 2^-60 |mu| (and s2 itself below 2^-26 |mu|, inside the quadratic regime), the next
        // evaluation of f could only confirm the root: stop here instead of paying for it.
        // The test runs on the binary exponents (integer operations, off the FP64 pipe):
        // v in [2^e, 2^(e+1)) bounds s2^3 / s1^2 below 2^(3 e2 + 3 - 2 e1)
        const int em = dexp(mu), e2 = dexp(step), e1 = dexp(prev_step);
        if (em > -600 && e2 <= em - 26 && 3 * e2 - 2 * e1 <= em - 63) stop = 1;
        prev_step = step;
      }
      mu_s = mu;
      done_s = stop;
    }
    __syncthreads();
    mu = mu_s;
    if (done_s) {
      conv = true;
      break;
    }
  }
  if (tid == 0) {
    if (!conv) atomicOr(&ctl->status, DEV_SECULAR);
    ws.sm.org[j] = o;
    ws.sm.mu[j] = mu;
    ws.sm.sig[j] = sqrt(fmax(dob * dob + mu, 0.0));
  }
}

__global__ void __launch_bounds__(kRootThreads) k_roots(const __grid_constant__ Ws ws) {
  roots_body(ws, cta_single());
}
__global__ void __launch_bounds__(kRootThreads) k_roots_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  roots_body(*t.ws[i], batch_pos(t, i));
}


// ---------------------------------------------------------------------------------------
// k_zhat: Loewner weights z^_i^2 = prod_k (lambda_k - d_i^2) / prod_{k != i} (d_k^2 - d_i^2),
// paired so every factor is O(1).  The last CTA of the grid orders all singular values of K.
// ---------------------------------------------------------------------------------------
constexpr int kZhatThreads = 64;

__device__ __forceinline__ void zhat_body(const Ws& ws, CtaPos cp) {
  pdl_wait();
  // after the wait, so that a successor placed now may read what any kernel before this one
  // wrote; it waits in its own pdl_wait for this grid, on the SMs this grid leaves free
  pdl_trigger();
  Ctl* ctl = ws.ctl;
  const int m = ctl->m;
  const int tid = threadIdx.x;
  if (cp.b == cp.g - 1) {  // the last CTA (kMaxN in an instance's own launch)
    // order roots (sig[0..m)) and deflated values (scaled diagonal at defl[k]), descending;
    // every value is >= 0, so its bit pattern orders it
    const int nd = ctl->ndefl;
    __shared__ double val[kMaxN];
    __shared__ long long key[kMaxN];
    __shared__ int code[kMaxN];
    const int tot = m + nd;
    for (int e = tid; e < tot; e += kZhatThreads) {
      double v;
      if (e < m) {
        v = ws.sm.sig[e];
        code[e] = e;
      } else {
        const int c = ws.sm.defl[e - m];
        v = ws.sm.dc[c];
        code[e] = -c - 1;
      }
      val[e] = v;
      key[e] = ord_key(v);
    }
    __syncthreads();
    long long kmax = 0;
    for (int e = 0; e < tot; ++e) kmax = max(kmax, key[e]);
    const double vmax = __longlong_as_double(kmax);
    const long long kcut = ord_key(ws.tau * vmax);
    for (int e = tid; e < tot; e += kZhatThreads) {
      int pos = 0;
      const long long ke = key[e];
      for (int f = 0; f < tot; ++f) pos += key[f] > ke || (key[f] == ke && f < e);
      ws.sm.src[pos] = code[e];
      ws.sm.sig[kMaxN + pos] = val[e];
    }
    if (tid == 0) {
      int keep = 0;
      if (vmax > 0.0)
        for (int e = 0; e < tot; ++e) keep += key[e] > kcut;
      ctl->rnew = min(keep, ws.rmax);
    }
    return;
  }
  const int i = cp.b;
  if (i >= m) return;
  const double* d = ws.sm.d;
  // the poles and the roots' origins and offsets into shared memory at once (asynchronous
  // copies), so that each factor's operands are one shared-memory read away
  __shared__ double sd[kMaxN], smu[kMaxN];
  __shared__ int sorg[kMaxN];
  for (int k = tid; k < m; k += kZhatThreads) {
    cp_async8(sd + k, d + k);
    cp_async8(smu + k, ws.sm.mu + k);
  }
  for (int k = tid; k < m; k += kZhatThreads) sorg[k] = ws.sm.org[k];
  cp_async_wait_all();
  __syncthreads();
  const double di = sd[i];
  double prod = 1.0;
  for (int k = tid; k < m; k += kZhatThreads) {
    const double dko = sd[sorg[k]];
    const double lam_m_di = smu[k] - (di - dko) * (di + dko);  // lambda_k - d_i^2
    double f;
    if (k == m - 1) {
      f = lam_m_di;
    } else {
      const double dk = sd[k < i ? k : k + 1];
      f = lam_m_di / ((dk - di) * (dk + di));
    }
    prod *= f;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) prod *= __shfl_xor_sync(0xffffffffu, prod, off);
  __shared__ double wp[kZhatThreads / 32];
  if ((tid & 31) == 0) wp[tid >> 5] = prod;
  __syncthreads();
  if (tid == 0) {
    double pr = wp[0];
    for (int w = 1; w < kZhatThreads / 32; ++w) pr *= wp[w];
    double zh = sqrt(pr > 0.0 ? pr : 0.0);
    if (ws.sm.z[i] < 0.0) zh = -zh;
    ws.sm.zhat[i] = zh;
  }
}

__global__ void __launch_bounds__(kZhatThreads) k_zhat(const __grid_constant__ Ws ws) {
  zhat_body(ws, cta_single());
}
__global__ void __launch_bounds__(kZhatThreads) k_zhat_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  zhat_body(*t.ws[i], batch_pos(t, i));
}


// ---------------------------------------------------------------------------------------
// k_vectors: kept column j -> u_j, v_j (core coordinates 0..r; r is the p/rho column)
// ---------------------------------------------------------------------------------------
constexpr int kVecThreads = 64;

__device__ __forceinline__ void vectors_body(const Ws& ws, CtaPos cp) {
  pdl_wait();
  // after the wait, so that a successor placed now may read what any kernel before this one
  // wrote; it waits in its own pdl_wait for this grid, on the SMs this grid leaves free
  pdl_trigger();
  Ctl* ctl = ws.ctl;
  const int j = cp.b;
  const int tid = threadIdx.x;
  const double* d = ws.sm.d;
  // this thread's first pole (the arrays hold kMaxN entries): loaded before the dependent
  // chain rnew -> src -> org -> d below, so that their latencies overlap
  const double d0 = d[tid], zh0 = ws.sm.zhat[tid];
  const int pole0 = ws.sm.pole[tid];
  if (j >= ctl->rnew) return;
  const int n = ctl->n, m = ctl->m, r = n - 1;
  const int code = ws.sm.src[j];
  __shared__ double u[kMaxN], v[kMaxN], red[4];
  for (int i = tid; i < n; i += kVecThreads) {
    u[i] = 0.0;
    v[i] = (code >= 0 && i == r) ? -1.0 : 0.0;  // v = (d_i u_i, -1) for a root
  }
  __syncthreads();
  if (code >= 0) {
    const double dob = d[ws.sm.org[code]];
    const double mu = ws.sm.mu[code];
    for (int i = tid; i < m; i += kVecThreads) {
      const bool first = i == tid;
      const double di = first ? d0 : d[i];
      const double ui = (first ? zh0 : ws.sm.zhat[i]) / ((di - dob) * (di + dob) - mu);  // z^_i / (d_i^2 - lambda)
      const int c = first ? pole0 : ws.sm.pole[i];
      u[c] = ui;
      if (c < r) v[c] = di * ui;
    }
    __syncthreads();
    double su = 0.0, sv = 0.0;
    for (int i = tid; i < n; i += kVecThreads) {
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
    __shared__ double inv_s[2];
    if (tid < 2)  // once: FP64 reciprocal square roots run at the FP64 rate
      inv_s[tid] = rsqrt(red[tid] + red[2 + tid]);
    __syncthreads();
    const double iu = inv_s[0], iv = inv_s[1];
    for (int i = tid; i < n; i += kVecThreads) {
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
  for (int i = tid; i < n; i += kVecThreads) {
    ws.sm.U[(size_t)j * kMaxN + i] = u[i];
    ws.sm.V[(size_t)j * kMaxN + i] = v[i];
  }
}

__global__ void __launch_bounds__(kVecThreads) k_vectors(const __grid_constant__ Ws ws) {
  vectors_body(ws, cta_single());
}
__global__ void __launch_bounds__(kVecThreads) k_vectors_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  vectors_body(*t.ws[i], batch_pos(t, i));
}


// ---------------------------------------------------------------------------------------
// k_apply: column j of the new small state (written to the other state buffer)
//   M'    = U'^T [[M, w], [rho r_last^T, gamma]] V'
//   Q'    = [[Q, q_n(0:r0)], [0, q_n(r0)]] U'     (rows: L0 coordinates incl. the append)
//   r_first' = [r_first, 0] V'  (= last row of V' when c is u^0),  r_last' = V'[r, :]
//   S' = sigma'[0:rnew] (unscaled);  a' = L0'^T x
// ---------------------------------------------------------------------------------------
constexpr int kApplyThreads = 256;
// shared regions of the bulk-staged arrays of k_apply, in doubles: one double longer than the
// array, rounded up to an even count (16-byte aligned), for the handle's r_max and cap
__host__ __device__ constexpr int apply_reg(int n) { return (n + 3) & ~1; }
__host__ __device__ constexpr int apply_reg_m(int rm) { return apply_reg(rm * rm); }
__host__ __device__ constexpr int apply_reg_q(int rm, int cap) { return apply_reg(rm * (cap + 1)); }
__host__ __device__ constexpr int apply_reg_u(int rm) { return apply_reg(rm * kMaxN); }
__host__ __device__ constexpr int apply_smem(int rm, int cap) {
  return (int)sizeof(double) * (apply_reg_m(rm) + apply_reg_q(rm, cap) + apply_reg_u(rm));
}

__device__ __forceinline__ int count4(int sub, int n) { return n > sub ? (n - sub + 3) >> 2 : 0; }

__device__ __forceinline__ void apply_body(const Ws& ws, CtaPos cp) {
  Ctl* ctl = ws.ctl;
  const int j = cp.b;
  const int tid = threadIdx.x;
  // Before the wait on the previous kernel (k_vectors) only what earlier kernels wrote is
  // read: the committed state, and the scalars and vectors of k_prep and k_zhat.  Nothing
  // is written before it.
  const int rnew = ctl->rnew;
  const int cur = ctl->cur;
  const StateBuf st = ws.st[cur], nx = ws.st[cur ^ 1];
  const int r = st.hdr->r, r0 = st.hdr->r0;
  const int r0e = ctl->r0e;
  const int cap = ws.cap;
  const bool compact = r0e > cap;
  const int append = ctl->append;
  const int n = r + 1;
  const int qld = cap + 1, rm = ws.rmax;
  const bool mine = j < rnew;  // this CTA forms column j
  // every product below runs from shared memory: M (r columns, ld rmax), Q (r columns, ld
  // cap + 1) and the kept left singular vectors U (rnew columns, ld kMaxN) by bulk copies
  // (regions of an even number of doubles, each one longer than its array), the short
  // vectors by 8-byte asynchronous copies
  extern __shared__ __align__(16) double asm_[];
  double* sM = bulk_dst(asm_, st.M);                                           // [k][i], ld rm
  double* sQ = bulk_dst(asm_ + apply_reg_m(rm), st.Q);                         // [k][i], ld qld
  double* sU = bulk_dst(asm_ + apply_reg_m(rm) + apply_reg_q(rm, cap), ws.sm.U);  // [i][k], ld kMaxN
  __shared__ double v[kMaxN], u[kMaxN], bv[kMaxN], qcol[kMaxCap + 1];
  __shared__ double sw[kMaxN], srl[kMaxN], srf[kMaxN], sqn[kMaxCap + 1], syx[kMaxCap + 1];
  __shared__ __align__(8) uint64_t sbar;
  const int nM = r * rm, nQ = r * qld, nU = rnew * kMaxN;
  int pairs = 0, sexp = 0;
  double sigj = 0.0, rho = 0.0, gamma = 0.0;
  if (mine) {
    if (tid == 0) {
      mbar_init(&sbar, 1);
      mbar_fence_init();
      const BulkSpan a = bulk_span(st.M, nM), b = bulk_span(st.Q, nQ), c = bulk_span(ws.sm.U, nU);
      mbar_arrive_expect_tx(&sbar, 8u * (uint32_t)(a.body + b.body + c.body));  // U joins after the wait
      bulk_issue(sM, st.M, a, &sbar);
      bulk_issue(sQ, st.Q, b, &sbar);
    }
    if (tid == 32) bulk_ends(sM, st.M, nM);
    if (tid == 64) bulk_ends(sQ, st.Q, nQ);
    stage_doubles(sw, ws.sm.w, r, tid, kApplyThreads);
    stage_doubles(srl, st.rl, r, tid, kApplyThreads);
    stage_doubles(srf, st.rf, r, tid, kApplyThreads);
    stage_doubles(sqn, ws.sm.qn, r0e, tid, kApplyThreads);
    if (compact) stage_doubles(syx, ws.sm.yext, r0e, tid, kApplyThreads);
    pairs = st.hdr->pairs;
    sexp = ctl->scale_exp;
    sigj = ws.sm.sig[kMaxN + j];
    rho = ctl->rho;
    gamma = ctl->gamma;
  }
  pdl_wait();
  pdl_trigger();  // the compaction kernel's CTAs are placed now (most return at once)
  // k_prep wrote the rest of the next state's header, its a and s (an update that does not
  // compact); an appended column is formed by the next tall pass (compaction forms it at once)
  if (j == 0 && tid == 0) {
    nx.hdr->r = rnew;
    if (compact) nx.hdr->r0 = rnew;
    ctl->mode = compact ? PB_COMPACT : (append ? PB_APPEND : PB_NONE);
  }
  if (mine) {
    // the singular vectors of k_vectors
    if (tid == 0) bulk_issue(sU, ws.sm.U, bulk_span(ws.sm.U, nU), &sbar);
    if (tid == 96) bulk_ends(sU, ws.sm.U, nU);
    stage_doubles(v, ws.sm.V + (size_t)j * kMaxN, n, tid, kApplyThreads);
    stage_doubles(u, ws.sm.U + (size_t)j * kMaxN, n, tid, kApplyThreads);
    cp_async_wait_all();
    __syncthreads();
    bulk_wait(&sbar, &ctl->status);
    // B v, rows 0..r-1: M v[0:r] + w v_r  (4 threads per row; r <= 64 rows)
    {
      const int i = tid >> 2, sub = tid & 3;
      double acc = 0.0;
      if (i < r)
        #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
        for (int k = sub; k < r; k += 4) acc = fma(sM[(size_t)k * rm + i], v[k], acc);
      acc = group4_sum_d(acc);
      if (i < r && sub == 0) bv[i] = fma(sw[i], v[r], acc);
    }
    // row r: rho (r_last . v[0:r]) + gamma v_r   (warp 7, which writes it itself)
    if ((tid >> 5) == 7) {
      const int lane = tid & 31;
      double t = 0.0;
      #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
      for (int k = lane; k < r; k += 32) t = fma(srl[k], v[k], t);
      t = warp_sum_d(t);
      if (lane == 0) bv[r] = fma(rho, t, gamma * v[r]);
    }
    // Q' column j (rows 0..r0e-1): Q u[0:r] + qn u_r
    for (int base = 0; base < 4 * r0e; base += kApplyThreads) {
      const int i = (base + tid) >> 2, sub = tid & 3;
      double acc = 0.0;
      if (i < r0)
        #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
        for (int k = sub; k < r; k += 4) acc = fma(sQ[(size_t)k * qld + i], u[k], acc);
      acc = group4_sum_d(acc);
      if (i < r0e && sub == 0) qcol[i] = fma(sqn[i], u[r], acc);
    }
    __syncthreads();
    // M' column j: U'^T (B v)   (4 threads per output row i < rnew)
    {
      const int i = tid >> 2, sub = tid & 3;
      double acc = 0.0;
      if (i < rnew)
        #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
        for (int k = sub; k < n; k += 4) acc = fma(sU[(size_t)i * kMaxN + k], bv[k], acc);
      acc = group4_sum_d(acc);
      if (i < rnew && sub == 0) nx.M[(size_t)j * rm + i] = acc;
    }
    if (compact) {
      for (int i = tid; i < r0e; i += kApplyThreads) ws.sm.QB[(size_t)j * qld + i] = d2f2(qcol[i]);
      for (int i = tid; i < rnew; i += kApplyThreads) nx.Q[(size_t)j * qld + i] = i == j ? 1.0 : 0.0;
    } else {
      for (int i = tid; i < r0e; i += kApplyThreads) nx.Q[(size_t)j * qld + i] = qcol[i];
    }
    // r_first', r_last', S', a' (compaction)  -- warp 0
    if (tid < 32) {
      const int lane = tid;
      double rf = 0.0;
      if (pairs != 0) {
        #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
        for (int k = lane; k < r; k += 32) rf = fma(srf[k], v[k], rf);
        rf = warp_sum_d(rf);
      }
      double a = 0.0;
      if (compact) {
        #pragma unroll 1  // a dependent chain: unrolling adds code, not speed
        for (int i = lane; i < r0e; i += 32) a = fma(qcol[i], syx[i], a);
        a = warp_sum_d(a);
      }
      if (lane == 0) {
        nx.rf[j] = pairs == 0 ? v[r] : rf;
        nx.rl[j] = v[r];
        nx.S[j] = sigj * __longlong_as_double((long long)(1023 + sexp) << 52);
        if (compact) nx.a[j] = d2f2(a);
      }
    }
  }
  // the last CTA commits the new state and snapshot buffers
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&ctl->ticket_b, 1u);
  __syncthreads();
  if (ticket != cp.g - 1) return;
  if (tid == 0) {
    __threadfence();
    ctl->cur = cur ^ 1;
    ctl->cur_c = ctl->cur_c ^ 1;
    ctl->eig_valid = 0;
    ctl->model_ver += 1ull;
    ctl->ticket_b = 0u;
  }
}

__global__ void __launch_bounds__(kApplyThreads) k_apply(const __grid_constant__ Ws ws) {
  apply_body(ws, cta_single());
}
__global__ void __launch_bounds__(kApplyThreads) k_apply_batch(const __grid_constant__ BatchTab t) {
  const int i = batch_find(t, blockIdx.x);
  apply_body(*t.ws[i], batch_pos(t, i));
}

// ---------------------------------------------------------------------------------------
static int prep_smem_cap(int cap) {
  const int qld = cap + 1;  // Q's region (bulk-copied: one double longer, kept even), then ac, yx, z, p, p2
  return (int)sizeof(double) * (qld * kMaxR + 2 + 3 * qld + 2 * kMaxN);
}

// staged M, Q and U of k_apply at the largest sizes (a batch's launch); a single handle's
// launch asks for its own r_max and cap only (apply_smem)
constexpr int kApplySmem = apply_smem(kMaxR, kMaxCap);

cudaError_t prepare_core() {
  cudaError_t e = cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, prep_smem_cap(kMaxCap));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prep_a, cudaFuncAttributeMaxDynamicSharedMemorySize, prep_smem_cap(kMaxCap));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prep_b, cudaFuncAttributeMaxDynamicSharedMemorySize, prep_smem_cap(kMaxCap));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmem);
  return e;
}

int prep_smem_of(int cap) { return prep_smem_cap(cap); }

cudaError_t prepare_core_batch() {
  cudaError_t e = cudaFuncSetAttribute(k_prep_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, prep_smem_cap(kMaxCap));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, kApplySmem);
  return e;
}

// the five small-solve kernels of a batch's update, each one launch over every instance: one
// CTA per instance for k_prep, kMaxN per instance for k_roots, k_vectors and k_apply, kMaxN + 1
// for k_zhat (the CTAs past an instance's own sizes return at once, as in its own launches)
cudaError_t launch_small_batch(const BatchTab& one, const BatchTab& per_root, const BatchTab& per_zhat, int prep_smem,
                               cudaStream_t s) {
  cudaError_t e = launch_dependent(k_prep_batch, one.first[one.ninst], kPrepThreads, prep_smem, s, one);
  if (e == cudaSuccess) e = launch_dependent(k_roots_batch, per_root.first[per_root.ninst], kRootThreads, 0, s, per_root);
  if (e == cudaSuccess) e = launch_dependent(k_zhat_batch, per_zhat.first[per_zhat.ninst], kZhatThreads, 0, s, per_zhat);
  if (e == cudaSuccess) e = launch_dependent(k_vectors_batch, per_root.first[per_root.ninst], kVecThreads, 0, s, per_root);
  if (e == cudaSuccess)
    e = launch_dependent(k_apply_batch, per_root.first[per_root.ninst], kApplyThreads, (size_t)kApplySmem, s, per_root);
  return e;
}

// the first part of k_prep alone: a pipelined update's last kernel (the next pass A waits
// for it; the rest of the update runs beside that pass)
cudaError_t launch_prep(const Ws& ws, cudaStream_t s) {
  return launch_dependent(k_prep_a, 1, kPrepThreads, prep_smem_cap(ws.cap), s, ws);
}
static cudaError_t launch_roots_to_apply(const Ws& ws, cudaStream_t s) {
  cudaError_t e = launch_dependent(k_roots, kMaxN, kRootThreads, 0, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_zhat, kMaxN + 1, kZhatThreads, 0, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_vectors, kMaxN, kVecThreads, 0, s, ws);
  if (e == cudaSuccess) e = launch_dependent(k_apply, kMaxN, kApplyThreads, (size_t)apply_smem(ws.rmax, ws.cap), s, ws);
  return e;
}
// the rest of an update after launch_prep: the second part of k_prep, then k_roots .. k_apply
cudaError_t launch_small_tail(const Ws& ws, cudaStream_t s) {
  cudaError_t e = launch_dependent(k_prep_b, 1, kPrepThreads, prep_smem_cap(ws.cap), s, ws);
  if (e == cudaSuccess) e = launch_roots_to_apply(ws, s);
  return e;
}
// the small solves of an update in one chain (k_prep whole)
cudaError_t launch_small(const Ws& ws, cudaStream_t s) {
  cudaError_t e = launch_dependent(k_prep, 1, kPrepThreads, prep_smem_cap(ws.cap), s, ws);
  if (e == cudaSuccess) e = launch_roots_to_apply(ws, s);
  return e;
}

}  // namespace odmd
