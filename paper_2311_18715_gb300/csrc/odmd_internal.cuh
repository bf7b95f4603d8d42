// Internal definitions shared by the CUDA translation units of libodmd.
//
// Numerics: GB300 issues FP32 FMAs ~70x faster than FP64 ones and converts between the
// two at the FP64 rate, so every pass over the tall basis works on floats: a basis
// element is an unevaluated sum hi + lo of two floats (48-bit significand) in the
// FP64-accuracy mode, products are formed exactly with FMA (two-product) and summed
// with Knuth's two-sum into a hi/lo accumulator.  Only O(r^2)..O(r^3) small solves run
// in native FP64.
#pragma once
#include <string>

#include "odmd.h"
#include "pair2d.cuh"
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace odmd {

constexpr int kThreads = 256;      // threads of every tall-pass CTA
constexpr int kTile = 64;          // rows per tile of a tall pass
constexpr int kStages = 4;         // TMA pipeline depth of a tall pass

constexpr int kMaxR = 64;          // largest r_max
constexpr int kMaxSlack = 32;      // largest slack
constexpr int kMaxCap = kMaxR + kMaxSlack;  // largest number of basis columns r0
constexpr int kMaxN = kMaxR + 1;   // largest core matrix order r + 1
constexpr int kMaxMaps = 13;       // tensor maps per plane and box height: widths of 1, 3, ..., 25 chunks
constexpr int kPassARows = 32;     // rows of a pass-A tile (its tensor maps' box height)
constexpr int kRollK = 64;         // horizons (columns) per rollout launch
constexpr int kGramCtas = 304;     // most CTAs of the Gram pass of the orthogonality refinement

enum Storage { ST_DD = 0, ST_F32 = 1, ST_BF16 = 2 };

// device status word bits
enum : int {
  DEV_NONFINITE = 1,   // a non-finite value reached a reduction or the small solve
  DEV_TIMEOUT = 2,     // a bounded wait on an mbarrier ran out
  DEV_EIG_NOCONV = 4,  // the Francis QR iteration did not converge
  DEV_EIG_COND = 8,    // the eigenvector matrix is singular to working precision
  DEV_SECULAR = 16,    // a secular-equation root failed to converge
  DEV_NOMODEL = 32     // predict/check/eig asked for with rank 0
};

// pass-B modes
enum : int { PB_NONE = 0, PB_APPEND = 1, PB_COMPACT = 2 };

// The small state that the update carries from one snapshot to the next (S, the rows of R,
// M, the factor Q of L = L0 Q) and the scratch of the core SVD are IEEE doubles; the vectors
// the tall passes read are double-float pairs (float2: hi, lo; see dd.cuh).

// Committed small state (two copies, selected by Ctl::cur).
struct StateHdr {
  int r;        // rank
  int r0;       // number of tall-basis columns in use
  int pairs;    // snapshot pairs ingested
  int compactions;
  int pend;     // 1: column r0-1 of L0 is not yet written (formed by the next tall pass)
  int pad_i;
  float2 cn2;   // ||c||^2 of the latest snapshot c
  float2 pinv;  // 1/rho0 of the pending column
};

struct StateBuf {
  StateHdr* hdr;
  double* S;    // r_max   singular values
  double* rf;   // r_max   first row of R
  double* rl;   // r_max   last row of R
  double* M;    // r_max x r_max, column-major, ld = r_max   (M = L^T U^+ R)
  double* Q;    // (cap+1) x r_max, column-major, ld = cap+1  (L = L0 Q), FP64
  float2* a;    // cap+1   L0^T c
  float2* ps;   // cap+1   coefficients s of the pending column: (e - L0 s) / rho0
};

// Control block: indices of the committed buffers, tickets, status, small scalars.
struct Ctl {
  int cur;          // committed StateBuf
  int cur_c;        // committed snapshot buffer (holds c)
  int status;       // DEV_* bits
  unsigned ticket_a, ticket_b, ticket_r;
  int mode;         // pass-B mode for the update in flight
  int r0e;          // basis columns after the (optional) append
  int rnew;         // rank after the update
  int append;       // 1 if the update appends a column to L0
  int n;            // core order r + 1
  int m;            // non-deflated poles of the secular problem
  int ndefl;        // deflated singular values
  int nrot;         // Givens rotations used by the deflation
  int eig_valid;    // eigen-cache matches the committed state
  int eig_r;        // rank the eigen-cache was built for
  int scale_exp;    // the core matrix is scaled by 2^-scale_exp for the secular solve
  int pipe_flag;    // 1: the update in flight compacts (a pipelined next tall pass must wait for it)
  double thr;       // tau * max(sigma_1, ||c||)
  double rho0;      // norm of the part of c outside span(L0)
  double rho;       // norm of the part of c outside span(L)
  double gamma;     // j^T x
  float2 check_num, check_den;  // reductions of the credibility check
  unsigned long long prof_r0_sum;  // sum of r0 over pass-A launches (for roofline accounting)
  unsigned long long prof_a;       // number of pass-A launches
  unsigned long long model_ver;    // advanced by every commit of a new model (update, refinement)
  unsigned long long pc_ver;       // model_ver + 1 of the vectors in Small::pc (0: none)
  double pc_t[2];                  // their horizons: the first and the last of the call that made them
};

// Scratch of the small solve (single copy).
struct Small {
  float2* red;      // 2*cap+3 reduced tall sums: s (r0), y (r0), eta, ex, xi
  double* ac;       // cap+1   corrected projection of c onto L0 (a + s)
  double* yext;     // cap+1   L0_ext^T x
  double* qn;       // cap+1   new unit direction in L0_ext coordinates
  double* p;        // kMaxN   L^T c
  double* w;        // kMaxN   L^T x
  double* d;        // kMaxN   poles (ascending) of the secular problem, as scaled singular values
  double* z;        // kMaxN   scaled weights at those poles
  int* pole;        // kMaxN   core coordinate of each pole
  double* dc;       // kMaxN   scaled diagonal of the core in core coordinates (S, 0)
  int* defl;        // kMaxN   deflated core coordinates
  int* rot_i;       // kMaxN
  int* rot_j;
  double* rot_c;
  double* rot_s;
  int* org;         // kMaxN   origin pole of each root
  double* mu;       // kMaxN   root minus its origin pole (scaled, squared units)
  double* zhat;     // kMaxN   Loewner weights
  double* sig;      // 2 kMaxN singular values of the core: roots, then the sorted list
  int* src;         // kMaxN   source of output column j: >=0 root index, <0: -(defl idx)-1
  double* U;        // kMaxN x kMaxN, column-major   left singular vectors of K (kept)
  double* V;        // kMaxN x kMaxN                   right singular vectors of K (kept)
  float2* QB;       // (cap+1) x r_max, col-major ld cap+1: pass-B rotation (compaction)
  float2* coef;     // (cap+1) x kRollK rollout coefficients in L0 coordinates
  float2* pc;       // 2 x kMaxN: A~^{pc_t[s]} y, s = 0, 1, of the model of version pc_ver - 1 (see Ctl)
};

// Eigen-cache.
struct Eig {
  float2* lre;      // r_max eigenvalues
  float2* lim;
  float2* Vre;      // r_max x r_max eigenvectors (column-major, unit 2-norm)
  float2* Vim;
  float2* bre;      // r_max  b = V^{-1} (S * r_first)
  float2* bim;
};

// Box width (in 16-byte chunks, always odd) used for r0 active columns of esz bytes:
// an odd number of chunks per shared-memory row keeps row-wise float4 reads and
// column-wise scalar reads of a dense TMA tile free of bank conflicts.
__host__ __device__ inline int box_chunks(int r0, int esz) {
  int c = (r0 * esz + 15) / 16;
  return (c & 1) ? c : c + 1;
}

struct Ws {
  int64_t n;        // rows
  int64_t npad;     // rows rounded up to kTile
  int rmax, cap, ldg, prec, gridA;
  int stagesA;      // TMA pipeline depth of pass A (as many stages as shared memory holds)
  int shards;       // row shards a reduction pass is split into (1: one launch; see tall.cu)
  int gridG;        // Gram pass grid: two CTAs per SM, at most kGramCtas
  float tau_h, tau_l;  // truncation tolerance as a double-float
  double tau;          // truncation tolerance
  Ctl* ctl;
  void* Lh;         // hi plane (float) / bf16 plane
  float* Ll;        // lo plane (FP64 mode only)
  void* cbuf[2];    // snapshot buffers (npad elements: float pairs in FP64 mode, else floats)
  void* xbuf;       // scratch snapshot (check input copy), same format
  float2* ebuf;     // first-pass residual e = c - L0 a of the update in flight (hi, lo)
  const CUtensorMap* maps;  // [2 plane + p][k] for box heights (kTile, kPassARows) x planes:
                            // 2-D maps of the basis planes, boxes of (2k+1) chunks; plane 1
                            // only in FP64 mode
  float2* part;     // per-CTA partial sums: gridA x (2*cap+3)
  float2* gpart;    // refinement: per-CTA Gram partials, kGramCtas x cap(cap+1)/2 (or null)
  float2* rscr;     // refinement: small matrices (or null)
  StateBuf st[2];
  Small sm;
  Eig eig;
  float2* out2;     // 4 double-floats for host read-back
};

// ------------------------------------------------------------------ multi-instance launches
// Where a CTA sits within its instance: its index b and the instance's grid size g.  A
// kernel of one instance takes blockIdx.x and gridDim.x; a kernel over many instances (one
// launch for the same step of every instance of a batch) maps its grid onto the instances
// of a table, instance i owning CTAs [first[i], first[i + 1]).
struct CtaPos {
  int b, g;
};
__device__ __forceinline__ CtaPos cta_single() { return CtaPos{(int)blockIdx.x, (int)gridDim.x}; }

constexpr int kMaxBatch = 64;  // instances per multi-instance launch
// passed by value (under 1 KB of kernel parameters): each instance's workspace view lives
// in its own workspace (written at create), so a batch needs no memory of its own
struct BatchTab {
  const Ws* ws[kMaxBatch];     // the instances' workspace views (device memory)
  int first[kMaxBatch + 1];    // first CTA of each instance in the launch's grid
  int ninst;
};
// the instance that owns CTA blk (binary search over the prefix sums)
__device__ __forceinline__ int batch_find(const BatchTab& t, int blk) {
  int lo = 0, hi = t.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.first[mid] <= blk)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ CtaPos batch_pos(const BatchTab& t, int i) {
  return CtaPos{(int)blockIdx.x - t.first[i], t.first[i + 1] - t.first[i]};
}
// the snapshots of a batch's update: instance i's n[i] elements from src[i] into dst[i];
// first[] are prefix sums of the element pairs
struct IngestTab {
  const void* src[kMaxBatch];
  void* dst[kMaxBatch];
  int64_t n[kMaxBatch];
  int64_t first[kMaxBatch + 1];
  int ninst;
};

// ------------------------------------------------------------------ dependent launches
// The kernels of an update run back to back in one CUDA graph.  Each is launched with
// programmatic stream serialisation, so the grid is set up while its predecessor finishes;
// its first statement waits for the predecessor's completion and memory (and returns at
// once when the kernel was launched without the attribute).  Every kernel that can be
// launched this way begins with pdl_wait.  (Letting every kernel trigger its successor at
// its start, so that the successor's CTAs are placed while it runs, measured slower: 5,926
// against 6,362 snapshot updates/s; the small-solve kernels, whose grids leave most SMs
// free, do trigger, after their own wait: see pdl_trigger.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the successor's CTAs be placed now (they still wait for this grid's completion in
// their pdl_wait): used only by the small-solve kernels, whose grids leave most SMs free,
// and only after their own pdl_wait, so that whatever a successor reads before its wait
// was written by kernels that have completed.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ float-float arithmetic
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Running sum h + l; l collects rounding errors and small cross terms lazily.
struct Acc {
  float h, l;
};

__device__ __forceinline__ Acc acc_zero() { return Acc{0.f, 0.f}; }

// A += (xh + xl) * (yh + yl), dropping xl*yl (2^-48 relative).
__device__ __forceinline__ void acc_fma(Acc& A, float xh, float xl, float yh, float yl) {
  float p = __fmul_rn(xh, yh);
  float pe = __fmaf_rn(xh, yh, -p);
  pe = __fmaf_rn(xh, yl, pe);
  pe = __fmaf_rn(xl, yh, pe);
  float s, e;
  two_sum(A.h, p, s, e);
  A.h = s;
  A.l = __fadd_rn(A.l, __fadd_rn(e, pe));
}

__device__ __forceinline__ void acc_add(Acc& A, float bh, float bl) {
  float s, e;
  two_sum(A.h, bh, s, e);
  A.h = s;
  A.l = __fadd_rn(A.l, __fadd_rn(e, bl));
}

__device__ __forceinline__ Acc acc_norm(Acc A) {
  float s = __fadd_rn(A.h, A.l);
  float e = __fsub_rn(A.l, __fsub_rn(s, A.h));
  return Acc{s, e};
}

// ---- packed pairs: two floats in one 64-bit register pair, operated on by the FP32x2
// instructions of sm_100 and later (one issue slot for two lanes of work).  The double-float
// accumulate below performs, lane by lane, exactly the operations of acc_fma, so a packed
// and a scalar accumulation give bitwise equal results.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2x_pack(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2x_unpack(f2x v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
#ifndef ODMD_SCALAR_PAIRS
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
#else
// the same operations lane by lane on scalar FP32 instructions
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  float a0, a1, b0, b1;
  f2x_unpack(a, a0, a1);
  f2x_unpack(b, b0, b1);
  return f2x_pack(__fadd_rn(a0, b0), __fadd_rn(a1, b1));
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  float a0, a1, b0, b1;
  f2x_unpack(a, a0, a1);
  f2x_unpack(b, b0, b1);
  return f2x_pack(__fsub_rn(a0, b0), __fsub_rn(a1, b1));
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  float a0, a1, b0, b1;
  f2x_unpack(a, a0, a1);
  f2x_unpack(b, b0, b1);
  return f2x_pack(__fmul_rn(a0, b0), __fmul_rn(a1, b1));
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  float a0, a1, b0, b1, c0, c1;
  f2x_unpack(a, a0, a1);
  f2x_unpack(b, b0, b1);
  f2x_unpack(c, c0, c1);
  return f2x_pack(__fmaf_rn(a0, b0, c0), __fmaf_rn(a1, b1, c1));
}
#endif

struct Acc2 {
  f2x h, l;
};
__device__ __forceinline__ Acc2 acc2_zero() { return Acc2{0ull, 0ull}; }

// A += (xh + xl) * (yh + yl) in both lanes, given nyh = -yh: the product's rounding error
// (xh*yh - p) + xh*yl + xl*yh is formed with FMAs and the high part p is added with
// two-sum, the same steps as acc_fma.
__device__ __forceinline__ void acc2_fma(Acc2& A, f2x xh, f2x xl, f2x yh, f2x nyh, f2x yl) {
  const f2x np = mul2(xh, nyh);     // -p
  f2x pe = fma2(xh, yh, np);        // xh*yh - p
  pe = fma2(xh, yl, pe);
  pe = fma2(xl, yh, pe);
  const f2x s = sub2(A.h, np);      // two-sum of A.h and p
  const f2x bb = sub2(s, A.h);
  const f2x e = sub2(sub2(A.h, sub2(s, bb)), add2(np, bb));
  A.h = s;
  A.l = add2(A.l, add2(e, pe));
}

// the two lanes of A as scalar accumulators
__device__ __forceinline__ void acc2_split(Acc2 A, Acc& a0, Acc& a1) {
  f2x_unpack(A.h, a0.h, a1.h);
  f2x_unpack(A.l, a0.l, a1.l);
}

// h = RN(x), l = RN(x - h): by integer operations on x's bits (pair2d.cuh), by conversions
// (FP64 rate) when a part leaves the normal float range
__device__ __forceinline__ void split_double(double x, float& h, float& l) {
  if (!double_to_pair_fast(x, h, l)) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
  }
}

__device__ __forceinline__ double join_double(float h, float l) { return (double)h + (double)l; }

// ------------------------------------------------------------------ TMA bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// one arrival (release semantics: this thread's earlier shared-memory writes are visible to
// whoever completes its wait on the phase)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for an mbarrier phase with a time limit (2 s).  On timeout the status word gets
// DEV_TIMEOUT and false is returned; the caller skips its compute for that tile.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 2000000000ull) {
      atomicOr(status, DEV_TIMEOUT);
      return false;
    }
  }
}

// After a timeout: give the copies still in flight for stages [li, li + depth) up to
// 0.5 s in total to land before the CTA leaves, so no copy outlives its shared memory.
__device__ __forceinline__ void mbar_drain(uint64_t* bars, int stages, int li, int my_tiles) {
  const uint64_t t0 = global_ns();
  for (int l = li; l < my_tiles && l < li + stages; ++l) {
    const uint32_t par = (uint32_t)((l / stages) & 1);
    while (!mbar_try_wait(&bars[l % stages], par)) {
      if (global_ns() - t0 > 500000000ull) return;
    }
  }
}

// 2-D tiled TMA load of box (x, y) of `map` into shared memory, counted on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// The same load with an L2 eviction-priority hint (a policy from l2_evict_first_policy).
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3}], [%4], %5;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// 1-D bulk copy global -> shared (TMA), completion counted on `bar` in bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// The same copy with an L2 eviction-priority hint (a policy from l2_evict_first_policy):
// data streamed once should not push reused lines (code, small state) out of L2.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ Acc warp_sum_acc(Acc a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float h = __shfl_xor_sync(0xffffffffu, a.h, o);
    float l = __shfl_xor_sync(0xffffffffu, a.l, o);
    acc_add(a, h, l);
  }
  return a;
}

// ------------------------------------------------------------------ launchers (per unit)
// tall.cu
cudaError_t launch_pass_a(const Ws& ws, cudaStream_t s);
cudaError_t launch_pass_b(const Ws& ws, cudaStream_t s);
cudaError_t launch_flush(const Ws& ws, cudaStream_t s);  // write a pending basis column
cudaError_t launch_first(const Ws& ws, cudaStream_t s);
int launches_per_reduction(const Ws& ws);  // kernel launches of one pass A, check or first-norm
cudaError_t launch_ingest(const Ws& ws, const void* src, void* dst, cudaStream_t s);  // snapshot -> workspace
const void* ingest_kernel(int prec);  // the kernel launch_ingest uses (graph node lookup)
cudaError_t prepare_tall(const Ws& ws);
cudaError_t prepare_small(const Ws& ws);
cudaError_t prepare_core();
// multi-instance launches (one per step of the update over every instance of a batch)
cudaError_t launch_ingest_batch(const IngestTab& t, int prec, cudaStream_t s);
cudaError_t launch_pass_a_batch(const BatchTab& t, int prec, int smem, cudaStream_t s);
cudaError_t launch_pass_b_batch(const BatchTab& t, int prec, int smem, cudaStream_t s);
cudaError_t launch_small_batch(const BatchTab& one, const BatchTab& per_root, const BatchTab& per_zhat,
                               int prep_smem, cudaStream_t s);
cudaError_t launch_split_compact_batch(const BatchTab& t, int prec, cudaStream_t s);
int split_grid_of(const Ws& ws, int sms);
int pass_a_smem(int prec, int cap);
int pass_b_smem(int prec, int cap);
int prep_smem_of(int cap);
cudaError_t prepare_tall_batch();
cudaError_t prepare_core_batch();
cudaError_t prepare_split_batch();  // shared-memory limits of the FP64 small solves of the update
bool split_rollout_ok(const Ws& ws, int kcols);       // the tensor-core rollout takes this call
cudaError_t prepare_split(const Ws& ws);
cudaError_t launch_split_rollout(const Ws& ws, int kcols, double* out, int64_t ld, int sms, cudaStream_t s);
bool split_compact_ok(const Ws& ws);               // compaction of this handle on the tensor cores
cudaError_t launch_split_compact(const Ws& ws, int sms, cudaStream_t s);
cudaError_t launch_rollout(const Ws& ws, const double* coef_src, int kcols, void* out, int64_t ld,
                           int coef_mode, cudaStream_t s);
cudaError_t launch_check(const Ws& ws, cudaStream_t s);
int tall_smem_bytes(int prec);
int stages_a(int prec, int cap);  // pass A pipeline depth for this storage format and cap
// small.cu
cudaError_t launch_small(const Ws& ws, cudaStream_t s);
cudaError_t launch_prep(const Ws& ws, cudaStream_t s);        // the first part of k_prep (pipelined)
cudaError_t launch_small_tail(const Ws& ws, cudaStream_t s);  // the rest: k_prep part 2, k_roots .. k_apply
cudaError_t launch_pass_a_sel(const Ws& ws, int sel, cudaStream_t s);  // pipelined pass A (tall.cu)
cudaError_t prepare_refine();
cudaError_t launch_norm_ratio(const Ws& ws, const void* r, const void* b, cudaStream_t s);  // sum r^2, sum b^2 -> out2
cudaError_t launch_refine(const Ws& ws, int cur, cudaStream_t s);  // Gram pass + small refinement
cudaError_t launch_eig(const Ws& ws, cudaStream_t s);
cudaError_t launch_coef(const Ws& ws, const double* t_host, int k, cudaStream_t s);  // k <= kRollK, t on the host
cudaError_t launch_coef_pow(const Ws& ws, const double* t_host, int k, cudaStream_t s);  // integer t only
cudaError_t launch_basis_coef(const Ws& ws, cudaStream_t s);
cudaError_t launch_init(const Ws& ws, cudaStream_t s);

// Record `msg` as the message of odmd_last_error(NULL) and return `s` (for entry points
// that have no handle).
odmd_status report_global_error(odmd_status s, const std::string& msg);

}  // namespace odmd
