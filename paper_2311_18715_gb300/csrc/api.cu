// C ABI of libodmd: argument checks, workspace layout, call sequencing.  Every O(N)
// or O(r^3) step runs in the kernels of tall.cu and small.cu; this file only decides
// which kernels to enqueue and carries a few bytes between host and device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/odmd.h"
#include "odmd_internal.cuh"

using namespace odmd;

struct odmd_instance {
  odmd_config cfg;
  Ws ws;
  cudaStream_t stream;
  int device;
  int64_t nsnap;       // snapshots received
  int64_t compactions; // host mirror is refreshed at sync points
  int cur_h;           // host mirror of Ctl::cur (flips on every update after the first)
  int curc_h;          // host mirror of Ctl::cur_c
  bool eig_dirty;
  double* pinned;      // 8 doubles of pinned host memory for read-backs
  std::string err;
  // observability
  bool prof_on;
  double prof_ms[ODMD_K_COUNT];
  long long launches[ODMD_K_COUNT];
  struct Pending {
    int cls;
    cudaEvent_t a, b;
    bool owned = true;  // false: the events also belong to another entry (returned by that one)
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  unsigned long long r0_base[2];  // device pass-A counters at enable time
  std::vector<CUtensorMap> maps_host;  // source of the tensor maps copied into the workspace
  // CUDA graphs of the update sequence, per snapshot-buffer parity and profiling mode:
  // ingest -> pass A -> small solves (5 kernels) -> pass B; the only argument that changes
  // between calls is the snapshot pointer of the ingest node.
  struct UpdGraph {
    cudaGraph_t graph = nullptr;      // kept alive: its node handles address the exec's nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ingest = nullptr;
    cudaKernelNodeParams kp{};
    const void* src = nullptr;
    void* dst = nullptr;
    int64_t n = 0;
    void* args[3] = {nullptr, nullptr, nullptr};
    cudaGraphNode_t ev[6] = {};
    cudaEvent_t ph[6] = {};           // events recorded by the nodes at capture (kept alive)
  };
  UpdGraph ug[2][2];
  // Pipelined updates: the graph of update k + 1 runs its ingest and pass A on one branch and
  // the SVD tail of update k (k_roots .. k_apply, the compaction kernel) on another, joined
  // before its k_prep; update k + 1's own tail then waits for the next update or a settle.
  // pg[cur][curc][tail]: the state and snapshot buffers of update k + 1, with or without a
  // previous tail to run; tg: a pending tail alone.
  UpdGraph pg[2][2][2];
  UpdGraph tg;
  cudaStream_t cap2 = nullptr;  // the forked branch while a pipelined graph is captured
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool pipe = true;             // pipelined updates wherever the graph path runs
  bool tail_pending = false;    // the last update's tail has not been enqueued yet
  cudaStream_t cap = nullptr;
  bool use_graphs = true;
  bool use_tc = true;   // multi-horizon rollouts on the tensor cores where split.cu takes them
  // false once nothing can be pending: the last call that changed the state was followed by
  // a flush or a tensor-core rollout (which write the pending basis column)
  bool maybe_pend = true;
  int sms = 0;          // streaming multiprocessors of the handle's device
  // odmd_update_host: two staging slots in the workspace, filled on a copy stream of their
  // own; a slot is refilled only after the update that read it
  unsigned char* stage[2] = {nullptr, nullptr};
  cudaStream_t copy = nullptr;
  // multi-instance updates (odmd_update_batch): this handle's Ws in its own workspace, a
  // process-unique serial that names it in cached batch plans, an event for their ordering
  Ws* wsv = nullptr;
  unsigned long long serial = 0;
  cudaEvent_t ev_batch = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  bool stage_used[2] = {false, false};
  int stage_next = 0;
};

namespace {

thread_local std::string g_err;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
  size_t total;
  size_t off_gpart = 0, off_rscr = 0;  // refinement scratch (refine_every > 0 only)
  size_t off_stage[2] = {0, 0};  // staging of snapshots read from host memory
  size_t off_wsv = 0;            // the handle's workspace view (Ws), read by multi-instance launches
  size_t off_ctl, off_hdr[2], off_state[2], off_small, off_eig, off_out2, off_part, off_Lh, off_Ll, off_c[2],
      off_x, off_e, off_maps;
  size_t state_doubles, small_bytes, eig_doubles;
  int64_t npad;
  int ldg, cap, rmax, partrows;
};

constexpr int kPartRows = 512;

int esz_of(int prec) { return prec == ODMD_BF16 ? 2 : 4; }
int vsz_of(int prec) { return prec == ODMD_FP64 ? 8 : 4; }

odmd_status check_cfg(const odmd_config* c, std::string& why) {
  if (!c) {
    why = "config is NULL";
    return ODMD_ERR_ARG;
  }
  if (c->n < 1 || c->n > 2147483647LL) {
    why = "n out of range [1, 2^31-1]";
    return ODMD_ERR_ARG;
  }
  if (c->r_max < 1 || c->r_max > kMaxR) {
    why = "r_max out of range [1, 64]";
    return ODMD_ERR_ARG;
  }
  if (c->slack < 0 || c->slack > kMaxSlack) {
    why = "slack out of range [0, 32]";
    return ODMD_ERR_ARG;
  }
  if (!(c->trunc_tol >= 1e-13 && c->trunc_tol < 1.0)) {
    why = "trunc_tol out of range [1e-13, 1)";
    return ODMD_ERR_ARG;
  }
  if (c->prec != ODMD_FP64 && c->prec != ODMD_FP32 && c->prec != ODMD_BF16) {
    why = "unknown precision";
    return ODMD_ERR_ARG;
  }
  if (c->prec == ODMD_BF16) {
    // an 8-bit significand cannot hold the basis orthonormal to the accuracy the rank-1
    // update assumes (measured: ||L^T L - I|| reaches ~1 at the first truncation)
    why = "ODMD_BF16 basis storage is not supported by the rank-1 update; use ODMD_FP32";
    return ODMD_ERR_ARG;
  }
  if ((c->flags & ~(ODMD_CUDA_CORES | ODMD_NO_PIPELINE)) != 0) {
    why = "unknown flags (only ODMD_CUDA_CORES and ODMD_NO_PIPELINE are defined)";
    return ODMD_ERR_ARG;
  }
  if (c->refine_every < 0) {
    why = "refine_every must be >= 0";
    return ODMD_ERR_ARG;
  }
  return ODMD_OK;
}

Layout make_layout(const odmd_config& c) {
  Layout L{};
  L.cap = c.r_max + c.slack;
  L.rmax = c.r_max;
  // row stride: an odd number of 16-byte chunks, the widest TMA box
  L.ldg = box_chunks(L.cap, esz_of(c.prec)) * 16 / esz_of(c.prec);
  L.npad = (int64_t)align_up((size_t)c.n, kTile);
  L.partrows = kPartRows;
  const int qld = L.cap + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.off_ctl = take(sizeof(Ctl));
  L.off_maps = take(4 * kMaxMaps * sizeof(CUtensorMap));
  L.off_hdr[0] = take(sizeof(StateHdr));
  L.off_hdr[1] = take(sizeof(StateHdr));
  L.state_doubles = 3 * (size_t)L.rmax + (size_t)L.rmax * L.rmax + (size_t)qld * L.rmax + 2 * (size_t)qld;
  L.off_state[0] = take(L.state_doubles * sizeof(float2));
  L.off_state[1] = take(L.state_doubles * sizeof(float2));
  // small scratch: double-floats then ints
  const size_t nd = (2 * (size_t)L.cap + 3) + 3 * (size_t)qld + 10 * (size_t)kMaxN + 2 * (size_t)kMaxN +
                    2 * (size_t)kMaxN * kMaxN + (size_t)qld * L.rmax + (size_t)qld * kRollK + 2 * (size_t)kMaxN;
  const size_t ni = 6 * (size_t)kMaxN;
  L.small_bytes = nd * sizeof(float2) + ni * 4;
  L.off_small = take(L.small_bytes);
  L.eig_doubles = 4 * (size_t)L.rmax + 2 * (size_t)L.rmax * L.rmax;
  L.off_eig = take(L.eig_doubles * sizeof(float2));
  L.off_out2 = take(8 * 8);
  L.off_part = take((size_t)L.partrows * (2 * L.cap + 3) * sizeof(float2));
  if (c.refine_every > 0) {
    L.off_gpart = take((size_t)kGramCtas * L.cap * (L.cap + 1) / 2 * sizeof(float2));
    L.off_rscr = take(((size_t)L.cap * L.cap + 3 * (size_t)L.rmax * L.rmax + 2 * (size_t)L.rmax + 2) * sizeof(float2));
  }
  const size_t plane = (size_t)L.npad * L.ldg * esz_of(c.prec);
  L.off_Lh = take(plane);
  L.off_Ll = c.prec == ODMD_FP64 ? take(plane) : 0;
  const size_t snap = (size_t)L.npad * vsz_of(c.prec);
  L.off_c[0] = take(snap);
  L.off_c[1] = take(snap);
  L.off_x = take(snap);
  L.off_e = take((size_t)L.npad * sizeof(float2));
  L.off_stage[0] = take(snap);
  L.off_stage[1] = take(snap);
  L.off_wsv = take(sizeof(Ws));
  L.total = o;
  return L;
}

odmd_status fail(odmd_t h, odmd_status s, const std::string& msg);

void carve(Ws& ws, const Layout& L, unsigned char* base, const odmd_config& c, int gridA) {
  ws.n = c.n;
  ws.npad = L.npad;
  ws.rmax = L.rmax;
  ws.cap = L.cap;
  ws.ldg = L.ldg;
  ws.prec = (int)c.prec;
  ws.gridA = gridA;
  ws.stagesA = stages_a((int)c.prec, L.cap);
  ws.tau_h = (float)c.trunc_tol;
  ws.tau_l = (float)(c.trunc_tol - (double)ws.tau_h);
  ws.tau = c.trunc_tol;
  ws.ctl = reinterpret_cast<Ctl*>(base + L.off_ctl);
  const int qld = L.cap + 1;
  for (int b = 0; b < 2; ++b) {
    StateBuf& s = ws.st[b];
    s.hdr = reinterpret_cast<StateHdr*>(base + L.off_hdr[b]);
    float2* d = reinterpret_cast<float2*>(base + L.off_state[b]);
    // S, rf, rl, M are doubles: the same 8 bytes per value as a float pair
    s.S = reinterpret_cast<double*>(d);
    d += L.rmax;
    s.rf = reinterpret_cast<double*>(d);
    d += L.rmax;
    s.rl = reinterpret_cast<double*>(d);
    d += L.rmax;
    s.M = reinterpret_cast<double*>(d);
    d += (size_t)L.rmax * L.rmax;
    s.Q = reinterpret_cast<double*>(d);
    d += (size_t)qld * L.rmax;
    s.a = d;
    d += qld;
    s.ps = d;
  }
  float2* d = reinterpret_cast<float2*>(base + L.off_small);
  Small& sm = ws.sm;
  sm.red = d;
  d += 2 * L.cap + 3;
  // the core-SVD scratch is doubles (8 bytes per value, like a float pair)
  auto dbl = [](float2* q) { return reinterpret_cast<double*>(q); };
  sm.ac = dbl(d);
  d += qld;
  sm.yext = dbl(d);
  d += qld;
  sm.qn = dbl(d);
  d += qld;
  sm.p = dbl(d);
  d += kMaxN;
  sm.w = dbl(d);
  d += kMaxN;
  sm.d = dbl(d);
  d += kMaxN;
  sm.z = dbl(d);
  d += kMaxN;
  sm.dc = dbl(d);
  d += kMaxN;
  sm.rot_c = dbl(d);
  d += kMaxN;
  sm.rot_s = dbl(d);
  d += kMaxN;
  sm.mu = dbl(d);
  d += kMaxN;
  sm.zhat = dbl(d);
  d += kMaxN;
  sm.sig = dbl(d);
  d += 2 * kMaxN;
  sm.U = dbl(d);
  d += (size_t)kMaxN * kMaxN;
  sm.V = dbl(d);
  d += (size_t)kMaxN * kMaxN;
  sm.QB = d;
  d += (size_t)qld * L.rmax;
  sm.coef = d;
  d += (size_t)qld * kRollK;
  sm.pc = d;
  d += 2 * kMaxN;
  int* ip = reinterpret_cast<int*>(d);
  sm.pole = ip;
  ip += kMaxN;
  sm.defl = ip;
  ip += kMaxN;
  sm.rot_i = ip;
  ip += kMaxN;
  sm.rot_j = ip;
  ip += kMaxN;
  sm.org = ip;
  ip += kMaxN;
  sm.src = ip;
  float2* e = reinterpret_cast<float2*>(base + L.off_eig);
  ws.eig.lre = e;
  e += L.rmax;
  ws.eig.lim = e;
  e += L.rmax;
  ws.eig.bre = e;
  e += L.rmax;
  ws.eig.bim = e;
  e += L.rmax;
  ws.eig.Vre = e;
  e += (size_t)L.rmax * L.rmax;
  ws.eig.Vim = e;
  ws.out2 = reinterpret_cast<float2*>(base + L.off_out2);
  ws.part = reinterpret_cast<float2*>(base + L.off_part);
  ws.gpart = L.off_gpart ? reinterpret_cast<float2*>(base + L.off_gpart) : nullptr;
  ws.rscr = L.off_rscr ? reinterpret_cast<float2*>(base + L.off_rscr) : nullptr;
  ws.Lh = base + L.off_Lh;
  ws.Ll = c.prec == ODMD_FP64 ? reinterpret_cast<float*>(base + L.off_Ll) : nullptr;
  ws.cbuf[0] = base + L.off_c[0];
  ws.cbuf[1] = base + L.off_c[1];
  ws.xbuf = base + L.off_x;
  ws.ebuf = reinterpret_cast<float2*>(base + L.off_e);
  ws.maps = reinterpret_cast<const CUtensorMap*>(base + L.off_maps);
}

// 2-D tile maps of the basis planes: dims {ldg, npad}, box {(2k+1) chunks, kTile rows}.
odmd_status encode_maps(odmd_t h, const Layout& L) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(h, ODMD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int esz = esz_of(h->cfg.prec);
  const int planes = h->cfg.prec == ODMD_FP64 ? 2 : 1;
  const int maxc = box_chunks(L.cap, esz);
  h->maps_host.assign(4 * kMaxMaps, CUtensorMap{});
  const CUtensorMapDataType dt = h->cfg.prec == ODMD_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  // boxes of kTile rows (the tile passes) and of kPassARows rows (pass A), per plane, for
  // every odd chunk width up to the widest basis
  for (int hh = 0; hh < 2; ++hh)
    for (int pl = 0; pl < planes; ++pl) {
      void* gaddr = pl == 0 ? h->ws.Lh : (void*)h->ws.Ll;
      for (int k = 0; k < kMaxMaps; ++k) {
        const int c = 2 * k + 1;
        if (c > maxc) break;
        const cuuint64_t dims[2] = {(cuuint64_t)L.ldg, (cuuint64_t)L.npad};
        const cuuint64_t strides[1] = {(cuuint64_t)L.ldg * esz};
        const cuuint32_t box[2] = {(cuuint32_t)(c * 16 / esz), (cuuint32_t)(hh == 0 ? kTile : kPassARows)};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&h->maps_host[(2 * hh + pl) * kMaxMaps + k], dt, 2, gaddr, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
          char buf[96];
          std::snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for box %d", (int)r, c);
          return fail(h, ODMD_ERR_CUDA, buf);
        }
      }
    }
  return ODMD_OK;
}

odmd_status fail(odmd_t h, odmd_status s, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_err = msg;
  return s;
}

odmd_status cuda_fail(odmd_t h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, ODMD_ERR_CUDA, m);
}

#define CK(h, call, where)                          \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

// Read and clear the device status word (synchronises the stream).
odmd_status device_status(odmd_t h) {
  CK(h, cudaMemcpyAsync(h->pinned + 7, &h->ws.ctl->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
     "status read");
  CK(h, cudaStreamSynchronize(h->stream), "stream sync");
  int st = 0;
  std::memcpy(&st, h->pinned + 7, sizeof(int));
  if (st == 0) return ODMD_OK;
  CK(h, cudaMemsetAsync(&h->ws.ctl->status, 0, sizeof(int), h->stream), "status clear");
  char buf[160];
  std::snprintf(buf, sizeof buf, "device status 0x%x (%s%s%s%s%s%s)", st, (st & DEV_NONFINITE) ? "non-finite " : "",
                (st & DEV_TIMEOUT) ? "timeout " : "", (st & DEV_EIG_NOCONV) ? "eig-no-convergence " : "",
                (st & DEV_EIG_COND) ? "singular-eigenbasis " : "", (st & DEV_SECULAR) ? "secular-no-convergence " : "",
                (st & DEV_NOMODEL) ? "no-model" : "");
  if (st & DEV_TIMEOUT) return fail(h, ODMD_ERR_TIMEOUT, buf);
  if (st & DEV_NOMODEL) return fail(h, ODMD_ERR_STATE, buf);
  return fail(h, ODMD_ERR_NUMERIC, buf);
}

// Bracket a kernel group with events when profiling; count its kernels always.
struct ProfScope {
  odmd_t h;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  bool graph_recorded = false;  // the events are recorded by graph nodes
  ProfScope(odmd_t h_, int cls_, int kernels) : h(h_), cls(cls_) {
    h->launches[cls] += kernels;
    if (!h->prof_on) return;
    a = take();
    b = take();
    if (a && kernels > 0) cudaEventRecord(a, h->stream);
  }
  void defer() { graph_recorded = true; }
  cudaEvent_t take() {
    if (!h->pool.empty()) {
      cudaEvent_t e = h->pool.back();
      h->pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  ~ProfScope() {
    if (!h->prof_on || !a || !b) return;
    if (!graph_recorded) cudaEventRecord(b, h->stream);
    h->pending.push_back({cls, a, b});
  }
};

void prof_collect(odmd_t h) {
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      h->prof_ms[p.cls] += ms;
    if (p.owned) {
      h->pool.push_back(p.a);
      h->pool.push_back(p.b);
    }
  }
  h->pending.clear();
}

// Capture the update sequence for snapshot-buffer parity `par` (the new snapshot goes to
// cbuf[par ^ 1]); with `prof`, event-record nodes bracket the three kernel groups.
odmd_status finish_graph(odmd_t h, odmd_instance::UpdGraph& G, cudaGraph_t graph, bool want_ingest);

odmd_status build_update_graph(odmd_t h, int par, int prof) {
  odmd_instance::UpdGraph& G = h->ug[par][prof];
  if (G.exec) return ODMD_OK;
  cudaEvent_t* ph = G.ph;
  if (prof)
    for (int i = 0; i < 6; ++i) CK(h, cudaEventCreate(&ph[i]), "graph events");
  cudaGraph_t graph = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = launch_ingest(h->ws, h->ws.cbuf[par], h->ws.cbuf[par ^ 1], h->cap);
  if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(ph[0], h->cap, cudaEventRecordExternal);
  if (e == cudaSuccess) e = launch_pass_a(h->ws, h->cap);
  if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(ph[1], h->cap, cudaEventRecordExternal);
  if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(ph[2], h->cap, cudaEventRecordExternal);
  if (e == cudaSuccess) e = launch_small(h->ws, h->cap);
  if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(ph[3], h->cap, cudaEventRecordExternal);
  if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(ph[4], h->cap, cudaEventRecordExternal);
  if (e == cudaSuccess)
    e = (h->use_tc && split_compact_ok(h->ws)) ? launch_split_compact(h->ws, h->sms, h->cap) : launch_pass_b(h->ws, h->cap);
  if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(ph[5], h->cap, cudaEventRecordExternal);
  cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, e, "update graph capture");
  }
  return finish_graph(h, G, graph, true);
}

// Keep a captured graph in G: find its ingest node (the snapshot pointer changes every
// update; want_ingest) and its event nodes, and instantiate it.  The graph is released on
// every way out that does not keep it.
odmd_status finish_graph(odmd_t h, odmd_instance::UpdGraph& G, cudaGraph_t graph, bool want_ingest) {
  cudaEvent_t* ph = G.ph;
  cudaError_t e = cudaSuccess;
  size_t nn = 0;
  e = cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(e == cudaSuccess ? nn : 0);
  if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
  const void* ingest_fn = ingest_kernel(h->ws.prec);
  for (size_t i = 0; e == cudaSuccess && i < nodes.size(); ++i) {
    cudaGraphNode_t nd = nodes[i];
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nd, &t);
    if (e != cudaSuccess) break;
    if (t == cudaGraphNodeTypeKernel) {
      cudaKernelNodeParams kp{};
      e = cudaGraphKernelNodeGetParams(nd, &kp);
      if (e == cudaSuccess && kp.func == ingest_fn) {
        G.ingest = nd;
        G.kp = kp;
      }
    } else if (t == cudaGraphNodeTypeEventRecord) {
      cudaEvent_t ev;
      e = cudaGraphEventRecordNodeGetEvent(nd, &ev);
      for (int k = 0; e == cudaSuccess && k < 6; ++k)
        if (ev == ph[k]) G.ev[k] = nd;
    }
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    G.ingest = nullptr;
    return cuda_fail(h, e, "update graph nodes");
  }
  if (want_ingest && !G.ingest) {
    cudaGraphDestroy(graph);
    return fail(h, ODMD_ERR_CUDA, "update graph: ingest node not found");
  }
  e = cudaGraphInstantiate(&G.exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    G.exec = nullptr;
    return cuda_fail(h, e, "update graph instantiate");
  }
  G.graph = graph;
  G.args[0] = &G.src;
  G.args[1] = &G.dst;
  G.args[2] = &G.n;
  G.kp.kernelParams = G.args;
  G.kp.extra = nullptr;
  return ODMD_OK;
}

// the SVD tail of an update on stream s: k_roots .. k_apply, then the compaction kernel
// (which returns at once unless the update compacts)
cudaError_t launch_update_tail(odmd_t h, cudaStream_t s) {
  cudaError_t e = launch_small_tail(h->ws, s);
  if (e == cudaSuccess)
    e = (h->use_tc && split_compact_ok(h->ws)) ? launch_split_compact(h->ws, h->sms, s) : launch_pass_b(h->ws, s);
  return e;
}

// Capture the pipelined update for state buffer `cur` and snapshot parity `curc` (its new
// snapshot goes to cbuf[curc ^ 1]).  With `tail` the previous update's tail runs on a forked
// branch beside this update's ingest and pass A; that pass A returns at once if the previous
// update compacts and runs again after the join in that case (pass_a_body's gate).
odmd_status build_pipe_graph(odmd_t h, int cur, int curc, int tail) {
  odmd_instance::UpdGraph& G = h->pg[cur][curc][tail];
  if (G.exec) return ODMD_OK;
  if (!h->cap2) {
    CK(h, cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking), "pipeline capture stream");
    CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "pipeline events");
    CK(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "pipeline events");
  }
  const int sel = cur | (curc << 1);
  cudaGraph_t graph = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaSuccess;
  if (tail) {
    e = cudaEventRecord(h->ev_fork, h->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cap2, h->ev_fork, 0);
  }
  if (e == cudaSuccess) e = launch_ingest(h->ws, h->ws.cbuf[curc], h->ws.cbuf[curc ^ 1], h->cap);
  if (e == cudaSuccess) e = launch_pass_a_sel(h->ws, sel | ((tail ? 1 : 0) << 2), h->cap);
  if (tail) {
    if (e == cudaSuccess) e = launch_update_tail(h, h->cap2);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->cap2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cap, h->ev_join, 0);
    if (e == cudaSuccess) e = launch_pass_a_sel(h->ws, sel | (2 << 2), h->cap);
  }
  if (e == cudaSuccess) e = launch_prep(h->ws, h->cap);
  cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, e, "pipelined update graph capture");
  }
  return finish_graph(h, G, graph, true);
}

// Enqueue the tail of the last pipelined update, if it has not run yet; every call that
// reads or changes the model other than an update begins with this.
odmd_status settle(odmd_t h) {
  if (!h->tail_pending) return ODMD_OK;
  odmd_instance::UpdGraph& G = h->tg;
  if (!G.exec) {
    cudaGraph_t graph = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = launch_update_tail(h, h->cap);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(h, e, "update tail graph capture");
    }
    if (odmd_status st = finish_graph(h, G, graph, false)) return st;
  }
  CK(h, cudaGraphLaunch(G.exec, h->stream), "update tail launch");
  h->launches[ODMD_K_SMALL] += 5;  // k_prep_b, k_roots .. k_apply
  h->launches[ODMD_K_PASS_B] += 1;
  h->tail_pending = false;
  return ODMD_OK;
}

// Write the column appended by the last update if the next tall pass has not yet done
// so (the kernel returns at once when nothing is pending).
odmd_status flush_pending(odmd_t h) {
  if (h->nsnap < 2 || !h->maybe_pend) return ODMD_OK;
  ProfScope ps(h, ODMD_K_PASS_B, 1);
  CK(h, launch_flush(h->ws, h->stream), "flush launch");
  h->maybe_pend = false;
  return ODMD_OK;
}

odmd_status ensure_eig(odmd_t h) {
  if (!h->eig_dirty) return ODMD_OK;
  {
    ProfScope ps(h, ODMD_K_EIG, 1);
    CK(h, launch_eig(h->ws, h->stream), "eig launch");
  }
  h->eig_dirty = false;
  return ODMD_OK;
}

// Integer horizons (the common case: states at time steps) take the coefficients from powers
// of the reduced operator, A~^t (S * r_first), which equals V Lambda^t b exactly; any other
// horizon takes them from the eigen-cache.
bool integer_horizons(const double* t, int k) {
  for (int i = 0; i < k; ++i)
    if (!(t[i] == std::floor(t[i])) || t[i] > 1e12) return false;
  return true;
}

odmd_status launch_coefficients(odmd_t h, const double* t, int k, bool by_powers) {
  ProfScope ps(h, ODMD_K_COEF, 1);
  if (by_powers) {
    CK(h, launch_coef_pow(h->ws, t, k, h->stream), "coef launch");
  } else {
    CK(h, launch_coef(h->ws, t, k, h->stream), "coef launch");
  }
  return ODMD_OK;
}

void* base_of(odmd_t h, const Layout&) { return const_cast<CUtensorMap*>(h->ws.maps); }

double join(float2 v) { return (double)v.x + (double)v.y; }

size_t snap_bytes(const odmd_t h) { return (size_t)h->cfg.n * vsz_of(h->cfg.prec); }

}  // namespace

extern "C" {

odmd_status odmd_config_default(odmd_config* cfg, int64_t n, int32_t r_max) {
  if (!cfg) return fail(nullptr, ODMD_ERR_ARG, "config is NULL");
  std::memset(cfg, 0, sizeof *cfg);
  cfg->n = n;
  cfg->r_max = r_max;
  cfg->slack = 16;
  cfg->trunc_tol = 1e-10;
  cfg->check_tol = 1e-5;
  cfg->prec = ODMD_FP64;
  cfg->refine_every = 0;
  cfg->flags = 0;
  return ODMD_OK;
}

odmd_status odmd_footprint(const odmd_config* cfg, size_t* device_bytes) {
  std::string why;
  if (odmd_status s = check_cfg(cfg, why)) return fail(nullptr, s, why);
  if (!device_bytes) return fail(nullptr, ODMD_ERR_ARG, "device_bytes is NULL");
  *device_bytes = make_layout(*cfg).total;
  return ODMD_OK;
}

odmd_status odmd_create(const odmd_config* cfg, void* workspace_dev, size_t bytes, void* stream, odmd_t* out) {
  std::string why;
  if (odmd_status s = check_cfg(cfg, why)) return fail(nullptr, s, why);
  if (!out) return fail(nullptr, ODMD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!workspace_dev) return fail(nullptr, ODMD_ERR_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0)
    return fail(nullptr, ODMD_ERR_ARG, "workspace must be 256-byte aligned");
  const Layout L = make_layout(*cfg);
  if (bytes < L.total) return fail(nullptr, ODMD_ERR_NOMEM, "workspace smaller than odmd_footprint()");
  odmd_instance* h = new (std::nothrow) odmd_instance();
  if (!h) return fail(nullptr, ODMD_ERR_NOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->nsnap = 0;
  h->compactions = 0;
  h->cur_h = 0;
  h->curc_h = 0;
  h->eig_dirty = true;
  h->maybe_pend = true;
  h->prof_on = false;
  for (int i = 0; i < ODMD_K_COUNT; ++i) {
    h->prof_ms[i] = 0.0;
    h->launches[i] = 0;
  }
  h->r0_base[0] = h->r0_base[1] = 0;
  cudaError_t e = cudaGetDevice(&h->device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->pinned), 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::string m = std::string("create: ") + cudaGetErrorString(e);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
    return fail(nullptr, ODMD_ERR_CUDA, m);
  }
  const int64_t ntiles = (cfg->n + kTile - 1) / kTile;
  int gridA = (int)(ntiles < sms ? ntiles : sms);
  if (gridA > kPartRows) gridA = kPartRows;
  if (gridA < 1) gridA = 1;
  carve(h->ws, L, reinterpret_cast<unsigned char*>(workspace_dev), *cfg, gridA);
  h->stage[0] = reinterpret_cast<unsigned char*>(workspace_dev) + L.off_stage[0];
  h->stage[1] = reinterpret_cast<unsigned char*>(workspace_dev) + L.off_stage[1];
  h->wsv = reinterpret_cast<Ws*>(reinterpret_cast<unsigned char*>(workspace_dev) + L.off_wsv);
  {
    static std::atomic<unsigned long long> serials{0};
    h->serial = ++serials;
  }
  {
    h->ws.shards = 1;
    h->ws.gridG = 2 * sms < kGramCtas ? 2 * sms : kGramCtas;
    if (h->ws.gridG < 1) h->ws.gridG = 1;
  }
  if (e == cudaSuccess) e = prepare_tall(h->ws);
  if (e == cudaSuccess) e = prepare_small(h->ws);
  if (e == cudaSuccess) e = prepare_core();
  if (e == cudaSuccess) e = prepare_split(h->ws);
  h->sms = sms;
  h->use_tc = (cfg->flags & ODMD_CUDA_CORES) == 0;
  h->pipe = (cfg->flags & ODMD_NO_PIPELINE) == 0;
  if (e == cudaSuccess && cfg->refine_every > 0) e = prepare_refine();
  if (e == cudaSuccess) e = cudaMemsetAsync(workspace_dev, 0, L.total, h->stream);
  if (e == cudaSuccess) {
    if (encode_maps(h, L) != ODMD_OK) {
      std::string m = h->err;
      cudaFreeHost(h->pinned);
      cudaStreamDestroy(h->cap);
      delete h;
      return fail(nullptr, ODMD_ERR_CUDA, m);
    }
    e = cudaMemcpyAsync(base_of(h, L), h->maps_host.data(), h->maps_host.size() * sizeof(CUtensorMap),
                        cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->wsv, &h->ws, sizeof(Ws), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaFreeHost(h->pinned);
    cudaStreamDestroy(h->cap);
    std::string m = std::string("create: ") + cudaGetErrorString(e);
    delete h;
    return fail(nullptr, ODMD_ERR_CUDA, m);
  }
  *out = h;
  return ODMD_OK;
}

// one update; `may_pipe`: it may leave its tail to the next call (odmd_update).  The
// hybrid loops, which read the model right after every update, run it to its end instead:
// a pipelined update there would only add the settle's launch.
static odmd_status update_impl(odmd_t h, const void* x_dev, bool may_pipe);

odmd_status odmd_update(odmd_t h, const void* x_dev) { return update_impl(h, x_dev, true); }

static odmd_status update_impl(odmd_t h, const void* x_dev, bool may_pipe) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (!x_dev) return fail(h, ODMD_ERR_ARG, "x is NULL");
  if (h->nsnap == 0) {
    CK(h, launch_ingest(h->ws, x_dev, h->ws.cbuf[h->curc_h], h->stream), "copy u0");
    ProfScope ps(h, ODMD_K_FIRST, launches_per_reduction(h->ws));
    CK(h, launch_first(h->ws, h->stream), "first launch");
    h->nsnap = 1;
    return ODMD_OK;
  }
  bool graphed = false;
  if (may_pipe && h->use_graphs && h->pipe && !h->prof_on && h->ws.shards == 1) {
    // pipelined: this update's ingest and pass A beside the last update's tail
    const int tail = h->tail_pending ? 1 : 0;
    if (odmd_status st = build_pipe_graph(h, h->cur_h, h->curc_h, tail)) return st;
    odmd_instance::UpdGraph& G = h->pg[h->cur_h][h->curc_h][tail];
    G.src = x_dev;
    G.dst = h->ws.cbuf[h->curc_h ^ 1];
    G.n = h->cfg.n;
    CK(h, cudaGraphExecKernelNodeSetParams(G.exec, G.ingest, &G.kp), "graph ingest params");
    CK(h, cudaGraphLaunch(G.exec, h->stream), "pipelined update graph launch");
    h->launches[ODMD_K_PASS_A] += 1 + tail;
    h->launches[ODMD_K_SMALL] += 1 + 5 * tail;
    h->launches[ODMD_K_PASS_B] += tail;
    h->tail_pending = true;
    graphed = true;
  } else if (odmd_status st = settle(h)) {
    return st;
  }
  if (!graphed && h->use_graphs) {
    const int par = h->curc_h, prof = h->prof_on ? 1 : 0;
    if (odmd_status st = build_update_graph(h, par, prof)) return st;
    odmd_instance::UpdGraph& G = h->ug[par][prof];
    G.src = x_dev;
    G.dst = h->ws.cbuf[par ^ 1];
    G.n = h->cfg.n;
    CK(h, cudaGraphExecKernelNodeSetParams(G.exec, G.ingest, &G.kp), "graph ingest params");
    bool ok = true;
    if (prof) {
      // point the graph's event nodes at fresh pool events (on failure this update runs
      // through the plain launch path below)
      cudaEvent_t evs[6] = {};
      for (int i = 0; i < 6 && ok; ++i) {
        if (!h->pool.empty()) {
          evs[i] = h->pool.back();
          h->pool.pop_back();
        } else if (cudaEventCreate(&evs[i]) != cudaSuccess) {
          evs[i] = nullptr;
        }
        if (!evs[i] || !G.ev[i] ||
            cudaGraphExecEventRecordNodeSetEvent(G.exec, G.ev[i], evs[i]) != cudaSuccess)
          ok = false;
      }
      cudaGetLastError();
      if (ok) {
        h->pending.push_back({ODMD_K_PASS_A, evs[0], evs[1]});
        h->pending.push_back({ODMD_K_SMALL, evs[2], evs[3]});
        h->pending.push_back({ODMD_K_PASS_B, evs[4], evs[5]});
        // the empty intervals between the groups: the graph's own timing overhead
        h->pending.push_back({ODMD_K_GAP, evs[1], evs[2], false});
        h->pending.push_back({ODMD_K_GAP, evs[3], evs[4], false});
      } else {
        for (cudaEvent_t ev : evs)
          if (ev) h->pool.push_back(ev);
      }
    }
    if (ok) {
      CK(h, cudaGraphLaunch(G.exec, h->stream), "update graph launch");
      h->launches[ODMD_K_PASS_A] += launches_per_reduction(h->ws);
      h->launches[ODMD_K_SMALL] += 5;
      h->launches[ODMD_K_PASS_B] += 1;
      graphed = true;
    }
  }
  if (!graphed) {
    CK(h, launch_ingest(h->ws, x_dev, h->ws.cbuf[h->curc_h ^ 1], h->stream), "copy x");
    {
      ProfScope ps(h, ODMD_K_PASS_A, launches_per_reduction(h->ws));
      CK(h, launch_pass_a(h->ws, h->stream), "pass A launch");
    }
    {
      ProfScope ps(h, ODMD_K_SMALL, 5);
      CK(h, launch_small(h->ws, h->stream), "small solve launch");
    }
    {
      ProfScope ps(h, ODMD_K_PASS_B, 1);
      CK(h, (h->use_tc && split_compact_ok(h->ws)) ? launch_split_compact(h->ws, h->sms, h->stream)
                                                    : launch_pass_b(h->ws, h->stream),
         "pass B launch");
    }
  }
  h->cur_h ^= 1;
  h->curc_h ^= 1;
  h->nsnap += 1;
  h->eig_dirty = true;
  h->maybe_pend = true;
  // periodic orthogonality refinement, every refine_every snapshot pairs
  if (h->cfg.refine_every > 0 && (h->nsnap - 1) % h->cfg.refine_every == 0) return odmd_refine(h);
  return ODMD_OK;
}

odmd_status odmd_predict(odmd_t h, const double* t_host, int32_t k, void* out_dev, int64_t ld) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (k < 0 || (k > 0 && (!t_host || !out_dev))) return fail(h, ODMD_ERR_ARG, "bad t/out/k");
  if (ld < h->cfg.n) return fail(h, ODMD_ERR_ARG, "ld < n");
  if (h->nsnap < 2) return fail(h, ODMD_ERR_STATE, "predict needs two snapshots");
  for (int i = 0; i < k; ++i)
    if (!(t_host[i] >= 0.0) || !std::isfinite(t_host[i])) return fail(h, ODMD_ERR_ARG, "t must be finite and >= 0");
  const bool by_powers = integer_horizons(t_host, k);
  if (!by_powers)
    if (odmd_status s = ensure_eig(h)) return s;
  // the tensor-core rollout forms a pending basis column itself; the other form reads L0
  // as it is, so the column is written first
  const bool tc_first = k > 0 && h->use_tc && split_rollout_ok(h->ws, k < kRollK ? k : kRollK);
  if (!tc_first) {
    if (odmd_status s = flush_pending(h)) return s;
  } else {
    h->maybe_pend = false;  // the first launch below writes the column
  }
  const size_t vs = (size_t)vsz_of(h->cfg.prec);
  for (int j0 = 0; j0 < k; j0 += kRollK) {
    const int kk = (k - j0) < kRollK ? (k - j0) : kRollK;
    if (odmd_status s = launch_coefficients(h, t_host + j0, kk, by_powers)) return s;
    ProfScope ps(h, ODMD_K_ROLLOUT, 1);
    unsigned char* o = static_cast<unsigned char*>(out_dev) + (size_t)j0 * ld * vs;
    if (h->use_tc && split_rollout_ok(h->ws, kk)) {
      // eight or more states: the contraction on the tensor cores (split.cu)
      CK(h, launch_split_rollout(h->ws, kk, reinterpret_cast<double*>(o), ld, h->sms, h->stream), "rollout launch");
    } else {
      CK(h, launch_rollout(h->ws, nullptr, kk, o, ld, 0, h->stream), "rollout launch");
    }
  }
  return ODMD_OK;
}

odmd_status odmd_check(odmd_t h, double t, const void* x_fom_dev, double tol, double* rel_err, int32_t* pass) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!x_fom_dev) return fail(h, ODMD_ERR_ARG, "x_fom is NULL");
  if (!(t >= 0.0) || !std::isfinite(t)) return fail(h, ODMD_ERR_ARG, "t must be finite and >= 0");
  if (h->nsnap < 2) return fail(h, ODMD_ERR_STATE, "check needs two snapshots");
  if (tol <= 0.0) tol = h->cfg.check_tol;
  CK(h, launch_ingest(h->ws, x_fom_dev, h->ws.xbuf, h->stream), "copy x_fom");
  const bool by_powers = integer_horizons(&t, 1);
  if (!by_powers)
    if (odmd_status s = ensure_eig(h)) return s;
  if (odmd_status s = launch_coefficients(h, &t, 1, by_powers)) return s;
  if (odmd_status s = flush_pending(h)) return s;
  {
    ProfScope ps(h, ODMD_K_CHECK, launches_per_reduction(h->ws));
    CK(h, launch_check(h->ws, h->stream), "check launch");
  }
  CK(h, cudaMemcpyAsync(h->pinned, h->ws.out2, 2 * sizeof(float2), cudaMemcpyDeviceToHost, h->stream), "read back");
  if (odmd_status s = device_status(h)) return s;
  float2 nd[2];
  std::memcpy(nd, h->pinned, sizeof nd);
  const double num = join(nd[0]), den = join(nd[1]);
  double err;
  if (den == 0.0)
    err = num == 0.0 ? 0.0 : INFINITY;
  else
    err = std::sqrt(num / den);
  if (rel_err) *rel_err = err;
  if (pass) *pass = err <= tol ? 1 : 0;
  return ODMD_OK;
}

odmd_status odmd_refine(odmd_t h) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!h->ws.gpart) return fail(h, ODMD_ERR_STATE, "refinement scratch not reserved: create with refine_every > 0");
  if (h->nsnap < 2) return ODMD_OK;  // no basis yet
  if (odmd_status s = flush_pending(h)) return s;
  {
    ProfScope ps(h, ODMD_K_REFINE, 5);
    CK(h, launch_refine(h->ws, h->cur_h, h->stream), "refine launch");
  }
  h->cur_h ^= 1;
  h->eig_dirty = true;
  h->maybe_pend = true;
  return ODMD_OK;
}

// ---- checkpoint / resume
// A checkpoint is a header followed by the raw bytes of every part of the workspace that
// survives from one call to the next: the control block, the two committed-state buffers
// with the small and eigen scratch after them, the rows 0..n-1 of the tall factor L0
// (each plane), both snapshot slots and the stored residual.  The tensor maps (they hold
// device addresses) and the per-call scratch are not saved.  A checkpoint loads into any
// handle created with the same n, r_max, precision and slack on a device of the same
// kind; the resumed model then continues bit for bit as the saved one would have.
namespace {
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int64_t n;
  int32_t r_max, prec, slack, cap, ldg, ctl_bytes;
  int64_t nsnap;
  int32_t cur_h, curc_h;
  uint64_t region[6];  // bytes: control block, state block, L0 hi rows, L0 lo rows, snapshots, residual
  uint64_t checksum;   // FNV-1a (8-byte words) over this header (checksum field zero), then the regions
};
// version 2: the small state (S, rows of R, M) is FP64 and the header is covered by the checksum
constexpr uint32_t kCkptVersion = 2;
constexpr char kCkptMagic[8] = {'O', 'D', 'M', 'D', 'C', 'K', 'P', '1'};

struct CkptRegion {
  size_t off, bytes;
};

void ckpt_regions(const odmd_t h, CkptRegion out[7]) {
  const Layout L = make_layout(h->cfg);
  const size_t n = (size_t)h->cfg.n;
  const size_t row = (size_t)L.ldg * esz_of(h->cfg.prec);
  const size_t snap = n * vsz_of(h->cfg.prec);
  out[0] = {L.off_ctl, sizeof(Ctl)};
  out[1] = {L.off_hdr[0], L.off_part - L.off_hdr[0]};
  out[2] = {L.off_Lh, n * row};
  out[3] = {L.off_Ll, h->cfg.prec == ODMD_FP64 ? n * row : 0};
  out[4] = {L.off_c[0], snap};
  out[5] = {L.off_c[1], snap};
  out[6] = {L.off_e, n * sizeof(float2)};
}

// FNV-1a over 8-byte little-endian words (then the tail bytes)
uint64_t fnv1a(uint64_t hsh, const unsigned char* p, size_t bytes) {
  size_t i = 0;
  for (; i + 8 <= bytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    hsh ^= w;
    hsh *= 1099511628211ull;
  }
  for (; i < bytes; ++i) {
    hsh ^= p[i];
    hsh *= 1099511628211ull;
  }
  return hsh;
}

size_t ckpt_bytes(const odmd_t h) {
  CkptRegion R[7];
  ckpt_regions(h, R);
  size_t b = sizeof(CkptHeader);
  for (const CkptRegion& r : R) b += r.bytes;
  return b;
}
}  // namespace

odmd_status odmd_checkpoint_size(odmd_t h, size_t* bytes) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (!bytes) return fail(h, ODMD_ERR_ARG, "bytes must not be NULL");
  *bytes = ckpt_bytes(h);
  return ODMD_OK;
}

odmd_status odmd_save(odmd_t h, void* host_buf, size_t bytes) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!host_buf) return fail(h, ODMD_ERR_ARG, "host buffer must not be NULL");
  const size_t need = ckpt_bytes(h);
  if (bytes < need) return fail(h, ODMD_ERR_ARG, "checkpoint buffer of " + std::to_string(bytes) +
                                                   " bytes is smaller than the " + std::to_string(need) + " needed");
  CK(h, cudaStreamSynchronize(h->stream), "save: sync");
  CkptRegion R[7];
  ckpt_regions(h, R);
  const Layout L = make_layout(h->cfg);
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.header_bytes = sizeof(CkptHeader);
  hd.n = h->cfg.n;
  hd.r_max = h->cfg.r_max;
  hd.prec = h->cfg.prec;
  hd.slack = h->cfg.slack;
  hd.cap = L.cap;
  hd.ldg = L.ldg;
  hd.ctl_bytes = (int32_t)sizeof(Ctl);
  hd.nsnap = h->nsnap;
  hd.cur_h = h->cur_h;
  hd.curc_h = h->curc_h;
  hd.region[0] = R[0].bytes;
  hd.region[1] = R[1].bytes;
  hd.region[2] = R[2].bytes;
  hd.region[3] = R[3].bytes;
  hd.region[4] = R[4].bytes + R[5].bytes;
  hd.region[5] = R[6].bytes;
  unsigned char* out = static_cast<unsigned char*>(host_buf) + sizeof(CkptHeader);
  const unsigned char* base = reinterpret_cast<const unsigned char*>(h->ws.ctl) - L.off_ctl;  // workspace start
  hd.checksum = 0;
  uint64_t hsh = fnv1a(1469598103934665603ull, reinterpret_cast<const unsigned char*>(&hd), sizeof hd);
  for (const CkptRegion& r : R) {
    if (r.bytes) CK(h, cudaMemcpy(out, base + r.off, r.bytes, cudaMemcpyDeviceToHost), "save: copy");
    hsh = fnv1a(hsh, out, r.bytes);
    out += r.bytes;
  }
  hd.checksum = hsh;
  std::memcpy(host_buf, &hd, sizeof hd);
  return ODMD_OK;
}

odmd_status odmd_load(odmd_t h, const void* host_buf, size_t bytes) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!host_buf) return fail(h, ODMD_ERR_ARG, "host buffer must not be NULL");
  if (bytes < sizeof(CkptHeader)) return fail(h, ODMD_ERR_ARG, "checkpoint shorter than its header");
  CkptHeader hd;
  std::memcpy(&hd, host_buf, sizeof hd);
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion || hd.header_bytes != sizeof(CkptHeader))
    return fail(h, ODMD_ERR_ARG, "not a checkpoint of this library version");
  // the scalars that select buffers are checked before anything else uses them
  if ((hd.cur_h != 0 && hd.cur_h != 1) || (hd.curc_h != 0 && hd.curc_h != 1) || hd.nsnap < 0)
    return fail(h, ODMD_ERR_ARG, "checkpoint header out of range (buffer indices or snapshot count)");
  const Layout L = make_layout(h->cfg);
  if (hd.n != h->cfg.n || hd.r_max != h->cfg.r_max || hd.prec != h->cfg.prec || hd.slack != h->cfg.slack ||
      hd.cap != L.cap || hd.ldg != L.ldg || hd.ctl_bytes != (int32_t)sizeof(Ctl))
    return fail(h, ODMD_ERR_ARG, "checkpoint of a different configuration (n, r_max, precision or slack)");
  if (bytes < ckpt_bytes(h)) return fail(h, ODMD_ERR_ARG, "checkpoint truncated");
  CkptRegion R[7];
  ckpt_regions(h, R);
  if (hd.region[0] != R[0].bytes || hd.region[1] != R[1].bytes || hd.region[2] != R[2].bytes ||
      hd.region[3] != R[3].bytes || hd.region[4] != R[4].bytes + R[5].bytes || hd.region[5] != R[6].bytes)
    return fail(h, ODMD_ERR_ARG, "checkpoint regions do not match this handle's layout");
  const unsigned char* in = static_cast<const unsigned char*>(host_buf) + sizeof(CkptHeader);
  CkptHeader hz = hd;
  hz.checksum = 0;
  uint64_t hsh = fnv1a(1469598103934665603ull, reinterpret_cast<const unsigned char*>(&hz), sizeof hz);
  {
    const unsigned char* p = in;
    for (const CkptRegion& r : R) {
      hsh = fnv1a(hsh, p, r.bytes);
      p += r.bytes;
    }
  }
  if (hsh != hd.checksum) return fail(h, ODMD_ERR_ARG, "checkpoint checksum mismatch (corrupted data)");
  {
    Ctl saved;
    std::memcpy(&saved, in, sizeof saved);  // region 0 is the control block
    if (saved.cur != hd.cur_h || saved.cur_c != hd.curc_h)
      return fail(h, ODMD_ERR_ARG, "checkpoint control block disagrees with its header");
  }
  CK(h, cudaStreamSynchronize(h->stream), "load: sync");
  unsigned char* base = reinterpret_cast<unsigned char*>(h->ws.ctl) - L.off_ctl;
  for (const CkptRegion& r : R) {
    if (r.bytes) CK(h, cudaMemcpy(base + r.off, in, r.bytes, cudaMemcpyHostToDevice), "load: copy");
    in += r.bytes;
  }
  h->nsnap = hd.nsnap;
  h->cur_h = hd.cur_h;
  h->curc_h = hd.curc_h;
  h->eig_dirty = true;
  h->maybe_pend = true;
  return ODMD_OK;
}

odmd_status odmd_hybrid_step(odmd_t h, const void* x_fom_dev, double tol, void* state_out_dev, int32_t* accepted,
                             double* rel_err) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!x_fom_dev || !state_out_dev) return fail(h, ODMD_ERR_ARG, "x_fom and state_out must not be NULL");
  if (state_out_dev == x_fom_dev) return fail(h, ODMD_ERR_ARG, "state_out must not alias x_fom");
  int32_t acc = 0;
  double err = INFINITY;
  const double t = (double)h->nsnap;  // the step about to be taken, counted from u^0
  if (h->nsnap >= 2) {
    odmd_status s = odmd_check(h, t, x_fom_dev, tol, &err, &acc);
    if (s == ODMD_ERR_STATE) {  // no model yet (every snapshot so far was zero): the FOM decides
      acc = 0;
      err = INFINITY;
    } else if (s != ODMD_OK) {
      return s;
    }
  }
  if (acc) {
    if (odmd_status s = odmd_predict(h, &t, 1, state_out_dev, h->cfg.n)) return s;
  } else {
    CK(h, cudaMemcpyAsync(state_out_dev, x_fom_dev, snap_bytes(h), cudaMemcpyDeviceToDevice, h->stream),
       "copy the FOM state");
  }
  // the state taken, accepted prediction or FOM state, joins the snapshot stream
  if (odmd_status s = update_impl(h, state_out_dev, false)) return s;
  if (accepted) *accepted = acc;
  if (rel_err) *rel_err = err;
  return ODMD_OK;
}

static odmd_status read_hdr(odmd_t h, StateHdr* hdr);

odmd_status odmd_hybrid_step_residual(odmd_t h, odmd_residual_fn residual, odmd_fom_fn fom, void* user, double tol,
                                      void* state_out_dev, void* r_dev, void* b_dev, int32_t* accepted,
                                      double* rel_res) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!residual || !fom) return fail(h, ODMD_ERR_ARG, "the residual and FOM callbacks must not be NULL");
  if (!state_out_dev || !r_dev || !b_dev) return fail(h, ODMD_ERR_ARG, "state_out, r and b must not be NULL");
  if (state_out_dev == r_dev || state_out_dev == b_dev || r_dev == b_dev)
    return fail(h, ODMD_ERR_ARG, "state_out, r and b must be three different buffers");
  if (tol <= 0.0) tol = h->cfg.check_tol;
  const int64_t step = h->nsnap;  // the step about to be taken, counted from u^0
  int32_t acc = 0;
  double rel = INFINITY;
  StateHdr hdr{};
  if (h->nsnap >= 2)
    if (odmd_status s = read_hdr(h, &hdr)) return s;
  if (h->nsnap >= 2 && hdr.r > 0) {  // (rank 0: no model yet, every snapshot so far was zero)
    const double t = (double)step;
    if (odmd_status s = odmd_predict(h, &t, 1, state_out_dev, h->cfg.n)) return s;
    if (residual(user, step, state_out_dev, r_dev, b_dev, h->stream) != 0)
      return fail(h, ODMD_ERR_STATE, "residual callback reported a failure");
    CK(h, launch_norm_ratio(h->ws, r_dev, b_dev, h->stream), "residual norm launch");
    CK(h, cudaMemcpyAsync(h->pinned, h->ws.out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
       "read back");
    if (odmd_status s = device_status(h)) return s;
    const double num = h->pinned[0], den = h->pinned[1];
    rel = den > 0.0 ? std::sqrt(num / den) : (num == 0.0 ? 0.0 : INFINITY);
    acc = rel <= tol ? 1 : 0;
  }
  if (!acc && fom(user, step, state_out_dev, h->stream) != 0)
    return fail(h, ODMD_ERR_STATE, "FOM callback reported a failure");
  // the state taken, accepted prediction or FOM state, joins the snapshot stream
  if (odmd_status s = update_impl(h, state_out_dev, false)) return s;
  if (accepted) *accepted = acc;
  if (rel_res) *rel_res = rel;
  return ODMD_OK;
}

namespace {
// DMD eigenvalues of the modes that carry the field (amplitude >= 1e-6 of the largest, the
// threshold below which parity of noise-subspace modes is not asked), host copies
odmd_status strong_eigs(odmd_t h, std::vector<double>& re, std::vector<double>& im, int32_t* rank) {
  double lr[kMaxR], li[kMaxR], am[kMaxR];
  if (odmd_status s = odmd_get_eigs(h, lr, li, am, kMaxR, rank)) return s;
  double amax = 0.0;
  for (int i = 0; i < *rank; ++i) amax = am[i] > amax ? am[i] : amax;
  re.clear();
  im.clear();
  for (int i = 0; i < *rank; ++i)
    if (am[i] >= 1e-6 * amax) {
      re.push_back(lr[i]);
      im.push_back(li[i]);
    }
  return ODMD_OK;
}

// largest distance from an eigenvalue of one set to the nearest of the other (both ways)
double eig_shift(const std::vector<double>& ar, const std::vector<double>& ai, const std::vector<double>& br,
                 const std::vector<double>& bi) {
  double worst = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    const auto& xr = pass ? br : ar;
    const auto& xi = pass ? bi : ai;
    const auto& yr = pass ? ar : br;
    const auto& yi = pass ? ai : bi;
    for (size_t i = 0; i < xr.size(); ++i) {
      double best = INFINITY;
      for (size_t j = 0; j < yr.size(); ++j) best = std::fmin(best, std::hypot(xr[i] - yr[j], xi[i] - yi[j]));
      worst = std::fmax(worst, best);
    }
  }
  return worst;
}
}  // namespace

odmd_status odmd_hybrid_run(odmd_t h, odmd_residual_fn residual, odmd_fom_fn fom, void* user, double tol,
                            int64_t t_final, int32_t check_every, int32_t conv_checks, double conv_tol,
                            void* state_out_dev, void* prev_dev, void* r_dev, void* b_dev, odmd_run_report* report) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (!prev_dev || prev_dev == state_out_dev || prev_dev == r_dev || prev_dev == b_dev)
    return fail(h, ODMD_ERR_ARG, "prev must be a buffer of its own");
  if (t_final < h->nsnap) return fail(h, ODMD_ERR_ARG, "t_final lies before the next step");
  if (check_every < 1 || conv_checks < 1 || !(conv_tol > 0.0))
    return fail(h, ODMD_ERR_ARG, "check_every and conv_checks must be >= 1 and conv_tol > 0");
  odmd_run_report rep{};
  rep.converged_at = -1;
  std::vector<double> pre, pim, cre, cim;
  int32_t prank = -1, streak = 0;
  while (h->nsnap <= t_final) {
    const int64_t t = h->nsnap;
    int32_t acc = 0;
    if (odmd_status s = odmd_hybrid_step_residual(h, residual, fom, user, tol, state_out_dev, r_dev, b_dev, &acc,
                                                  nullptr))
      return s;
    ++rep.steps;
    rep.accepted += acc;
    rep.fom_calls += acc ? 0 : 1;
    if (t == t_final) break;
    // the callbacks of the next step see the state taken at this one
    CK(h, cudaMemcpyAsync(prev_dev, state_out_dev, snap_bytes(h), cudaMemcpyDeviceToDevice, h->stream),
       "copy the state taken");
    if (t % check_every != 0 || h->nsnap < 2) continue;
    // convergence (reading of Sec. 2.1, whose criterion is not given): conv_checks consecutive
    // checks with the rank unchanged and no strong eigenvalue moved by more than conv_tol
    int32_t rank = 0;
    odmd_status s = strong_eigs(h, cre, cim, &rank);
    if (s == ODMD_ERR_STATE || s == ODMD_ERR_NUMERIC) {
      // no model yet, or an eigensolve that did not converge or met an ill-conditioned
      // eigenbasis: not converged at this check; the run goes on
      prank = -1;
      streak = 0;
      continue;
    }
    if (s) return s;
    const bool same = rank == prank && cre.size() == pre.size() && eig_shift(cre, cim, pre, pim) <= conv_tol;
    streak = same ? streak + 1 : 0;
    pre.swap(cre);
    pim.swap(cim);
    prank = rank;
    if (streak >= conv_checks) {
      const double tf = (double)t_final;
      if (odmd_status s2 = odmd_predict(h, &tf, 1, state_out_dev, h->cfg.n)) return s2;
      rep.converged = 1;
      rep.converged_at = t;
      rep.skipped = t_final - t;
      break;
    }
  }
  if (report) *report = rep;
  return ODMD_OK;
}

odmd_status odmd_update_host(odmd_t h, const void* host, int64_t count, int64_t ld) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (count < 0 || (count > 0 && !host)) return fail(h, ODMD_ERR_ARG, "bad host buffer or count");
  if (ld < h->cfg.n) return fail(h, ODMD_ERR_ARG, "ld < n");
  if (!h->copy) {
    CK(h, cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking), "copy stream");
    for (int b = 0; b < 2; ++b) {
      CK(h, cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming), "staging events");
      CK(h, cudaEventCreateWithFlags(&h->ev_used[b], cudaEventDisableTiming), "staging events");
    }
  }
  const size_t esz = (size_t)vsz_of(h->cfg.prec), bytes = (size_t)h->cfg.n * esz;
  const unsigned char* src = static_cast<const unsigned char*>(host);
  for (int64_t k = 0; k < count; ++k) {
    const int b = h->stage_next;
    if (h->stage_used[b]) CK(h, cudaStreamWaitEvent(h->copy, h->ev_used[b], 0), "wait for the slot");
    CK(h, cudaMemcpyAsync(h->stage[b], src + (size_t)k * (size_t)ld * esz, bytes, cudaMemcpyHostToDevice, h->copy),
       "host copy");
    CK(h, cudaEventRecord(h->ev_copied[b], h->copy), "record copy");
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0), "wait for the copy");
    if (odmd_status s = odmd_update(h, h->stage[b])) return s;
    CK(h, cudaEventRecord(h->ev_used[b], h->stream), "record use");
    h->stage_used[b] = true;
    h->stage_next ^= 1;
  }
  return ODMD_OK;
}

// ---------------------------------------------------------------- multi-instance updates
// odmd_update_batch runs the update of many instances as one launch per step: ingest (kernel
// parameters carry the snapshot pointers), then a CUDA graph of pass A, the five small-solve
// kernels and the compaction, each a single launch over every instance of the batch (each
// CTA finds its instance and its place in that instance's own grid; instance i's work is
// exactly that of its own update, so the results are bitwise those of odmd_update).  The
// graph is captured once per set of handles and kept in a plan; plans are dropped when one
// of their handles is destroyed or changes its row shards.
namespace {
// one multi-instance launch sequence over a subset of a batch, on its own stream
struct SubPlan {
  std::vector<odmd_t> hs;
  int prec = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
// A batch (a set of handles) as S sub-batches balanced by rows, each a graph on its own
// stream, so that one sub-batch's latency-bound small solves overlap another's tall passes.
// The split S is picked by timing: the first calls of a plan try each candidate on the
// caller's own updates (the results do not depend on S), then the fastest is kept.
struct BatchPlan {
  std::vector<unsigned long long> serials;  // the instances, in call order
  std::vector<odmd_t> hs;
  std::vector<int> cand;                    // candidate splits S
  std::vector<std::vector<SubPlan*>> subs;  // per candidate, built on first use
  std::vector<float> best_ms;               // per candidate, best step time seen
  int tried = 0;                            // tuning calls made so far
  int chosen = -1;                          // index into cand once tuning is done
  cudaStream_t lead = nullptr;              // orders the sub-batches and times a step
  cudaEvent_t t0 = nullptr, t1 = nullptr, joined = nullptr;
};
constexpr int kTuneRounds = 2;  // timed calls per candidate
std::mutex g_plans_mu;
std::vector<BatchPlan*> g_plans;

void free_sub(SubPlan* p) {
  if (p->s) cudaStreamSynchronize(p->s);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->done) cudaEventDestroy(p->done);
  if (p->s) cudaStreamDestroy(p->s);
  delete p;
}
void free_plan(BatchPlan* p) {
  for (auto& v : p->subs)
    for (SubPlan* q : v) free_sub(q);
  if (p->lead) cudaStreamSynchronize(p->lead);
  for (cudaEvent_t e : {p->t0, p->t1, p->joined})
    if (e) cudaEventDestroy(e);
  if (p->lead) cudaStreamDestroy(p->lead);
  delete p;
}

// the compaction of an instance on the tensor cores (else the CUDA-core pass B)
bool split_compaction(odmd_t h) { return h->use_tc && split_compact_ok(h->ws); }

// an update of h can join a multi-instance launch
bool batchable(odmd_t h, int device) {
  return h->use_graphs && h->ws.shards == 1 && h->nsnap >= 1 && !h->prof_on && h->device == device;
}

BatchTab tab_of(const std::vector<odmd_t>& hs, const std::vector<int>& per) {
  BatchTab t{};
  int f = 0;
  for (size_t i = 0; i < hs.size(); ++i) {
    t.ws[i] = hs[i]->wsv;
    t.first[i] = f;
    f += per[i];
  }
  t.first[hs.size()] = f;
  t.ninst = (int)hs.size();
  return t;
}

odmd_status build_sub(const std::vector<odmd_t>& hs, SubPlan** out) {
  odmd_t h0 = hs[0];
  SubPlan* p = new SubPlan;
  p->hs = hs;
  p->prec = h0->ws.prec;
  const bool split = split_compaction(h0);
  const size_t n = hs.size();
  // the small solves' CTAs per instance are bounded by its own r_max (roots and columns of
  // a core of order r + 1 <= r_max + 1; k_zhat's ordering CTA is its last)
  std::vector<int> pa(n), pc(n), one(n, 1), root(n), zhat(n);
  int sa = 0, sb = 0, sp = 0;
  for (size_t i = 0; i < n; ++i) {
    const Ws& w = hs[i]->ws;
    pa[i] = w.gridA;
    pc[i] = split ? split_grid_of(w, hs[i]->sms) : w.gridA;
    root[i] = w.rmax + 1;
    zhat[i] = w.rmax + 2;
    sa = std::max(sa, pass_a_smem(w.prec, w.cap));
    sb = std::max(sb, pass_b_smem(w.prec, w.cap));
    sp = std::max(sp, prep_smem_of(w.cap));
  }
  cudaError_t e = prepare_tall_batch();
  if (e == cudaSuccess) e = prepare_core_batch();
  if (e == cudaSuccess) e = prepare_split_batch();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = launch_pass_a_batch(tab_of(hs, pa), p->prec, sa, p->s);
    if (e == cudaSuccess) e = launch_small_batch(tab_of(hs, one), tab_of(hs, root), tab_of(hs, zhat), sp, p->s);
    if (e == cudaSuccess)
      e = split ? launch_split_compact_batch(tab_of(hs, pc), p->prec, p->s) : launch_pass_b_batch(tab_of(hs, pc), p->prec, sb, p->s);
    const cudaError_t e2 = cudaStreamEndCapture(p->s, &p->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (e != cudaSuccess) {
    free_sub(p);
    return fail(nullptr, ODMD_ERR_CUDA, std::string("update_batch: plan: ") + cudaGetErrorString(e));
  }
  *out = p;
  return ODMD_OK;
}

// S sub-batches balanced by rows: instances in decreasing n, each to the lightest sub-batch
odmd_status build_split(const std::vector<odmd_t>& hs, int S, std::vector<SubPlan*>& out) {
  std::vector<int> order(hs.size());
  for (size_t i = 0; i < hs.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->cfg.n > hs[b]->cfg.n; });
  std::vector<std::vector<odmd_t>> parts(S);
  std::vector<int64_t> load(S, 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    parts[k].push_back(hs[i]);
    load[k] += hs[i]->cfg.n;
  }
  for (auto& part : parts) {
    if (part.empty()) continue;
    SubPlan* q = nullptr;
    if (odmd_status st = build_sub(part, &q)) return st;
    out.push_back(q);
  }
  return ODMD_OK;
}

BatchPlan* find_plan(const std::vector<odmd_t>& hs) {
  for (BatchPlan* p : g_plans) {
    if (p->serials.size() != hs.size()) continue;
    bool same = true;
    for (size_t i = 0; i < hs.size() && same; ++i) same = p->serials[i] == hs[i]->serial && p->hs[i] == hs[i];
    if (same) return p;
  }
  return nullptr;
}

odmd_status new_plan(const std::vector<odmd_t>& hs, BatchPlan** out) {
  BatchPlan* p = new BatchPlan;
  p->hs = hs;
  for (odmd_t h : hs) p->serials.push_back(h->serial);
  for (int S : {1, 2, 4, 8})
    if (S == 1 || (size_t)S * 2 <= hs.size()) p->cand.push_back(S);
  p->subs.resize(p->cand.size());
  p->best_ms.assign(p->cand.size(), 1e30f);
  cudaError_t e = cudaStreamCreateWithFlags(&p->lead, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&p->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&p->t1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->joined, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_plan(p);
    return fail(nullptr, ODMD_ERR_CUDA, std::string("update_batch: plan: ") + cudaGetErrorString(e));
  }
  *out = p;
  return ODMD_OK;
}

// one multi-instance update of hs (all batchable, one precision and compaction kind)
odmd_status run_batch(const std::vector<odmd_t>& hs, const std::vector<const void*>& xs) {
  BatchPlan* p = nullptr;
  std::lock_guard<std::mutex> lk(g_plans_mu);
  p = find_plan(hs);
  if (!p) {
    if (odmd_status st = new_plan(hs, &p)) return st;
    g_plans.push_back(p);
  }
  const bool tuning = p->chosen < 0;
  const int ci = tuning ? p->tried % (int)p->cand.size() : p->chosen;
  if (p->subs[ci].empty())
    if (odmd_status st = build_split(hs, p->cand[ci], p->subs[ci])) return st;
  odmd_t h0 = hs[0];
  // the lead stream waits for each instance's earlier work; the sub-batches wait for it
  for (odmd_t h : hs) {
    if (!h->ev_batch) CK(h, cudaEventCreateWithFlags(&h->ev_batch, cudaEventDisableTiming), "batch event");
    CK(h, cudaEventRecord(h->ev_batch, h->stream), "batch order");
    CK(h, cudaStreamWaitEvent(p->lead, h->ev_batch, 0), "batch order");
  }
  CK(h0, cudaEventRecord(p->t0, p->lead), "batch order");
  for (SubPlan* q : p->subs[ci]) {
    CK(h0, cudaStreamWaitEvent(q->s, p->t0, 0), "batch order");
    IngestTab it{};
    int64_t f = 0;
    for (size_t i = 0; i < q->hs.size(); ++i) {
      odmd_t h = q->hs[i];
      const size_t k = (size_t)(std::find(hs.begin(), hs.end(), h) - hs.begin());
      it.src[i] = xs[k];
      it.dst[i] = h->ws.cbuf[h->curc_h ^ 1];
      it.n[i] = h->cfg.n;
      it.first[i] = f;
      f += (h->cfg.n + 1) / 2;
    }
    it.first[q->hs.size()] = f;
    it.ninst = (int)q->hs.size();
    CK(h0, launch_ingest_batch(it, q->prec, q->s), "batch ingest");
    CK(h0, cudaGraphLaunch(q->exec, q->s), "batch graph launch");
    CK(h0, cudaEventRecord(q->done, q->s), "batch order");
    CK(h0, cudaStreamWaitEvent(p->lead, q->done, 0), "batch order");
  }
  CK(h0, cudaEventRecord(p->t1, p->lead), "batch order");
  for (odmd_t h : hs) {
    CK(h, cudaStreamWaitEvent(h->stream, p->t1, 0), "batch order");
    h->launches[ODMD_K_PASS_A] += 1;
    h->launches[ODMD_K_SMALL] += 5;
    h->launches[ODMD_K_PASS_B] += 1;
    h->cur_h ^= 1;
    h->curc_h ^= 1;
    h->nsnap += 1;
    h->eig_dirty = true;
    h->maybe_pend = true;
  }
  if (tuning) {
    // the tuning calls wait for their own step to time it (the first calls of a plan only)
    CK(h0, cudaEventSynchronize(p->t1), "batch tuning");
    float ms = 0.f;
    CK(h0, cudaEventElapsedTime(&ms, p->t0, p->t1), "batch tuning");
    p->best_ms[ci] = std::min(p->best_ms[ci], ms);
    if (++p->tried >= kTuneRounds * (int)p->cand.size()) {
      p->chosen = (int)(std::min_element(p->best_ms.begin(), p->best_ms.end()) - p->best_ms.begin());
      for (size_t c = 0; c < p->subs.size(); ++c)  // the other splits' graphs are not needed
        if ((int)c != p->chosen) {
          for (SubPlan* q : p->subs[c]) free_sub(q);
          p->subs[c].clear();
        }
    }
  }
  for (odmd_t h : hs)
    if (h->cfg.refine_every > 0 && (h->nsnap - 1) % h->cfg.refine_every == 0)
      if (odmd_status st = odmd_refine(h)) return st;
  return ODMD_OK;
}
}  // namespace

odmd_status odmd_get_batch_split(odmd_t* hs, int32_t count, int32_t* split) {
  if (count < 0 || !split || (count > 0 && !hs)) return fail(nullptr, ODMD_ERR_ARG, "get_batch_split: bad arguments");
  std::lock_guard<std::mutex> lk(g_plans_mu);
  std::vector<odmd_t> v(hs, hs + count);
  BatchPlan* p = find_plan(v);
  *split = p ? (p->chosen >= 0 ? p->cand[p->chosen] : 0) : -1;
  return ODMD_OK;
}

static void drop_batch_plans(odmd_t h) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  for (size_t i = 0; i < g_plans.size();) {
    BatchPlan* p = g_plans[i];
    if (std::find(p->serials.begin(), p->serials.end(), h->serial) != p->serials.end()) {
      free_plan(p);
      g_plans.erase(g_plans.begin() + (long)i);
    } else {
      ++i;
    }
  }
}

odmd_status odmd_update_batch(odmd_t* hs, const void* const* xs, int32_t count) {
  if (count < 0 || (count > 0 && (!hs || !xs))) return fail(nullptr, ODMD_ERR_ARG, "update_batch: bad arguments");
  for (int32_t i = 0; i < count; ++i) {
    if (!hs[i]) return fail(nullptr, ODMD_ERR_ARG, "update_batch: handle " + std::to_string(i) + " is NULL");
    if (!xs[i]) return fail(nullptr, ODMD_ERR_ARG, "update_batch: snapshot " + std::to_string(i) + " is NULL");
    for (int32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i])
        return fail(nullptr, ODMD_ERR_ARG, "update_batch: handle " + std::to_string(i) + " repeats handle " +
                                               std::to_string(j));
  }
  if (count == 0) return ODMD_OK;
  for (int32_t i = 0; i < count; ++i)  // any pipelined tail first
    if (odmd_status s = settle(hs[i])) return fail(nullptr, s, "update_batch: instance " + std::to_string(i) + ": " + hs[i]->err);
  // instances that can share launches, grouped by storage format and compaction kind, in
  // groups of at most kMaxBatch; the others (first snapshot, profiling on, row shards, no
  // graphs, another device) update one by one
  const int dev = hs[0]->device;
  std::vector<std::vector<int>> groups;
  std::vector<int> solo;
  for (int32_t i = 0; i < count; ++i) {
    if (!batchable(hs[i], dev)) {
      solo.push_back(i);
      continue;
    }
    bool placed = false;
    for (auto& g : groups) {
      odmd_t a = hs[g[0]];
      if ((int)g.size() < kMaxBatch && a->ws.prec == hs[i]->ws.prec && split_compaction(a) == split_compaction(hs[i])) {
        g.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back({i});
  }
  for (auto& g : groups) {
    if (g.size() == 1) {
      solo.push_back(g[0]);
      continue;
    }
    std::vector<odmd_t> gh;
    std::vector<const void*> gx;
    for (int i : g) {
      gh.push_back(hs[i]);
      gx.push_back(xs[i]);
    }
    if (odmd_status st = run_batch(gh, gx)) return fail(nullptr, st, "update_batch: " + g_err);
  }
  for (int i : solo)
    if (odmd_status s = odmd_update(hs[i], xs[i]))
      return fail(nullptr, s, "update_batch: instance " + std::to_string(i) + ": " + hs[i]->err);
  return ODMD_OK;
}

odmd_status odmd_predict_batch(odmd_t* hs, const double* const* ts, const int32_t* ks, void* const* outs,
                               const int64_t* lds, int32_t count) {
  if (count < 0 || (count > 0 && (!hs || !ts || !ks || !outs || !lds)))
    return fail(nullptr, ODMD_ERR_ARG, "predict_batch: bad arguments");
  for (int32_t i = 0; i < count; ++i)
    if (!hs[i]) return fail(nullptr, ODMD_ERR_ARG, "predict_batch: handle " + std::to_string(i) + " is NULL");
  for (int32_t i = 0; i < count; ++i)
    if (odmd_status s = odmd_predict(hs[i], ts[i], ks[i], outs[i], lds[i]))
      return fail(nullptr, s, "predict_batch: instance " + std::to_string(i) + ": " + hs[i]->err);
  return ODMD_OK;
}

odmd_status odmd_sync(odmd_t h) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  return device_status(h);
}

static odmd_status read_hdr(odmd_t h, StateHdr* hdr) {
  CK(h, cudaMemcpyAsync(h->pinned, h->ws.st[h->cur_h].hdr, sizeof(StateHdr), cudaMemcpyDeviceToHost, h->stream),
     "header read");
  if (odmd_status s = device_status(h)) return s;
  std::memcpy(hdr, h->pinned, sizeof(StateHdr));
  h->compactions = hdr->compactions;
  return ODMD_OK;
}

odmd_status odmd_get_rank(odmd_t h, int32_t* r) {
  if (!h || !r) return fail(h, ODMD_ERR_ARG, "NULL argument");
  if (odmd_status st_ = settle(h)) return st_;
  StateHdr hdr;
  if (odmd_status s = read_hdr(h, &hdr)) return s;
  *r = hdr.r;
  return ODMD_OK;
}

odmd_status odmd_get_singular_values(odmd_t h, double* s_host, int32_t cap, int32_t* r) {
  if (!h || !r || (cap > 0 && !s_host)) return fail(h, ODMD_ERR_ARG, "NULL argument");
  if (odmd_status st_ = settle(h)) return st_;
  StateHdr hdr;
  if (odmd_status s = read_hdr(h, &hdr)) return s;
  *r = hdr.r;
  const int nc = hdr.r < cap ? hdr.r : cap;
  if (nc > 0) {
    CK(h, cudaMemcpy(s_host, h->ws.st[h->cur_h].S, nc * sizeof(double), cudaMemcpyDeviceToHost), "S read");
  }
  return ODMD_OK;
}

odmd_status odmd_get_eigs(odmd_t h, double* re_host, double* im_host, double* amp_host, int32_t cap, int32_t* r) {
  if (!h || !r || (cap > 0 && (!re_host || !im_host))) return fail(h, ODMD_ERR_ARG, "NULL argument");
  if (odmd_status st_ = settle(h)) return st_;
  if (h->nsnap < 2) return fail(h, ODMD_ERR_STATE, "no model yet");
  if (odmd_status s = ensure_eig(h)) return s;
  StateHdr hdr;
  if (odmd_status s = read_hdr(h, &hdr)) return s;
  *r = hdr.r;
  const int nc = hdr.r < cap ? hdr.r : cap;
  if (nc > 0) {
    float2 br[kMaxR], bi[kMaxR];
    CK(h, cudaMemcpy(br, h->ws.eig.lre, nc * sizeof(float2), cudaMemcpyDeviceToHost), "eig read");
    CK(h, cudaMemcpy(bi, h->ws.eig.lim, nc * sizeof(float2), cudaMemcpyDeviceToHost), "eig read");
    for (int i = 0; i < nc; ++i) {
      re_host[i] = join(br[i]);
      im_host[i] = join(bi[i]);
    }
    if (amp_host) {
      CK(h, cudaMemcpy(br, h->ws.eig.bre, nc * sizeof(float2), cudaMemcpyDeviceToHost), "b read");
      CK(h, cudaMemcpy(bi, h->ws.eig.bim, nc * sizeof(float2), cudaMemcpyDeviceToHost), "b read");
      for (int i = 0; i < nc; ++i) amp_host[i] = std::hypot(join(br[i]), join(bi[i]));
    }
  }
  return ODMD_OK;
}

odmd_status odmd_get_basis(odmd_t h, void* out_dev, int64_t ld, int32_t* r) {
  if (!h || !out_dev || !r) return fail(h, ODMD_ERR_ARG, "NULL argument");
  if (odmd_status st_ = settle(h)) return st_;
  if (ld < h->cfg.n) return fail(h, ODMD_ERR_ARG, "ld < n");
  StateHdr hdr;
  if (odmd_status s = read_hdr(h, &hdr)) return s;
  *r = hdr.r;
  if (hdr.r == 0) return ODMD_OK;
  if (odmd_status s = flush_pending(h)) return s;
  {
    ProfScope ps(h, ODMD_K_COEF, 1);
    CK(h, launch_basis_coef(h->ws, h->stream), "basis coef launch");
  }
  {
    ProfScope ps(h, ODMD_K_ROLLOUT, 1);
    CK(h, launch_rollout(h->ws, nullptr, hdr.r, out_dev, ld, 0, h->stream), "basis launch");
  }
  return device_status(h);
}

odmd_status odmd_get_counts(odmd_t h, int64_t* snapshots, int64_t* compactions) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (snapshots) *snapshots = h->nsnap;
  if (compactions) {
    StateHdr hdr;
    if (odmd_status s = read_hdr(h, &hdr)) return s;
    *compactions = hdr.compactions;
  }
  return ODMD_OK;
}

static odmd_status read_prof_counters(odmd_t h, unsigned long long* out2) {
  CK(h, cudaMemcpyAsync(h->pinned, &h->ws.ctl->prof_r0_sum, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        h->stream),
     "profile counters");
  CK(h, cudaStreamSynchronize(h->stream), "stream sync");
  std::memcpy(out2, h->pinned, 2 * sizeof(unsigned long long));
  return ODMD_OK;
}

odmd_status odmd_profile_enable(odmd_t h, int32_t enable) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  prof_collect(h);
  for (int i = 0; i < ODMD_K_COUNT; ++i) h->prof_ms[i] = 0.0;
  if (odmd_status s = read_prof_counters(h, h->r0_base)) return s;
  h->prof_on = enable != 0;
  return ODMD_OK;
}

odmd_status odmd_profile_read(odmd_t h, double* ms_total, int64_t* launches, int32_t cap, double* mean_r0) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (odmd_status s = device_status(h)) return s;
  prof_collect(h);
  const int nc = cap < ODMD_K_COUNT ? cap : ODMD_K_COUNT;
  for (int i = 0; i < nc; ++i) {
    if (ms_total) ms_total[i] = h->prof_ms[i];
    if (launches) launches[i] = h->launches[i];
  }
  if (mean_r0) {
    unsigned long long now[2];
    if (odmd_status s = read_prof_counters(h, now)) return s;
    const unsigned long long na = now[1] - h->r0_base[1];
    *mean_r0 = na ? (double)(now[0] - h->r0_base[0]) / (double)na : 0.0;
  }
  return ODMD_OK;
}

// release the captured update graphs (they are captured again on the next update)
static void drop_graph(odmd_instance::UpdGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  for (cudaEvent_t ev : g.ph)
    if (ev) cudaEventDestroy(ev);
  g = odmd_instance::UpdGraph{};
}
static void drop_update_graphs(odmd_t h) {
  for (auto& row : h->ug)
    for (auto& g : row) drop_graph(g);
  for (auto& a : h->pg)
    for (auto& b : a)
      for (auto& g : b) drop_graph(g);
  drop_graph(h->tg);
}

odmd_status odmd_set_row_shards(odmd_t h, int32_t shards) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  if (odmd_status st_ = settle(h)) return st_;
  if (shards < 1 || shards > h->ws.gridA)
    return fail(h, ODMD_ERR_ARG, "shards must lie in [1, " + std::to_string(h->ws.gridA) + "] (the row blocks)");
  if (shards == h->ws.shards) return ODMD_OK;
  CK(h, cudaStreamSynchronize(h->stream), "shards: sync");
  drop_update_graphs(h);
  drop_batch_plans(h);
  h->ws.shards = shards;
  CK(h, cudaMemcpy(h->wsv, &h->ws, sizeof(Ws), cudaMemcpyHostToDevice), "shards: workspace view");
  return ODMD_OK;
}

odmd_status odmd_get_row_blocks(odmd_t h, int32_t* blocks, int64_t* rows_host, int32_t cap) {
  if (!h || !blocks) return fail(h, ODMD_ERR_ARG, "NULL argument");
  const int B = h->ws.gridA;
  *blocks = B;
  if (rows_host && cap > 0) {
    const int64_t T = (h->cfg.n + kTile - 1) / kTile;
    for (int b = 0; b <= B && b < cap; ++b) {
      const int64_t r = (int64_t)b * T / B * kTile;
      rows_host[b] = r < h->cfg.n ? r : h->cfg.n;
    }
  }
  return ODMD_OK;
}

odmd_status odmd_destroy(odmd_t h) {
  if (!h) return fail(nullptr, ODMD_ERR_ARG, "handle is NULL");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  prof_collect(h);
  for (cudaEvent_t ev : h->pool) cudaEventDestroy(ev);
  drop_update_graphs(h);
  drop_batch_plans(h);
  if (h->ev_batch) cudaEventDestroy(h->ev_batch);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap2) cudaStreamDestroy(h->cap2);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (int b = 0; b < 2; ++b) {
    if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
    if (h->ev_used[b]) cudaEventDestroy(h->ev_used[b]);
  }
  if (h->copy) cudaStreamDestroy(h->copy);
  cudaFreeHost(h->pinned);
  delete h;
  if (e != cudaSuccess) return fail(nullptr, ODMD_ERR_CUDA, std::string("destroy: ") + cudaGetErrorString(e));
  return ODMD_OK;
}

const char* odmd_last_error(odmd_t h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"

namespace odmd {
odmd_status report_global_error(odmd_status s, const std::string& msg) { return fail(nullptr, s, msg); }
}  // namespace odmd
