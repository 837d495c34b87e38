// C ABI of the reconstruction library: contexts, resident circuits, query
// planning (merge descriptors, contraction order, layouts) and the
// per-query launch sequence.  See include/sqc.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "../../include/sqc.h"
#include "internal.h"
#include "launch.cuh"

using namespace sqc;

namespace sqc {
bool& pdl_flag() {
  static thread_local bool on = false;
  return on;
}
}  // namespace sqc

namespace {

thread_local std::string g_create_error;

constexpr int kBinBase = 1 << 16;   // layout codes: edge bit = 2*eid + (hi?1:0); bin bit = kBinBase + position
constexpr int kMaxK = 16;           // cut edges per subcircuit
constexpr int kMaxSub = 64;

struct Circuit {
  int n_qubits = 0, nC = 0, K = 0;
  std::vector<int> eu, ed, ndata, dq_flat;
  std::vector<std::vector<int>> dq, inc, ins, outs;
  std::vector<int64_t> V;        // 4^k_i
  std::vector<int> w;            // n_i + kout_i
  std::vector<float*> A;         // [V_i][2^n_i], data index bit-reversed
  // merge pyramid (cfg.merge_pyramid): level m = 1..n_i of subcircuit i at
  // pyr[i] + V_i (2^n_i - 2^(n_i-m+1)), [V_i][2^(n_i-m)], the sums of A_i
  // over its m lowest storage bits
  std::vector<float*> pyr;
  void* staging = nullptr;       // device copy of one subcircuit's host input
  size_t staging_bytes = 0;
  float* scratch = nullptr;      // fold output for subcircuits with incoming edges
  size_t scratch_floats = 0;
  size_t bytes = 0;
};

constexpr int kPad = -1;           // layout code of a padding bit (never written, zero)

struct Tensor {
  std::vector<int> bits;         // unordered set of logical bit codes
  std::set<int> edges;           // open cut edges
  std::vector<int> layout;       // layout[p] = code stored at address bit p (kPad: padding)
  int producer_sub = -1;         // merge of this subcircuit, or
  int producer_step = -1;        // output of this step
  int kind = OUT_F32;            // storage: FP32, or three BF16 planes for a tensor-core step
  int64_t plane_stride = 0;      // elements per BF16 plane
  void* buf = nullptr;
  size_t bytes = 0;
};

struct Step {
  int x = -1, y = -1, z = -1;    // operand tensors (x = A rows, y = B cols after layout) and result
  std::vector<int> shared;       // shared edge ids
  int64_t M = 1, N = 1, Kd = 1;
  bool tc = false;               // split-BF16 on tcgen05
  int64_t Kp = 1;                // shared index padded to the tensor-core K block
  uint64_t* rowmap = nullptr;    // device
  uint64_t* colmap = nullptr;
  int vec4 = 0;
  int contig16 = 0;           // colmap runs of 16 consecutive, 4-aligned offsets; rowmap 4-aligned
};

// Everything one precision needs to run a query: contraction order, layouts,
// maps, buffers.  Built on first use of that precision.
// What a plan's device part (workspace allocation, uploads) needs from its
// host part; kept between the two when they run on different threads.
struct PlanDraft {
  size_t off_desc = 0, off_maps = 0, off_part = 0, off_cnt = 0, zero_begin = 0, zero_end = 0;
  std::vector<size_t> off_tensor;
  std::vector<uint64_t> maps;
  std::vector<std::pair<size_t, size_t>> step_map_off, merge_map_off;
  std::vector<size_t> rowsel_off;
  std::vector<char> has_rowsel;
  std::vector<std::vector<std::pair<int, int>>> slice_pos;
};

struct Plan {
  bool built = false;
  std::unique_ptr<PlanDraft> draft;   // host part done, device part pending
  bool split = false;
  std::vector<Tensor> tensors;
  std::vector<Step> steps;
  int final_tensor = -1;
  std::vector<MergeDesc> merge_host;
  MergeDesc* merge_dev = nullptr;
  int64_t merge_blocks = 0;
  void* work = nullptr;
  size_t work_bytes = 0;
  double* partials = nullptr;
  unsigned* counter = nullptr;
  int* err = nullptr;            // set by bounded device waits that gave up
  double flops = 0.0;
  std::vector<int> sliced;       // first-level sliced edges (Section 6.3), in greedy order
  int64_t n_slices = 1;          // 4^{sliced edges}: merge descriptor sets, one per slice
  int order = 0;                 // contraction order the plan follows (SQC_ORDER_*)
  // FP32 plans: the steps and selection in one cooperative launch
  // (launch_select_tail); tail.P, total, alpha are set per call
  bool tail_ok = false;
  TailArgs tail{};
};

struct Batch {
  void* work = nullptr;
  size_t work_bytes = 0;
  BatchLaunch L{};                   // phase 0 (the only phase of an FP32 batch)
  int grid = 0;
  std::vector<sqc_query_id> queries;
  std::vector<unsigned> expected;    // host copy of the completion targets
  // split-BF16: the persistent launch of every phase, then that phase's
  // tensor-core steps
  std::vector<BatchLaunch> phases;
  std::vector<int> phase_grid;
  std::vector<std::vector<GemmTcArgs>> tc;
  int n_tc = 0;
};

struct Query {
  sqc_circuit_id circuit = 0;
  int order = -1;                // contraction order of its plans (SQC_ORDER_*; -1: the context's)
  std::vector<int8_t> roles;
  int n_active = 0;
  int64_t out_elems = 1;
  Plan plans[2];                 // [SQC_PREC_FP32], [SQC_PREC_SPLIT_BF16]
  void* sel_mem = nullptr;       // cooperative selection workspace (+ error flag)
  size_t sel_bytes = 0;
  int sel_grid = 0;
  double merge_bytes = 0.0;
  // single-launch FP32 reconstruction (merge and every step in one
  // persistent launch), one per output format [OUT_F32], [OUT_F64]; built
  // by the first FP32 reconstruct into that format
  std::unique_ptr<Batch> solo[2];
};

}  // namespace

struct StageMark {
  int stage;
  cudaEvent_t start, stop;
};

struct sqc_ctx {
  int device = 0;
  // stream-ordered allocation and uploads (the serving loop): when set, every
  // device allocation, upload and free of the context is issued on this
  // stream and nothing synchronises the device
  cudaStream_t alloc_stream = nullptr;
  bool async_alloc = false;
  bool prof = false;
  bool prof_keep = false;       // marks belong to a captured graph: keep them across reads
  std::vector<StageMark> marks;
  std::vector<cudaEvent_t> event_pool;
  int64_t launches = 0;
  sqc_config cfg{};
  std::string err;
  size_t bytes = 0;
  int64_t next_id = 1;
  int batch_policy = 0;          // tile policy of new batches (sqc_batch_autotune)
  std::map<int64_t, std::unique_ptr<Circuit>> circuits;
  std::map<int64_t, std::unique_ptr<Query>> queries;
  std::map<int64_t, std::unique_ptr<Batch>> batches;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Host-only planning on a worker thread reports into its own string
// instead of the context's (which another thread may be using).
thread_local std::string* t_err_sink = nullptr;

sqc_status fail(sqc_ctx* ctx, sqc_status st, const std::string& msg) {
  if (t_err_sink) *t_err_sink = msg;
  else if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return st;
}

sqc_status cuda_fail(sqc_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, SQC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);       \
  } while (0)

cudaEvent_t take_event(sqc_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Scope that brackets one stage with events when timing is on.
struct StageScope {
  sqc_ctx* ctx;
  cudaStream_t s;
  int stage;
  cudaEvent_t a = nullptr, b = nullptr;
  // inside a stream capture the records become graph nodes that must be
  // observable outside the graph (external event records)
  static void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s);
  }
  StageScope(sqc_ctx* c, cudaStream_t st, int stg) : ctx(c), s(st), stage(stg) {
    if (ctx->prof) {
      a = take_event(ctx);
      b = take_event(ctx);
      if (a) record(a, s);
    }
  }
  ~StageScope() {
    if (a && b) {
      record(b, s);
      ctx->marks.push_back({stage, a, b});
    }
  }
};

sqc_status dev_alloc(sqc_ctx* ctx, void** p, size_t bytes, bool admit = true) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (admit && ctx->cfg.hbm_budget_bytes && ctx->bytes + bytes > ctx->cfg.hbm_budget_bytes)
    return fail(ctx, SQC_EBUSY, "HBM budget exceeded: " + std::to_string(ctx->bytes + bytes) + " > " +
                                     std::to_string(ctx->cfg.hbm_budget_bytes) + " bytes");
  cudaError_t e = ctx->async_alloc ? cudaMallocAsync(p, bytes, ctx->alloc_stream) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, SQC_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  ctx->bytes += bytes;
  return SQC_OK;
}

void dev_free(sqc_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->async_alloc) cudaFreeAsync(p, ctx->alloc_stream); else cudaFree(p);
  ctx->bytes = ctx->bytes >= bytes ? ctx->bytes - bytes : 0;
}

cudaError_t upload(sqc_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (ctx->async_alloc) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->alloc_stream);
  return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}

cudaError_t zero(sqc_ctx* ctx, void* dst, size_t bytes) {
  if (ctx->async_alloc) return cudaMemsetAsync(dst, 0, bytes, ctx->alloc_stream);
  return cudaMemset(dst, 0, bytes);
}

inline int popc32(uint32_t x) { return __builtin_popcount(x); }

// Limit of every bounded device wait, from the configuration.
uint64_t wait_ns(const sqc_ctx* ctx) {
  const int ms = ctx->cfg.wait_limit_ms > 0 ? ctx->cfg.wait_limit_ms : 2000;
  return uint64_t(ms) * 1000000ull;
}

// ---- graph validation ---------------------------------------------------------

sqc_status build_circuit(sqc_ctx* ctx, const sqc_graph* g, Circuit* c) {
  if (!g || g->n_qubits < 1 || g->n_subcircuits < 1 || g->n_edges < 0)
    return fail(ctx, SQC_EINVAL, "graph: need n_qubits >= 1, n_subcircuits >= 1, n_edges >= 0");
  if (g->n_subcircuits > kMaxSub) return fail(ctx, SQC_ESHAPE, "graph: more than 64 subcircuits");
  if (g->n_edges > 60) return fail(ctx, SQC_ESHAPE, "graph: more than 60 cut edges");
  if (!g->n_data || !g->data_qubit || (g->n_edges > 0 && (!g->edge_up || !g->edge_down)))
    return fail(ctx, SQC_EINVAL, "graph: null array");
  c->n_qubits = g->n_qubits;
  c->nC = g->n_subcircuits;
  c->K = g->n_edges;
  c->eu.assign(g->edge_up, g->edge_up + g->n_edges);
  c->ed.assign(g->edge_down, g->edge_down + g->n_edges);
  c->ndata.assign(g->n_data, g->n_data + g->n_subcircuits);
  int64_t tot = 0;
  for (int i = 0; i < c->nC; ++i) {
    if (c->ndata[i] < 0 || c->ndata[i] > 30) return fail(ctx, SQC_ESHAPE, "graph: n_data[i] must be in [0, 30]");
    tot += c->ndata[i];
  }
  if (tot != c->n_qubits) return fail(ctx, SQC_EINVAL, "graph: sum of n_data must equal n_qubits");
  c->dq_flat.assign(g->data_qubit, g->data_qubit + c->n_qubits);
  std::vector<int> seen(c->n_qubits, 0);
  c->dq.resize(c->nC);
  int off = 0;
  for (int i = 0; i < c->nC; ++i) {
    for (int t = 0; t < c->ndata[i]; ++t) {
      const int q = c->dq_flat[off + t];
      if (q < 0 || q >= c->n_qubits || seen[q]) return fail(ctx, SQC_EINVAL, "graph: data_qubit must be a permutation of 0..n_qubits-1");
      seen[q] = 1;
      c->dq[i].push_back(q);
    }
    off += c->ndata[i];
  }
  c->inc.assign(c->nC, {});
  c->ins.assign(c->nC, {});
  c->outs.assign(c->nC, {});
  for (int e = 0; e < c->K; ++e) {
    const int u = c->eu[e], d = c->ed[e];
    if (u < 0 || u >= c->nC || d < 0 || d >= c->nC) return fail(ctx, SQC_EINVAL, "graph: edge endpoint out of range");
    if (u == d) return fail(ctx, SQC_EINVAL, "graph: an edge must join two different subcircuits");
    c->outs[u].push_back(e);
    c->ins[d].push_back(e);
  }
  c->V.resize(c->nC);
  c->w.resize(c->nC);
  for (int i = 0; i < c->nC; ++i) {
    std::set<int> s(c->ins[i].begin(), c->ins[i].end());
    s.insert(c->outs[i].begin(), c->outs[i].end());
    c->inc[i].assign(s.begin(), s.end());
    const int k = int(c->inc[i].size());
    if (k > kMaxK) return fail(ctx, SQC_ESHAPE, "graph: more than 16 cut edges on one subcircuit");
    c->V[i] = int64_t(1) << (2 * k);
    c->w[i] = c->ndata[i] + int(c->outs[i].size());
    if (2 * k + c->w[i] >= 40) return fail(ctx, SQC_ESHAPE, "graph: subcircuit input beyond 2^40 values");
  }
  return SQC_OK;
}

int digit_shift(const Circuit& c, int i, int eid) {
  const auto& inc = c.inc[i];
  const int k = int(inc.size());
  const int p = int(std::find(inc.begin(), inc.end(), eid) - inc.begin());
  return 2 * (k - 1 - p);
}

// Host inputs staged back to back in the circuit's staging buffer; src[i]
// receives each one's device address.  Mapped pinned host memory (every
// buffer 16-byte aligned, sizes multiples of 16) is copied by the SMs in one
// launch -- many loads in flight over the host link, 1.2x faster end to end
// on the 2^20-bin step than one copy-engine transfer per buffer -- other
// host memory by copies.
sqc_status stage_host_inputs(sqc_ctx* ctx, Circuit& c, const void* const* probs, size_t esz, cudaStream_t s,
                             std::vector<const void*>* src) {
  StageCopy sc{};
  bool sm_copy = c.nC <= kAttrPerLaunch;
  std::vector<const void*> mapped(c.nC, nullptr);
  for (int i = 0; i < c.nC && sm_copy; ++i) {
    const size_t nbytes = size_t(c.V[i]) * (size_t(1) << c.w[i]) * esz;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, probs[i]) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
        !pa.devicePointer || (reinterpret_cast<uintptr_t>(pa.devicePointer) & 15) || (nbytes & 15)) {
      cudaGetLastError();
      sm_copy = false;
    } else {
      mapped[i] = pa.devicePointer;
    }
  }
  size_t off = 0;
  for (int i = 0; i < c.nC; ++i) {
    const size_t nbytes = size_t(c.V[i]) * (size_t(1) << c.w[i]) * esz;
    if (off + nbytes > c.staging_bytes) return fail(ctx, SQC_ESHAPE, "staging buffer too small for these inputs");
    char* dst = static_cast<char*>(c.staging) + off;
    if (sm_copy) {
      sc.src[sc.n] = mapped[i];
      sc.dst[sc.n] = dst;
      sc.words[sc.n] = nbytes / 16;
      ++sc.n;
    } else {
      CK(cudaMemcpyAsync(dst, probs[i], nbytes, cudaMemcpyHostToDevice, s));
    }
    (*src)[i] = dst;
    off += (nbytes + 255) & ~size_t(255);
  }
  if (sc.n > 0) {
    PdlScope pdl(ctx->cfg.pdl != 0);
    CK(launch_stage_copy(sc, s));
    ctx->launches += 1;
  }
  return SQC_OK;
}

sqc_status attribute_all(sqc_ctx* ctx, Circuit* c, const void* const* probs, sqc_dtype dtype, int on_device,
                         cudaStream_t s) {
  const size_t esz = dtype == SQC_F64 ? 8 : 4;
  for (int i = 0; i < c->nC; ++i)
    if (!probs[i]) return fail(ctx, SQC_EINVAL, "probs[i] is null");
  StageScope scope(ctx, s, SQC_STAGE_ATTRIBUTE);
  // device addresses of every subcircuit's input (host inputs are staged
  // back to back so that one launch can attribute all subcircuits)
  std::vector<const void*> src(c->nC);
  if (on_device) {
    for (int i = 0; i < c->nC; ++i) src[i] = probs[i];
  } else {
    const sqc_status st = stage_host_inputs(ctx, *c, probs, esz, s, &src);
    if (st != SQC_OK) return st;
  }
  AttrLaunch L{};
  int64_t blocks = 0;
  int smem = 0;
  auto flush = [&]() -> sqc_status {
    if (L.n == 0) return SQC_OK;
    CK(launch_attr_fused(L, blocks, smem, s));
    ctx->launches += 1;
    L = AttrLaunch{};
    blocks = 0;
    smem = 0;
    return SQC_OK;
  };
  for (int i = 0; i < c->nC; ++i) {
    const int n = c->ndata[i];
    const int kin = int(c->ins[i].size());
    const int kout = int(c->outs[i].size());
    if (kin <= kMaxFusedIn) {
      AttrDesc& d = L.d[L.n];
      d.p = src[i];
      d.A = c->A[i];
      d.in_f64 = dtype == SQC_F64;
      d.n = n;
      d.kin = kin;
      d.kout = kout;
      // x tile: 2^L1 consecutive low values (read runs) x 2^L2 top-bit
      // values (write runs of the bit-reversed A).  Start at 8 x 2; grow
      // toward 32 x 8 (128-byte reads, whole 32-byte write sectors) while
      // the subcircuit still has kAttrTileTarget tiles, so that small
      // subcircuits keep enough CTAs and large ones amortise each tile's
      // shared-memory passes over more data.
      int L2 = std::min(1, n / 2), L1 = std::min(3, n - L2);
      const int64_t S = int64_t(1) << (2 * kin);
      while ((S << (L1 + L2)) > kAttrSmemMax / 4) {
        if (L1 >= L2 && L1 > 0) --L1;
        else if (L2 > 0) --L2;
        else break;
      }
      constexpr int64_t kAttrTileTarget = 4096;
      for (;;) {
        const int64_t tiles_next = ((int64_t(1) << (n - L1 - L2)) << (2 * kout)) >> 1;
        if (L1 + L2 >= n || tiles_next < kAttrTileTarget || (S << (L1 + L2 + 1)) > kAttrSmemMax / 4) break;
        if (L2 < 3) ++L2;
        else if (L1 < 5) ++L1;
        else break;
      }
      d.L1 = L1;
      d.L2 = L2;
      d.vec = L1 == 5 && L2 == 3 && dtype != SQC_F64 && (reinterpret_cast<uintptr_t>(src[i]) % 16) == 0;
      d.async2 = d.vec && kout == 0 && kin >= 1 && S <= 32;
      // without outgoing edges A_i is as large as p_i and the bit-reversed
      // write runs (2^L2 states) set the speed: the double-buffered form
      // takes 16 x 32 tiles (64-byte reads, 128-byte writes) in a ring of
      // two buffers, three CTAs per SM.  At 592 MB per step: 136.2 us,
      // against 149.4 us for 8 x 32 (32-byte reads), 148.5 us for 16 x 32
      // in a ring of three (two CTAs per SM), 167.1 us for 16 x 16 and
      // 248 us for 32 x 8 (32-byte writes).  With outgoing edges the reads
      // dominate and the 128-byte read runs of 32 x 8 measured faster.
      if (d.async2) {
        d.L1 = kRingL1;
        d.L2 = kRingL2;
      } else if (d.vec && kin > 0) {
        // the other 4-state form with incoming edges: 16 x 16 tiles, whose
        // 64-byte write runs beat the 32-byte runs of 32 x 8 while the reads
        // stream as fast in 64-byte runs (1.08 GB with incoming and
        // outgoing edges on one subcircuit: 360 -> 286 us)
        d.L1 = 4;
        d.L2 = 4;
      }
      for (int t = 0; t < kin; ++t) d.inshift[t] = digit_shift(*c, i, c->ins[i][t]);
      for (int u = 0; u < kout; ++u) d.outshift[u] = digit_shift(*c, i, c->outs[i][u]);
      d.block_begin = blocks;
      // a 4-state-per-thread CTA takes 4 tiles at once when there is a
      // single prepared-state row (no incoming edges): one per 64 threads
      const int64_t tiles_i = (int64_t(1) << (n - d.L1 - d.L2)) << (2 * kout);
      blocks += (d.vec && kin == 0) ? tiles_i / 4 : tiles_i;
      d.block_end = blocks;
      smem = std::max(smem, int((d.vec && kin == 0 ? 4 : (d.async2 ? kAttrRing * S : S)) << (d.L1 + d.L2)) * 4);
      if (++L.n == kAttrPerLaunch) {
        sqc_status st = flush();
        if (st != SQC_OK) return st;
      }
      continue;
    }
    // many incoming edges: outcome fold, then a per-output prepared-state mix
    FoldArgs fa{};
    fa.p = src[i];
    fa.in_f64 = dtype == SQC_F64;
    fa.V = c->V[i];
    fa.n = n;
    fa.kout = kout;
    for (int u = 0; u < kout; ++u) fa.outshift[u] = digit_shift(*c, i, c->outs[i][u]);
    fa.B = c->scratch;
    CK(launch_fold(fa, s));
    MixArgs ma{};
    ma.B = c->scratch;
    ma.A = c->A[i];
    ma.rows = c->V[i];
    ma.n = n;
    ma.kin = kin;
    for (int t = 0; t < kin; ++t) ma.inshift[t] = digit_shift(*c, i, c->ins[i][t]);
    CK(launch_mix(ma, s));
    ctx->launches += 2;
  }
  sqc_status st = flush();
  if (st != SQC_OK) return st;
  for (size_t i = 0; i < c->pyr.size(); ++i)
    if (c->pyr[i]) {
      CK(launch_pyramid(c->A[i], c->pyr[i], c->V[i], c->ndata[i], s));
      ctx->launches += (c->ndata[i] + kPyramidLevelsPerPass - 1) / kPyramidLevelsPerPass;
    }
  if (!on_device) {
    // host inputs: the caller may reuse its buffers on return, except while
    // the stream is captured into a graph (no synchronisation is allowed
    // there; the graph's copies then read the pinned buffers at every replay)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) CK(cudaStreamSynchronize(s));
  }
  return SQC_OK;
}

void free_plan(sqc_ctx* ctx, Plan* p) {
  dev_free(ctx, p->work, p->work_bytes);
  *p = Plan{};
}

void free_query(sqc_ctx* ctx, Query* q) {
  for (auto& b : q->solo)
    if (b) {
      dev_free(ctx, b->work, b->work_bytes);
      b.reset();
    }
  for (Plan& p : q->plans) free_plan(ctx, &p);
  dev_free(ctx, q->sel_mem, q->sel_bytes);
  q->sel_mem = nullptr;
}

void free_circuit(sqc_ctx* ctx, Circuit* c) {
  for (int i = 0; i < c->nC; ++i)
    if (c->A[i]) dev_free(ctx, c->A[i], size_t(c->V[i]) * (size_t(1) << c->ndata[i]) * 4);
  for (size_t i = 0; i < c->pyr.size(); ++i)
    if (c->pyr[i]) dev_free(ctx, c->pyr[i], size_t(c->V[i]) * (size_t(1) << c->ndata[i]) * 4);
  dev_free(ctx, c->staging, c->staging_bytes);
  dev_free(ctx, c->scratch, c->scratch_floats * 4);
}

// ---- planning -------------------------------------------------------------------

struct MapBuild {
  std::vector<uint64_t> host;   // all maps, concatenated
  size_t add(const std::vector<uint64_t>& m) {
    const size_t off = host.size();
    host.insert(host.end(), m.begin(), m.end());
    return off;
  }
};

// offset contribution of an index whose bit p holds logical code codes[p]
std::vector<uint64_t> make_map(const std::vector<int>& codes, const std::map<int, int>& pos) {
  const size_t n = size_t(1) << codes.size();
  std::vector<uint64_t> m(n, 0);
  std::vector<uint64_t> w(codes.size());
  for (size_t p = 0; p < codes.size(); ++p) w[p] = uint64_t(1) << pos.at(codes[p]);
  for (size_t i = 1; i < n; ++i) m[i] = m[i & (i - 1)] | w[size_t(__builtin_ctzll(i))];
  return m;
}

std::map<int, int> positions(const std::vector<int>& layout) {
  std::map<int, int> pos;
  for (size_t p = 0; p < layout.size(); ++p)
    if (layout[p] != kPad) pos[layout[p]] = int(p);
  return pos;
}

int ilog2(int64_t x) { return 63 - __builtin_clzll(uint64_t(x)); }

// Per-query roles: the bins (canonical positions) and, per subcircuit, the
// merge masks in storage order.
void resolve_roles(const Circuit& c, Query* q) {
  int na = 0;
  for (int qb = 0; qb < c.n_qubits; ++qb) na += q->roles[qb] == SQC_ROLE_ACTIVE;
  q->n_active = na;
  q->out_elems = int64_t(1) << na;
}

sqc_status finalize_plan(sqc_ctx* ctx, Plan* P);

// The pairwise contraction order with the fewest multiplications (Section
// 6.2 cost: a step costs the product of all its index dimensions) over every
// contraction tree, by dynamic programming over subsets of the subcircuit
// tensors.  emask[i]: open cut edges of T_i; bins[i]: its bin bits.  A
// subset's result keeps the edges that join it to the rest (each edge joins
// two tensors, so the XOR of the members' masks) and all their bins.  Ties:
// the smaller largest intermediate, then the first split found.  Returns the
// pairs in execution order (tensor indices, intermediates numbered n, n+1,
// ... as they are made), or nothing when n is beyond kMaxMinMultSub.
constexpr int kMaxMinMultSub = 14;
std::vector<std::pair<int, int>> min_mult_order(const std::vector<uint64_t>& emask, const std::vector<int>& bins) {
  const int n = int(emask.size());
  std::vector<std::pair<int, int>> pairs;
  if (n < 2 || n > kMaxMinMultSub) return pairs;
  const uint32_t full = (1u << n) - 1u;
  std::vector<uint64_t> open(size_t(1) << n, 0);
  std::vector<int> bits(size_t(1) << n, 0);
  for (uint32_t S = 1; S <= full; ++S) {
    const int low = __builtin_ctz(S);
    const uint32_t rest = S & (S - 1);
    open[S] = open[rest] ^ emask[low];
    bits[S] = bits[rest] + bins[low];
  }
  for (uint32_t S = 1; S <= full; ++S) bits[S] += 2 * __builtin_popcountll(open[S]);
  std::vector<double> best(size_t(1) << n, 0.0), peak(size_t(1) << n, 0.0);
  std::vector<uint32_t> split(size_t(1) << n, 0);
  for (uint32_t S = 1; S <= full; ++S) {
    if ((S & (S - 1)) == 0) continue;               // one tensor: nothing to do
    const uint32_t low = S & (0u - S);
    bool have = false;
    // every split into A (holding S's lowest member) and B = S \ A
    for (uint32_t A = (S - 1) & S; A; A = (A - 1) & S) {
      if (!(A & low)) continue;
      const uint32_t B = S ^ A;
      if (!B) continue;
      const int sh = __builtin_popcountll(open[A] & open[B]);
      const double c = std::ldexp(1.0, bits[A] + bits[B] - 2 * sh);
      const double tot = best[A] + best[B] + c;
      const double pk = std::max({peak[A], peak[B], std::ldexp(1.0, bits[S])});
      if (!have || tot < best[S] || (tot == best[S] && pk < peak[S])) {
        best[S] = tot;
        peak[S] = pk;
        split[S] = A;
        have = true;
      }
    }
  }
  // post-order: both halves first, then the pair that joins them
  std::function<int(uint32_t)> emit = [&](uint32_t S) -> int {
    if ((S & (S - 1)) == 0) return __builtin_ctz(S);
    const int a = emit(split[S]);
    const int b = emit(S ^ split[S]);
    pairs.push_back({a, b});
    return n + int(pairs.size()) - 1;
  };
  emit(full);
  return pairs;
}

// Host part of a plan; with defer the device part (finalize_plan) is left
// for the caller.
sqc_status build_plan(sqc_ctx* ctx, const Circuit& c, Query* q, bool split, Plan* P, bool defer = false) {
  const int nC = c.nC;
  std::vector<int> canon(c.n_qubits, -1);
  int na = 0;
  for (int qb = 0; qb < c.n_qubits; ++qb)
    if (q->roles[qb] == SQC_ROLE_ACTIVE) canon[qb] = na++;

  // first-level slicing (Section 6.3): write out cfg.slice_edges cut edges,
  // each time the one whose slicing shrinks sum_i 4^{k_i} 2^{a_i} most
  // (ties: lowest edge id)
  std::vector<int> a_of(nC, 0);
  for (int i = 0; i < nC; ++i)
    for (int t = 0; t < c.ndata[i]; ++t) a_of[i] += q->roles[c.dq[i][t]] == SQC_ROLE_ACTIVE;
  std::set<int> sliced;
  P->sliced.clear();
  auto total_size = [&](const std::set<int>& sl) {
    double tot = 0;
    for (int i = 0; i < nC; ++i) {
      int k = 0;
      for (int e : c.inc[i]) k += !sl.count(e);
      tot += std::ldexp(1.0, 2 * k + a_of[i]);
    }
    return tot;
  };
  auto slice_one = [&]() {
    int best = -1;
    double best_size = 0;
    for (int e = 0; e < c.K; ++e) {
      if (sliced.count(e)) continue;
      std::set<int> t = sliced;
      t.insert(e);
      const double sz = total_size(t);
      if (best < 0 || sz < best_size) { best = e; best_size = sz; }
    }
    sliced.insert(best);
    P->sliced.push_back(best);
  };
  for (int sidx = 0; sidx < ctx->cfg.slice_edges && int(sliced.size()) < c.K; ++sidx) slice_one();
  constexpr int kMaxSliced = 8;
  // first level by budget: the paper's rule (slice until the inputs fit)
  if (ctx->cfg.slice_input_log2 > 0) {
    const double budget = std::ldexp(1.0, ctx->cfg.slice_input_log2);
    while (total_size(sliced) > budget) {
      if (int(sliced.size()) >= std::min(c.K, kMaxSliced))
        return fail(ctx, SQC_ESHAPE, "slicing: the input budget needs more than 8 sliced edges");
      slice_one();
    }
  }
  // second level: the largest intermediate of the greedy contraction order
  // (the same rule as below, on tensor summaries: open edges, bins)
  auto max_intermediate = [&](const std::set<int>& sl) {
    struct Sum { std::set<int> edges; int bins; };
    std::vector<Sum> alive_t;
    for (int i = 0; i < nC; ++i) {
      Sum s{{}, a_of[i]};
      for (int e : c.inc[i]) if (!sl.count(e)) s.edges.insert(e);
      alive_t.push_back(s);
    }
    double worst = 0;
    while (alive_t.size() > 1) {
      int bx = -1, by = -1;
      double best = 0, best_out = 0;
      bool best_conn = false;
      for (size_t x = 0; x < alive_t.size(); ++x)
        for (size_t y = x + 1; y < alive_t.size(); ++y) {
          int sh = 0;
          for (int e : alive_t[x].edges) sh += int(alive_t[y].edges.count(e));
          const bool conn = sh > 0;
          const double fx = 2.0 * double(alive_t[x].edges.size()) + alive_t[x].bins - 2.0 * sh;
          const double fy = 2.0 * double(alive_t[y].edges.size()) + alive_t[y].bins - 2.0 * sh;
          const double out = std::ldexp(1.0, int(fx + fy));
          const double cost = std::ldexp(1.0, int(fx + fy + 2 * sh));
          bool better;
          if (bx < 0) better = true;
          else if (conn != best_conn) better = conn;
          else better = cost < best || (cost == best && out < best_out);
          if (better) { bx = int(x); by = int(y); best = cost; best_out = out; best_conn = conn; }
        }
      Sum z{{}, alive_t[bx].bins + alive_t[by].bins};
      for (int e : alive_t[bx].edges) if (!alive_t[by].edges.count(e)) z.edges.insert(e);
      for (int e : alive_t[by].edges) if (!alive_t[bx].edges.count(e)) z.edges.insert(e);
      alive_t.erase(alive_t.begin() + by);
      alive_t.erase(alive_t.begin() + bx);
      if (!alive_t.empty()) worst = std::max(worst, std::ldexp(1.0, 2 * int(z.edges.size()) + z.bins));
      alive_t.push_back(z);
    }
    return worst;
  };
  if (ctx->cfg.slice_intermediate_log2 > 0) {
    const double budget = std::ldexp(1.0, ctx->cfg.slice_intermediate_log2);
    while (max_intermediate(sliced) > budget) {
      if (int(sliced.size()) >= std::min(c.K, kMaxSliced))
        return fail(ctx, SQC_ESHAPE, "slicing: the intermediate budget needs more than 8 sliced edges");
      int best = -1;
      double best_mi = 0, best_in = 0;
      for (int e = 0; e < c.K; ++e) {
        if (sliced.count(e)) continue;
        std::set<int> t = sliced;
        t.insert(e);
        const double mi = max_intermediate(t), in = total_size(t);
        if (best < 0 || mi < best_mi || (mi == best_mi && in < best_in)) { best = e; best_mi = mi; best_in = in; }
      }
      sliced.insert(best);
      P->sliced.push_back(best);
    }
  }
  P->n_slices = int64_t(1) << (2 * sliced.size());

  // subcircuit tensors T_i and the merge index codes
  P->split = split;
  P->tensors.assign(nC, Tensor{});
  std::vector<std::vector<int>> row_codes(nC), col_codes(nC);
  std::vector<std::vector<uint64_t>> rowsel(nC);
  std::vector<std::vector<std::pair<int, int>>> slice_pos(nC);   // (digit shift in A's row, sliced index)
  P->merge_host.assign(nC, MergeDesc{});
  double merge_bytes = 0.0;
  for (int i = 0; i < nC; ++i) {
    const int n = c.ndata[i];
    const int k = int(c.inc[i].size());
    uint32_t act = 0, mer = 0, zval = 0;
    for (int t = 0; t < n; ++t) {
      const int qb = c.dq[i][t];
      const uint32_t bit = 1u << (n - 1 - t);   // storage order is bit-reversed
      switch (q->roles[qb]) {
        case SQC_ROLE_ACTIVE: act |= bit; break;
        case SQC_ROLE_MERGED: mer |= bit; break;
        case SQC_ROLE_ZOOM1: zval |= bit; break;
        default: break;
      }
    }
    Tensor& T = P->tensors[i];
    T.producer_sub = i;
    // row index e of A_i: incident edge p's digit at bits 2(k-1-p) (lo) and
    // 2(k-1-p)+1 (hi).  Sliced edges leave T_i: its rows run over the other
    // edges (kept in A's digit order) and rowsel maps them back to A's rows.
    std::vector<int> kept_shift;
    for (int p = k - 1; p >= 0; --p) {           // least significant digit first
      const int eid = c.inc[i][p];
      const int shift = 2 * (k - 1 - p);
      if (sliced.count(eid)) {
        const int sidx = int(std::find(P->sliced.begin(), P->sliced.end(), eid) - P->sliced.begin());
        slice_pos[i].push_back({shift, sidx});
        continue;
      }
      row_codes[i].push_back(2 * eid);
      row_codes[i].push_back(2 * eid + 1);
      kept_shift.push_back(shift);
      T.edges.insert(eid);
    }
    if (!slice_pos[i].empty()) {
      rowsel[i].assign(size_t(1) << (2 * kept_shift.size()), 0);
      for (size_t r = 0; r < rowsel[i].size(); ++r) {
        uint64_t e = 0;
        for (size_t t = 0; t < kept_shift.size(); ++t) e |= uint64_t((r >> (2 * t)) & 3) << kept_shift[t];
        rowsel[i][r] = e;
      }
    }
    // column index b: u-th lowest active storage bit
    for (int sp = 0; sp < n; ++sp)
      if ((act >> sp) & 1) col_codes[i].push_back(kBinBase + canon[c.dq[i][n - 1 - sp]]);
    T.bits = row_codes[i];
    T.bits.insert(T.bits.end(), col_codes[i].begin(), col_codes[i].end());
    MergeDesc& d = P->merge_host[i];
    d.A = c.A[i];
    d.rows = int64_t(1) << row_codes[i].size();
    d.n = n;
    d.act_mask = act;
    d.mer_mask = mer;
    d.zoom_val = zval;
    d.a = popc32(act);
    d.m = popc32(mer);
    d.fast = (mer == ((1u << d.m) - 1u)) && (act == (((1u << d.a) - 1u) << d.m));
    if (d.fast && d.m > 0 && i < int(c.pyr.size()) && c.pyr[i]) {
      // read the pyramid level holding the sums over the m merged bits
      const int m = d.m;
      d.A = c.pyr[i] + size_t(c.V[i]) * ((size_t(1) << n) - (size_t(1) << (n - m + 1)));
      d.n = n - m;
      d.act_mask = act >> m;
      d.mer_mask = 0;
      d.zoom_val = zval >> m;
      d.m = 0;
    }
    const uint32_t run = 1u << d.m;
    int lanes = d.fast ? int(run / 16) : int(run / 4);
    d.lanes = std::max(1, std::min(32, lanes));
    d.alpha = 1.0;
    merge_bytes += double(d.rows) * double(int64_t(1) << (d.a + d.m)) * 4.0 + double(d.rows << d.a) * 4.0;
  }
  q->merge_bytes = merge_bytes;

  // contraction order on the Section 6.2 cost (multiplications): greedy
  // pair by pair, or the fewest multiplications over all pairwise trees;
  // open edges as 64-bit masks (K <= 60) so that a pair's shared edges are
  // one popcount
  std::vector<int> alive;
  std::vector<uint64_t> emask;
  auto mask_of = [](const std::set<int>& edges) {
    uint64_t m = 0;
    for (int e : edges) m |= uint64_t(1) << e;
    return m;
  };
  for (int i = 0; i < nC; ++i) {
    alive.push_back(i);
    emask.push_back(mask_of(P->tensors[i].edges));
  }
  const int order = q->order >= 0 ? q->order : ctx->cfg.contraction_order;
  std::vector<std::pair<int, int>> schedule;      // the pairs in execution order (fewest multiplications)
  if (order == SQC_ORDER_MIN_MULT && nC > 2) {
    std::vector<int> nbits(nC);
    for (int i = 0; i < nC; ++i) nbits[i] = int(P->tensors[i].bits.size()) - 2 * int(P->tensors[i].edges.size());
    schedule = min_mult_order(emask, nbits);
  }
  P->order = schedule.empty() ? SQC_ORDER_GREEDY : SQC_ORDER_MIN_MULT;
  while (alive.size() > 1) {
    int bx = -1, by = -1;
    double best = 0, best_out = 0;
    bool best_conn = false;
    if (!schedule.empty()) {
      bx = schedule[P->steps.size()].first;
      by = schedule[P->steps.size()].second;
    }
    for (size_t a = 0; a < alive.size() && schedule.empty(); ++a)
      for (size_t b = a + 1; b < alive.size(); ++b) {
        const Tensor& X = P->tensors[alive[a]];
        const Tensor& Y = P->tensors[alive[b]];
        const int sh = __builtin_popcountll(emask[alive[a]] & emask[alive[b]]);
        const bool conn = sh > 0;
        const double fx = double(X.bits.size()) - 2.0 * sh, fy = double(Y.bits.size()) - 2.0 * sh;
        const double out = std::ldexp(1.0, int(fx + fy));
        const double cost = std::ldexp(1.0, int(fx + fy + 2 * sh));
        bool better;
        if (bx < 0) better = true;
        else if (conn != best_conn) better = conn;
        else better = cost < best || (cost == best && out < best_out);
        if (better) {
          bx = alive[a]; by = alive[b]; best = cost; best_out = out; best_conn = conn;
        }
      }
    Step st;
    st.x = bx;
    st.y = by;
    Tensor Z;
    const Tensor& X = P->tensors[bx];
    const Tensor& Y = P->tensors[by];
    for (int e : X.edges)
      if (Y.edges.count(e)) st.shared.push_back(e);
    std::set<int> shcodes;
    for (int e : st.shared) { shcodes.insert(2 * e); shcodes.insert(2 * e + 1); }
    for (int b : X.bits) if (!shcodes.count(b)) Z.bits.push_back(b);
    for (int b : Y.bits) if (!shcodes.count(b)) Z.bits.push_back(b);
    for (int e : X.edges) if (!Y.edges.count(e)) Z.edges.insert(e);
    for (int e : Y.edges) if (!X.edges.count(e)) Z.edges.insert(e);
    Z.producer_step = int(P->steps.size());
    st.z = int(P->tensors.size());
    emask.push_back(mask_of(Z.edges));
    P->tensors.push_back(Z);
    P->steps.push_back(st);
    alive.erase(std::find(alive.begin(), alive.end(), bx));
    alive.erase(std::find(alive.begin(), alive.end(), by));
    alive.push_back(st.z);
  }
  P->final_tensor = alive[0];
  {
    Tensor& F = P->tensors[P->final_tensor];
    if (!F.edges.empty()) return fail(ctx, SQC_EINVAL, "plan: open edges left after contraction");
    F.layout.resize(na);
    for (int p = 0; p < na; ++p) F.layout[p] = kBinBase + p;
    if (int(F.bits.size()) != na) return fail(ctx, SQC_EINVAL, "plan: result bits do not match active qubits");
  }

  // layouts, from the result backwards; maps and dimensions of every step
  const bool tc_ok = split && gemm_tc_available();
  MapBuild maps;
  std::vector<std::pair<size_t, size_t>> step_map_off(P->steps.size());
  for (int s = int(P->steps.size()) - 1; s >= 0; --s) {
    Step& st = P->steps[s];
    const Tensor& Z = P->tensors[st.z];
    const std::map<int, int> zpos = positions(Z.layout);
    std::set<int> shcodes;
    for (int e : st.shared) { shcodes.insert(2 * e); shcodes.insert(2 * e + 1); }
    auto free_of = [&](int t) {
      std::vector<int> f;
      for (int b : P->tensors[t].bits) if (!shcodes.count(b)) f.push_back(b);
      std::sort(f.begin(), f.end(), [&](int a, int b) { return zpos.at(a) < zpos.at(b); });
      return f;
    };
    std::vector<int> fx = free_of(st.x), fy = free_of(st.y);
    // B (columns) = the operand that owns the result's lowest address bit,
    // so that consecutive columns land on consecutive addresses
    bool swap = false;
    int low = kPad;
    for (int code : Z.layout)
      if (code != kPad) { low = code; break; }
    if (low != kPad) swap = std::find(fx.begin(), fx.end(), low) != fx.end();
    else swap = fx.size() < fy.size();
    if (swap) { std::swap(st.x, st.y); std::swap(fx, fy); }
    std::vector<int> sh(shcodes.begin(), shcodes.end());
    st.Kd = int64_t(1) << sh.size();
    st.M = int64_t(1) << fx.size();
    st.N = int64_t(1) << fy.size();
    // tensor cores for the big steps: M, N >= 128 (one UMMA tile) and
    // enough work to amortise a tensor-core launch -- at least 2^21 outputs,
    // or a shared index of 256 or more (contraction-bound) with at least 2^14
    // outputs.  Smaller split-BF16 steps run FP32 on the SIMT cores (as
    // accurate): measured, a 2^20-output step with a 16-term shared index
    // took 12 us in FP32 against 17 us on tcgen05, and 2^18-output
    // intermediates about 3x longer on tcgen05.  The kernel sums a long
    // shared index in FP32 passes added in FP64 and adds later slices into
    // the output itself.
    const int64_t outs_mn = st.M * st.N;
    st.tc = tc_ok && st.M >= gemm_tc_min_rows() && st.N >= gemm_tc_min_rows() &&
            (outs_mn >= (int64_t(1) << 21) || (st.Kd >= 256 && outs_mn >= (int64_t(1) << 14)));
    st.Kp = st.tc ? std::max<int64_t>(st.Kd, gemm_tc_k_align()) : st.Kd;
    std::vector<int> lay = sh;
    for (int p = ilog2(st.Kd); p < ilog2(st.Kp); ++p) lay.push_back(kPad);
    for (Tensor* T : {&P->tensors[st.x], &P->tensors[st.y]}) {
      T->layout = lay;
      const std::vector<int>& f = (T == &P->tensors[st.x]) ? fx : fy;
      T->layout.insert(T->layout.end(), f.begin(), f.end());
      T->kind = st.tc ? OUT_BF16X3 : OUT_F32;
      T->plane_stride = int64_t(1) << T->layout.size();
    }
    const std::vector<uint64_t> rm = make_map(fx, zpos), cm = make_map(fy, zpos);
    bool v4 = st.N % 4 == 0;
    for (size_t j = 0; v4 && j < cm.size(); ++j)
      if (cm[j] != cm[j & ~size_t(3)] + (j & 3) || (cm[j & ~size_t(3)] & 3)) v4 = false;
    for (size_t i = 0; v4 && i < rm.size(); ++i)
      if (rm[i] & 3) v4 = false;
    st.vec4 = v4;
    bool c16 = st.N % 16 == 0;
    for (size_t j = 0; c16 && j < cm.size(); ++j)
      if (cm[j] != cm[j & ~size_t(15)] + (j & 15) || (cm[j & ~size_t(15)] & 3)) c16 = false;
    for (size_t i = 0; c16 && i < rm.size(); ++i)
      if (rm[i] & 3) c16 = false;
    st.contig16 = c16;
    step_map_off[s] = {maps.add(rm), maps.add(cm)};
    P->flops += 2.0 * double(st.M) * double(st.N) * double(st.Kd);
  }
  std::vector<std::pair<size_t, size_t>> merge_map_off(nC);
  std::vector<size_t> rowsel_off(nC, 0);
  for (int i = 0; i < nC; ++i) {
    const std::map<int, int> tpos = positions(P->tensors[i].layout);
    merge_map_off[i] = {maps.add(make_map(row_codes[i], tpos)), maps.add(make_map(col_codes[i], tpos))};
    if (!rowsel[i].empty()) rowsel_off[i] = maps.add(rowsel[i]);
  }

  // workspace: descriptors | maps | tensors | partials + counter + error flag
  auto align = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  size_t off = 0;
  const size_t off_desc = off; off = align(off + sizeof(MergeDesc) * nC * size_t(P->n_slices));
  const size_t off_maps = off; off = align(off + sizeof(uint64_t) * maps.host.size());
  std::vector<size_t> off_tensor(P->tensors.size(), 0);
  size_t zero_begin = 0, zero_end = 0;
  for (size_t t = 0; t < P->tensors.size(); ++t) {
    Tensor& T = P->tensors[t];
    if (int(t) == P->final_tensor) continue;
    const size_t elems = size_t(1) << T.layout.size();
    T.bytes = T.kind == OUT_BF16X3 ? 3 * elems * 2 : elems * 4;
    off_tensor[t] = off;
    if (T.kind == OUT_BF16X3) {
      if (!zero_end) zero_begin = off;
      zero_end = off + T.bytes;
    }
    off = align(off + T.bytes);
  }
  int64_t max_tiles = 1024;
  for (const Step& st : P->steps) max_tiles = std::max<int64_t>(max_tiles, ((st.M + 31) / 32) * ((st.N + 31) / 32));
  const size_t off_part = off; off = align(off + sizeof(double) * size_t(max_tiles));
  const size_t off_cnt = off; off = align(off + 64);
  P->work_bytes = off;
  auto D = std::make_unique<PlanDraft>();
  D->off_desc = off_desc;
  D->off_maps = off_maps;
  D->off_part = off_part;
  D->off_cnt = off_cnt;
  D->zero_begin = zero_begin;
  D->zero_end = zero_end;
  D->off_tensor = std::move(off_tensor);
  D->maps = std::move(maps.host);
  D->step_map_off = std::move(step_map_off);
  D->merge_map_off = std::move(merge_map_off);
  D->rowsel_off = std::move(rowsel_off);
  D->has_rowsel.resize(nC);
  for (int i = 0; i < nC; ++i) D->has_rowsel[i] = !rowsel[i].empty();
  D->slice_pos = std::move(slice_pos);
  P->draft = std::move(D);
  return defer ? SQC_OK : finalize_plan(ctx, P);
}

// Runs of consecutive bit positions of a deposit map m[0..cnt) (m[i] = the
// bits of i spread over fixed positions, in order): false if m is not one or
// needs more than kTailMaxRuns runs.
bool pext_of_map(const uint64_t* m, int64_t cnt, TailPext* r) {
  *r = TailPext{};
  if (cnt < 1 || (cnt & (cnt - 1)) || m[0] != 0) return false;
  const int nbits = ilog2(cnt);
  std::vector<int> pos(nbits);
  for (int t = 0; t < nbits; ++t) {
    const uint64_t v = m[int64_t(1) << t];
    if (!v || (v & (v - 1))) return false;
    pos[t] = __builtin_ctzll(v);
  }
  for (int64_t i = 1; i < cnt; ++i)
    if (m[i] != (m[i & (i - 1)] | m[i & -i])) return false;
  for (int t = 0; t < nbits;) {
    int e = t + 1;
    while (e < nbits && pos[e] == pos[e - 1] + 1) ++e;
    if (r->n == kTailMaxRuns) return false;
    r->pos[r->n] = static_cast<unsigned char>(pos[t]);
    r->len[r->n] = static_cast<unsigned char>(e - t);
    r->out[r->n] = static_cast<unsigned char>(t);
    ++r->n;
    t = e;
  }
  return true;
}

// The fused contraction + selection launch of an FP32 plan (P->tail): the
// steps before the last, ordered by dependency level with their tile
// shapes (passed as kernel parameters), and the last step's operands and
// bin-index runs.  Leaves P->tail_ok false when the plan does not fit the
// launch: sliced, a shared index of the last step above 64, more than
// kTailMaxLevels levels or kTailMaxPre steps before the last, or bin maps
// with too many runs.
cudaError_t prepare_tail(Plan* P, const PlanDraft& D) {
  P->tail_ok = false;
  P->tail = TailArgs{};
  if (P->split || P->n_slices != 1 || P->steps.empty()) return cudaSuccess;
  const int grid = select_resident_grid();
  if (grid <= 0) return cudaSuccess;
  const size_t ns = P->steps.size();
  const Step& fin = P->steps.back();
  if (fin.tc || fin.Kd > 64) return cudaSuccess;
  TailArgs& T = P->tail;
  if (!pext_of_map(D.maps.data() + D.step_map_off[ns - 1].first, fin.M, &T.rows) ||
      !pext_of_map(D.maps.data() + D.step_map_off[ns - 1].second, fin.N, &T.cols))
    return cudaSuccess;
  // dependency levels: merged subcircuit tensors 0, a step 1 + its inputs'
  std::vector<int> level(P->tensors.size(), 0);
  int top = 0;
  for (size_t si = 0; si + 1 < ns; ++si) {
    const Step& st = P->steps[si];
    if (st.tc) return cudaSuccess;
    level[st.z] = 1 + std::max(level[st.x], level[st.y]);
    top = std::max(top, level[st.z]);
  }
  if (top > kTailMaxLevels || ns - 1 > size_t(kTailMaxPre)) return cudaSuccess;
  std::vector<TailStep> pre;
  for (int l = 1; l <= top; ++l) {
    for (size_t si = 0; si + 1 < ns; ++si) {
      const Step& st = P->steps[si];
      if (level[st.z] != l) continue;
      TailStep ts{};
      GemmArgs& a = ts.a;
      a.A = static_cast<const float*>(P->tensors[st.x].buf);
      a.B = static_cast<const float*>(P->tensors[st.y].buf);
      a.M = st.M;
      a.N = st.N;
      a.K = st.Kd;
      a.rowmap = st.rowmap;
      a.colmap = st.colmap;
      a.vec4 = st.vec4;
      a.C = P->tensors[st.z].buf;
      a.kind = P->tensors[st.z].kind;
      a.plane_stride = P->tensors[st.z].plane_stride;
      a.alpha = 1.0;
      auto tiles = [&](int64_t b) { return ((st.M + b - 1) / b) * ((st.N + b - 1) / b); };
      ts.cfg = tiles(128) >= grid ? 2 : (tiles(64) >= grid ? 1 : 0);
      const int64_t edge = int64_t(32) << ts.cfg;
      ts.ntiles = tiles(edge);
      ts.tn_shift = ilog2((st.N + edge - 1) / edge);          // M, N and the edge are powers of two
      pre.push_back(ts);
    }
    T.level_end[l - 1] = int(pre.size());
  }
  T.n_levels = top;
  T.n_pre = int(pre.size());
  for (size_t j = 0; j < pre.size(); ++j) T.pre[j] = pre[j];
  // the operand with fewer rows is staged in shared memory (Y), the other
  // read from L2 (X); fmaf is symmetric in its factors, so the bins do not
  // depend on which is which
  const bool swap = fin.M < fin.N;
  if (swap) std::swap(T.rows, T.cols);
  T.X = static_cast<const float*>(P->tensors[swap ? fin.y : fin.x].buf);
  T.Y = static_cast<const float*>(P->tensors[swap ? fin.x : fin.y].buf);
  T.M = swap ? fin.N : fin.M;
  T.N = swap ? fin.M : fin.N;
  T.Kd = int(fin.Kd);
  T.ystride = fin.Kd >= 4 ? int(fin.Kd) + 4 : 1;
  {
    // a slice's X rows form a range when every bit X owns lies above every
    // bit Y owns
    int xlow = 64, yhigh = -1;
    for (int t = 0; t < T.rows.n; ++t) xlow = std::min<int>(xlow, T.rows.pos[t]);
    for (int t = 0; t < T.cols.n; ++t) yhigh = std::max<int>(yhigh, T.cols.pos[t] + T.cols.len[t] - 1);
    T.x_range = xlow > yhigh;
  }
  T.partials = P->partials;
  P->tail_ok = true;
  return cudaSuccess;
}

// Device part of a plan: allocate the workspace, point the steps and merge
// descriptors into it, upload maps and descriptors, zero what must start
// at zero.
sqc_status finalize_plan(sqc_ctx* ctx, Plan* P) {
  if (!P->draft) return fail(ctx, SQC_EINVAL, "plan: nothing to finalize");
  const PlanDraft& D = *P->draft;
  const int nC = int(P->merge_host.size());
  sqc_status st = dev_alloc(ctx, &P->work, P->work_bytes);
  if (st != SQC_OK) return st;
  char* base = static_cast<char*>(P->work);
  P->merge_dev = reinterpret_cast<MergeDesc*>(base + D.off_desc);
  uint64_t* maps_dev = reinterpret_cast<uint64_t*>(base + D.off_maps);
  for (size_t t = 0; t < P->tensors.size(); ++t)
    if (int(t) != P->final_tensor) P->tensors[t].buf = base + D.off_tensor[t];
  P->partials = reinterpret_cast<double*>(base + D.off_part);
  P->counter = reinterpret_cast<unsigned*>(base + D.off_cnt);
  P->err = reinterpret_cast<int*>(base + D.off_cnt + 16);

  for (size_t s = 0; s < P->steps.size(); ++s) {
    P->steps[s].rowmap = maps_dev + D.step_map_off[s].first;
    P->steps[s].colmap = maps_dev + D.step_map_off[s].second;
  }
  int64_t blocks = 0;
  for (int i = 0; i < nC; ++i) {
    MergeDesc& d = P->merge_host[i];
    d.rowmap = maps_dev + D.merge_map_off[i].first;
    d.colmap = maps_dev + D.merge_map_off[i].second;
    d.dst = P->tensors[i].buf;          // null for the result (set per call)
    d.kind = P->tensors[i].kind;
    d.plane_stride = P->tensors[i].plane_stride;
    d.rowsel = D.has_rowsel[i] ? maps_dev + D.rowsel_off[i] : nullptr;
    d.row_add = 0;
    d.block_begin = blocks;
    const int64_t outs = d.rows << d.a;
    const int64_t per = 256 / d.lanes;
    blocks += (outs + per - 1) / per;
  }
  P->merge_blocks = blocks;
  cudaError_t e = upload(ctx, maps_dev, D.maps.data(), sizeof(uint64_t) * D.maps.size());
  if (e == cudaSuccess && nC > 0) {
    // one descriptor set per slice: slice sigma fixes sliced edge j's digit
    // to (sigma >> 2j) & 3 in every A row it reads
    std::vector<MergeDesc> sets(size_t(nC) * size_t(P->n_slices));
    for (int64_t sg = 0; sg < P->n_slices; ++sg)
      for (int i = 0; i < nC; ++i) {
        MergeDesc d = P->merge_host[i];
        for (const auto& sp : D.slice_pos[i]) d.row_add += int64_t((sg >> (2 * sp.second)) & 3) << sp.first;
        sets[size_t(sg) * nC + i] = d;
      }
    e = upload(ctx, P->merge_dev, sets.data(), sizeof(MergeDesc) * sets.size());
  }
  if (e == cudaSuccess) e = zero(ctx, base + D.off_cnt, 64);
  if (e == cudaSuccess && !P->split) e = prepare_tail(P, D);
  // BF16 operand padding (shared-index columns beyond K) must read as zero
  if (e == cudaSuccess && D.zero_end > D.zero_begin) e = zero(ctx, base + D.zero_begin, D.zero_end - D.zero_begin);
  if (e != cudaSuccess) {
    free_plan(ctx, P);
    return cuda_fail(ctx, e, "plan upload");
  }
  P->draft.reset();
  P->built = true;
  return SQC_OK;
}

sqc_status ensure_select_work(sqc_ctx* ctx, Query* q) {
  if (q->sel_mem) return SQC_OK;
  q->sel_grid = select_coop_grid();
  q->sel_bytes = select_coop_bytes(q->sel_grid) + 64;
  sqc_status st = dev_alloc(ctx, &q->sel_mem, q->sel_bytes);
  if (st != SQC_OK) return st;
  cudaError_t e = zero(ctx, q->sel_mem, q->sel_bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "selection workspace");
  return SQC_OK;
}

// The fused attribution + merge of query q on fresh outputs src[i] (device
// pointers, FP64 if in_f64): one descriptor per subcircuit, the tile shape
// per subcircuit.  Returns false (with the reason) when some subcircuit's
// roles do not follow the recursion's pattern (zoomed lowest, active next,
// at most 8 merged highest), it has more than kMaxFusedIn incoming edges,
// its tile does not fit shared memory, or the query is sliced.
bool build_attr_merge(const Circuit& c, const Query& q, const Plan& P, const void* const* src, int in_f64,
                      void* out_bins, int out_kind, double alpha, std::vector<AttrMergeLaunch>* launches,
                      std::vector<int64_t>* blocks, std::vector<int>* smem, std::string* why) {
  if (P.n_slices != 1) {
    *why = "sliced queries take sqc_update_subcircuit_outputs + sqc_reconstruct";
    return false;
  }
  launches->assign(1, AttrMergeLaunch{});
  blocks->assign(1, 0);
  smem->assign(1, 0);
  for (int i = 0; i < c.nC; ++i) {
    const int n = c.ndata[i], kin = int(c.ins[i].size()), kout = int(c.outs[i].size());
    if (kin > kMaxFusedIn) {
      *why = "a subcircuit has more than 7 incoming cut edges";
      return false;
    }
    // roles in data-index order: zoomed, then active, then merged
    int z = 0, a = 0, m = 0, t = 0;
    uint32_t zval = 0;
    for (; t < n && (q.roles[c.dq[i][t]] == SQC_ROLE_ZOOM0 || q.roles[c.dq[i][t]] == SQC_ROLE_ZOOM1); ++t, ++z)
      if (q.roles[c.dq[i][t]] == SQC_ROLE_ZOOM1) zval |= 1u << t;
    for (; t < n && q.roles[c.dq[i][t]] == SQC_ROLE_ACTIVE; ++t) ++a;
    for (; t < n && q.roles[c.dq[i][t]] == SQC_ROLE_MERGED; ++t) ++m;
    if (t != n || m > 8) {
      *why = "the roles of a subcircuit do not follow the recursion's pattern (zoomed lowest data qubits, "
             "then active, then at most 8 merged)";
      return false;
    }
    const int64_t S = int64_t(1) << (2 * kin);
    int L1 = std::min(a, 8 - m);
    while (L1 > 0 && (S << (L1 + m)) > kAttrSmemMax / 4) --L1;
    if ((S << (L1 + m)) > kAttrSmemMax / 4) {
      *why = "a subcircuit's attribution tile does not fit shared memory";
      return false;
    }
    AttrMergeLaunch& L = launches->back();
    AttrMergeDesc& d = L.d[L.n];
    d.p = src[i];
    d.in_f64 = in_f64;
    d.n = n;
    d.kin = kin;
    d.kout = kout;
    d.z = z;
    d.a = a;
    d.zval = zval;
    d.L1 = L1;
    d.L2 = m;
    for (int u = 0; u < kin; ++u) d.inshift[u] = digit_shift(c, i, c.ins[i][u]);
    for (int u = 0; u < kout; ++u) d.outshift[u] = digit_shift(c, i, c.outs[i][u]);
    const MergeDesc& md = P.merge_host[i];
    d.rowmap = md.rowmap;
    d.colmap = md.colmap;
    const bool direct = P.steps.empty();
    d.dst = direct ? out_bins : P.tensors[i].buf;
    d.kind = direct ? out_kind : P.tensors[i].kind;
    d.plane_stride = direct ? 0 : P.tensors[i].plane_stride;
    d.alpha = float(direct ? alpha : 1.0);
    if (++L.n == kAttrPerLaunch && i + 1 < c.nC) {
      launches->push_back(AttrMergeLaunch{});
      blocks->push_back(0);
      smem->push_back(0);
    }
  }
  // Tile sizes per launch.  A tile's reads are latency-bound chains of
  // 4^kin 2^(L1 + m) 2^kout loads over 256 threads, and the launch ends
  // with its slowest CTA: starting from the fewest tiles, the subcircuit
  // with the longest tiles is split in two (L1 - 1) while the launch still
  // fits one wave of resident CTAs, down to runs of 2 consecutive reads
  // (L1 = 1) and no further once a tile is one load per thread.
  for (size_t j = 0; j < launches->size(); ++j) {
    AttrMergeLaunch& L = (*launches)[j];
    auto tiles = [&](const AttrMergeDesc& d) { return (int64_t(1) << (d.a - d.L1)) << (2 * d.kout); };
    auto work = [&](const AttrMergeDesc& d) { return (int64_t(1) << (2 * d.kin + d.L1 + d.L2)) << d.kout; };
    auto tile_smem = [&](const AttrMergeDesc& d) { return int((int64_t(1) << (2 * d.kin + d.L1 + d.L2)) * 4); };
    int64_t total = 0;
    for (int u = 0; u < L.n; ++u) total += tiles(L.d[u]);
    bool any64 = false;
    for (int u = 0; u < L.n; ++u) any64 = any64 || L.d[u].in_f64;
    for (;;) {
      int best = -1;
      int64_t best_work = 256;
      for (int u = 0; u < L.n; ++u) {
        const AttrMergeDesc& d = L.d[u];
        if (d.L1 > 1 && work(d) > best_work) {
          // the split must keep the launch within one wave
          int sm = 0;
          for (int v = 0; v < L.n; ++v) sm = std::max(sm, v == u ? tile_smem(d) / 2 : tile_smem(L.d[v]));
          if (total + tiles(d) <= attr_merge_wave(any64, sm)) {
            best = u;
            best_work = work(d);
          }
        }
      }
      if (best < 0) break;
      total += tiles(L.d[best]);
      --L.d[best].L1;
    }
    int64_t b = 0;
    int sm = 0;
    for (int u = 0; u < L.n; ++u) {
      AttrMergeDesc& d = L.d[u];
      d.block_begin = b;
      b += tiles(d);
      d.block_end = b;
      sm = std::max(sm, tile_smem(d));
    }
    (*blocks)[j] = b;
    (*smem)[j] = sm;
  }
  return true;
}

// Plan query q again under contraction order `order` (SQC_ORDER_*): its
// plans and single-launch work lists are freed, the FP32 plan is rebuilt
// (the split-BF16 plan is rebuilt by the next split-BF16 reconstruct).
sqc_status replan(sqc_ctx* ctx, Query& q, int order) {
  auto cit = ctx->circuits.find(q.circuit);
  if (cit == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "circuit of the query was unloaded");
  if (!ctx->async_alloc) cudaDeviceSynchronize();
  for (auto& b : q.solo)
    if (b) {
      dev_free(ctx, b->work, b->work_bytes);
      b.reset();
    }
  for (Plan& p : q.plans) free_plan(ctx, &p);
  q.order = order;
  return build_plan(ctx, *cit->second, &q, false, &q.plans[SQC_PREC_FP32]);
}

// Work lists of the persistent launches over the plans of n queries
// (shared by sqc_batch_create and the single-query launch of
// sqc_reconstruct).  solo: one query whose output and probability sum are
// named per launch (BatchLaunch::out / total) instead of being baked in.
// A split-BF16 plan's tensor-core steps run as their own launches between
// phases: phase j is one persistent batch launch (merges in phase 0, and
// every SIMT step whose inputs are complete by then, waiting on the
// in-launch completion counters of the tensors it reads) followed by the
// tensor-core steps whose inputs are complete after it.
sqc_status build_batch(sqc_ctx* ctx, int32_t n, Query* const* qv, void* const* outs, int out_kind, double* totals,
                       bool solo, std::unique_ptr<Batch>* out_b, int precision = SQC_PREC_FP32) {
  std::vector<MergeDesc> mdescs;
  std::vector<BatchStep> steps;
  std::vector<unsigned> expected;            // per tensor slot (all phases)
  std::vector<int> slot_phase;               // the batch phase that produces each slot
  struct Pending { BatchItem it; int level; int phase; };
  std::vector<Pending> items;
  std::vector<int64_t> part_off;             // per batch step with a probability sum: offset into partials
  int64_t n_parts = 0;
  struct TcPending { GemmTcArgs a; int phase; bool sums; int query; };
  std::vector<TcPending> tcs;
  int n_phases = 1;
  for (int j = 0; j < n; ++j) {
    Query& q = *qv[j];
    auto cit = ctx->circuits.find(q.circuit);
    if (cit == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "batch: circuit of a query was unloaded");
    const Circuit& c = *cit->second;
    Plan& P = q.plans[precision];
    if (!P.built) {
      sqc_status st = build_plan(ctx, c, &q, precision == SQC_PREC_SPLIT_BF16, &P);
      if (st != SQC_OK) return st;
    }
    if (P.steps.empty()) return fail(ctx, SQC_EINVAL, "batch: every query needs at least two subcircuits");
    if (P.n_slices > 1) return fail(ctx, SQC_EINVAL, "batch: sliced queries (cfg.slice_edges > 0) run one at a time");
    if (!solo && !outs[j]) return fail(ctx, SQC_EINVAL, "batch: null output");
    // tensor slots of this query; the phase after which a tensor is
    // complete for a SIMT reader (same phase: wait on its counter) and for
    // a tensor-core reader
    std::vector<int> slot(P.tensors.size(), -1), level(P.tensors.size(), 0);
    std::vector<int> av_simt(P.tensors.size(), 0), av_tc(P.tensors.size(), 0);
    std::vector<char> by_tc(P.tensors.size(), 0);
    for (size_t t = 0; t < P.tensors.size(); ++t) {
      if (int(t) == P.final_tensor) continue;
      slot[t] = int(expected.size());
      expected.push_back(0);
      slot_phase.push_back(0);
    }
    for (int i = 0; i < c.nC; ++i) {
      const int di = int(mdescs.size());
      mdescs.push_back(P.merge_host[i]);
      const MergeDesc& d = P.merge_host[i];
      const int64_t per = 256 / d.lanes;
      const int64_t nblk = ((d.rows << d.a) + per - 1) / per;
      for (int64_t b = 0; b < nblk; ++b) items.push_back({{kItemMerge, di, b, -1, -1, slot[i]}, 0, 0});
      expected[slot[i]] = unsigned(nblk);
    }
    const double alpha = std::ldexp(1.0, -c.K);
    for (size_t si = 0; si < P.steps.size(); ++si) {
      const Step& st = P.steps[si];
      const bool last = si + 1 == P.steps.size();
      const Tensor& Z = P.tensors[st.z];
      void* C = last ? (solo ? nullptr : outs[j]) : Z.buf;
      const int kind = last ? out_kind : Z.kind;
      const int64_t pstride = last ? 0 : Z.plane_stride;
      if (st.tc) {
        const int ph = std::max(av_tc[st.x], av_tc[st.y]);
        GemmTcArgs a{};
        a.A = P.tensors[st.x].buf;
        a.B = P.tensors[st.y].buf;
        a.M = st.M; a.N = st.N; a.K = st.Kd;
        a.Mp = st.M; a.Np = st.N; a.Kp = st.Kp;
        a.rowmap = st.rowmap;
        a.colmap = st.colmap;
        a.C = C;
        a.kind = kind;
        a.plane_stride = pstride;
        a.alpha = last ? alpha : 1.0;
        a.chunk = (last && out_kind == OUT_F64 && c.K >= ctx->cfg.fp64_chunk_min_edges &&
                   st.Kd > ctx->cfg.chunk_terms) ? ctx->cfg.chunk_terms : 0;
        a.err = P.err;
        a.contig16 = st.contig16;
        a.pairs = ctx->cfg.tc_pairs;
        a.wait_ns = wait_ns(ctx);
        if (solo && last) return fail(ctx, SQC_EINVAL, "batch: a single-query launch runs FP32 steps only");
        tcs.push_back({a, ph, last && totals != nullptr, j});
        av_simt[st.z] = av_tc[st.z] = ph + 1;
        by_tc[st.z] = 1;
        n_phases = std::max(n_phases, ph + 2);
        if (!last) {
          slot_phase[slot[st.z]] = -1;             // written by a tensor-core launch, not counted
          expected[slot[st.z]] = 0;
        }
        continue;
      }
      const int ph = std::max(av_simt[st.x], av_simt[st.y]);
      BatchStep bs{};
      GemmArgs& a = bs.a;
      a.A = static_cast<const float*>(P.tensors[st.x].buf);
      a.B = static_cast<const float*>(P.tensors[st.y].buf);
      a.M = st.M;
      a.N = st.N;
      a.K = st.Kd;
      a.rowmap = st.rowmap;
      a.colmap = st.colmap;
      a.vec4 = st.vec4;
      a.C = C;
      a.kind = kind;
      a.plane_stride = pstride;
      a.alpha = last ? alpha : 1.0;
      a.chunk = (last && out_kind == OUT_F64 && c.K >= ctx->cfg.fp64_chunk_min_edges)
                    ? std::min<int64_t>(ctx->cfg.chunk_terms, st.Kd < 16 ? 16 : st.Kd)
                    : 0;
      bs.from_launch = last && solo;
      int64_t bm = 0, bn = 0;
      bs.cfg = batch_tile_cfg(a.M, a.N, a.K, a.chunk > 0, a.chunk, &bm, &bn, ctx->batch_policy);
      bs.ntiles = ((a.M + bm - 1) / bm) * ((a.N + bn - 1) / bn);
      if (last && (totals || solo)) {
        part_off.push_back(n_parts);
        bs.total = solo ? nullptr : totals + j;
        n_parts += bs.ntiles;
      } else {
        part_off.push_back(-1);
      }
      const int lvl = 1 + std::max(level[st.x], level[st.y]);
      level[st.z] = lvl;
      const int si_b = int(steps.size());
      steps.push_back(bs);
      // inputs made earlier in this phase by batch items are waited on; a
      // tensor-core result or an earlier phase's tensor is complete already
      auto dep = [&](int t) { return (!by_tc[t] && av_simt[t] == ph) ? slot[t] : -1; };
      for (int64_t t = 0; t < bs.ntiles; ++t)
        items.push_back({{kItemGemm, si_b, t, dep(st.x), dep(st.y), last ? -1 : slot[st.z]}, lvl, ph});
      if (!last) {
        expected[slot[st.z]] = unsigned(bs.ntiles);
        slot_phase[slot[st.z]] = ph;
      }
      av_simt[st.z] = ph;
      av_tc[st.z] = ph;
    }
  }
  // per phase, dependency order: merges, then steps level by level (stable)
  std::stable_sort(items.begin(), items.end(), [](const Pending& a, const Pending& b) {
    return a.phase != b.phase ? a.phase < b.phase : a.level < b.level;
  });
  std::vector<int64_t> ph_begin(n_phases + 1, 0);
  for (const Pending& p : items) ph_begin[p.phase + 1] += 1;
  for (int j = 0; j < n_phases; ++j) ph_begin[j + 1] += ph_begin[j];

  auto B = std::make_unique<Batch>();
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_items = off; off = align(off + sizeof(BatchItem) * std::max<size_t>(items.size(), 1));
  const size_t o_md = off; off = align(off + sizeof(MergeDesc) * mdescs.size());
  const size_t o_st = off; off = align(off + sizeof(BatchStep) * std::max<size_t>(steps.size(), 1));
  const size_t o_cnt = off; off = align(off + sizeof(unsigned) * expected.size());
  const size_t o_exp = off; off = align(off + sizeof(unsigned) * expected.size());
  const size_t o_part = off; off = align(off + sizeof(double) * size_t(std::max<int64_t>(n_parts, 1)));
  const size_t o_pc = off; off = align(off + sizeof(unsigned) * std::max<size_t>(steps.size(), 1));
  const size_t o_ctl = off; off = align(off + 64 * size_t(n_phases));
  const size_t o_tcp = off; off = align(off + sizeof(double) * 256 * tcs.size());   // tensor-core step partials
  const size_t o_tcc = off; off = align(off + 64 * tcs.size());                      // and counters
  B->work_bytes = off;
  sqc_status st = dev_alloc(ctx, &B->work, off);
  if (st != SQC_OK) return st;
  char* base = static_cast<char*>(B->work);
  for (size_t k = 0; k < steps.size(); ++k) {
    steps[k].counter = reinterpret_cast<unsigned*>(base + o_pc) + k;
    if (part_off[k] >= 0) {
      steps[k].partials = reinterpret_cast<double*>(base + o_part) + part_off[k];
      steps[k].a.partials = steps[k].partials;     // marks the query's last step
      steps[k].a.counter = steps[k].counter;
      steps[k].a.total = steps[k].total;
    }
  }
  std::vector<BatchItem> flat(items.size());
  for (size_t k = 0; k < items.size(); ++k) flat[k] = items[k].it;
  cudaError_t e = flat.empty() ? cudaSuccess : upload(ctx, base + o_items, flat.data(), sizeof(BatchItem) * flat.size());
  if (e == cudaSuccess && !mdescs.empty()) e = upload(ctx, base + o_md, mdescs.data(), sizeof(MergeDesc) * mdescs.size());
  if (e == cudaSuccess && !steps.empty()) e = upload(ctx, base + o_st, steps.data(), sizeof(BatchStep) * steps.size());
  if (e == cudaSuccess) e = upload(ctx, base + o_exp, expected.data(), sizeof(unsigned) * expected.size());
  if (e == cudaSuccess) e = zero(ctx, base + o_cnt, sizeof(unsigned) * expected.size());
  if (e == cudaSuccess && !steps.empty()) e = zero(ctx, base + o_pc, sizeof(unsigned) * steps.size());
  if (e == cudaSuccess) e = zero(ctx, base + o_ctl, 64 * size_t(n_phases));
  if (e == cudaSuccess && !tcs.empty()) e = zero(ctx, base + o_tcc, 64 * tcs.size());
  if (e != cudaSuccess) {
    dev_free(ctx, B->work, B->work_bytes);
    return cuda_fail(ctx, e, "batch upload");
  }
  int sms = 152, per = 2;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  B->phases.assign(n_phases, BatchLaunch{});
  B->phase_grid.assign(n_phases, 0);
  B->tc.assign(n_phases, {});
  for (int j = 0; j < n_phases; ++j) {
    BatchLaunch& L = B->phases[j];
    L.items = reinterpret_cast<const BatchItem*>(base + o_items) + ph_begin[j];
    L.n_items = ph_begin[j + 1] - ph_begin[j];
    L.mdescs = reinterpret_cast<const MergeDesc*>(base + o_md);
    L.steps = reinterpret_cast<const BatchStep*>(base + o_st);
    L.counts = reinterpret_cast<unsigned*>(base + o_cnt);
    L.expected = reinterpret_cast<const unsigned*>(base + o_exp);
    L.n_slots = int64_t(expected.size());
    char* ctl = base + o_ctl + 64 * size_t(j);
    L.head = reinterpret_cast<unsigned long long*>(ctl);
    L.done = reinterpret_cast<unsigned*>(ctl + 8);
    L.abort = reinterpret_cast<int*>(ctl + 16);
    L.err = reinterpret_cast<int*>(ctl + 20);
    L.wait_ns = wait_ns(ctx);
    B->phase_grid[j] = int(std::min<int64_t>(int64_t(sms) * per, std::max<int64_t>(L.n_items, 1)));
  }
  for (size_t k = 0; k < tcs.size(); ++k) {
    GemmTcArgs a = tcs[k].a;
    if (tcs[k].sums) {
      a.partials = reinterpret_cast<double*>(base + o_tcp) + 256 * k;
      a.counter = reinterpret_cast<unsigned*>(base + o_tcc + 64 * k);
      a.total = totals + tcs[k].query;
    }
    B->tc[tcs[k].phase].push_back(a);
    B->n_tc += 1;
  }
  // the last phase's counters re-arm every slot (they all start at zero)
  B->L = B->phases[0];
  B->grid = B->phase_grid[0];
  B->expected = std::move(expected);
  *out_b = std::move(B);
  return SQC_OK;
}


}  // namespace

// Hooks for the serving loop (server.cu), which drives a context from its
// own thread.
namespace sqc {
struct QueryDraft {
  int64_t circuit_id = 0;
  std::unique_ptr<Query> q;
};

const void* ctx_circuit(sqc_ctx* ctx, int64_t circuit) {
  auto it = ctx->circuits.find(circuit);
  return it == ctx->circuits.end() ? nullptr : it->second.get();
}

int32_t query_draft(const sqc_ctx* cctx, int64_t circuit_id, const void* circuit, const int8_t* roles,
                    QueryDraft** out, std::string* err) {
  sqc_ctx* ctx = const_cast<sqc_ctx*>(cctx);      // read only: configuration (errors go to *err)
  t_err_sink = err;
  *out = nullptr;
  const Circuit& c = *static_cast<const Circuit*>(circuit);
  sqc_status st = SQC_OK;
  int na = 0;
  for (int qb = 0; qb < c.n_qubits && st == SQC_OK; ++qb) {
    if (roles[qb] < SQC_ROLE_ACTIVE || roles[qb] > SQC_ROLE_ZOOM1) st = fail(ctx, SQC_EINVAL, "role out of range");
    na += roles[qb] == SQC_ROLE_ACTIVE;
  }
  if (st == SQC_OK && na > ctx->cfg.max_active_qubits)
    st = fail(ctx, SQC_ESHAPE, "active qubits " + std::to_string(na) + " > max_active_qubits");
  auto d = std::make_unique<QueryDraft>();
  if (st == SQC_OK) {
    d->circuit_id = circuit_id;
    d->q = std::make_unique<Query>();
    d->q->circuit = circuit_id;
    d->q->roles.assign(roles, roles + c.n_qubits);
    resolve_roles(c, d->q.get());
    st = build_plan(ctx, c, d->q.get(), false, &d->q->plans[SQC_PREC_FP32], true);
  }
  t_err_sink = nullptr;
  if (st == SQC_OK) *out = d.release();
  return st;
}

int32_t query_commit(sqc_ctx* ctx, QueryDraft* d, int64_t* query, int32_t* n_active) {
  std::unique_ptr<QueryDraft> own(d);
  if (!ctx->circuits.count(d->circuit_id)) return fail(ctx, SQC_ENOTFOUND, "circuit of a drafted query was unloaded");
  DeviceGuard g(ctx->device);
  sqc_status st = finalize_plan(ctx, &d->q->plans[SQC_PREC_FP32]);
  if (st != SQC_OK) {
    free_query(ctx, d->q.get());
    return st;
  }
  const int64_t qid = ctx->next_id++;
  if (n_active) *n_active = d->q->n_active;
  ctx->queries[qid] = std::move(d->q);
  *query = qid;
  return SQC_OK;
}

void query_draft_free(QueryDraft* d) { delete d; }

void ctx_set_alloc_stream(sqc_ctx* ctx, cudaStream_t s) {
  ctx->alloc_stream = s;
  ctx->async_alloc = s != nullptr;
}
int ctx_device(const sqc_ctx* ctx) { return ctx->device; }
void ctx_set_fused(sqc_ctx* ctx, bool on) { ctx->cfg.fused_query = on ? 1 : 0; }
sqc_status ctx_alloc(sqc_ctx* ctx, void** p, size_t bytes) { return dev_alloc(ctx, p, bytes); }
void ctx_free(sqc_ctx* ctx, void* p, size_t bytes) { dev_free(ctx, p, bytes); }
sqc_status ctx_fail(sqc_ctx* ctx, sqc_status st, const char* msg) { return fail(ctx, st, msg); }
}  // namespace sqc

namespace {
// Why a configuration is invalid (empty: it is valid).
std::string config_error(const sqc_config& c) {
  if (c.max_active_qubits < 0 || c.max_active_qubits > 40) return "max_active_qubits must be in [0, 40]";
  if (c.chunk_terms < 16 || (c.chunk_terms & (c.chunk_terms - 1))) return "chunk_terms must be a power of two >= 16";
  if (c.slice_edges < 0 || c.slice_edges > 8) return "slice_edges must be in [0, 8]";
  if (c.select_resident != 0 && c.select_resident != 1) return "select_resident must be 0 or 1";
  if (c.merge_pyramid != 0 && c.merge_pyramid != 1) return "merge_pyramid must be 0 or 1";
  if (c.tc_pairs != 0 && c.tc_pairs != 1) return "tc_pairs must be 0 or 1";
  if (c.wait_limit_ms < 0 || c.wait_limit_ms > 600000) return "wait_limit_ms must be in [0, 600000]";
  if (c.fused_query != 0 && c.fused_query != 1) return "fused_query must be 0 or 1";
  if (c.pdl != 0 && c.pdl != 1) return "pdl must be 0 or 1";
  if (c.fused_select != 0 && c.fused_select != 1) return "fused_select must be 0 or 1";
  if (c.contraction_order != SQC_ORDER_GREEDY && c.contraction_order != SQC_ORDER_MIN_MULT)
    return "contraction_order must be SQC_ORDER_GREEDY or SQC_ORDER_MIN_MULT";
  if (c.slice_input_log2 < 0 || c.slice_input_log2 > 62 || c.slice_intermediate_log2 < 0 ||
      c.slice_intermediate_log2 > 62)
    return "slice_input_log2 and slice_intermediate_log2 must be in [0, 62]";
  return {};
}
}  // namespace

// ================================================================ C ABI =====

extern "C" {

SQC_API void sqc_default_config(sqc_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->hbm_budget_bytes = 0;
  cfg->max_active_qubits = 32;
  cfg->fp64_chunk_min_edges = 12;
  cfg->chunk_terms = 256;
  cfg->select_resident = 1;
  cfg->fused_query = 0;
  cfg->pdl = 1;
  cfg->fused_select = 1;
}

SQC_API const char* sqc_last_error(const sqc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

SQC_API sqc_status sqc_create(sqc_ctx** out, int device, const sqc_config* cfg) {
  if (!out) return fail(nullptr, SQC_EINVAL, "out is null");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(nullptr, SQC_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) return fail(nullptr, SQC_EINVAL, "device index out of range");
  cudaDeviceProp prop{};
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return fail(nullptr, SQC_ECUDA, cudaGetErrorString(e));
  if (prop.major < 10) return fail(nullptr, SQC_ECUDA, std::string("device is not a Blackwell GPU: ") + prop.name);
  auto ctx = std::make_unique<sqc_ctx>();
  ctx->device = device;
  sqc_default_config(&ctx->cfg);
  if (cfg) ctx->cfg = *cfg;
  const std::string ce = config_error(ctx->cfg);
  if (!ce.empty()) return fail(nullptr, SQC_EINVAL, ce);
  DeviceGuard g(device);
  e = select_configure();
  if (e == cudaSuccess) e = attr_configure();
  if (e == cudaSuccess) e = gemm_tc_configure();
  if (e == cudaSuccess) e = batch_configure();
  if (e != cudaSuccess) return fail(nullptr, SQC_ECUDA, std::string("kernel setup: ") + cudaGetErrorString(e));
  *out = ctx.release();
  return SQC_OK;
}

SQC_API void sqc_destroy(sqc_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->queries) free_query(ctx, kv.second.get());
    for (auto& kv : ctx->circuits) free_circuit(ctx, kv.second.get());
    for (auto& kv : ctx->batches) dev_free(ctx, kv.second->work, kv.second->work_bytes);
    for (auto& m : ctx->marks) {
      cudaEventDestroy(m.start);
      cudaEventDestroy(m.stop);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  }
  delete ctx;
}

SQC_API sqc_status sqc_load_subcircuit_outputs(sqc_ctx* ctx, const sqc_graph* graph, const void* const* probs,
                                               sqc_dtype dtype, int probs_on_device, sqc_circuit_id* out_id,
                                               void* stream) {
  if (!ctx || !out_id || !probs) return fail(ctx, SQC_EINVAL, "null argument");
  if (dtype != SQC_F32 && dtype != SQC_F64) return fail(ctx, SQC_EINVAL, "dtype must be SQC_F32 or SQC_F64");
  DeviceGuard g(ctx->device);
  PdlScope pdl(ctx->cfg.pdl != 0);
  auto c = std::make_unique<Circuit>();
  sqc_status st = build_circuit(ctx, graph, c.get());
  if (st != SQC_OK) return st;
  c->A.assign(c->nC, nullptr);
  size_t stage = 0, scratch = 0;
  for (int i = 0; i < c->nC; ++i) {
    stage += (size_t(c->V[i]) * (size_t(1) << c->w[i]) * (dtype == SQC_F64 ? 8 : 4) + 255) & ~size_t(255);
    if (int(c->ins[i].size()) > kMaxFusedIn) scratch = std::max(scratch, size_t(c->V[i]) << c->ndata[i]);
  }
  auto cleanup = [&](sqc_status s) {
    free_circuit(ctx, c.get());
    return s;
  };
  for (int i = 0; i < c->nC; ++i) {
    void* p = nullptr;
    st = dev_alloc(ctx, &p, size_t(c->V[i]) * (size_t(1) << c->ndata[i]) * 4);
    if (st != SQC_OK) return cleanup(st);
    c->A[i] = static_cast<float*>(p);
  }
  if (ctx->cfg.merge_pyramid) {
    c->pyr.assign(c->nC, nullptr);
    for (int i = 0; i < c->nC; ++i) {
      if (c->ndata[i] == 0) continue;
      void* p = nullptr;
      st = dev_alloc(ctx, &p, size_t(c->V[i]) * (size_t(1) << c->ndata[i]) * 4);
      if (st != SQC_OK) return cleanup(st);
      c->pyr[i] = static_cast<float*>(p);
    }
  }
  if (!probs_on_device) {
    c->staging_bytes = stage;
    st = dev_alloc(ctx, &c->staging, stage);
    if (st != SQC_OK) return cleanup(st);
  }
  if (scratch) {
    c->scratch_floats = scratch;
    void* p = nullptr;
    st = dev_alloc(ctx, &p, scratch * 4);
    if (st != SQC_OK) return cleanup(st);
    c->scratch = static_cast<float*>(p);
  }
  st = attribute_all(ctx, c.get(), probs, dtype, probs_on_device, static_cast<cudaStream_t>(stream));
  if (st != SQC_OK) return cleanup(st);
  const int64_t id = ctx->next_id++;
  ctx->circuits[id] = std::move(c);
  *out_id = id;
  return SQC_OK;
}

SQC_API sqc_status sqc_update_subcircuit_outputs(sqc_ctx* ctx, sqc_circuit_id id, const void* const* probs,
                                                 sqc_dtype dtype, int probs_on_device, void* stream) {
  if (!ctx || !probs) return fail(ctx, SQC_EINVAL, "null argument");
  auto it = ctx->circuits.find(id);
  if (it == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "unknown circuit");
  Circuit* c = it->second.get();
  if (dtype != SQC_F32 && dtype != SQC_F64) return fail(ctx, SQC_EINVAL, "dtype must be SQC_F32 or SQC_F64");
  if (!probs_on_device) {
    size_t need = 0;
    for (int i = 0; i < c->nC; ++i)
      need += (size_t(c->V[i]) * (size_t(1) << c->w[i]) * (dtype == SQC_F64 ? 8 : 4) + 255) & ~size_t(255);
    if (need > c->staging_bytes)
      return fail(ctx, SQC_ESHAPE, "host-input update needs the circuit loaded from host data in this dtype");
  }
  DeviceGuard g(ctx->device);
  PdlScope pdl(ctx->cfg.pdl != 0);
  return attribute_all(ctx, c, probs, dtype, probs_on_device, static_cast<cudaStream_t>(stream));
}

SQC_API sqc_status sqc_unload(sqc_ctx* ctx, sqc_circuit_id id) {
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->circuits.find(id);
  if (it == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "unknown circuit");
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (auto q = ctx->queries.begin(); q != ctx->queries.end();) {
    if (q->second->circuit == id) {
      free_query(ctx, q->second.get());
      q = ctx->queries.erase(q);
    } else {
      ++q;
    }
  }
  free_circuit(ctx, it->second.get());
  ctx->circuits.erase(it);
  return SQC_OK;
}

SQC_API sqc_status sqc_set_qubit_roles(sqc_ctx* ctx, sqc_circuit_id id, const int8_t* roles, sqc_query_id* out_q,
                                       int32_t* n_active) {
  if (!ctx || !roles || !out_q) return fail(ctx, SQC_EINVAL, "null argument");
  auto it = ctx->circuits.find(id);
  if (it == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "unknown circuit");
  sqc::QueryDraft* d = nullptr;
  std::string err;
  sqc_status st = sqc::query_draft(ctx, id, it->second.get(), roles, &d, &err);
  if (st != SQC_OK) return fail(ctx, st, err);
  int64_t q = 0;
  st = sqc::query_commit(ctx, d, &q, n_active);
  if (st == SQC_OK) *out_q = q;
  return st;
}

SQC_API sqc_status sqc_release_query(sqc_ctx* ctx, sqc_query_id qid) {
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  DeviceGuard g(ctx->device);
  if (!ctx->async_alloc) cudaDeviceSynchronize();   // stream-ordered frees need no device sync
  free_query(ctx, it->second.get());
  ctx->queries.erase(it);
  return SQC_OK;
}

SQC_API sqc_status sqc_query_info(const sqc_ctx* cctx, sqc_query_id qid, int32_t* n_steps, double* flops,
                                  double* merge_bytes, uint64_t* work_bytes) {
  sqc_ctx* ctx = const_cast<sqc_ctx*>(cctx);
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  const Query& q = *it->second;
  const Plan& P = q.plans[SQC_PREC_FP32];
  if (n_steps) *n_steps = int32_t(P.steps.size());
  if (flops) *flops = P.flops;
  if (merge_bytes) *merge_bytes = q.merge_bytes;
  if (work_bytes) *work_bytes = q.plans[0].work_bytes + q.plans[1].work_bytes + q.sel_bytes;
  return SQC_OK;
}

SQC_API sqc_status sqc_query_slices(const sqc_ctx* cctx, sqc_query_id qid, int32_t* n_sliced, int32_t* edges,
                                    int32_t cap) {
  sqc_ctx* ctx = const_cast<sqc_ctx*>(cctx);
  if (!ctx || !n_sliced) return SQC_EINVAL;
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  const Plan& P = it->second->plans[SQC_PREC_FP32];
  *n_sliced = int32_t(P.sliced.size());
  for (size_t j = 0; j < P.sliced.size() && edges && int32_t(j) < cap; ++j) edges[j] = P.sliced[j];
  return SQC_OK;
}

SQC_API sqc_status sqc_memory_info(const sqc_ctx* ctx, uint64_t* held_bytes, uint64_t* budget_bytes) {
  if (!ctx) return SQC_EINVAL;
  if (held_bytes) *held_bytes = ctx->bytes;
  if (budget_bytes) *budget_bytes = ctx->cfg.hbm_budget_bytes;
  return SQC_OK;
}

SQC_API sqc_status sqc_query_step(const sqc_ctx* cctx, sqc_query_id qid, int32_t step, int64_t* M, int64_t* N,
                                  int64_t* Kd) {
  sqc_ctx* ctx = const_cast<sqc_ctx*>(cctx);
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  const Plan& P = it->second->plans[SQC_PREC_FP32];
  if (step < 0 || step >= int32_t(P.steps.size())) return fail(ctx, SQC_EINVAL, "step out of range");
  if (M) *M = P.steps[step].M;
  if (N) *N = P.steps[step].N;
  if (Kd) *Kd = P.steps[step].Kd;
  return SQC_OK;
}

SQC_API sqc_status sqc_query_tc_steps(const sqc_ctx* cctx, sqc_query_id qid, int32_t* n_tc, int32_t* n_steps) {
  sqc_ctx* ctx = const_cast<sqc_ctx*>(cctx);
  if (!ctx || !n_tc) return SQC_EINVAL;
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  const Plan& P = it->second->plans[SQC_PREC_SPLIT_BF16];
  int32_t k = 0;
  for (const Step& st : P.steps) k += st.tc ? 1 : 0;
  *n_tc = k;
  if (n_steps) *n_steps = P.built ? int32_t(P.steps.size()) : 0;
  return SQC_OK;
}

}  // extern "C"

namespace {
// Fresh subcircuit outputs for a fused attribution + merge (device
// pointers; FP64 if in_f64).
struct FusedSrc {
  const void* const* src;
  int in_f64;
};

// Selection of the largest bins after a reconstruction (sqc_top_bins'
// arguments).
struct SelectReq {
  int k;
  double threshold;
  unsigned long long* bins;
  double* probs;
  int* n_found;
};

sqc_status reconstruct_core(sqc_ctx* ctx, sqc_query_id qid, sqc_precision precision, void* out_bins,
                            sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob, void* stream,
                            const FusedSrc* fused, const SelectReq* sel = nullptr, bool* selected = nullptr);

// Select bins of query q's output (the body of sqc_top_bins).
sqc_status select_bins(sqc_ctx* ctx, Query& q, const void* probs, bool is_f64, uint64_t n, const SelectReq& r,
                       cudaStream_t s) {
  {
    // the first selection on a query allocates its workspace
    sqc_status st = ensure_select_work(ctx, &q);
    if (st != SQC_OK) return st;
  }
  StageScope scope(ctx, s, SQC_STAGE_SELECT);
  ctx->launches += 1;
  int* err = reinterpret_cast<int*>(static_cast<char*>(q.sel_mem) + q.sel_bytes - 64);
  const int rgrid = ctx->cfg.select_resident ? select_resident_grid() : 0;
  if (rgrid > 0 && select_resident_smem(n, is_f64, rgrid, nullptr))
    CK(launch_select_resident(q.sel_mem, rgrid, probs, is_f64, n, r.k, r.threshold, r.bins, r.probs, r.n_found, err,
                              s));
  else
    CK(launch_select_coop(q.sel_mem, q.sel_grid, probs, is_f64, n, r.k, r.threshold, r.bins, r.probs, r.n_found,
                          err, s));
  return SQC_OK;
}
}  // namespace

extern "C" {

SQC_API sqc_status sqc_reconstruct(sqc_ctx* ctx, sqc_query_id qid, sqc_precision precision, void* out_bins,
                                   sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob, void* stream) {
  return reconstruct_core(ctx, qid, precision, out_bins, out_dtype, out_bytes, total_prob, stream, nullptr);
}

}  // extern "C"

namespace {
// sqc_reconstruct_outputs (sel null) and sqc_reconstruct_select on fresh
// outputs.
sqc_status reconstruct_fresh(sqc_ctx* ctx, sqc_query_id qid, const void* const* probs, sqc_dtype dtype,
                             int probs_on_device, sqc_precision precision, void* out_bins, sqc_dtype out_dtype,
                             uint64_t out_bytes, double* total_prob, void* stream, const SelectReq* sel) {
  if (!ctx || !probs || !out_bins) return fail(ctx, SQC_EINVAL, "null argument");
  if (dtype != SQC_F32 && dtype != SQC_F64) return fail(ctx, SQC_EINVAL, "dtype must be F32 or F64");
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  auto cit = ctx->circuits.find(it->second->circuit);
  if (cit == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "circuit of the query was unloaded");
  Circuit& c = *cit->second;
  for (int i = 0; i < c.nC; ++i)
    if (!probs[i]) return fail(ctx, SQC_EINVAL, "probs[i] is null");
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // host inputs are staged back to back in the circuit's staging buffer
  // (as in an update)
  const size_t esz = dtype == SQC_F64 ? 8 : 4;
  std::vector<const void*> src(c.nC);
  if (probs_on_device < 0 || probs_on_device > 2) return fail(ctx, SQC_EINVAL, "probs_on_device must be 0, 1 or 2");
  if (probs_on_device == 1) {
    for (int i = 0; i < c.nC; ++i) src[i] = probs[i];
  } else if (probs_on_device == 2) {
    // host memory the device reads in place (pinned and mapped): the
    // attribution reads the kept states straight from it, no staging copy
    for (int i = 0; i < c.nC; ++i) {
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, probs[i]) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
          !pa.devicePointer) {
        cudaGetLastError();
        return fail(ctx, SQC_EINVAL, "probs[i] is not host memory mapped for the device (probs_on_device == 2)");
      }
      src[i] = pa.devicePointer;
    }
  } else {
    const sqc_status st = stage_host_inputs(ctx, c, probs, esz, s, &src);
    if (st != SQC_OK) return st;
  }
  const FusedSrc fs{src.data(), dtype == SQC_F64};
  sqc_status st =
      reconstruct_core(ctx, qid, precision, out_bins, out_dtype, out_bytes, total_prob, stream, &fs, sel);
  if (st == SQC_OK && probs_on_device == 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) CK(cudaStreamSynchronize(s));
  }
  return st;
}

// Checks of sqc_top_bins' arguments shared by sqc_reconstruct_select.
sqc_status check_select_args(sqc_ctx* ctx, int32_t k, double threshold, const void* bins_out, const void* probs_out,
                             const void* n_found) {
  if (k < 1 || k > kSelectMaxK) return fail(ctx, SQC_ESHAPE, "k must be in [1, 4096]");
  if (!bins_out || !probs_out || !n_found) return fail(ctx, SQC_EINVAL, "null argument");
  if (std::isnan(threshold)) return fail(ctx, SQC_EINVAL, "threshold is NaN");
  return SQC_OK;
}
}  // namespace

extern "C" {

SQC_API sqc_status sqc_reconstruct_outputs(sqc_ctx* ctx, sqc_query_id qid, const void* const* probs,
                                           sqc_dtype dtype, int probs_on_device, sqc_precision precision,
                                           void* out_bins, sqc_dtype out_dtype, uint64_t out_bytes,
                                           double* total_prob, void* stream) {
  return reconstruct_fresh(ctx, qid, probs, dtype, probs_on_device, precision, out_bins, out_dtype, out_bytes,
                           total_prob, stream, nullptr);
}

SQC_API sqc_status sqc_reconstruct_select(sqc_ctx* ctx, sqc_query_id qid, const void* const* probs,
                                          sqc_dtype dtype, int probs_on_device, sqc_precision precision,
                                          void* out_bins, sqc_dtype out_dtype, uint64_t out_bytes,
                                          double* total_prob, int32_t k, double threshold, uint64_t* bins_out,
                                          double* probs_out, int32_t* n_found, void* stream) {
  if (!ctx) return SQC_EINVAL;
  {
    const sqc_status st = check_select_args(ctx, k, threshold, bins_out, probs_out, n_found);
    if (st != SQC_OK) return st;
  }
  const SelectReq r{k, threshold, reinterpret_cast<unsigned long long*>(bins_out), probs_out, n_found};
  if (probs)
    return reconstruct_fresh(ctx, qid, probs, dtype, probs_on_device, precision, out_bins, out_dtype, out_bytes,
                             total_prob, stream, &r);
  return reconstruct_core(ctx, qid, precision, out_bins, out_dtype, out_bytes, total_prob, stream, nullptr, &r);
}

SQC_API sqc_status sqc_query_fused_select(sqc_ctx* ctx, sqc_query_id qid, int32_t* n_steps) {
  if (!ctx || !n_steps) return fail(ctx, SQC_EINVAL, "null argument");
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  const Query& q = *it->second;
  const Plan& P = q.plans[SQC_PREC_FP32];
  *n_steps = 0;
  if (!P.built || !P.tail_ok || !ctx->cfg.fused_select || !ctx->cfg.select_resident) return SQC_OK;
  DeviceGuard g(ctx->device);
  const int rgrid = select_resident_grid();
  if (rgrid > 0 && select_tail_smem(uint64_t(q.out_elems), P.tail, rgrid, nullptr)) *n_steps = P.tail.n_pre + 1;
  return SQC_OK;
}

}  // extern "C"

namespace {
sqc_status reconstruct_stages(sqc_ctx* ctx, sqc_query_id qid, sqc_precision precision, void* out_bins,
                              sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob, void* stream,
                              const FusedSrc* fused, const SelectReq* sel, bool* selected);

// A reconstruction, then (sel) the selection of its largest bins: in one
// launch with the contraction steps when the plan allows it, else as
// sqc_top_bins on the written bins.
sqc_status reconstruct_core(sqc_ctx* ctx, sqc_query_id qid, sqc_precision precision, void* out_bins,
                            sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob, void* stream,
                            const FusedSrc* fused, const SelectReq* sel, bool* selected) {
  bool done = false;
  sqc_status st = reconstruct_stages(ctx, qid, precision, out_bins, out_dtype, out_bytes, total_prob, stream, fused,
                                     sel, &done);
  if (st == SQC_OK && sel && !done) {
    Query& q = *ctx->queries.find(qid)->second;
    PdlScope pdl(ctx->cfg.pdl != 0);
    st = select_bins(ctx, q, out_bins, out_dtype == SQC_F64, uint64_t(q.out_elems), *sel,
                     static_cast<cudaStream_t>(stream));
  }
  if (selected) *selected = done;
  return st;
}

sqc_status reconstruct_stages(sqc_ctx* ctx, sqc_query_id qid, sqc_precision precision, void* out_bins,
                              sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob, void* stream,
                              const FusedSrc* fused, const SelectReq* sel, bool* selected) {
  if (!ctx || !out_bins) return fail(ctx, SQC_EINVAL, "null argument");
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  Query& q = *it->second;
  auto cit = ctx->circuits.find(q.circuit);
  if (cit == ctx->circuits.end()) return fail(ctx, SQC_ENOTFOUND, "circuit of the query was unloaded");
  const Circuit& c = *cit->second;
  if (out_dtype != SQC_F32 && out_dtype != SQC_F64) return fail(ctx, SQC_EINVAL, "out_dtype must be F32 or F64");
  if (precision != SQC_PREC_FP32 && precision != SQC_PREC_SPLIT_BF16)
    return fail(ctx, SQC_EINVAL, "precision must be SQC_PREC_FP32 or SQC_PREC_SPLIT_BF16");
  const uint64_t need = uint64_t(q.out_elems) * (out_dtype == SQC_F64 ? 8 : 4);
  if (out_bytes < need)
    return fail(ctx, SQC_ESHAPE, "out_bytes " + std::to_string(out_bytes) + " < " + std::to_string(need));
  DeviceGuard g(ctx->device);
  PdlScope pdl(ctx->cfg.pdl != 0);
  Plan& P = q.plans[precision];
  if (!P.built) {
    // the first split-BF16 call on a query plans that precision (allocates)
    sqc_status st = build_plan(ctx, c, &q, precision == SQC_PREC_SPLIT_BF16, &P);
    if (st != SQC_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int out_kind = out_dtype == SQC_F64 ? OUT_F64 : OUT_F32;
  const double alpha = std::ldexp(1.0, -c.K);

  // fresh outputs: attribution fused into the merge replaces the merge launch
  std::vector<AttrMergeLaunch> am;
  std::vector<int64_t> am_blocks;
  std::vector<int> am_smem;
  if (fused) {
    std::string why;
    if (!build_attr_merge(c, q, P, fused->src, fused->in_f64, out_bins, out_kind, alpha, &am, &am_blocks, &am_smem,
                          &why))
      return fail(ctx, SQC_EINVAL, "sqc_reconstruct_outputs: " + why);
  }
  auto run_merge = [&](const MergeDesc* descs, int nd) -> sqc_status {
    StageScope scope(ctx, s, SQC_STAGE_MERGE);
    if (fused) {
      for (size_t j = 0; j < am.size(); ++j) {
        CK(launch_attr_merge(am[j], am_blocks[j], am_smem[j], s));
        ctx->launches += 1;
      }
      return SQC_OK;
    }
    CK(launch_merge_blocks(descs, nd, P.merge_blocks, s));
    ctx->launches += 1;
    return SQC_OK;
  };

  if (sel && ctx->cfg.fused_select && precision == SQC_PREC_FP32 && out_kind == OUT_F32 && P.tail_ok &&
      ctx->cfg.select_resident) {
    const int rgrid = select_resident_grid();
    const uint64_t n = uint64_t(q.out_elems);
    if (rgrid > 0 && select_tail_smem(n, P.tail, rgrid, nullptr)) {
      // merges, then the contraction steps, the bins and their selection in
      // one cooperative launch
      sqc_status st = ensure_select_work(ctx, &q);
      if (st != SQC_OK) return st;
      st = run_merge(P.merge_dev, int(P.merge_host.size()));
      if (st != SQC_OK) return st;
      TailArgs T = P.tail;
      T.alpha = float(alpha);
      T.P = static_cast<float*>(out_bins);
      T.total = total_prob;
      int* err = reinterpret_cast<int*>(static_cast<char*>(q.sel_mem) + q.sel_bytes - 64);
      StageScope scope(ctx, s, SQC_STAGE_SELECT);
      CK(launch_select_tail(q.sel_mem, rgrid, T, n, sel->k, sel->threshold, sel->bins, sel->probs, sel->n_found,
                            err, s));
      ctx->launches += 1;
      *selected = true;
      return SQC_OK;
    }
  }

  if (!fused && precision == SQC_PREC_FP32 && ctx->cfg.fused_query && P.n_slices == 1 && !P.steps.empty()) {
    // the merge and every contraction step in ONE persistent launch: merge
    // blocks and step tiles form a dependency-ordered work list, each item
    // waiting only for the tensors it reads (the batched level's kernel
    // with one query); the same bins as the per-step launches below
    std::unique_ptr<Batch>& sb = q.solo[out_kind];
    if (!sb) {
      Query* qp = &q;
      sqc_status st = build_batch(ctx, 1, &qp, nullptr, out_kind, nullptr, true, &sb);
      if (st != SQC_OK) return st;
    }
    BatchLaunch L = sb->L;
    L.out = out_bins;
    L.total = total_prob;
    StageScope scope(ctx, s, SQC_STAGE_CONTRACT);
    CK(launch_batch(L, sb->grid, s));
    ctx->launches += 1;
    return SQC_OK;
  }

  if (P.steps.empty()) {
    // one subcircuit: the merge writes the bins directly
    if (!fused) {
      MergeDesc d = P.merge_host[0];
      d.dst = out_bins;
      d.kind = out_kind;
      d.alpha = alpha;
      CK(cudaMemcpyAsync(P.merge_dev, &d, sizeof(MergeDesc), cudaMemcpyHostToDevice, s));
    }
    {
      const sqc_status ms = run_merge(P.merge_dev, int(P.merge_host.size()));
      if (ms != SQC_OK) return ms;
    }
    if (total_prob) {
      StageScope scope(ctx, s, SQC_STAGE_FINAL);
      CK(launch_sum(out_bins, out_dtype == SQC_F64, uint64_t(q.out_elems), P.partials, P.counter, total_prob, s));
      ctx->launches += 1;
    }
    return SQC_OK;
  }
  // first-level slices (Section 6.3): every slice runs the whole merge and
  // contraction over the unsliced edges and adds its bins into the output
  const int nCm = int(P.merge_host.size());
  for (int64_t sg = 0; sg < P.n_slices; ++sg) {
    {
      const sqc_status ms = run_merge(P.merge_dev + sg * nCm, nCm);
      if (ms != SQC_OK) return ms;
    }
    for (size_t si = 0; si < P.steps.size(); ++si) {
      const Step& st = P.steps[si];
      const bool last = int(si) == int(P.steps.size()) - 1;
      const Tensor& Z = P.tensors[st.z];
      void* C = last ? out_bins : Z.buf;
      const int kind = last ? out_kind : Z.kind;
      const bool sums_here = last && total_prob && P.n_slices == 1;
      StageScope scope(ctx, s, last ? SQC_STAGE_FINAL : SQC_STAGE_CONTRACT);
      if (st.tc) {
        GemmTcArgs a{};
        a.A = P.tensors[st.x].buf;
        a.B = P.tensors[st.y].buf;
        a.M = st.M;
        a.N = st.N;
        a.K = st.Kd;
        a.Mp = st.M;
        a.Np = st.N;
        a.Kp = st.Kp;
        a.rowmap = st.rowmap;
        a.colmap = st.colmap;
        a.C = C;
        a.kind = kind;
        a.plane_stride = last ? 0 : Z.plane_stride;
        a.alpha = last ? alpha : 1.0;
        // the cross-chunk FP64 sum (Section 6.3): same rule as the SIMT path
        a.chunk = (last && out_kind == OUT_F64 && c.K >= ctx->cfg.fp64_chunk_min_edges &&
                   st.Kd > ctx->cfg.chunk_terms)
                      ? ctx->cfg.chunk_terms
                      : 0;
        a.accumulate = last && sg > 0;
        a.partials = sums_here ? P.partials : nullptr;
        a.counter = P.counter;
        a.total = total_prob;
        a.err = P.err;
        a.contig16 = st.contig16;
        a.pairs = ctx->cfg.tc_pairs;
        a.wait_ns = wait_ns(ctx);
        CK(launch_gemm_tc(a, s));
      } else {
        GemmArgs a{};
        a.A = static_cast<const float*>(P.tensors[st.x].buf);
        a.B = static_cast<const float*>(P.tensors[st.y].buf);
        a.M = st.M;
        a.N = st.N;
        a.K = st.Kd;
        a.rowmap = st.rowmap;
        a.colmap = st.colmap;
        a.vec4 = st.vec4;
        a.C = C;
        a.kind = kind;
        a.plane_stride = last ? 0 : Z.plane_stride;
        if (last) {
          a.alpha = alpha;
          a.chunk = (out_kind == OUT_F64 && c.K >= ctx->cfg.fp64_chunk_min_edges)
                        ? std::min<int64_t>(ctx->cfg.chunk_terms, st.Kd < 16 ? 16 : st.Kd)
                        : 0;
          a.accumulate = sg > 0;
          a.partials = sums_here ? P.partials : nullptr;
          a.counter = P.counter;
          a.total = total_prob;
        } else {
          a.alpha = 1.0;
          a.chunk = 0;
        }
        CK(launch_gemm_simt(a, s));
      }
      ctx->launches += 1;
    }
  }
  if (total_prob && P.n_slices > 1) {
    StageScope scope(ctx, s, SQC_STAGE_FINAL);
    CK(launch_sum(out_bins, out_dtype == SQC_F64, uint64_t(q.out_elems), P.partials, P.counter, total_prob, s));
    ctx->launches += 1;
  }
  return SQC_OK;
}

}  // namespace

extern "C" {

SQC_API sqc_status sqc_top_bins(sqc_ctx* ctx, sqc_query_id qid, const void* probs, sqc_dtype dtype, uint64_t n,
                                int32_t k, double threshold, uint64_t* bins_out, double* probs_out, int32_t* n_found,
                                void* stream) {
  if (!ctx) return SQC_EINVAL;
  if (k < 1 || k > kSelectMaxK) return fail(ctx, SQC_ESHAPE, "k must be in [1, 4096]");
  if (!probs || !bins_out || !probs_out || !n_found) return fail(ctx, SQC_EINVAL, "null argument");
  if (dtype != SQC_F32 && dtype != SQC_F64) return fail(ctx, SQC_EINVAL, "dtype must be F32 or F64");
  if (std::isnan(threshold)) return fail(ctx, SQC_EINVAL, "threshold is NaN");
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  DeviceGuard g(ctx->device);
  PdlScope pdl(ctx->cfg.pdl != 0);
  const SelectReq r{k, threshold, reinterpret_cast<unsigned long long*>(bins_out), probs_out, n_found};
  return select_bins(ctx, *it->second, probs, dtype == SQC_F64, n, r, static_cast<cudaStream_t>(stream));
}

SQC_API sqc_status sqc_batch_create(sqc_ctx* ctx, int32_t n, const sqc_query_id* qs, void* const* outs,
                                    sqc_dtype out_dtype, double* totals, sqc_precision precision,
                                    sqc_batch_id* out_b) {
  if (!ctx || !qs || !outs || !out_b || n < 1) return fail(ctx, SQC_EINVAL, "batch: null argument or n < 1");
  if (out_dtype != SQC_F32 && out_dtype != SQC_F64) return fail(ctx, SQC_EINVAL, "out_dtype must be F32 or F64");
  if (precision != SQC_PREC_FP32 && precision != SQC_PREC_SPLIT_BF16)
    return fail(ctx, SQC_EINVAL, "precision must be SQC_PREC_FP32 or SQC_PREC_SPLIT_BF16");
  DeviceGuard g(ctx->device);
  std::vector<Query*> qv(n);
  for (int j = 0; j < n; ++j) {
    auto it = ctx->queries.find(qs[j]);
    if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "batch: unknown query");
    qv[j] = it->second.get();
  }
  std::unique_ptr<Batch> B;
  sqc_status st =
      build_batch(ctx, n, qv.data(), outs, out_dtype == SQC_F64 ? OUT_F64 : OUT_F32, totals, false, &B, precision);
  if (st != SQC_OK) return st;
  B->queries.assign(qs, qs + n);
  const int64_t id = ctx->next_id++;
  ctx->batches[id] = std::move(B);
  *out_b = id;
  return SQC_OK;
}

SQC_API sqc_status sqc_batch_run(sqc_ctx* ctx, sqc_batch_id b, void* stream) {
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->batches.find(b);
  if (it == ctx->batches.end()) return fail(ctx, SQC_ENOTFOUND, "unknown batch");
  DeviceGuard g(ctx->device);
  PdlScope pdl(ctx->cfg.pdl != 0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StageScope scope(ctx, s, SQC_STAGE_CONTRACT);
  const Batch& B = *it->second;
  for (size_t j = 0; j < B.phases.size(); ++j) {
    if (B.phases[j].n_items > 0) {
      CK(launch_batch(B.phases[j], B.phase_grid[j], s));
      ctx->launches += 1;
    }
    for (const GemmTcArgs& a : B.tc[j]) {
      CK(launch_gemm_tc(a, s));
      ctx->launches += 1;
    }
  }
  return SQC_OK;
}

SQC_API sqc_status sqc_batch_status(sqc_ctx* ctx, sqc_batch_id b) {
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->batches.find(b);
  if (it == ctx->batches.end()) return fail(ctx, SQC_ENOTFOUND, "unknown batch");
  DeviceGuard g(ctx->device);
  CK(cudaDeviceSynchronize());
  // every phase's flag and every tensor-core step's flag (cleared once read)
  std::vector<int*> flags;
  for (const BatchLaunch& L : it->second->phases) flags.push_back(L.err);
  for (const auto& ph : it->second->tc)
    for (const GemmTcArgs& a : ph)
      if (a.err && std::find(flags.begin(), flags.end(), a.err) == flags.end()) flags.push_back(a.err);
  bool any = false;
  for (int* f : flags) {
    int err = 0;
    CK(cudaMemcpy(&err, f, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      any = true;
      const int zero = 0;
      CK(cudaMemcpy(f, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  if (any) return fail(ctx, SQC_ETIMEOUT, "batch: a bounded device wait gave up");
  return SQC_OK;
}

SQC_API sqc_status sqc_batch_inject_stall(sqc_ctx* ctx, sqc_batch_id b, int32_t on) {
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->batches.find(b);
  if (it == ctx->batches.end()) return fail(ctx, SQC_ENOTFOUND, "unknown batch");
  Batch& B = *it->second;
  if (B.expected.empty()) return fail(ctx, SQC_EINVAL, "batch has no intermediate tensor to stall");
  DeviceGuard g(ctx->device);
  std::vector<unsigned> e = B.expected;
  if (on) e.back() += 1u;        // one completion more than its producers will ever deliver
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(const_cast<unsigned*>(B.L.expected), e.data(), sizeof(unsigned) * e.size(),
                cudaMemcpyHostToDevice));
  return SQC_OK;
}

SQC_API sqc_status sqc_batch_release(sqc_ctx* ctx, sqc_batch_id b) {
  if (!ctx) return SQC_EINVAL;
  auto it = ctx->batches.find(b);
  if (it == ctx->batches.end()) return fail(ctx, SQC_ENOTFOUND, "unknown batch");
  DeviceGuard g(ctx->device);
  if (!ctx->async_alloc) cudaDeviceSynchronize();
  dev_free(ctx, it->second->work, it->second->work_bytes);
  ctx->batches.erase(it);
  return SQC_OK;
}

}  // extern "C"

namespace {
// The batched launch of n queries (their current plans) under every tile
// policy: mean ms per launch into ms[kBatchPolicies], the fastest into
// *best_policy; leaves ctx->batch_policy as it found it.
sqc_status batch_autotune_tiles(sqc_ctx* ctx, int32_t n, const sqc_query_id* qs, void* const* outs,
                                sqc_dtype out_dtype, double* totals, int32_t reps, int32_t* best_policy, float* ms) {
  const int saved = ctx->batch_policy;
  int best = -1;
  float best_ms = 0.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  const cudaError_t ee = cudaEventCreate(&e1);
  if (ee != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, ee, "batch autotune events");
  }
  sqc_status st = SQC_OK;
  for (int p = 0; p < kBatchPolicies && st == SQC_OK; ++p) {
    ctx->batch_policy = p;
    sqc_batch_id b = 0;
    st = sqc_batch_create(ctx, n, qs, outs, out_dtype, totals, SQC_PREC_FP32, &b);
    if (st != SQC_OK) break;
    st = sqc_batch_run(ctx, b, nullptr);                       // warm-up
    cudaError_t e = cudaSuccess;
    if (st == SQC_OK) e = cudaEventRecord(e0, nullptr);
    for (int r = 0; r < reps && st == SQC_OK && e == cudaSuccess; ++r) st = sqc_batch_run(ctx, b, nullptr);
    if (st == SQC_OK && e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
    if (st == SQC_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (st == SQC_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (st == SQC_OK) st = sqc_batch_status(ctx, b);
    const sqc_status rs = sqc_batch_release(ctx, b);
    if (st == SQC_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "batch autotune timing");
    if (st == SQC_OK) st = rs;
    if (st != SQC_OK) break;
    t /= float(reps);
    if (ms) ms[p] = t;
    if (best < 0 || t < best_ms) { best = p; best_ms = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->batch_policy = saved;
  if (st == SQC_OK) *best_policy = best;
  return st;
}
}  // namespace

extern "C" {

SQC_API sqc_status sqc_batch_autotune(sqc_ctx* ctx, int32_t n, const sqc_query_id* qs, void* const* outs,
                                      sqc_dtype out_dtype, double* totals, int32_t reps, int32_t* best_policy,
                                      int32_t* best_order, float* ms) {
  if (!ctx || !best_policy || !best_order || reps < 1 || n < 1 || !qs)
    return fail(ctx, SQC_EINVAL, "batch autotune: null argument, n < 1 or reps < 1");
  DeviceGuard g(ctx->device);
  std::vector<Query*> qv(n);
  for (int j = 0; j < n; ++j) {
    auto it = ctx->queries.find(qs[j]);
    if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "batch autotune: unknown query");
    qv[j] = it->second.get();
  }
  const int saved = ctx->batch_policy;
  int best = -1, best_o = SQC_ORDER_GREEDY;
  float best_ms = 0.f;
  sqc_status st = SQC_OK;
  for (int o = 0; o < 2 && st == SQC_OK; ++o) {
    for (Query* q : qv)
      if (st == SQC_OK && (q->plans[SQC_PREC_FP32].order != o || !q->plans[SQC_PREC_FP32].built)) st = replan(ctx, *q, o);
    if (st != SQC_OK) break;
    int32_t pol = -1;
    float t3[kBatchPolicies] = {0.f, 0.f, 0.f};
    st = batch_autotune_tiles(ctx, n, qs, outs, out_dtype, totals, reps, &pol, t3);
    if (st != SQC_OK) break;
    for (int p = 0; p < kBatchPolicies; ++p) {
      if (ms) ms[o * kBatchPolicies + p] = t3[p];
      if (best < 0 || t3[p] < best_ms) { best = p; best_ms = t3[p]; best_o = o; }
    }
  }
  if (st == SQC_OK) {
    for (Query* q : qv)
      if (st == SQC_OK && q->plans[SQC_PREC_FP32].order != best_o) st = replan(ctx, *q, best_o);
  }
  ctx->batch_policy = st == SQC_OK ? best : saved;
  if (st == SQC_OK) {
    // the outputs and totals end as the chosen order and policy write them
    sqc_batch_id b = 0;
    st = sqc_batch_create(ctx, n, qs, outs, out_dtype, totals, SQC_PREC_FP32, &b);
    if (st == SQC_OK) {
      st = sqc_batch_run(ctx, b, nullptr);
      if (st == SQC_OK) st = sqc_batch_status(ctx, b);
      const sqc_status rs = sqc_batch_release(ctx, b);
      if (st == SQC_OK) st = rs;
    }
    if (st != SQC_OK) ctx->batch_policy = saved;
  }
  if (st == SQC_OK) {
    *best_policy = best;
    *best_order = best_o;
  }
  return st;
}


SQC_API sqc_status sqc_query_autotune(sqc_ctx* ctx, sqc_query_id qid, sqc_precision precision, void* out_bins,
                                      sqc_dtype out_dtype, uint64_t out_bytes, int32_t reps, int32_t* best_order,
                                      float* ms) {
  if (!ctx || !best_order || !out_bins || reps < 1)
    return fail(ctx, SQC_EINVAL, "query autotune: null argument or reps < 1");
  auto it = ctx->queries.find(qid);
  if (it == ctx->queries.end()) return fail(ctx, SQC_ENOTFOUND, "unknown query");
  Query& q = *it->second;
  DeviceGuard g(ctx->device);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  const cudaError_t ee = cudaEventCreate(&e1);
  if (ee != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, ee, "query autotune events");
  }
  const int orders[2] = {SQC_ORDER_GREEDY, SQC_ORDER_MIN_MULT};
  float t_of[2] = {0.f, 0.f};
  int planned[2] = {-1, -1};          // the order each candidate's plan actually followed
  sqc_status st = SQC_OK;
  for (int j = 0; j < 2 && st == SQC_OK; ++j) {
    st = replan(ctx, q, orders[j]);
    if (st != SQC_OK) break;
    planned[j] = q.plans[SQC_PREC_FP32].order;
    if (j == 1 && planned[1] != SQC_ORDER_MIN_MULT) {   // too many subcircuits: the same greedy plan
      t_of[1] = t_of[0];
      break;
    }
    st = sqc_reconstruct(ctx, qid, precision, out_bins, out_dtype, out_bytes, nullptr, nullptr);   // warm-up
    cudaError_t e = cudaSuccess;
    if (st == SQC_OK) e = cudaEventRecord(e0, nullptr);
    for (int r = 0; r < reps && st == SQC_OK && e == cudaSuccess; ++r)
      st = sqc_reconstruct(ctx, qid, precision, out_bins, out_dtype, out_bytes, nullptr, nullptr);
    if (st == SQC_OK && e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
    if (st == SQC_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (st == SQC_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t_of[j], e0, e1);
    if (st == SQC_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "query autotune timing");
    t_of[j] /= float(reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SQC_OK) return st;
  const int best = (planned[1] == SQC_ORDER_MIN_MULT && t_of[1] < t_of[0]) ? SQC_ORDER_MIN_MULT : SQC_ORDER_GREEDY;
  if (ms) {
    ms[0] = t_of[0];
    ms[1] = t_of[1];
  }
  if (q.plans[SQC_PREC_FP32].order != best || q.order != best) st = replan(ctx, q, best);
  if (st == SQC_OK) *best_order = best;
  return st;
}

SQC_API sqc_status sqc_plan_preview(const sqc_graph* graph, const int8_t* roles, const sqc_config* cfg,
                                    int32_t* n_steps, int64_t* steps, int32_t cap_steps, int32_t* n_sliced,
                                    int32_t* sliced, int32_t cap_sliced, double* flops, uint64_t* work_bytes,
                                    char* err, int32_t err_len) {
  std::string msg;
  sqc_status st = SQC_OK;
  {
    // a context holding only the configuration: planning is host work and
    // nothing here touches a device
    sqc_ctx ctx;
    sqc_default_config(&ctx.cfg);
    if (cfg) ctx.cfg = *cfg;
    t_err_sink = &msg;
    if (!graph || !roles || !n_steps || !n_sliced) st = fail(nullptr, SQC_EINVAL, "null argument");
    if (st == SQC_OK) {
      const std::string ce = config_error(ctx.cfg);
      if (!ce.empty()) st = fail(nullptr, SQC_EINVAL, ce);
    }
    Circuit c;
    if (st == SQC_OK) st = build_circuit(&ctx, graph, &c);
    c.A.assign(c.nC, nullptr);          // no resident tensors: the plan only records their addresses
    t_err_sink = nullptr;
    sqc::QueryDraft* d = nullptr;
    if (st == SQC_OK) st = sqc::query_draft(&ctx, 0, &c, roles, &d, &msg);
    if (st == SQC_OK) {
      const Plan& P = d->q->plans[SQC_PREC_FP32];
      *n_steps = int32_t(P.steps.size());
      for (size_t s = 0; steps && s < P.steps.size() && int32_t(s) < cap_steps; ++s) {
        steps[3 * s] = P.steps[s].M;
        steps[3 * s + 1] = P.steps[s].N;
        steps[3 * s + 2] = P.steps[s].Kd;
      }
      *n_sliced = int32_t(P.sliced.size());
      for (size_t j = 0; sliced && j < P.sliced.size() && int32_t(j) < cap_sliced; ++j) sliced[j] = P.sliced[j];
      if (flops) *flops = P.flops;
      if (work_bytes) *work_bytes = P.work_bytes;
    }
    sqc::query_draft_free(d);
  }
  if (err && err_len > 0) {
    const size_t n = std::min(msg.size(), size_t(err_len - 1));
    std::memcpy(err, msg.data(), n);
    err[n] = '\0';
  }
  return st;
}

SQC_API sqc_status sqc_top_bins_noalloc(int device, const void* probs, sqc_dtype dtype, uint64_t n, int32_t k,
                                        double threshold, uint64_t* bins_out, double* probs_out, int32_t* n_found,
                                        void* stream) {
  if (k < 1 || k > kSelectMaxK)
    return fail(nullptr, SQC_ESHAPE, "k must be in [1, 4096]: the static scratch holds at most 4096 selected bins");
  if (!probs || !bins_out || !probs_out || !n_found) return fail(nullptr, SQC_EINVAL, "null argument");
  if (dtype != SQC_F32 && dtype != SQC_F64) return fail(nullptr, SQC_EINVAL, "dtype must be F32 or F64");
  if (std::isnan(threshold)) return fail(nullptr, SQC_EINVAL, "threshold is NaN");
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return fail(nullptr, e != cudaSuccess ? SQC_ECUDA : SQC_EINVAL, "no such CUDA device");
  }
  DeviceGuard g(device);
  e = launch_select_static(device, probs, dtype == SQC_F64, n, k, threshold,
                           reinterpret_cast<unsigned long long*>(bins_out), probs_out, n_found,
                           static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, SQC_ECUDA, std::string("selection: ") + cudaGetErrorString(e));
  return SQC_OK;
}

SQC_API sqc_status sqc_profile_enable(sqc_ctx* ctx, int on) {
  if (!ctx) return SQC_EINVAL;
  DeviceGuard g(ctx->device);
  for (auto& m : ctx->marks) {
    cudaEventSynchronize(m.stop);
    ctx->event_pool.push_back(m.start);
    ctx->event_pool.push_back(m.stop);
  }
  ctx->marks.clear();
  ctx->launches = 0;
  ctx->prof = on != 0;
  ctx->prof_keep = on == 2;
  return SQC_OK;
}

SQC_API sqc_status sqc_profile_read(sqc_ctx* ctx, double* ms, int64_t* calls, int64_t* launches) {
  if (!ctx) return SQC_EINVAL;
  DeviceGuard g(ctx->device);
  double acc[SQC_STAGE_COUNT] = {0};
  int64_t cnt[SQC_STAGE_COUNT] = {0};
  for (auto& m : ctx->marks) {
    cudaError_t e = cudaEventSynchronize(m.stop);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, m.start, m.stop);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventElapsedTime");
    if (m.stage >= 0 && m.stage < SQC_STAGE_COUNT) {
      acc[m.stage] += t;
      cnt[m.stage] += 1;
    }
    if (!ctx->prof_keep) {
      ctx->event_pool.push_back(m.start);
      ctx->event_pool.push_back(m.stop);
    }
  }
  if (!ctx->prof_keep) ctx->marks.clear();
  if (ms) for (int i = 0; i < SQC_STAGE_COUNT; ++i) ms[i] = acc[i];
  if (calls) for (int i = 0; i < SQC_STAGE_COUNT; ++i) calls[i] = cnt[i];
  if (launches) *launches = ctx->launches;
  if (!ctx->prof_keep) ctx->launches = 0;
  return SQC_OK;
}

}  // extern "C"
