// Serving loop: continuous batching of zoom queries.
//
// Clients submit queries (a loaded circuit + qubit roles) from any thread;
// one server thread owns the context and repeatedly
//   1. retires launches whose completion event has fired (their requests are
//      done; their plans and batch state are freed, stream-ordered),
//   2. copies the retired requests' bins to host memory and frees their
//      device outputs at once (so memory held for results never blocks
//      admission), and forgets the requests clients have collected,
//   3. for every idle launch slot (a non-blocking stream), admits waiting
//      requests in arrival order as long as their plans and outputs fit the
//      context's HBM budget (a plan that does not fit leaves the request
//      waiting: admission by footprint), and launches all admitted requests
//      of the slot as one persistent batch -- or, in plain mode, one
//      reconstruction per request -- then records the slot's event.
// Requests that arrive while launches are on the GPU are admitted into the
// next idle slot, so several batches overlap on the device.  Allocations,
// uploads and frees are stream-ordered on the slot's stream: the loop never
// synchronises the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sqc.h"
#include "internal.h"

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { WAITING = 0, RUNNING = 1, DONE = 2, FAILED = 3, COLLECTED = 4 };

struct Request {
  sqc_circuit_id circuit = 0;
  std::vector<int8_t> roles;
  double t_submit = 0, t_launch = 0, t_done = 0;
  int state = WAITING;
  sqc_status status = SQC_OK;
  sqc_query_id q = 0;
  int32_t n_active = 0;
  void* out = nullptr;
  size_t out_bytes = 0;
  std::vector<float> host;   // the bins, copied out when the launch retires
  int slot = -1;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  bool has_batch = false;
  sqc_batch_id b = 0;
  std::vector<int64_t> tickets;
};

}  // namespace

struct sqc_server {
  sqc_ctx* ctx = nullptr;
  sqc_server_config cfg{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<int64_t> submitted;   // guarded by mu
  std::map<int64_t, Request> reqs; // guarded by mu
  std::vector<int64_t> to_free;    // collected outputs, guarded by mu
  int64_t next_ticket = 1;
  std::vector<Slot> slots;         // server thread only
  std::deque<int64_t> waiting;     // server thread only
  int64_t launches = 0, admitted = 0, busy_refusals = 0;
  size_t planner_threads = 1;      // host planning threads per dispatch
  std::string err;

  void loop();
  bool retire();
  bool dispatch(Slot& sl, int idx);
};

bool sqc_server::retire() {
  bool any = false;
  for (size_t i = 0; i < slots.size(); ++i) {
    Slot& sl = slots[i];
    if (!sl.busy || cudaEventQuery(sl.ev) != cudaSuccess) continue;
    const double t = now_us();
    sqc::ctx_set_alloc_stream(ctx, sl.s);
    if (sl.has_batch) sqc_batch_release(ctx, sl.b);
    // copy every result to the host right away so that its HBM is free for
    // the next admissions whether or not the client has collected it yet
    for (int64_t tk : sl.tickets) {
      Request* r;
      {
        std::lock_guard<std::mutex> lk(mu);
        r = &reqs[tk];
      }
      std::vector<float> host(r->out_bytes / 4);
      const cudaError_t e = cudaMemcpy(host.data(), r->out, r->out_bytes, cudaMemcpyDeviceToHost);
      sqc::ctx_free(ctx, r->out, r->out_bytes);
      sqc_release_query(ctx, r->q);
      std::lock_guard<std::mutex> lk(mu);
      r->out = nullptr;
      r->host.swap(host);
      r->t_done = t;
      r->state = e == cudaSuccess ? DONE : FAILED;
      r->status = e == cudaSuccess ? SQC_OK : SQC_ECUDA;
    }
    sl.busy = false;
    sl.has_batch = false;
    sl.tickets.clear();
    any = true;
  }
  cv.notify_all();
  return any;
}

bool sqc_server::dispatch(Slot& sl, int idx) {
  if (waiting.empty()) return false;
  sqc::ctx_set_alloc_stream(ctx, sl.s);
  std::vector<int64_t> taken;
  std::vector<sqc_query_id> qs;
  std::vector<void*> outs;
  std::vector<int32_t> nas;
  const int limit = cfg.max_batch > 0 ? cfg.max_batch : 256;
  // the host part of the next waiting requests' plans, on planner threads
  // (it reads only the configuration and the circuits); the device part
  // and the admission below stay on this thread, in arrival order
  const size_t nd = std::min(waiting.size(), size_t(limit));
  std::vector<int64_t> cand(waiting.begin(), waiting.begin() + std::ptrdiff_t(nd));
  std::vector<Request*> rp(nd);
  {
    std::lock_guard<std::mutex> lk(mu);
    for (size_t j = 0; j < nd; ++j) rp[j] = &reqs[cand[j]];
  }
  std::vector<const void*> circ(nd);
  for (size_t j = 0; j < nd; ++j) circ[j] = sqc::ctx_circuit(ctx, rp[j]->circuit);
  std::vector<sqc::QueryDraft*> drafts(nd, nullptr);
  std::vector<sqc_status> dst(nd, SQC_OK);
  std::vector<std::string> derr(nd);
  auto draft = [&](size_t j0, size_t step) {
    for (size_t j = j0; j < nd; j += step) {
      if (!circ[j]) {
        dst[j] = SQC_ENOTFOUND;
        continue;
      }
      dst[j] = sqc::query_draft(ctx, rp[j]->circuit, circ[j], rp[j]->roles.data(), &drafts[j], &derr[j]);
    }
  };
  const size_t nt = nd >= 4 ? std::min<size_t>(nd / 2, planner_threads) : 1;
  if (nt <= 1) {
    draft(0, 1);
  } else {
    std::vector<std::thread> ts;
    for (size_t t = 1; t < nt; ++t) ts.emplace_back(draft, t, nt);
    draft(0, nt);
    for (std::thread& t : ts) t.join();
  }
  size_t j = 0;
  for (; j < nd && int(taken.size()) < limit; ++j) {
    const int64_t tk = cand[j];
    Request* r = rp[j];
    sqc_query_id q = 0;
    int32_t na = 0;
    // nothing else holds request memory: a request that does not fit now
    // never will
    bool alone = taken.empty();
    for (const Slot& o : slots) alone = alone && !o.busy;
    sqc_status st = dst[j];
    if (st == SQC_OK) {
      st = sqc::query_commit(ctx, drafts[j], &q, &na);   // consumes the draft
      drafts[j] = nullptr;
    }
    void* out = nullptr;
    const size_t ob = size_t(4) << na;
    if (st == SQC_OK) {
      st = sqc::ctx_alloc(ctx, &out, ob);
      if (st != SQC_OK) sqc_release_query(ctx, q);
    }
    if (st == SQC_EBUSY && !alone) {
      ++busy_refusals;
      break;                                   // not enough HBM now: wait for launches to retire
    }
    waiting.pop_front();
    std::lock_guard<std::mutex> lk(mu);
    if (st != SQC_OK) {
      r->state = FAILED;
      r->status = st;
      continue;
    }
    r->q = q;
    r->n_active = na;
    r->out = out;
    r->out_bytes = ob;
    r->slot = idx;
    taken.push_back(tk);
    qs.push_back(q);
    outs.push_back(out);
    nas.push_back(na);
  }
  // drafts of requests left waiting are dropped (planned again later)
  for (; j < nd; ++j)
    if (drafts[j]) sqc::query_draft_free(drafts[j]);
  if (taken.empty()) return false;
  const double t = now_us();
  sqc_status st = SQC_OK;
  if (cfg.plain) {
    for (size_t j = 0; j < qs.size() && st == SQC_OK; ++j)
      st = sqc_reconstruct(ctx, qs[j], SQC_PREC_FP32, outs[j], SQC_F32, size_t(4) << nas[j], nullptr, sl.s);
  } else {
    // the batch's own state is allocated last: if it does not fit, hand the
    // most recently admitted requests back to the queue and retry
    for (;;) {
      st = sqc_batch_create(ctx, int32_t(qs.size()), qs.data(), outs.data(), SQC_F32, nullptr, SQC_PREC_FP32, &sl.b);
      if (st != SQC_EBUSY || qs.size() == 1) break;
      ++busy_refusals;
      sqc::ctx_free(ctx, outs.back(), size_t(4) << nas.back());
      sqc_release_query(ctx, qs.back());
      {
        std::lock_guard<std::mutex> lk(mu);
        Request& r = reqs[taken.back()];
        r.out = nullptr;
        r.q = 0;
        r.slot = -1;
      }
      waiting.push_front(taken.back());
      taken.pop_back();
      qs.pop_back();
      outs.pop_back();
      nas.pop_back();
    }
    if (st == SQC_OK) {
      sl.has_batch = true;
      st = sqc_batch_run(ctx, sl.b, sl.s);
    }
  }
  if (st == SQC_OK && cudaEventRecord(sl.ev, sl.s) != cudaSuccess) st = SQC_ECUDA;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int64_t tk : taken) {
      Request& r = reqs[tk];
      r.t_launch = t;
      r.state = st == SQC_OK ? RUNNING : FAILED;
      r.status = st;
    }
  }
  if (st != SQC_OK) {
    err = sqc_last_error(ctx);
    cudaStreamSynchronize(sl.s);
    if (sl.has_batch) sqc_batch_release(ctx, sl.b);
    for (sqc_query_id q : qs) sqc_release_query(ctx, q);
    sl.has_batch = false;
    return false;
  }
  sl.busy = true;
  sl.tickets = taken;
  ++launches;
  admitted += int64_t(taken.size());
  return true;
}

void sqc_server::loop() {
  cudaSetDevice(sqc::ctx_device(ctx));
  for (;;) {
    bool stopping;
    std::vector<int64_t> frees;
    {
      std::unique_lock<std::mutex> lk(mu);
      while (!submitted.empty()) {
        waiting.push_back(submitted.front());
        submitted.pop_front();
      }
      frees.swap(to_free);
      stopping = stop;
    }
    bool progress = retire();
    if (stopping && !waiting.empty()) {
      // shutting down: requests not yet admitted are cancelled
      std::lock_guard<std::mutex> lk(mu);
      for (int64_t tk : waiting) {
        reqs[tk].state = FAILED;
        reqs[tk].status = SQC_EBUSY;
      }
      waiting.clear();
      cv.notify_all();
    }
    if (!frees.empty()) {
      std::lock_guard<std::mutex> lk(mu);
      for (int64_t tk : frees) reqs.erase(tk);     // collected: forget the request
      progress = true;
    }
    for (size_t i = 0; i < slots.size(); ++i)
      if (!slots[i].busy) progress |= dispatch(slots[i], int(i));
    bool idle = waiting.empty();
    for (const Slot& sl : slots) idle = idle && !sl.busy;
    if (stopping && idle) break;
    if (!progress) {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::microseconds(idle ? 500 : 20),
                  [&] { return stop || !submitted.empty() || !to_free.empty(); });
    }
  }
  sqc::ctx_set_alloc_stream(ctx, nullptr);
}

extern "C" {

SQC_API void sqc_server_default_config(sqc_server_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_batch = 64;
  cfg->n_streams = 4;
  cfg->plain = 0;
}

SQC_API sqc_status sqc_server_create(sqc_ctx* ctx, const sqc_server_config* cfg, sqc_server** out) {
  if (!ctx || !out) return SQC_EINVAL;
  *out = nullptr;
  auto srv = new sqc_server();
  srv->ctx = ctx;
  sqc_server_default_config(&srv->cfg);
  if (cfg) srv->cfg = *cfg;
  if (srv->cfg.n_streams < 1 || srv->cfg.n_streams > 32 || srv->cfg.max_batch < 1) {
    delete srv;
    return sqc::ctx_fail(ctx, SQC_EINVAL, "server: n_streams in [1, 32] and max_batch >= 1");
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(sqc::ctx_device(ctx));
  srv->slots.resize(srv->cfg.n_streams);
  for (Slot& sl : srv->slots) {
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaSetDevice(prev);
      delete srv;
      return sqc::ctx_fail(ctx, SQC_ECUDA, "server: stream or event creation failed");
    }
  }
  cudaSetDevice(prev);
  {
    const unsigned hc = std::thread::hardware_concurrency();
    srv->planner_threads = hc >= 4 ? std::min<size_t>(8, hc / 2) : 1;
  }
  // the plain baseline keeps one launch per stage for every request
  if (srv->cfg.plain) sqc::ctx_set_fused(ctx, false);
  srv->th = std::thread([srv] { srv->loop(); });
  *out = srv;
  return SQC_OK;
}

SQC_API sqc_status sqc_server_submit(sqc_server* srv, sqc_circuit_id circuit, const int8_t* roles, int32_t n_qubits,
                                     int64_t* ticket) {
  if (!srv || !roles || !ticket || n_qubits < 1) return SQC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return SQC_EINVAL;
  const int64_t tk = srv->next_ticket++;
  Request& r = srv->reqs[tk];
  r.circuit = circuit;
  r.roles.assign(roles, roles + n_qubits);
  r.t_submit = now_us();
  srv->submitted.push_back(tk);
  *ticket = tk;
  srv->cv.notify_all();
  return SQC_OK;
}

SQC_API sqc_status sqc_server_poll(sqc_server* srv, int64_t ticket, int32_t* state, double* latency_us,
                                   int32_t* n_active) {
  if (!srv || !state) return SQC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return SQC_ENOTFOUND;
  const Request& r = it->second;
  *state = r.state;
  if (latency_us) *latency_us = r.state == DONE ? r.t_done - r.t_submit : -1.0;
  if (n_active) *n_active = r.n_active;
  return r.state == FAILED ? r.status : SQC_OK;
}

SQC_API sqc_status sqc_server_result(sqc_server* srv, int64_t ticket, float* host_out, uint64_t capacity) {
  if (!srv || !host_out) return SQC_EINVAL;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return SQC_ENOTFOUND;
    Request& r = it->second;
    if (r.state != DONE) return r.state == FAILED ? r.status : SQC_EBUSY;
    if (capacity < (uint64_t(1) << r.n_active)) return SQC_ESHAPE;
    std::memcpy(host_out, r.host.data(), r.host.size() * sizeof(float));
    r.host.clear();
    r.host.shrink_to_fit();
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->reqs[ticket].state = COLLECTED;
  srv->to_free.push_back(ticket);
  srv->cv.notify_all();
  return SQC_OK;
}

SQC_API sqc_status sqc_server_drain(sqc_server* srv, double timeout_s) {
  if (!srv) return SQC_EINVAL;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    bool pending = !srv->submitted.empty();
    for (auto& kv : srv->reqs) pending = pending || kv.second.state == WAITING || kv.second.state == RUNNING;
    if (!pending) return SQC_OK;
    if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout) return SQC_ETIMEOUT;
  }
}

SQC_API sqc_status sqc_server_stats(sqc_server* srv, int64_t* launches, int64_t* admitted, int64_t* busy_refusals) {
  if (!srv) return SQC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (launches) *launches = srv->launches;
  if (admitted) *admitted = srv->admitted;
  if (busy_refusals) *busy_refusals = srv->busy_refusals;
  return SQC_OK;
}

SQC_API void sqc_server_destroy(sqc_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  if (srv->th.joinable()) srv->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(sqc::ctx_device(srv->ctx));
  for (Slot& sl : srv->slots) cudaStreamSynchronize(sl.s);
  for (auto& kv : srv->reqs)
    if (kv.second.out) sqc::ctx_free(srv->ctx, kv.second.out, kv.second.out_bytes);
  sqc::ctx_set_alloc_stream(srv->ctx, nullptr);
  cudaDeviceSynchronize();
  for (Slot& sl : srv->slots) {
    cudaEventDestroy(sl.ev);
    cudaStreamDestroy(sl.s);
  }
  cudaSetDevice(prev);
  delete srv;
}

}  // extern "C"
