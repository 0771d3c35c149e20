// kc_serve.cu -- the serving loop of libkc.so (kc_serve_* in kclique.h).
//
// Continuous batching over the batched-count path: submitted requests wait
// in one FIFO queue; each of `lanes` worker threads owns a private context
// (device scratch, streams) and, whenever it is free, takes every queued
// request that fits the batch size and the device-memory admission cap and
// counts them together (run_batch).  Arrivals during a batch go to the next
// free lane, so batches of different lanes overlap on the GPU.  Host-side
// code only; the counting itself runs in the kernels of kc_enum.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "kc_internal.cuh"

namespace kc {

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct ServeReq {
  uint64_t ticket = 0;
  uint32_t k = 0;
  BatchQuery q{};             // resident graph; q.n = 0 when answered without enumeration
  bool host_answer = false;   // count known at submission (k <= 2, or k - 1 above every out-degree)
  uint64_t host_count = 0;
  bool inline_csr = false;    // graph given as a host CSR, uploaded by the lane
  uint32_t n = 0, flags = 0;
  std::vector<uint64_t> rowptr;
  std::vector<uint32_t> col;
  uint64_t bytes = 0;         // device bytes reserved while admitted
  uint64_t t_submit = 0;
  int status = KC_OK;
};

}  // namespace

struct Server {
  kc_ctx* owner = nullptr;
  kc_serve_opts opts{};
  bool memo = true, prune = true;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeReq> queue;
  std::unordered_set<uint64_t> live;                   // submitted, not yet complete
  std::unordered_map<uint64_t, kc_serve_result> done;  // complete, not yet collected
  uint64_t next_ticket = 1;
  uint64_t reserved = 0, peak_reserved = 0;
  bool running = false, stopping = false;
  std::vector<kc_ctx*> lanes;
  std::vector<std::thread> workers;
  // statistics since start
  uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_reqs = 0, cliques = 0;
  uint64_t first_submit = 0, last_done = 0;
  std::vector<double> lat_ms;
};

namespace {

// Device bytes a request holds while admitted: its root lists in the batch
// (two words per vertex) and, for an inline graph, its upload footprint
// (input copy, peel work arrays, DAG and order arrays).
uint64_t request_bytes(uint32_t n, uint64_t nnz, bool inline_csr) {
  uint64_t b = 8ull * n + 64;
  if (inline_csr) b += 48ull * n + 8ull * nnz + 64;
  return b;
}

// Records a finished request (lock held).
void finish(Server* S, const ServeReq& r, uint64_t count, int status, uint32_t batch, uint64_t t_start,
            uint64_t t_done) {
  kc_serve_result res{};
  res.count = count;
  res.status = status;
  res.batch_size = batch;
  res.t_submit_ns = r.t_submit;
  res.t_start_ns = t_start;
  res.t_done_ns = t_done;
  S->done[r.ticket] = res;
  S->live.erase(r.ticket);
  S->completed++;
  if (status != KC_OK) S->failed++;
  else S->cliques += count;
  S->last_done = std::max(S->last_done, t_done);
  S->lat_ms.push_back((double)(t_done - r.t_submit) * 1e-6);
}

void lane_loop(Server* S, int li) {
  kc_ctx* lane = S->lanes[li];
  cudaSetDevice(lane->device);
  std::vector<ServeReq> batch;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      const uint64_t cap = S->opts.mem_cap_bytes;
      S->cv_work.wait(lk, [&] {
        return S->stopping || (!S->queue.empty() && (S->queue.front().bytes > cap ||
                                                     S->reserved + S->queue.front().bytes <= cap));
      });
      if (S->stopping) return;
      // admit in arrival order while the batch and the memory cap allow
      while (!S->queue.empty() && batch.size() < S->opts.max_batch) {
        ServeReq& r = S->queue.front();
        if (r.bytes > cap) {  // can never fit
          const uint64_t t = now_ns();
          finish(S, r, 0, KC_E_OOM, 1, t, t);
          S->queue.pop_front();
          S->cv_done.notify_all();
          continue;
        }
        if (S->reserved + r.bytes > cap) break;
        S->reserved += r.bytes;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
        batch.push_back(std::move(r));
        S->queue.pop_front();
      }
    }
    if (batch.empty()) continue;
    const uint64_t t_start = now_ns();
    // inline graphs: upload on this lane
    std::vector<kc_graph> uploaded(batch.size(), 0);
    for (size_t i = 0; i < batch.size(); i++) {
      ServeReq& r = batch[i];
      if (!r.inline_csr) continue;
      kc_graph h = 0;
      r.status = kc_upload(lane, r.n, r.rowptr.data(), r.col.empty() ? nullptr : r.col.data(),
                           KC_HOST_PTRS | r.flags, &h, nullptr);
      if (r.status != KC_OK) continue;
      uploaded[i] = h;
      const DevGraph& g = lane->graphs[h];
      r.q = BatchQuery{g.orow, g.ocol, g.vert, g.n, r.k};
      if (r.k == 1 || r.k == 2 || (uint64_t)r.k - 1 > g.max_out) {
        r.host_answer = true;
        r.host_count = r.k == 1 ? g.n : (r.k == 2 ? g.m : 0);
      }
    }
    std::vector<BatchQuery> qs;
    std::vector<size_t> slot(batch.size(), SIZE_MAX);
    for (size_t i = 0; i < batch.size(); i++) {
      if (batch[i].status != KC_OK || batch[i].host_answer) continue;
      slot[i] = qs.size();
      qs.push_back(batch[i].q);
    }
    std::vector<uint64_t> counts(std::max<size_t>(qs.size(), 1), 0);
    int st = KC_OK;
    if (!qs.empty()) st = run_batch(lane, qs.data(), (uint32_t)qs.size(), S->memo, S->prune, counts.data(),
                                    lane->own_stream);
    for (size_t i = 0; i < batch.size(); i++)
      if (uploaded[i]) kc_free_graph(lane, uploaded[i]);
    const uint64_t t_done = now_ns();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (size_t i = 0; i < batch.size(); i++) {
        const ServeReq& r = batch[i];
        int rs = r.status;
        uint64_t c = r.host_count;
        if (rs == KC_OK && !r.host_answer) {
          rs = st;
          c = st == KC_OK ? counts[slot[i]] : 0;
        }
        finish(S, r, c, rs, (uint32_t)batch.size(), t_start, t_done);
        S->reserved -= r.bytes;
      }
      S->batches++;
      S->batched_reqs += batch.size();
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();  // freed memory may admit what waits
  }
}

int enqueue(kc_ctx* ctx, ServeReq&& r, uint64_t* ticket) {
  Server* S = ctx->server;
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->running || S->stopping) return KC_E_BUSY;
  r.ticket = S->next_ticket++;
  r.t_submit = now_ns();
  if (S->submitted == 0) S->first_submit = r.t_submit;
  S->submitted++;
  S->live.insert(r.ticket);
  *ticket = r.ticket;
  if (r.host_answer) {
    finish(S, r, r.host_count, KC_OK, 1, r.t_submit, r.t_submit);
    S->cv_done.notify_all();
    return KC_OK;
  }
  S->queue.push_back(std::move(r));
  S->cv_work.notify_one();
  return KC_OK;
}

}  // namespace

void serve_shutdown(kc_ctx* ctx) {
  Server* S = ctx->server;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->running) return;
    S->stopping = true;
    const uint64_t t = now_ns();
    while (!S->queue.empty()) {
      finish(S, S->queue.front(), 0, KC_E_BUSY, 0, t, t);
      S->queue.pop_front();
    }
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& w : S->workers) w.join();
  S->workers.clear();
  for (kc_ctx* l : S->lanes) kc_destroy(l);
  S->lanes.clear();
  std::lock_guard<std::mutex> lk(S->mu);
  S->running = false;
  S->stopping = false;
}

void serve_release(kc_ctx* ctx) {
  serve_shutdown(ctx);
  delete ctx->server;
  ctx->server = nullptr;
}

}  // namespace kc

using namespace kc;

extern "C" {

int kc_serve_start(kc_ctx* ctx, const kc_serve_opts* opts) {
  if (!ctx) return KC_E_INVALID_ARG;
  if (ctx->server && ctx->server->running) return KC_E_BUSY;
  kc_serve_opts o{};
  if (opts) {
    if (opts->struct_size != 0 && opts->struct_size < sizeof(uint32_t)) return KC_E_INVALID_ARG;
    const size_t nb = opts->struct_size ? std::min<size_t>(opts->struct_size, sizeof(kc_serve_opts))
                                        : sizeof(kc_serve_opts);
    std::memcpy(&o, opts, nb);
  }
  o.struct_size = sizeof(kc_serve_opts);
  if (!o.lanes) o.lanes = 2;
  if (!o.max_batch) o.max_batch = 4096;
  if (!o.mem_cap_bytes) o.mem_cap_bytes = 64ull << 30;
  if (o.lanes > 16) return KC_E_INVALID_ARG;
  serve_release(ctx);  // results of an earlier run are dropped
  Server* S = new (std::nothrow) Server();
  if (!S) return KC_E_OOM;
  S->owner = ctx;
  S->opts = o;
  S->memo = ctx->opts.no_memo == 0;
  S->prune = ctx->opts.no_prune == 0;
  for (uint32_t i = 0; i < o.lanes; i++) {
    kc_ctx* l = nullptr;
    const int st = kc_create(&l, ctx->device, &ctx->opts);
    if (st != KC_OK) {
      for (kc_ctx* x : S->lanes) kc_destroy(x);
      delete S;
      return st;
    }
    S->lanes.push_back(l);
  }
  S->running = true;
  ctx->server = S;
  for (uint32_t i = 0; i < o.lanes; i++) S->workers.emplace_back(lane_loop, S, (int)i);
  return KC_OK;
}

int kc_serve_submit(kc_ctx* ctx, kc_graph g, uint32_t k, uint32_t mode, uint64_t* ticket) {
  if (!ctx || !ticket || k == 0 || mode != KC_SERVE_COUNT) return KC_E_INVALID_ARG;
  if (k > KC_MAX_K) return KC_E_UNSUPPORTED;
  if (!ctx->server || !ctx->server->running) return KC_E_BUSY;
  auto it = ctx->graphs.find(g);  // read-only while serving
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  const DevGraph& dg = it->second;
  ServeReq r;
  r.k = k;
  r.q = BatchQuery{dg.orow, dg.ocol, dg.vert, dg.n, k};
  if (k == 1 || k == 2 || (uint64_t)k - 1 > dg.max_out) {
    r.host_answer = true;
    r.host_count = k == 1 ? dg.n : (k == 2 ? dg.m : 0);
  }
  r.bytes = request_bytes(dg.n, 0, false);
  return enqueue(ctx, std::move(r), ticket);
}

int kc_serve_submit_csr(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr, const uint32_t* col, uint32_t flags,
                        uint32_t k, uint32_t mode, uint64_t* ticket) {
  if (!ctx || !ticket || !rowptr || k == 0 || mode != KC_SERVE_COUNT) return KC_E_INVALID_ARG;
  if (flags & ~(uint32_t)(KC_HOST_PTRS | KC_CANONICALIZE)) return KC_E_INVALID_ARG;
  if (k > KC_MAX_K || n == 0xFFFFFFFFu) return KC_E_UNSUPPORTED;
  if (!ctx->server || !ctx->server->running) return KC_E_BUSY;
  const uint64_t nnz = rowptr[n];
  if (nnz > 0 && !col) return KC_E_INVALID_ARG;
  ServeReq r;
  r.k = k;
  r.inline_csr = true;
  r.n = n;
  r.flags = flags & KC_CANONICALIZE;
  r.rowptr.assign(rowptr, rowptr + (size_t)n + 1);
  if (nnz) r.col.assign(col, col + nnz);
  r.bytes = request_bytes(n, nnz, true);
  return enqueue(ctx, std::move(r), ticket);
}

int kc_serve_poll(kc_ctx* ctx, uint64_t ticket, kc_serve_result* out) {
  if (!ctx || !out) return KC_E_INVALID_ARG;
  Server* S = ctx->server;
  if (!S) return KC_E_NOT_FOUND;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it != S->done.end()) {
    *out = it->second;
    S->done.erase(it);
    return KC_OK;
  }
  return S->live.count(ticket) ? KC_E_BUSY : KC_E_NOT_FOUND;
}

int kc_serve_wait(kc_ctx* ctx, uint64_t ticket, int64_t timeout_ms, kc_serve_result* out) {
  if (!ctx || !out) return KC_E_INVALID_ARG;
  Server* S = ctx->server;
  if (!S) return KC_E_NOT_FOUND;
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&] { return S->done.count(ticket) || !S->live.count(ticket); };
  if (timeout_ms < 0) S->cv_done.wait(lk, ready);
  else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  auto it = S->done.find(ticket);
  if (it != S->done.end()) {
    *out = it->second;
    S->done.erase(it);
    return KC_OK;
  }
  return S->live.count(ticket) ? KC_E_BUSY : KC_E_NOT_FOUND;
}

int kc_serve_stats_get(kc_ctx* ctx, kc_serve_stats* out) {
  if (!ctx || !out) return KC_E_INVALID_ARG;
  *out = kc_serve_stats{};
  Server* S = ctx->server;
  if (!S) return KC_OK;
  std::lock_guard<std::mutex> lk(S->mu);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->batches = S->batches;
  out->mean_batch = S->batches ? (double)S->batched_reqs / (double)S->batches : 0.0;
  out->peak_reserved_bytes = S->peak_reserved;
  if (!S->lat_ms.empty()) {
    std::vector<double> v = S->lat_ms;
    auto pct = [&](double p) {
      const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + i, v.end());
      return v[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
  }
  if (S->last_done > S->first_submit) {
    const double sec = (double)(S->last_done - S->first_submit) * 1e-9;
    out->req_per_s = (double)S->completed / sec;
    out->cliques_per_s = (double)S->cliques / sec;
  }
  return KC_OK;
}

int kc_serve_stop(kc_ctx* ctx) {
  if (!ctx) return KC_E_INVALID_ARG;
  if (!ctx->server || !ctx->server->running) return KC_E_NOT_FOUND;
  serve_shutdown(ctx);
  return KC_OK;
}

}  // extern "C"
