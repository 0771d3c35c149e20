// kc_serve.cu -- the serving loop of libkc.so (kc_serve_* in kclique.h).
//
// Continuous batching over the batched-count path: submitted requests wait
// in one FIFO queue; each of `lanes` worker threads owns a private context
// (device scratch, streams) and, whenever it is free, takes every queued
// request that fits the batch size and the device-memory admission cap and
// enumerates them together (run_batch: the counts of one batch in one set of
// tier launches, the listings -- count and checksum -- in another).
// Arrivals during a batch go to the next free lane, so batches of different
// lanes overlap on the GPU.  Host-side code only; the enumeration itself runs
// in the kernels of kc_enum.cu.
//
// Device memory under the cap: admitted requests may reserve half of it (the
// bytes of a request bound everything a batch allocates for it: root lists,
// the heavy-root arena and task queue of its width tiers, an inline graph's
// upload); the lanes' own scratch (memo tables and per-warp state, planned
// within a budget of cap / (2 lanes) each) takes the other half.  A lane that
// holds more than its share after a batch releases its scratch.
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
  uint32_t mode = KC_SERVE_COUNT;
  BatchQuery q{};             // resident graph; q.n = 0 when answered without enumeration
  bool host_answer = false;   // result known at submission (counting k <= 2; k - 1 above every out-degree)
  uint64_t host_count = 0;
  uint32_t tier_roots[kTiers] = {};  // vertices per width tier (bound of the split path's scratch)
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
  std::vector<double> lat_enum_ms;                     // requests the GPU enumerated
  uint64_t lane_budget = 0;                            // scratch bytes each lane may keep between batches
  std::vector<uint64_t> lane_scratch;                  // scratch each lane holds (updated after its batches)
};

namespace {

// Device bytes a request holds while admitted: its root lists in the batch
// (two words per vertex), its query record, the heavy-root arena and task
// queue of the width tiers its roots fall in (tiers of two words and more,
// by the graph's tier histogram) and, for an inline graph, its upload
// footprint (input copy, peel work arrays, DAG and order arrays).  An inline
// graph's tiers are bounded before its upload from its degrees.
uint64_t request_bytes(uint32_t n, uint64_t nnz, bool inline_csr, const uint32_t* tier_roots) {
  uint64_t b = 8ull * n + 128;
  for (int t = 1; t < kTiers; t++) {
    const uint64_t W = 1ull << t;
    const uint64_t roots = tier_roots[t];
    const uint64_t unit = ((16 + 128 * W + 128 * W * W + 32 * W + 15) / 16) * 16;  // one published root
    b += roots * (unit + 8 * 32 * W);                                            // and its tasks
  }
  // upload of an inline graph: input copy, canonicalisation, peel and sort
  // work arrays, and the graph's own order and DAG arrays
  if (inline_csr) b += 96ull * n + 24ull * nnz + 1024;
  return b;
}

uint64_t lanes_scratch(const Server* S) {
  uint64_t t = 0;
  for (uint64_t x : S->lane_scratch) t += x;
  return t;
}

// Records a finished request (lock held).
void finish(Server* S, const ServeReq& r, uint64_t count, uint64_t checksum, int status, uint32_t batch,
            uint64_t t_start, uint64_t t_done, bool enumerated) {
  kc_serve_result res{};
  res.count = count;
  res.checksum = checksum;
  res.mode = r.mode;
  res.enumerated = enumerated ? 1u : 0u;
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
  if (enumerated) S->lat_enum_ms.push_back((double)(t_done - r.t_submit) * 1e-6);
}

// Frees every scratch buffer of a lane (between its batches).
void release_scratch(kc_ctx* lane) {
  for (auto& sc : lane->scratch)
    if (sc.p) cudaFreeAsync(sc.p, lane->own_stream);
  cudaStreamSynchronize(lane->own_stream);
  lane->scratch.clear();
  lane->scratch_bytes = 0;
}

void lane_loop(Server* S, int li) {
  kc_ctx* lane = S->lanes[li];
  cudaSetDevice(lane->device);
  std::vector<ServeReq> batch;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      const uint64_t rcap = S->opts.mem_cap_bytes / 2;  // the requests' half of the cap
      S->cv_work.wait(lk, [&] {
        return S->stopping || (!S->queue.empty() && (S->queue.front().bytes > rcap ||
                                                     S->reserved + S->queue.front().bytes <= rcap));
      });
      if (S->stopping) return;
      // admit in arrival order while the batch and the memory cap allow
      while (!S->queue.empty() && batch.size() < S->opts.max_batch) {
        ServeReq& r = S->queue.front();
        if (r.bytes > rcap) {  // can never fit
          const uint64_t t = now_ns();
          finish(S, r, 0, 0, KC_E_OOM, 1, t, t, false);
          S->queue.pop_front();
          S->cv_done.notify_all();
          continue;
        }
        if (S->reserved + r.bytes > rcap) break;
        S->reserved += r.bytes;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved + S->lane_budget * S->lanes.size());
        batch.push_back(std::move(r));
        S->queue.pop_front();
      }
    }
    if (batch.empty()) continue;
    const uint64_t t_start = now_ns();
    // inline graphs: upload on this lane
    std::vector<kc_graph> uploaded(batch.size(), 0);
    std::vector<const DevGraph*> graph(batch.size(), nullptr);
    for (size_t i = 0; i < batch.size(); i++) {
      ServeReq& r = batch[i];
      if (!r.inline_csr) continue;
      kc_graph h = 0;
      r.status = kc_upload(lane, r.n, r.rowptr.data(), r.col.empty() ? nullptr : r.col.data(),
                           KC_HOST_PTRS | r.flags, &h, nullptr);
      if (r.status != KC_OK) continue;
      uploaded[i] = h;
      const DevGraph& g = lane->graphs[h];
      graph[i] = &g;
      r.q = BatchQuery{g.orow, g.ocol, g.vert, g.n, r.k};
      if ((uint64_t)r.k - 1 > g.max_out && r.k >= 2) {
        r.host_answer = true;
        r.host_count = 0;
      } else if (r.mode == KC_SERVE_COUNT && r.k <= 2) {
        r.host_answer = true;
        r.host_count = r.k == 1 ? g.n : g.m;
      }
    }
    // counts in one batch, listings (count and checksum) in another, k = 1 listings one by one
    std::vector<BatchQuery> qc, ql;
    std::vector<size_t> slot(batch.size(), SIZE_MAX);
    std::vector<uint64_t> single_cnt(batch.size(), 0), single_sum(batch.size(), 0);
    int st1 = KC_OK;
    for (size_t i = 0; i < batch.size(); i++) {
      ServeReq& r = batch[i];
      if (r.status != KC_OK || r.host_answer) continue;
      if (r.mode == KC_SERVE_LIST && r.k == 1) {
        const DevGraph* g = graph[i];
        DevGraph tmp{};
        if (!g) {  // resident graph: its arrays, read only
          tmp.n = r.q.n;
          tmp.vert = const_cast<uint32_t*>(r.q.vert);
          g = &tmp;
        }
        EnumArgs ea;
        ea.k = 1;
        ea.mode = 1;
        ea.root_lo = 0;
        ea.root_hi = g->n;
        const int st = run_enum(lane, *g, ea, lane->own_stream);
        if (st != KC_OK) st1 = st;
        single_cnt[i] = lane->h_acc[kAccCount];
        single_sum[i] = lane->h_acc[kAccChecksum];
        continue;
      }
      if (r.mode == KC_SERVE_LIST) {
        slot[i] = ql.size();
        ql.push_back(r.q);
      } else {
        slot[i] = qc.size();
        qc.push_back(r.q);
      }
    }
    std::vector<uint64_t> ccounts(std::max<size_t>(qc.size(), 1), 0);
    std::vector<uint64_t> lcounts(std::max<size_t>(ql.size(), 1), 0), lsums(std::max<size_t>(ql.size(), 1), 0);
    int stc = KC_OK, stl = KC_OK;
    if (!qc.empty()) stc = run_batch(lane, qc.data(), (uint32_t)qc.size(), S->memo, S->prune, ccounts.data(),
                                     lane->own_stream);
    if (!ql.empty()) stl = run_batch(lane, ql.data(), (uint32_t)ql.size(), S->memo, S->prune, lcounts.data(),
                                     lane->own_stream, lsums.data());
    for (size_t i = 0; i < batch.size(); i++)
      if (uploaded[i]) kc_free_graph(lane, uploaded[i]);
    const uint64_t t_done = now_ns();
    if (lane->scratch_bytes > S->lane_budget) release_scratch(lane);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (size_t i = 0; i < batch.size(); i++) {
        const ServeReq& r = batch[i];
        int rs = r.status;
        uint64_t c = r.host_count, h = 0;
        bool enumerated = false;
        if (rs == KC_OK && !r.host_answer) {
          enumerated = true;
          if (r.mode == KC_SERVE_LIST && r.k == 1) {
            rs = st1;
            c = single_cnt[i];
            h = single_sum[i];
          } else if (r.mode == KC_SERVE_LIST) {
            rs = stl;
            c = stl == KC_OK ? lcounts[slot[i]] : 0;
            h = stl == KC_OK ? lsums[slot[i]] : 0;
          } else {
            rs = stc;
            c = stc == KC_OK ? ccounts[slot[i]] : 0;
          }
          if (rs != KC_OK) c = h = 0;
        }
        finish(S, r, c, h, rs, (uint32_t)batch.size(), t_start, t_done, enumerated);
        S->reserved -= r.bytes;
      }
      S->lane_scratch[li] = lane->scratch_bytes;
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
    finish(S, r, r.host_count, 0, KC_OK, 1, r.t_submit, r.t_submit, false);
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
      finish(S, S->queue.front(), 0, 0, KC_E_BUSY, 0, t, t, false);
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
  // each lane plans its memo tables (half) and the per-warp state of the two
  // widest tiers (a quarter each) within its share of the lanes' half of the cap
  S->lane_budget = o.mem_cap_bytes / 2 / o.lanes;
  kc_opts lo = ctx->opts;
  const uint64_t memo_default = 1ull << 30;
  lo.memo_bytes = std::min<uint64_t>(lo.memo_bytes ? lo.memo_bytes : memo_default, S->lane_budget / 2);
  for (uint32_t i = 0; i < o.lanes; i++) {
    kc_ctx* l = nullptr;
    const int st = kc_create(&l, ctx->device, &lo);
    if (st != KC_OK) {
      for (kc_ctx* x : S->lanes) kc_destroy(x);
      delete S;
      return st;
    }
    l->gstate_budget = std::max<uint64_t>(1, S->lane_budget / 4);
    S->lanes.push_back(l);
  }
  S->lane_scratch.assign(o.lanes, 0);
  S->running = true;
  ctx->server = S;
  for (uint32_t i = 0; i < o.lanes; i++) S->workers.emplace_back(lane_loop, S, (int)i);
  return KC_OK;
}

int kc_serve_submit(kc_ctx* ctx, kc_graph g, uint32_t k, uint32_t mode, uint64_t* ticket) {
  if (!ctx || !ticket || k == 0 || (mode != KC_SERVE_COUNT && mode != KC_SERVE_LIST)) return KC_E_INVALID_ARG;
  if (k > KC_MAX_K) return KC_E_UNSUPPORTED;
  if (!ctx->server || !ctx->server->running) return KC_E_BUSY;
  auto it = ctx->graphs.find(g);  // read-only while serving
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  const DevGraph& dg = it->second;
  ServeReq r;
  r.k = k;
  r.mode = mode;
  r.q = BatchQuery{dg.orow, dg.ocol, dg.vert, dg.n, k};
  if (k >= 2 && (uint64_t)k - 1 > dg.max_out) {  // no k-clique: count 0, checksum 0
    r.host_answer = true;
    r.host_count = 0;
  } else if (mode == KC_SERVE_COUNT && k <= 2) {
    r.host_answer = true;
    r.host_count = k == 1 ? dg.n : dg.m;
  }
  r.bytes = request_bytes(dg.n, 0, false, dg.tier_roots);
  return enqueue(ctx, std::move(r), ticket);
}

int kc_serve_submit_csr(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr, const uint32_t* col, uint32_t flags,
                        uint32_t k, uint32_t mode, uint64_t* ticket) {
  if (!ctx || !ticket || !rowptr || k == 0 || (mode != KC_SERVE_COUNT && mode != KC_SERVE_LIST))
    return KC_E_INVALID_ARG;
  if (flags & ~(uint32_t)(KC_HOST_PTRS | KC_CANONICALIZE)) return KC_E_INVALID_ARG;
  if (k > KC_MAX_K || n == 0xFFFFFFFFu) return KC_E_UNSUPPORTED;
  if (!ctx->server || !ctx->server->running) return KC_E_BUSY;
  const uint64_t nnz = rowptr[n];
  if (nnz > 0 && !col) return KC_E_INVALID_ARG;
  ServeReq r;
  r.k = k;
  r.mode = mode;
  r.inline_csr = true;
  r.n = n;
  r.flags = flags & KC_CANONICALIZE;
  r.rowptr.assign(rowptr, rowptr + (size_t)n + 1);
  if (nnz) r.col.assign(col, col + nnz);
  // tiers before the upload: a vertex's out-degree is at most its degree and at
  // most the degeneracy, which is below sqrt(2m) + 1 (m <= nnz edges)
  uint32_t tiers[kTiers] = {};
  uint64_t dmax = 1;
  while (dmax * dmax <= 2 * nnz) dmax++;
  for (uint32_t v = 0; v < n; v++) {
    const uint64_t d = std::min<uint64_t>(2 * (rowptr[v + 1] - rowptr[v]), dmax);  // raw rows may be one-sided
    if (!d) continue;
    const uint64_t words = (d + 31) >> 5;
    int t = 0;
    while (t < kTiers - 1 && (1ull << t) < words) t++;
    tiers[t]++;
  }
  r.bytes = request_bytes(n, nnz, true, tiers);
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
  if (!S->lat_enum_ms.empty()) {
    std::vector<double> v = S->lat_enum_ms;
    auto pct = [&](double p) {
      const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + i, v.end());
      return v[i];
    };
    out->p50_enum_ms = pct(0.50);
    out->p99_enum_ms = pct(0.99);
  }
  out->lane_scratch_bytes = lanes_scratch(S);
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
