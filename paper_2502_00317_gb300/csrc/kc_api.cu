// kc_api.cu -- the extern "C" boundary of libkc.so (declared in include/kclique.h).
// Argument checks, context and graph bookkeeping, scratch buffers; every step
// of the path itself runs in the kernels of kc_prep.cu and kc_enum.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "kc_internal.cuh"

namespace kc {

int cuda_fail(kc_ctx* ctx, cudaError_t e, const char* what) {
  if (ctx) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? KC_E_OOM : KC_E_CUDA;
}

// Scratch buffers come from the stream-ordered allocator on the stream of the
// running call (ctx->cur_stream): a buffer that must grow is released after
// the work already queued on that stream (which every launch that used it
// was joined back into) instead of after a device-wide synchronisation, so
// contexts that share the GPU (serving lanes) never wait for one another.
int scratch_get(kc_ctx* ctx, int slot, size_t bytes, void** out) {
  if ((int)ctx->scratch.size() <= slot) ctx->scratch.resize(slot + 1);
  Scratch& sc = ctx->scratch[slot];
  if (bytes == 0) bytes = 16;
  if (sc.bytes < bytes) {
    cudaStream_t s = ctx->cur_stream ? ctx->cur_stream : ctx->own_stream;
    if (sc.p) {
      KC_CUDA(cudaFreeAsync(sc.p, s));
      ctx->scratch_bytes -= sc.bytes;
      sc.p = nullptr;
      sc.bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    KC_CUDA(cudaMallocAsync(&sc.p, want, s));
    sc.bytes = want;
    ctx->scratch_bytes += want;
    ctx->scratch_peak = std::max(ctx->scratch_peak, ctx->scratch_bytes);
  }
  *out = sc.p;
  return KC_OK;
}

// Graph arrays come from the stream-ordered allocator too.  Every call that
// read them synchronised its stream before returning, so they are released
// in order on `s` without a device-wide synchronisation.
static void free_graph(DevGraph& g, cudaStream_t s) {
  for (void* p : {(void*)g.core, (void*)g.rank, (void*)g.vert, (void*)g.orow, (void*)g.ocol})
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  g = DevGraph{};
}

// The stream of a call (the context's own when the caller passes NULL); it
// also orders the call's scratch allocations.
static cudaStream_t pick_stream(kc_ctx* ctx, void* stream) {
  ctx->cur_stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return ctx->cur_stream;
}

}  // namespace kc

using namespace kc;

extern "C" {

const char* kc_strerror(int st) {
  switch (st) {
    case KC_OK: return "KC_OK";
    case KC_E_INVALID_ARG: return "KC_E_INVALID_ARG";
    case KC_E_INVALID_GRAPH: return "KC_E_INVALID_GRAPH";
    case KC_E_OOM: return "KC_E_OOM";
    case KC_E_CAPACITY: return "KC_E_CAPACITY";
    case KC_E_DEVICE_TIMEOUT: return "KC_E_DEVICE_TIMEOUT";
    case KC_E_CUDA: return "KC_E_CUDA";
    case KC_E_BUSY: return "KC_E_BUSY";
    case KC_E_UNSUPPORTED: return "KC_E_UNSUPPORTED";
    case KC_E_NOT_FOUND: return "KC_E_NOT_FOUND";
    default: return "KC_E_UNKNOWN";
  }
}

const char* kc_last_error(kc_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int kc_create(kc_ctx** out, int device, const kc_opts* opts) {
  if (!out) return KC_E_INVALID_ARG;
  *out = nullptr;
  kc_ctx* ctx = new (std::nothrow) kc_ctx();
  if (!ctx) return KC_E_OOM;
  if (opts) {
    if (opts->struct_size != 0 && opts->struct_size < sizeof(uint32_t)) {
      delete ctx;
      return KC_E_INVALID_ARG;
    }
    size_t n = opts->struct_size ? std::min<size_t>(opts->struct_size, sizeof(kc_opts)) : sizeof(kc_opts);
    std::memcpy(&ctx->opts, opts, n);
  }
  ctx->opts.struct_size = sizeof(kc_opts);
  if (ctx->opts.decomposition != KC_NODE_PARALLEL && ctx->opts.decomposition != KC_EDGE_PARALLEL) {
    delete ctx;
    return KC_E_INVALID_ARG;
  }
  if (!ctx->opts.spin_limit) ctx->opts.spin_limit = 2000000000ull;  // 2 s, in nanoseconds
  ctx->device = device;
  auto fail = [&](cudaError_t e, const char* what) {
    int st = cuda_fail(ctx, e, what);
    kc_destroy(ctx);
    return st;
  };
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(e, "cudaSetDevice");
  cudaDeviceProp prop{};
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return fail(e, "cudaGetDeviceProperties");
  ctx->num_sms = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  for (const char* c = prop.name; *c; c++) ctx->gpu_name.push_back(*c == ' ' ? '_' : *c);
  tune_load(ctx);
  ctx->opts.tune_cache = nullptr;  // the caller's string need not outlive kc_create
  if ((e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(e, "cudaStreamCreate");
  for (int t = 0; t < kTiers; t++) {
    if ((e = cudaStreamCreateWithFlags(&ctx->tier_stream[t], cudaStreamNonBlocking)) != cudaSuccess)
      return fail(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&ctx->ev_join[t], cudaEventDisableTiming)) != cudaSuccess)
      return fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ctx->ev_tier0[t])) != cudaSuccess) return fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ctx->ev_tier1[t])) != cudaSuccess) return fail(e, "cudaEventCreate");
  }
  if ((e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e, "cudaEventCreate");
  for (auto& ev : ctx->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e, "cudaEventCreate");
  if ((e = cudaMalloc(&ctx->d_status, 64)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->d_acc, kAccSlots * sizeof(unsigned long long))) != cudaSuccess)
    return fail(e, "cudaMalloc");
  if ((e = cudaMallocHost(&ctx->h_acc, kAccSlots * sizeof(unsigned long long))) != cudaSuccess)
    return fail(e, "cudaMallocHost");
  cudaMemset(ctx->d_status, 0, 64);
  {
    // Pascal's triangle mod 2^64 (unsigned wrap-around is exact modular arithmetic)
    const size_t rows = KC_MAX_OUTDEG + 1, cols = KC_MAX_K + 1;
    std::vector<unsigned long long> tab(rows * cols, 0ull);
    for (size_t n = 0; n < rows; n++) {
      tab[n * cols] = 1ull;
      for (size_t j = 1; j < cols && j <= n; j++) tab[n * cols + j] = tab[(n - 1) * cols + j - 1] + tab[(n - 1) * cols + j];
    }
    if ((e = cudaMalloc(&ctx->d_binom, tab.size() * sizeof(unsigned long long))) != cudaSuccess)
      return fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(ctx->d_binom, tab.data(), tab.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return fail(e, "cudaMemcpy");
  }
  *out = ctx;
  return KC_OK;
}

int kc_destroy(kc_ctx* ctx) {
  if (!ctx) return KC_E_INVALID_ARG;
  serve_release(ctx);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->graphs) free_graph(kv.second, ctx->own_stream);
  ctx->graphs.clear();
  for (auto& sc : ctx->scratch)
    if (sc.p) cudaFreeAsync(sc.p, ctx->own_stream);
  if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
  ctx->scratch.clear();
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_acc) cudaFree(ctx->d_acc);
  if (ctx->d_binom) cudaFree(ctx->d_binom);
  if (ctx->h_acc) cudaFreeHost(ctx->h_acc);
  for (auto& ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  for (int t = 0; t < kTiers; t++) {
    if (ctx->ev_join[t]) cudaEventDestroy(ctx->ev_join[t]);
    if (ctx->ev_tier0[t]) cudaEventDestroy(ctx->ev_tier0[t]);
    if (ctx->ev_tier1[t]) cudaEventDestroy(ctx->ev_tier1[t]);
    if (ctx->tier_stream[t]) cudaStreamDestroy(ctx->tier_stream[t]);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
  return KC_OK;
}

int kc_upload(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr, const uint32_t* col, uint32_t flags, kc_graph* out,
              void* stream) {
  if (!ctx || !out || !rowptr) return KC_E_INVALID_ARG;
  const uint32_t where = flags & (KC_HOST_PTRS | KC_DEVICE_PTRS);
  if (where != KC_HOST_PTRS && where != KC_DEVICE_PTRS) return KC_E_INVALID_ARG;
  if (flags & ~(KC_HOST_PTRS | KC_DEVICE_PTRS | KC_CANONICALIZE)) return KC_E_INVALID_ARG;
  if (n == 0xFFFFFFFFu) return KC_E_UNSUPPORTED;
  *out = 0;
  KC_CUDA(cudaSetDevice(ctx->device));
  if ((flags & KC_HOST_PTRS) && rowptr[n] > 0 && !col) return KC_E_INVALID_ARG;
  if ((flags & KC_HOST_PTRS) && rowptr[0] != 0) return KC_E_INVALID_GRAPH;
  cudaStream_t s = pick_stream(ctx, stream);
  DevGraph g;
  int st = prep_graph(ctx, n, rowptr, col, flags, &g, s);
  if (st != KC_OK) {
    cudaStreamSynchronize(s);
    free_graph(g, s);
    return st;
  }
  uint32_t h = ctx->next_handle++;
  if (ctx->next_handle == 0) ctx->next_handle = 1;
  ctx->graphs[h] = g;
  *out = h;
  return KC_OK;
}

int kc_free_graph(kc_ctx* ctx, kc_graph h) {
  if (!ctx) return KC_E_INVALID_ARG;
  auto it = ctx->graphs.find(h);
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  KC_CUDA(cudaSetDevice(ctx->device));
  free_graph(it->second, ctx->own_stream);
  ctx->graphs.erase(it);
  return KC_OK;
}

int kc_graph_info_get(kc_ctx* ctx, kc_graph h, kc_graph_info* info) {
  if (!ctx || !info) return KC_E_INVALID_ARG;
  auto it = ctx->graphs.find(h);
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  const DevGraph& g = it->second;
  info->n = g.n;
  info->m = g.m;
  info->degeneracy = g.degeneracy;
  info->max_out_degree = g.max_out;
  info->peel_rounds = g.peel_rounds;
  return KC_OK;
}

int kc_export_dag(kc_ctx* ctx, kc_graph h, uint32_t* core, uint32_t* rank, uint64_t* orow, uint32_t* ocol) {
  if (!ctx) return KC_E_INVALID_ARG;
  auto it = ctx->graphs.find(h);
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  const DevGraph& g = it->second;
  KC_CUDA(cudaSetDevice(ctx->device));
  if (core && g.n) KC_CUDA(cudaMemcpy(core, g.core, (size_t)g.n * 4, cudaMemcpyDeviceToHost));
  if (rank && g.n) KC_CUDA(cudaMemcpy(rank, g.rank, (size_t)g.n * 4, cudaMemcpyDeviceToHost));
  if (orow) KC_CUDA(cudaMemcpy(orow, g.orow, ((size_t)g.n + 1) * 8, cudaMemcpyDeviceToHost));
  if (ocol && g.m) KC_CUDA(cudaMemcpy(ocol, g.ocol, (size_t)g.m * 4, cudaMemcpyDeviceToHost));
  return KC_OK;
}

static int enum_common(kc_ctx* ctx, kc_graph h, uint32_t k, int mode, uint32_t lo, uint32_t hi, uint32_t* d_buf,
                       uint64_t cap, uint64_t* written, uint64_t* total, uint64_t* checksum, void* stream) {
  auto it = ctx->graphs.find(h);
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  const DevGraph& g = it->second;
  if (k == 0) return KC_E_INVALID_ARG;
  if (k > KC_MAX_K) return KC_E_UNSUPPORTED;
  if (hi > g.n) hi = g.n;
  if (lo > hi) return KC_E_INVALID_ARG;
  KC_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, stream);
  ctx->last = kc_stats{};
  // no root has k-1 out-neighbours: nothing to enumerate
  if (k >= 2 && (uint64_t)k - 1 > g.max_out) {
    if (written) *written = 0;
    if (total) *total = 0;
    if (checksum) *checksum = 0;
    return KC_OK;
  }
  EnumArgs ea;
  ea.k = k;
  ea.mode = mode;
  ea.root_lo = lo;
  ea.root_hi = hi;
  ea.d_buf = d_buf;
  ea.cap = d_buf ? cap : 0;
  ea.memo = mode == 1 ? ctx->opts.no_memo == 0 : count_uses_memo(ctx, k);
  ea.prune = ctx->opts.no_prune == 0;
  KC_TRY(run_enum(ctx, g, ea, s));
  uint64_t tot = ctx->h_acc[kAccCount];
  if (total) *total = tot;
  if (checksum) *checksum = ctx->h_acc[kAccChecksum];
  uint64_t wr = std::min<uint64_t>(tot, ea.cap);
  if (written) *written = wr;
  if (mode == 1 && ea.cap > 0 && tot > ea.cap) return KC_E_CAPACITY;  // cap 0: total and checksum only
  return KC_OK;
}

int kc_count(kc_ctx* ctx, kc_graph h, uint32_t k, uint64_t* count, void* stream) {
  if (!ctx || !count) return KC_E_INVALID_ARG;
  auto it = ctx->graphs.find(h);
  if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
  if (k == 0) return KC_E_INVALID_ARG;
  if (k == 1) {
    ctx->last = kc_stats{};
    *count = it->second.n;
    return KC_OK;
  }
  if (k == 2) {
    ctx->last = kc_stats{};
    *count = it->second.m;
    return KC_OK;
  }
  if (ctx->opts.autotune && k <= KC_MAX_K && (uint64_t)k - 1 <= it->second.max_out) {
    KC_CUDA(cudaSetDevice(ctx->device));
    KC_TRY(tune_for_graph(ctx, it->second, k, pick_stream(ctx, stream)));
  }
  return enum_common(ctx, h, k, 0, 0, it->second.n, nullptr, 0, nullptr, count, nullptr, stream);
}

int kc_list(kc_ctx* ctx, kc_graph h, uint32_t k, uint32_t* d_buf, uint64_t cap, uint64_t* written, uint64_t* total,
            uint64_t* checksum, void* stream) {
  if (!ctx) return KC_E_INVALID_ARG;
  if (cap > 0 && !d_buf) return KC_E_INVALID_ARG;
  return enum_common(ctx, h, k, 1, 0, 0xFFFFFFFFu, d_buf, cap, written, total, checksum, stream);
}

int kc_list_range(kc_ctx* ctx, kc_graph h, uint32_t k, uint32_t root_lo, uint32_t root_hi, uint32_t* d_buf,
                  uint64_t cap, uint64_t* written, uint64_t* total, uint64_t* checksum, void* stream) {
  if (!ctx) return KC_E_INVALID_ARG;
  if (cap > 0 && !d_buf) return KC_E_INVALID_ARG;
  if (root_lo > root_hi) return KC_E_INVALID_ARG;
  return enum_common(ctx, h, k, 1, root_lo, root_hi, d_buf, cap, written, total, checksum, stream);
}

int kc_count_batched(kc_ctx* ctx, const kc_graph* graphs, const uint32_t* ks, uint32_t nq, uint64_t* counts,
                     void* stream) {
  if (!ctx || (nq > 0 && (!graphs || !ks || !counts))) return KC_E_INVALID_ARG;
  std::vector<BatchQuery> q(nq);
  for (uint32_t i = 0; i < nq; i++) {
    auto it = ctx->graphs.find(graphs[i]);
    if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
    const uint32_t k = ks[i];
    if (k == 0) return KC_E_INVALID_ARG;
    if (k > KC_MAX_K) return KC_E_UNSUPPORTED;
  }
  for (uint32_t i = 0; i < nq; i++) {
    const DevGraph& g = ctx->graphs.find(graphs[i])->second;
    const uint32_t k = ks[i];
    q[i] = BatchQuery{g.orow, g.ocol, g.vert, g.n, k};
    counts[i] = 0;
    if (k == 1) counts[i] = g.n;
    if (k == 2) counts[i] = g.m;
    // k <= 2, or no root with k-1 out-neighbours: answered here
    if (k <= 2 || (uint64_t)k - 1 > g.max_out) q[i].n = 0;
  }
  KC_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, stream);
  if (ctx->opts.autotune) {
    uint64_t tiers[kTiers] = {0};
    for (uint32_t i = 0; i < nq; i++) {
      if (!q[i].n) continue;
      const DevGraph& g = ctx->graphs.find(graphs[i])->second;
      for (int t = 0; t < kTiers; t++) tiers[t] += g.tier_roots[t];
    }
    KC_TRY(tune_for_batch(ctx, q.data(), nq, tiers, s, nullptr));
  }
  ctx->last = kc_stats{};
  std::vector<uint64_t> got(std::max<uint32_t>(nq, 1), 0);
  KC_TRY(run_batch(ctx, q.data(), nq, ctx->opts.no_memo == 0, ctx->opts.no_prune == 0, got.data(), s));
  for (uint32_t i = 0; i < nq; i++)
    if (q[i].n) counts[i] = got[i];
  return KC_OK;
}

int kc_last_stats(kc_ctx* ctx, kc_stats* out) {
  if (!ctx || !out) return KC_E_INVALID_ARG;
  *out = ctx->last;
  return KC_OK;
}

int kc_last_upload_stats(kc_ctx* ctx, kc_upload_stats* out) {
  if (!ctx || !out) return KC_E_INVALID_ARG;
  *out = ctx->last_up;
  return KC_OK;
}

}  // extern "C"
