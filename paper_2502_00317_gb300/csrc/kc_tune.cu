// kc_tune.cu -- the autotuner of libkc.so (kc_tune, and kc_opts.autotune for
// kc_count and kc_count_batched).  The settings it chooses have no
// counterpart in the paper and change no result, only the time: warps per
// block of the narrow (1-4 words) and wide (8-32 words) width tiers, the
// heavy-root split threshold, and the memo budget.  A choice is made per
// class of input -- the GPU, the size of the input, the k values asked for
// and the share of roots in each width tier -- by timing the input itself
// (or a sample of it) under candidate settings, and is cached in memory and,
// when a file is named, on disk.  Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kc_internal.cuh"

namespace kc {
namespace {

uint32_t log2_bucket(uint64_t x) {
  uint32_t b = 0;
  while (x > 1) {
    x >>= 1;
    b++;
  }
  return b;
}

// The class of a batch: GPU / log2 of its vertices / log2 of its queries /
// the k values present / the share of roots in each width tier, in eighths.
std::string class_key(const kc_ctx* ctx, const BatchQuery* hq, uint32_t nq, const uint64_t* tier_roots) {
  uint64_t sum_n = 0, kmask = 0, tot = 0;
  for (uint32_t q = 0; q < nq; q++) {
    sum_n += hq[q].n;
    if (hq[q].n) kmask |= 1ull << std::min<uint32_t>(hq[q].k, 63);
  }
  for (int t = 0; t < kTiers; t++) tot += tier_roots[t];
  char buf[160];
  int p = snprintf(buf, sizeof(buf), "%s/n%u/q%u/k%llx/t", ctx->gpu_name.c_str(), log2_bucket(sum_n),
                   log2_bucket(nq), (unsigned long long)kmask);
  for (int t = 0; t < kTiers && p > 0 && p < (int)sizeof(buf) - 2; t++)
    p += snprintf(buf + p, sizeof(buf) - p, "%u", tot ? (unsigned)((tier_roots[t] * 8 + tot - 1) / tot) : 0u);
  return std::string(buf);
}

// The timed work of a probe: a batched count of the sampled queries, or, for
// one large graph, the count of the roots in the top sixteenth of its order
// (the dense core, where the settings matter).
struct ProbeWork {
  std::vector<BatchQuery> qs;
  const DevGraph* g = nullptr;
  uint32_t k = 0, lo = 0, hi = 0;
};

int run_probe(kc_ctx* ctx, const ProbeWork& w, cudaStream_t s) {
  if (w.g) {
    EnumArgs ea;
    ea.k = w.k;
    ea.mode = 0;
    ea.root_lo = w.lo;
    ea.root_hi = w.hi;
    ea.memo = count_uses_memo(ctx, w.k);  // as kc_count would run it
    ea.prune = ctx->opts.no_prune == 0;
    return run_enum(ctx, *w.g, ea, s);
  }
  std::vector<uint64_t> counts(std::max<size_t>(w.qs.size(), 1));
  return run_batch(ctx, w.qs.data(), (uint32_t)w.qs.size(), ctx->opts.no_memo == 0, ctx->opts.no_prune == 0,
                   counts.data(), s);
}

// One timed run under settings t (twice: the first run sizes the scratch,
// the second is timed).  Returns the call's device time in ms.
float probe(kc_ctx* ctx, const ProbeWork& w, cudaStream_t s, const Tuning& t, int* status) {
  const Tuning save = ctx->tuning;
  ctx->tuning = t;
  float ms = 1e30f;
  for (int r = 0; r < 2 && *status == KC_OK; r++) {
    *status = run_probe(ctx, w, s);
    if (r == 1 && *status == KC_OK) ms = ctx->last.ms_total;
  }
  ctx->tuning = save;
  return ms;
}

void tune_store(kc_ctx* ctx, const std::string& key, const Tuning& t) {
  ctx->tune_table[key] = t;
  if (ctx->tune_path.empty()) return;
  FILE* f = fopen(ctx->tune_path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s %u %u %u %llu\n", key.c_str(), t.split, t.wpb_small, t.wpb_large, (unsigned long long)t.memo_bytes);
  fclose(f);
}

// Coordinate descent over the settings, each change kept when it is at
// least 3 % faster: split threshold, warps per block (narrow, then wide
// tiers), memo budget.
int tune_probe(kc_ctx* ctx, const ProbeWork& w, cudaStream_t s, Tuning* best, kc_tune_result* out) {
  int st = KC_OK;
  Tuning cur{};
  float tcur = probe(ctx, w, s, cur, &st);
  if (st != KC_OK) return st;
  const float t0 = tcur;
  uint32_t probes = 1;
  auto attempt = [&](Tuning cand) {
    const float tc = probe(ctx, w, s, cand, &st);
    probes++;
    if (st == KC_OK && tc < 0.97f * tcur) {
      cur = cand;
      tcur = tc;
    }
  };
  for (uint32_t split : {0xFFFFFFFFu, 4096u, 65536u}) {
    Tuning c = cur;
    c.split = split;
    attempt(c);
    if (st != KC_OK) return st;
  }
  {
    Tuning c = cur;
    c.wpb_small = 4;
    attempt(c);
  }
  {
    Tuning c = cur;
    c.wpb_large = 2;
    attempt(c);
  }
  for (uint64_t mb : {256ull << 20, 4ull << 30}) {
    Tuning c = cur;
    c.memo_bytes = mb;
    attempt(c);
    if (st != KC_OK) return st;
  }
  *best = cur;
  if (out) {
    out->ms_default = t0;
    out->ms_tuned = tcur;
    out->probes = probes;
  }
  return KC_OK;
}

void fill_result(kc_tune_result* out, const std::string& key, const Tuning& t, bool cached) {
  if (!out) return;
  out->split_threshold = t.split ? t.split : 16384u;
  out->warps_small = t.wpb_small ? t.wpb_small : 8u;
  out->warps_large = t.wpb_large ? t.wpb_large : 4u;
  out->memo_bytes = t.memo_bytes ? t.memo_bytes : (1ull << 30);
  out->cached = cached ? 1u : 0u;
  std::strncpy(out->key, key.c_str(), sizeof(out->key) - 1);
  out->key[sizeof(out->key) - 1] = 0;
}

}  // namespace

void tune_load(kc_ctx* ctx) {
  const char* path = ctx->opts.tune_cache ? ctx->opts.tune_cache : std::getenv("KC_TUNE_CACHE");
  ctx->tune_path = path ? path : "";
  if (ctx->tune_path.empty()) return;
  FILE* f = fopen(ctx->tune_path.c_str(), "r");
  if (!f) return;
  char key[256];
  unsigned split, ws, wl;
  unsigned long long mb;
  while (fscanf(f, "%255s %u %u %u %llu", key, &split, &ws, &wl, &mb) == 5) {
    Tuning t;
    t.split = split;
    t.wpb_small = ws <= 8 ? ws : 0;
    t.wpb_large = wl <= 4 ? wl : 0;
    t.memo_bytes = mb;
    ctx->tune_table[key] = t;  // a later line for the same class wins
  }
  fclose(f);
}

int tune_for_batch(kc_ctx* ctx, const BatchQuery* hq, uint32_t nq, const uint64_t* tier_roots, cudaStream_t s,
                   kc_tune_result* out) {
  const std::string key = class_key(ctx, hq, nq, tier_roots);
  auto it = ctx->tune_table.find(key);
  if (it != ctx->tune_table.end() && !out) {
    ctx->tuning = it->second;
    return KC_OK;
  }
  // the probe: every query, or about 512 of them evenly spaced
  ProbeWork w;
  const uint32_t stride = nq > 512 ? (nq + 511) / 512 : 1;
  for (uint32_t q = 0; q < nq; q += stride) w.qs.push_back(hq[q]);
  if (out) std::memset(out, 0, sizeof(*out));
  Tuning best{};
  KC_TRY(tune_probe(ctx, w, s, &best, out));
  tune_store(ctx, key, best);
  ctx->tuning = best;
  fill_result(out, key, best, false);
  return KC_OK;
}

int tune_for_graph(kc_ctx* ctx, const DevGraph& g, uint32_t k, cudaStream_t s) {
  uint64_t tiers[kTiers];
  for (int t = 0; t < kTiers; t++) tiers[t] = g.tier_roots[t];
  const BatchQuery bq{g.orow, g.ocol, g.vert, g.n, k};
  const std::string key = class_key(ctx, &bq, 1, tiers);
  auto it = ctx->tune_table.find(key);
  if (it != ctx->tune_table.end()) {
    ctx->tuning = it->second;
    return KC_OK;
  }
  ProbeWork w;
  w.g = &g;
  w.k = k;
  w.hi = g.n;
  w.lo = g.n - std::max<uint32_t>(std::min<uint32_t>(g.n, 4096u), g.n / 16);
  Tuning best{};
  KC_TRY(tune_probe(ctx, w, s, &best, nullptr));
  tune_store(ctx, key, best);
  ctx->tuning = best;
  return KC_OK;
}

}  // namespace kc

using namespace kc;

extern "C" int kc_tune(kc_ctx* ctx, const kc_graph* graphs, const uint32_t* ks, uint32_t nq, kc_tune_result* out) {
  if (!ctx || (nq > 0 && (!graphs || !ks))) return KC_E_INVALID_ARG;
  std::vector<BatchQuery> q(nq);
  uint64_t tiers[kTiers] = {0};
  for (uint32_t i = 0; i < nq; i++) {
    auto it = ctx->graphs.find(graphs[i]);
    if (it == ctx->graphs.end()) return KC_E_NOT_FOUND;
    if (ks[i] == 0) return KC_E_INVALID_ARG;
    if (ks[i] > KC_MAX_K) return KC_E_UNSUPPORTED;
    const DevGraph& g = it->second;
    q[i] = BatchQuery{g.orow, g.ocol, g.vert, g.n, ks[i]};
    if (ks[i] <= 2 || (uint64_t)ks[i] - 1 > g.max_out) q[i].n = 0;
    if (q[i].n)
      for (int t = 0; t < kTiers; t++) tiers[t] += g.tier_roots[t];
  }
  KC_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->own_stream;
  ctx->cur_stream = s;
  kc_tune_result local{};
  KC_TRY(tune_for_batch(ctx, q.data(), nq, tiers, s, out ? out : &local));
  return KC_OK;
}
