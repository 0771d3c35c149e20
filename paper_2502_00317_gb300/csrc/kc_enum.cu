// kc_enum.cu -- host side of the per-root enumeration of libkc.so: root
// binning, per-width launch plans, the tier launcher for kc_count / kc_list /
// kc_list_range and kc_count_batched, and the allocation-free count.  The
// enumerator kernels themselves are in kc_enum_dev.cuh, instantiated per width
// by kc_enum_w*.cu.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "kc_enum_dev.cuh"

namespace kc {

// k = 1 listing: every vertex of the rank range is a clique.
__global__ void k_list_singletons(const uint32_t* __restrict__ vert, uint32_t lo, uint32_t hi,
                                  uint32_t* __restrict__ out, unsigned long long cap, unsigned long long* acc) {
  unsigned long long s = 0, c = 0;
  for (uint64_t r = (uint64_t)lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < hi;
       r += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t id = vert[r];
    unsigned long long slot = r - lo;
    if (slot < cap) out[slot] = id;
    s += mix64(mix64(0x9E3779B97F4A7C15ull ^ 1ull) ^ (uint64_t)id);
    c++;
  }
  s = warp_sum(s);
  c = warp_sum(c);
  if (lane_id() == 0 && c) {
    atomicAdd(&acc[kAccChecksum], s);
    atomicAdd(&acc[kAccCount], c);
    atomicAdd(&acc[kAccWritten], c);
  }
}

// Roots of [lo, hi) with out-degree >= k-1, binned by bitmap width.

__global__ void k_bin_roots(const uint64_t* __restrict__ orow, uint32_t lo, uint32_t hi, uint32_t need,
                            uint32_t* __restrict__ lists, uint32_t list_cap, uint32_t* __restrict__ cnts,
                            unsigned long long* acc) {
  unsigned long long tot = 0;
  for (uint64_t r = (uint64_t)lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < hi;
       r += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = (uint32_t)(orow[r + 1] - orow[r]);
    if (d < need || d == 0) continue;
    tot++;
    uint32_t words = (d + 31) >> 5;
    int t = 0;
    while (t < kTiers && tier_words(t) < (int)words) t++;
    if (t < kTiers) {
      uint32_t p = atomicAdd(&cnts[t], 1u);
      lists[(size_t)t * list_cap + p] = (uint32_t)r;
    } else {
      atomicAdd(&cnts[kTiers], 1u);
    }
  }
  tot = warp_sum(tot);
  if (lane_id() == 0 && tot) atomicAdd(&acc[kAccRootsTotal], tot);
}

// --------------------------------------------------------------- launcher
struct TierPlan {
  int W = 0;
  int mode = 0;
  uint32_t nroots = 0;
  int warps_per_block = 0;
  size_t smem = 0;
  uint64_t blocks = 0;
  uint64_t gstate_bytes = 0;   // per-warp state in global memory (0: in shared memory)
  uint32_t depth = 0;          // stack depth of the per-warp states
  uint32_t sstride = 0;        // shared-memory bytes per warp
  uint32_t coff = 0;           // offset of the narrow branch state in them
  uint32_t soff_stats = 0;     // offset of the per-root counters
  uint32_t memo_cap = 0;       // entries per warp (0: no memo)
  uint32_t memo_cap2 = 0;      // and per warp for its narrow subproblems
  uint64_t memo_bytes = 0;
  uint32_t larena_bytes = 0;   // listing with the memo: arena bytes per warp
  bool split = false;          // heavy roots of this tier go to the split path
  uint64_t arena_units = 0;    // 16-byte units for published roots
  uint64_t task_cap = 0;       // (root, branch) task slots
  const void* fn = nullptr;
  const void* fn_tasks = nullptr;
};

// Bytes of one published root of width W: header, out-neighbours, bit-matrix rows, r values.
__host__ __device__ constexpr uint64_t published_root_units(int W) {
  return (16 + 32ull * W * 4 + 32ull * W * W * 4 + 32ull * W + 15) / 16;
}

// Enumerator and task kernels of tier t in a mode.
static void tier_kernels(int t, int mode, const void** fe, const void** ft) {
  switch (t) {
    case 0: tier_kernels_w1(mode, fe, ft); break;
    case 1: tier_kernels_w2(mode, fe, ft); break;
    case 2: tier_kernels_w4(mode, fe, ft); break;
    case 3: tier_kernels_w8(mode, fe, ft); break;
    case 4: tier_kernels_w16(mode, fe, ft); break;
    default: tier_kernels_w32(mode, fe, ft); break;
  }
}

static int plan_tier(kc_ctx* ctx, int t, int mode, uint32_t nroots, bool split, uint32_t depth, TierPlan* tp) {
  const int W = tier_words(t);
  const size_t wbytes = warp_state_stride(W, (int)depth);
  const bool in_smem = W <= 8;
  tp->W = W;
  tp->mode = mode;
  tp->nroots = nroots;
  tp->depth = depth;
  tp->sstride = (uint32_t)warp_smem_bytes(W, (int)depth);
  tp->soff_stats = tp->sstride - 64u;
  tp->coff = in_smem ? (uint32_t)wbytes : 0u;
  tier_kernels(t, mode, &tp->fn, &tp->fn_tasks);
  if (nroots == 0) return KC_OK;
  // warps per block: 8 and 4 by default, or the autotuner's choice (within the kernels' bounds)
  tp->warps_per_block = W <= 4 ? (ctx->tuning.wpb_small ? (int)ctx->tuning.wpb_small : 8)
                               : (ctx->tuning.wpb_large ? (int)ctx->tuning.wpb_large : 4);
  tp->smem = (size_t)tp->sstride * tp->warps_per_block;
  if (tp->smem > 48 * 1024) {
    KC_CUDA(cudaFuncSetAttribute(tp->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp->smem));
    KC_CUDA(cudaFuncSetAttribute(tp->fn_tasks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp->smem));
  }
  int per_sm = 0;
  KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tp->fn, tp->warps_per_block * 32, tp->smem));
  per_sm = std::max(per_sm, 1);
  uint64_t blocks = (uint64_t)ctx->num_sms * per_sm;
  uint64_t need_blocks = (nroots + tp->warps_per_block - 1) / tp->warps_per_block;
  // a split tier keeps the whole grid: its task phase has many more work items than roots
  if (!split) blocks = std::max<uint64_t>(1, std::min(blocks, need_blocks));
  tp->split = split;
  if (split) {
    tp->arena_units = (uint64_t)nroots * published_root_units(W);
    tp->task_cap = std::min<uint64_t>((uint64_t)nroots * 32 * W, 1ull << 26);
  }
  if (!in_smem) {
    // per-warp state in global memory: as many warps as the budget holds (at least one block)
    const uint64_t gbudget = ctx->gstate_budget ? ctx->gstate_budget : (1ull << 30);
    uint64_t max_warps = std::max<uint64_t>((uint64_t)tp->warps_per_block, gbudget / wbytes);
    blocks = std::max<uint64_t>(1, std::min<uint64_t>(blocks, max_warps / tp->warps_per_block));
    tp->gstate_bytes = wbytes;
  }
  tp->blocks = blocks;
  if (mode == 2 || mode == 3) {
    // per-warp memo tables within the budget (the tau of Sec. VI), shared by the tiers;
    // a window of 32 slots is the smallest table, and a tier that cannot get one counts without
    uint64_t warps = blocks * tp->warps_per_block;
    uint32_t cap = 1u << 12;
    uint64_t budget = ctx->tuning.memo_bytes ? ctx->tuning.memo_bytes
                      : (ctx->opts.memo_bytes ? ctx->opts.memo_bytes : (1ull << 30));
    uint64_t per_entry = 4 + 4ull * W + 8;
    // narrow subproblems get a table of their own, a quarter of the root's
    auto cap2_of = [&](uint32_t c) { return compact_width(W) ? std::max<uint32_t>(32, c / 4) : 0u; };
    while (cap > 32 && warps * (cap + cap2_of(cap)) * per_entry > budget / kTiers) cap >>= 1;
    if (warps * (cap + cap2_of(cap)) * per_entry > budget / kTiers) {
      tp->mode = mode == 3 ? 1 : 0;
      tier_kernels(t, tp->mode, &tp->fn, &tp->fn_tasks);
      if (tp->smem > 48 * 1024) {
        KC_CUDA(cudaFuncSetAttribute(tp->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp->smem));
        KC_CUDA(cudaFuncSetAttribute(tp->fn_tasks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp->smem));
      }
    } else {
      tp->memo_cap = cap;
      tp->memo_cap2 = cap2_of(cap);
      tp->memo_bytes = warps * (cap + tp->memo_cap2) * per_entry;
      if (mode == 3) {
        // the stored clique lists: up to four times the memo budget over the
        // tiers, 4 KiB to 256 KiB per warp
        const uint64_t per = std::min<uint64_t>(256 << 10, 4 * budget / kTiers / std::max<uint64_t>(warps, 1));
        tp->larena_bytes = (uint32_t)(per & ~(uint64_t)15);
        if (tp->larena_bytes < (4u << 10)) tp->larena_bytes = 0;  // too small to pay: plain listing tables only
      }
    }
  }
  return KC_OK;
}

// Every tier in one mode; width 1 is never split (its roots are light).
static int plan_all(kc_ctx* ctx, int mode, const uint32_t* hcnt, bool split, bool edge, uint32_t depth,
                    TierPlan* plans) {
  for (int t = 0; t < kTiers; t++)
    KC_TRY(plan_tier(ctx, t, mode, hcnt[t], (t > 0 || edge) && split, depth, &plans[t]));
  return KC_OK;
}

// Default split test: a root of a split tier is split when the wedge count of
// its G_u (sum over local vertices of C(out-degree, 2)) exceeds this.
constexpr uint32_t kDefaultSplitWedges = 16384;

// Plans and launches the enumerator of every non-empty width tier, each on
// its own stream (widest first), joined back into `s`.  troots[t] lists the
// tier's roots (troots_q[t] their queries in a batch, else nullptr).
static int launch_tiers(kc_ctx* ctx, const EnumKArgs& args, const uint32_t* hcnt, uint32_t* const* troots,
                        uint32_t* const* troots_q, int mode, bool split_ok, cudaStream_t s, uint32_t* launches,
                        uint32_t* enum_launches) {
  const uint32_t split_opt = ctx->tuning.split ? ctx->tuning.split : ctx->opts.split_threshold;
  const uint32_t split_wedges =
      split_opt == 0 ? kDefaultSplitWedges : (split_opt == 0xFFFFFFFFu ? 0u : split_opt);
  // the split path needs at least two levels below the first branch (k >= 5)
  // EdgeParallel decomposition (kc_opts.decomposition): every root of every
  // tier is split into its first-level branches, for any k >= 3
  const bool edge = ctx->opts.decomposition == KC_EDGE_PARALLEL;
  const bool split = (split_wedges != 0 && split_ok) || edge;
  TierPlan plans[kTiers];
  KC_TRY(plan_all(ctx, mode, hcnt, split, edge, args.depth, plans));
  // one scratch region for every tier's global state, memo tables, arena and task queue
  uint64_t total = 0;
  uint64_t goff[kTiers], moff[kTiers], loff[kTiers], aoff[kTiers], toff[kTiers];
  for (int t = 0; t < kTiers; t++) {
    goff[t] = total;
    total += (plans[t].gstate_bytes * plans[t].blocks * std::max(plans[t].warps_per_block, 1) + 255) & ~255ull;
    moff[t] = total;
    total += (plans[t].memo_bytes + 255) & ~255ull;
    loff[t] = total;
    total += ((uint64_t)plans[t].larena_bytes * plans[t].blocks * std::max(plans[t].warps_per_block, 1) + 255) & ~255ull;
    aoff[t] = total;
    total += (plans[t].arena_units * 16 + 255) & ~255ull;
    toff[t] = total;
    total += (plans[t].task_cap * 8 + 255) & ~255ull;
  }
  void* base = nullptr;
  if (total) KC_TRY(scratch_get(ctx, kScrEnum, total, &base));
  KC_CUDA(cudaEventRecord(ctx->ev_fork, s));
  for (int t = kTiers - 1; t >= 0; t--) {
    const TierPlan& tp = plans[t];
    if (tp.nroots == 0) continue;
    cudaStream_t ts = ctx->tier_stream[t];
    KC_CUDA(cudaStreamWaitEvent(ts, ctx->ev_fork, 0));
    EnumKArgs x = args;
    x.sstride = tp.sstride;
    x.coff = tp.coff;
    x.soff_stats = tp.soff_stats;
    x.roots = troots[t];
    x.roots_q = troots_q ? troots_q[t] : nullptr;
    x.nroots = tp.nroots;
    x.qctr = (unsigned int*)&ctx->d_acc[kAccQueue0 + t];
    if (tp.gstate_bytes) {
      x.gstate = (uint8_t*)base + goff[t];
      x.gstride = tp.gstate_bytes;
    }
    if (tp.memo_cap) {
      uint64_t warps = tp.blocks * tp.warps_per_block;
      uint8_t* mb = (uint8_t*)base + moff[t];
      const uint64_t slots = warps * (uint64_t)(tp.memo_cap + tp.memo_cap2);
      x.memo_vals = (unsigned long long*)mb;
      x.memo_tags = (uint32_t*)(mb + slots * 8);
      x.memo_keys = (uint32_t*)(mb + slots * 12);
      x.memo_cap = tp.memo_cap;
      x.memo_cap2 = tp.memo_cap2;
      KC_CUDA(cudaMemsetAsync(x.memo_tags, 0, slots * 4, ts));
    }
    if (tp.larena_bytes) {
      x.larena = (uint8_t*)base + loff[t];
      x.larena_bytes = tp.larena_bytes;
    }
    if (tp.split) {
      x.split_wedges = split_ok ? split_wedges : 0u;
      x.split_min_d = 32;
      x.edge_all = edge ? 1 : 0;
      x.arena = (uint8_t*)base + aoff[t];
      x.arena_units = tp.arena_units;
      x.arena_used = &ctx->d_acc[kAccArena0 + t];
      x.tasks = (unsigned long long*)((uint8_t*)base + toff[t]);
      x.task_cap = tp.task_cap;
      x.task_used = &ctx->d_acc[kAccTaskUsed0 + t];
      x.task_head = &ctx->d_acc[kAccTaskHead0 + t];
    }
    void* kargs[] = {&x};
    KC_CUDA(cudaEventRecord(ctx->ev_tier0[t], ts));
    KC_CUDA(cudaLaunchKernel(tp.fn, dim3((unsigned)tp.blocks), dim3(tp.warps_per_block * 32), kargs, tp.smem, ts));
    (*launches)++;
    (*enum_launches)++;
    if (tp.split) {
      // second phase: (root, first-level branch) tasks of the roots the first phase published
      KC_CUDA(cudaLaunchKernel(tp.fn_tasks, dim3((unsigned)tp.blocks), dim3(tp.warps_per_block * 32), kargs, tp.smem,
                               ts));
      (*launches)++;
      (*enum_launches)++;
    }
    KC_CUDA(cudaEventRecord(ctx->ev_tier1[t], ts));
    KC_CUDA(cudaEventRecord(ctx->ev_join[t], ts));
    KC_CUDA(cudaStreamWaitEvent(s, ctx->ev_join[t], 0));
  }
  return KC_OK;
}

int run_enum(kc_ctx* ctx, const DevGraph& g, const EnumArgs& ea, cudaStream_t s) {
  ctx->cur_stream = s;
  kc_stats stt{};
  uint32_t launches = 0, enum_launches = 0;
  uint32_t tier_roots[kTiers] = {0};
  cudaEvent_t* ev = ctx->ev;
  KC_CUDA(cudaEventRecord(ev[5], s));
  KC_CUDA(cudaMemsetAsync(ctx->d_acc, 0, kAccSlots * sizeof(unsigned long long), s));
  const uint32_t k = ea.k;
  const uint32_t lo = ea.root_lo, hi = ea.root_hi;
  if (k == 1) {
    if (ea.mode == 1 && hi > lo) {
      k_list_singletons<<<std::max<uint32_t>(1, std::min<uint32_t>((hi - lo + 255) / 256, ctx->num_sms * 8)), 256, 0,
                          s>>>(g.vert, lo, hi, ea.d_buf, ea.cap, ctx->d_acc);
      KC_CUDA(cudaGetLastError());
      launches++;
    }
    KC_CUDA(cudaEventRecord(ev[6], s));
    KC_CUDA(cudaEventRecord(ev[7], s));
  } else {
    uint32_t nr = hi > lo ? hi - lo : 0;
    uint32_t lcap = std::max<uint32_t>(nr, 1);
    void* lp = nullptr;
    KC_TRY(scratch_get(ctx, kScrRoots, ((size_t)kTiers * lcap + 16) * sizeof(uint32_t), &lp));
    uint32_t* lists = (uint32_t*)lp;
    uint32_t* cnts = lists + (size_t)kTiers * lcap;
    KC_CUDA(cudaMemsetAsync(cnts, 0, 16 * sizeof(uint32_t), s));
    if (nr) {
      unsigned blocks = std::max<uint32_t>(1, std::min<uint32_t>((nr + 255) / 256, ctx->num_sms * 8));
      k_bin_roots<<<blocks, 256, 0, s>>>(g.orow, lo, hi, k - 1, lists, lcap, cnts, ctx->d_acc);
      KC_CUDA(cudaGetLastError());
      launches++;
    }
    uint32_t hcnt[16] = {0};
    KC_CUDA(cudaMemcpyAsync(hcnt, cnts, sizeof(hcnt), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    KC_CUDA(cudaEventRecord(ev[6], s));
    if (hcnt[kTiers] != 0) return KC_E_UNSUPPORTED;  // out-degree above the widest tier
    // memo needs at least one level to split (k >= 3); k = 2 counts by popcount
    // listing uses the trie where Eq. (1) can hold below the first branch (k >= 6)
    const int mode = ea.mode == 1 ? ((ea.memo && k >= 6) ? 3 : 1) : ((ea.memo && k >= 3) ? 2 : 0);
    EnumKArgs args{};
    args.orow = g.orow;
    args.ocol = g.ocol;
    args.vert = g.vert;
    args.k = k;
    args.depth = k + 1;
    args.prune = ea.prune ? 1 : 0;
    args.memo = ea.memo ? 1 : 0;
    args.plex = (ea.mode != 1 && !ctx->opts.no_plex) ? 1 : 0;  // counting only
    args.binom = ctx->d_binom;
    args.out = ea.d_buf;
    args.cap = ea.cap;
    args.acc = ctx->d_acc;
    args.status = ctx->d_status;
    uint32_t* troots[kTiers];
    for (int t = 0; t < kTiers; t++) troots[t] = lists + (size_t)t * lcap;
    // the default split starts at k = 6: at k = 5 a heavy root's branches
    // hold too little below them to pay for publishing it (config 2: 6.6 ms
    // unsplit against 8.7 ms split); a threshold the caller or the autotuner
    // sets applies from k = 5
    const bool split_set = ctx->tuning.split != 0 || ctx->opts.split_threshold != 0;
    KC_TRY(launch_tiers(ctx, args, hcnt, troots, nullptr, mode, k >= (split_set ? 5u : 6u), s, &launches,
                        &enum_launches));
    for (int t = 0; t < kTiers; t++) tier_roots[t] = hcnt[t];
    KC_CUDA(cudaEventRecord(ev[7], s));
  }
  KC_CUDA(cudaMemcpyAsync(ctx->h_acc, ctx->d_acc, kAccSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaEventRecord(ev[8], s));
  KC_CUDA(cudaEventSynchronize(ev[8]));
  cudaEventElapsedTime(&stt.ms_bin, ev[5], ev[6]);
  cudaEventElapsedTime(&stt.ms_enum, ev[6], ev[7]);
  cudaEventElapsedTime(&stt.ms_total, ev[5], ev[8]);
  stt.enum_launches = enum_launches;
  stt.total_launches = launches;
  stt.roots_total = ctx->h_acc[kAccRootsTotal];
  stt.roots_pruned = ctx->h_acc[kAccRootsPruned];
  stt.build_words = ctx->h_acc[kAccBuildWords];
  stt.memo_hits = ctx->h_acc[kAccMemoHits];
  stt.memo_inserts = ctx->h_acc[kAccMemoInserts];
  stt.memo_full = ctx->h_acc[kAccMemoFull];
  stt.memo_frames = ctx->h_acc[kAccMemoFrames];
  stt.roots_heavy = ctx->h_acc[kAccRootsHeavy];
  stt.word_ops = ctx->h_acc[kAccWordOps];
  stt.warp_ns_build = ctx->h_acc[kAccBuildNs];
  stt.warp_ns_busy = ctx->h_acc[kAccBusyNs];
  stt.memo_peak = ctx->h_acc[kAccMemoPeak];
  stt.plex_frames = ctx->h_acc[kAccPlex];
  if (k >= 2) {
    for (int t = 0; t < kTiers; t++) {
      stt.roots_tier[t] = tier_roots[t];
      stt.ms_tier[t] = 0.f;
      if (tier_roots[t]) cudaEventElapsedTime(&stt.ms_tier[t], ctx->ev_tier0[t], ctx->ev_tier1[t]);
    }
  }
  ctx->last = stt;
  return KC_OK;
}


// ------------------------------------------------------------ batched count
// Roots of every query of a batch, binned by width: the flattened index g over
// all queries' ranks maps to (query, rank) by a binary search of the query
// offsets.  Pass 0 counts the roots of each tier, pass 1 writes them at the
// tier's offset (tier_off), warp-aggregated.
struct BinBatchArgs {
  const BatchQuery* bq;
  const uint64_t* qoff;  // [nq + 1] running sum of the queries' n
  uint32_t nq;
  uint64_t total;
  uint32_t* cnts;        // [16]: per-tier counts (pass 0) or cursors (pass 1); [kTiers] too wide
  uint32_t tier_off[kTiers];
  uint32_t* roots;
  uint32_t* roots_q;
  unsigned long long* acc;
  int pass;
  uint32_t kmin;         // smallest k enumerated (3 counting: k <= 2 is answered on the host; 2 listing)
};

__global__ void k_bin_batch(BinBatchArgs a) {
  const uint32_t lane = lane_id();
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long tot = 0;
  for (uint64_t w0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5; w0 < a.total; w0 += nw << 5) {
    const uint64_t g = w0 + lane;
    uint32_t t = 0xFFu, q = 0, r = 0;
    if (g < a.total) {
      uint32_t lo = 0, hi = a.nq;  // last query whose offset is <= g
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.qoff[mid] <= g) lo = mid;
        else hi = mid;
      }
      q = lo;
      r = (uint32_t)(g - a.qoff[q]);
      const BatchQuery bq = a.bq[q];
      const uint32_t d = (uint32_t)(bq.orow[r + 1] - bq.orow[r]);
      if (bq.k >= a.kmin && d >= bq.k - 1) {
        const uint32_t words = (d + 31) >> 5;
        t = 0;
        while (t < (uint32_t)kTiers && (uint32_t)tier_words((int)t) < words) t++;
        tot++;
      }
    }
    const uint32_t same = __match_any_sync(0xFFFFFFFFu, t);
    const uint32_t leader = __ffs(same) - 1;
    uint32_t basep = 0;
    if (lane == leader && t != 0xFFu) basep = atomicAdd(&a.cnts[t], (uint32_t)__popc(same));
    basep = __shfl_sync(0xFFFFFFFFu, basep, leader);
    if (a.pass == 1 && t < (uint32_t)kTiers) {
      const uint32_t pos = a.tier_off[t] + basep + __popc(same & lanemask_lt());
      a.roots[pos] = r;
      a.roots_q[pos] = q;
    }
  }
  tot = warp_sum(tot);
  if (a.pass == 0 && lane == 0 && tot) atomicAdd(&a.acc[kAccRootsTotal], tot);
}

int run_batch(kc_ctx* ctx, const BatchQuery* hq, uint32_t nq, bool memo, bool prune, uint64_t* counts,
              cudaStream_t s, uint64_t* checksums) {
  const bool list = checksums != nullptr;
  ctx->cur_stream = s;
  kc_stats stt{};
  uint32_t launches = 0, enum_launches = 0;
  cudaEvent_t* ev = ctx->ev;
  KC_CUDA(cudaEventRecord(ev[5], s));
  KC_CUDA(cudaMemsetAsync(ctx->d_acc, 0, kAccSlots * sizeof(unsigned long long), s));
  std::vector<uint64_t> qoff(nq + 1, 0);
  bool any5 = false;
  for (uint32_t q = 0; q < nq; q++) {
    qoff[q + 1] = qoff[q] + hq[q].n;
    any5 |= hq[q].k >= 5;
  }
  const uint64_t total = qoff[nq];
  // device copies of the queries, offsets, counts and tier counters
  const size_t qbytes = ((size_t)nq * sizeof(BatchQuery) + 255) & ~(size_t)255;
  const size_t obytes = (((size_t)nq + 1) * 8 + 255) & ~(size_t)255;
  const size_t cbytes = ((size_t)nq * 8 + 255) & ~(size_t)255;
  void* meta = nullptr;
  KC_TRY(scratch_get(ctx, kScrBatch, qbytes + obytes + 2 * cbytes + 256, &meta));
  BatchQuery* d_q = (BatchQuery*)meta;
  uint64_t* d_off = (uint64_t*)((uint8_t*)meta + qbytes);
  unsigned long long* d_cnt = (unsigned long long*)((uint8_t*)meta + qbytes + obytes);
  unsigned long long* d_sum = (unsigned long long*)((uint8_t*)meta + qbytes + obytes + cbytes);
  uint32_t* d_tc = (uint32_t*)((uint8_t*)meta + qbytes + obytes + 2 * cbytes);
  KC_CUDA(cudaMemcpyAsync(d_q, hq, (size_t)nq * sizeof(BatchQuery), cudaMemcpyHostToDevice, s));
  KC_CUDA(cudaMemcpyAsync(d_off, qoff.data(), ((size_t)nq + 1) * 8, cudaMemcpyHostToDevice, s));
  KC_CUDA(cudaMemsetAsync(d_cnt, 0, 2 * cbytes, s));
  KC_CUDA(cudaMemsetAsync(d_tc, 0, 256, s));
  BinBatchArgs ba{};
  ba.bq = d_q;
  ba.qoff = d_off;
  ba.nq = nq;
  ba.total = total;
  ba.cnts = d_tc;
  ba.acc = ctx->d_acc;
  ba.kmin = list ? 2u : 3u;
  const unsigned bb =
      (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->num_sms * 8));
  uint32_t hcnt[16] = {0};
  if (total) {
    ba.pass = 0;
    k_bin_batch<<<bb, 256, 0, s>>>(ba);
    KC_CUDA(cudaGetLastError());
    launches++;
    KC_CUDA(cudaMemcpyAsync(hcnt, d_tc, sizeof(hcnt), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
  }
  if (hcnt[kTiers] != 0) return KC_E_UNSUPPORTED;  // out-degree above the widest tier
  uint64_t nroots = 0;
  for (int t = 0; t < kTiers; t++) {
    ba.tier_off[t] = (uint32_t)nroots;
    nroots += hcnt[t];
  }
  if (nroots >= (1ull << 32)) return KC_E_UNSUPPORTED;
  void* lp = nullptr;
  KC_TRY(scratch_get(ctx, kScrRoots, (2 * std::max<uint64_t>(nroots, 1) + 16) * sizeof(uint32_t), &lp));
  ba.roots = (uint32_t*)lp;
  ba.roots_q = ba.roots + std::max<uint64_t>(nroots, 1);
  if (nroots) {
    KC_CUDA(cudaMemsetAsync(d_tc, 0, 64, s));
    ba.pass = 1;
    k_bin_batch<<<bb, 256, 0, s>>>(ba);
    KC_CUDA(cudaGetLastError());
    launches++;
  }
  KC_CUDA(cudaEventRecord(ev[6], s));
  if (nroots) {
    EnumKArgs args{};
    args.k = 3;  // per query through bq; this value is never used for a root
    uint32_t kmax = 3;
    for (uint32_t q = 0; q < nq; q++) kmax = std::max(kmax, hq[q].k);
    args.depth = kmax + 1;  // stacks deep enough for every query
    args.prune = prune ? 1 : 0;
    args.memo = memo ? 1 : 0;
    args.plex = (!list && !ctx->opts.no_plex) ? 1 : 0;  // counting only
    args.binom = ctx->d_binom;
    args.acc = ctx->d_acc;
    args.status = ctx->d_status;
    args.bq = d_q;
    args.bcount = d_cnt;
    args.bsum = d_sum;
    uint32_t* troots[kTiers];
    uint32_t* troots_q[kTiers];
    for (int t = 0; t < kTiers; t++) {
      troots[t] = ba.roots + ba.tier_off[t];
      troots_q[t] = ba.roots_q + ba.tier_off[t];
    }
    // listing (cap 0: counts and checksums only) or counting, with the memo where allowed
    const int mode = list ? 1 : (memo ? 2 : 0);
    KC_TRY(launch_tiers(ctx, args, hcnt, troots, troots_q, mode, any5, s, &launches, &enum_launches));
  }
  KC_CUDA(cudaEventRecord(ev[7], s));
  KC_CUDA(cudaMemcpyAsync(counts, d_cnt, (size_t)nq * 8, cudaMemcpyDeviceToHost, s));
  if (list) KC_CUDA(cudaMemcpyAsync(checksums, d_sum, (size_t)nq * 8, cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaMemcpyAsync(ctx->h_acc, ctx->d_acc, kAccSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaEventRecord(ev[8], s));
  KC_CUDA(cudaEventSynchronize(ev[8]));
  cudaEventElapsedTime(&stt.ms_bin, ev[5], ev[6]);
  cudaEventElapsedTime(&stt.ms_enum, ev[6], ev[7]);
  cudaEventElapsedTime(&stt.ms_total, ev[5], ev[8]);
  stt.enum_launches = enum_launches;
  stt.total_launches = launches;
  stt.roots_total = ctx->h_acc[kAccRootsTotal];
  stt.roots_pruned = ctx->h_acc[kAccRootsPruned];
  stt.roots_heavy = ctx->h_acc[kAccRootsHeavy];
  stt.build_words = ctx->h_acc[kAccBuildWords];
  stt.memo_hits = ctx->h_acc[kAccMemoHits];
  stt.memo_inserts = ctx->h_acc[kAccMemoInserts];
  stt.memo_full = ctx->h_acc[kAccMemoFull];
  stt.memo_frames = ctx->h_acc[kAccMemoFrames];
  stt.word_ops = ctx->h_acc[kAccWordOps];
  stt.warp_ns_build = ctx->h_acc[kAccBuildNs];
  stt.warp_ns_busy = ctx->h_acc[kAccBusyNs];
  stt.memo_peak = ctx->h_acc[kAccMemoPeak];
  stt.plex_frames = ctx->h_acc[kAccPlex];
  for (int t = 0; t < kTiers; t++) {
    stt.roots_tier[t] = hcnt[t];
    if (hcnt[t]) cudaEventElapsedTime(&stt.ms_tier[t], ctx->ev_tier0[t], ctx->ev_tier1[t]);
  }
  ctx->last = stt;
  return KC_OK;
}

}  // namespace kc

// ------------------------------------------- counting without allocating
// kc_count_dag_noalloc: the plain count of k_enum (mode 0, pruning on, no
// memo, no split) over a DAG the caller already holds on the device, with
// all of its scratch (accumulators, root lists) in one fixed device array.
// It exists for callers that must not allocate device memory; see the
// declaration in kclique.h for the contract.
namespace kc {
namespace {
constexpr uint32_t kStaticChunk = 1u << 17;  // roots binned per pass
constexpr size_t kStaticAccBytes = 512;      // accumulator slots
constexpr size_t kStaticCntBytes = 256;      // tier counts (16 words), status word
constexpr size_t kStaticListBytes = (size_t)kTiers * kStaticChunk * sizeof(uint32_t);
constexpr size_t kStaticBytes = kStaticAccBytes + kStaticCntBytes + kStaticListBytes;  // 3 MiB + 768 B
static_assert(kAccSlots * sizeof(unsigned long long) <= kStaticAccBytes, "accumulators do not fit");
constexpr int kStaticMaxDevices = 64;
}  // namespace
}  // namespace kc

// Shared by every call on a device; held by each GPU that loads the library until the process exits.
static __device__ __align__(256) uint8_t g_kc_static_scratch[kc::kStaticBytes];

namespace kc {
namespace {
std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices];  // device address of g_kc_static_scratch, per device

// Device address of the static scratch on device `dev` (the current device).
// Host code cannot use the symbol itself: it names a host-side shadow.
int static_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kStaticMaxDevices) return KC_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_kc_static_scratch);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return KC_OK;
}

// Rows must be strictly ascending, above their own rank and below n.
__global__ void k_check_dag(const uint64_t* __restrict__ orow, const uint32_t* __restrict__ ocol, uint32_t n,
                            uint64_t m, uint32_t* status) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = orow[r], e = orow[r + 1];
    if (e < b || e > m) {
      atomicOr(status, kStBadGraph);
      continue;
    }
    uint32_t prev = (uint32_t)r;
    for (uint64_t p = b; p < e; p++) {
      const uint32_t v = ocol[p];
      if (v <= prev || v >= n) {
        atomicOr(status, kStBadGraph);
        break;
      }
      prev = v;
    }
  }
}

int static_tier(int t, int num_sms, const EnumKArgs& x, cudaStream_t s) {
  kc_ctx* ctx = nullptr;  // for KC_CUDA: errors carry no context
  const int W = tier_words(t);
  const void* fe = nullptr;
  const void* ft = nullptr;
  tier_kernels(t, 0, &fe, &ft);
  const int wpb = W <= 4 ? 8 : 4;
  const size_t sstride = warp_smem_bytes(W, (int)x.depth);
  const size_t smem = sstride * wpb;
  if (smem > 48 * 1024) KC_CUDA(cudaFuncSetAttribute(fe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fe, wpb * 32, smem));
  uint64_t blocks = (uint64_t)num_sms * std::max(per_sm, 1);
  blocks = std::max<uint64_t>(1, std::min<uint64_t>(blocks, (x.nroots + wpb - 1) / wpb));
  EnumKArgs y = x;
  y.sstride = (uint32_t)sstride;
  y.coff = (uint32_t)warp_state_stride(W, (int)x.depth);
  y.soff_stats = (uint32_t)sstride - 64u;
  void* kargs[] = {&y};
  KC_CUDA(cudaLaunchKernel(fe, dim3((unsigned)blocks), dim3(wpb * 32), kargs, smem, s));
  return KC_OK;
}
}  // namespace
}  // namespace kc

extern "C" int kc_count_dag_noalloc(uint32_t n, const uint64_t* d_orow, const uint32_t* d_ocol, uint32_t k,
                                    uint64_t* count, void* stream) {
  using namespace kc;
  kc_ctx* ctx = nullptr;  // for KC_CUDA: errors carry no context
  if (!d_orow || !count || k == 0) return KC_E_INVALID_ARG;
  if (k > KC_MAX_K || n == 0xFFFFFFFFu) return KC_E_UNSUPPORTED;
  int dev = 0;
  KC_CUDA(cudaGetDevice(&dev));
  void* base = nullptr;
  KC_TRY(static_scratch(dev, &base));
  int num_sms = 0;
  KC_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* acc = (unsigned long long*)base;
  uint32_t* cnts = (uint32_t*)((uint8_t*)base + kStaticAccBytes);
  uint32_t* status = cnts + 16;
  uint32_t* lists = (uint32_t*)((uint8_t*)base + kStaticAccBytes + kStaticCntBytes);
  // the array keeps the previous call's contents: clear accumulators, counts and status
  KC_CUDA(cudaMemsetAsync(base, 0, kStaticAccBytes + kStaticCntBytes, s));
  uint64_t ends[2] = {0, 0};
  KC_CUDA(cudaMemcpyAsync(&ends[0], d_orow, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaMemcpyAsync(&ends[1], d_orow + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] >= (1ull << 40)) return KC_E_INVALID_GRAPH;
  const uint64_t m = ends[1];
  if (m > 0 && !d_ocol) return KC_E_INVALID_ARG;
  if (n > 0) {
    const unsigned cb = std::max<uint32_t>(1, std::min<uint32_t>((n + 255) / 256, (uint32_t)num_sms * 8));
    k_check_dag<<<cb, 256, 0, s>>>(d_orow, d_ocol, n, m, status);
    KC_CUDA(cudaGetLastError());
  }
  uint32_t hstatus = 0;
  KC_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  if (hstatus & kStBadGraph) return KC_E_INVALID_GRAPH;
  if (k == 1) {
    *count = n;
    return KC_OK;
  }
  if (k == 2) {
    *count = m;
    return KC_OK;
  }
  EnumKArgs x{};
  x.orow = d_orow;
  x.ocol = d_ocol;
  // no id map: the count kernel (mode 0) never reads vert, only listing does
  x.vert = nullptr;
  x.k = k;
  x.depth = k + 1;
  x.prune = 1;
  x.acc = acc;
  x.status = status;
  for (uint64_t lo = 0; lo < n; lo += kStaticChunk) {
    const uint32_t hi = (uint32_t)std::min<uint64_t>(n, lo + kStaticChunk);
    // per pass: tier counts and root-queue counters start at zero
    KC_CUDA(cudaMemsetAsync(cnts, 0, 16 * sizeof(uint32_t), s));
    KC_CUDA(cudaMemsetAsync(&acc[kAccQueue0], 0, kTiers * sizeof(unsigned long long), s));
    const unsigned bb = std::max<uint32_t>(1, std::min<uint32_t>((hi - (uint32_t)lo + 255) / 256, (uint32_t)num_sms * 8));
    k_bin_roots<<<bb, 256, 0, s>>>(d_orow, (uint32_t)lo, hi, k - 1, lists, kStaticChunk, cnts, acc);
    KC_CUDA(cudaGetLastError());
    uint32_t hcnt[16] = {0};
    KC_CUDA(cudaMemcpyAsync(hcnt, cnts, sizeof(hcnt), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    // out-degrees above 256 need per-warp state outside shared memory: not in this entry point
    if (hcnt[4] || hcnt[5] || hcnt[kTiers]) return KC_E_UNSUPPORTED;
    for (int t = 0; t < 4; t++) {
      if (!hcnt[t]) continue;
      EnumKArgs y = x;
      y.roots = lists + (size_t)t * kStaticChunk;
      y.nroots = hcnt[t];
      y.qctr = (unsigned int*)&acc[kAccQueue0 + t];
      KC_TRY(static_tier(t, num_sms, y, s));
    }
  }
  unsigned long long total = 0;
  KC_CUDA(cudaMemcpyAsync(&total, &acc[kAccCount], sizeof(total), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  *count = total;
  return KC_OK;
}
