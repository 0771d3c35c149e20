// kc_internal.cuh -- internal declarations shared by the libkc.so translation
// units (device helpers, context and graph records, kernel launchers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "kclique.h"

namespace kc {

constexpr uint32_t kAlive = 0xFFFFFFFFu;
constexpr int kWarp = 32;
constexpr int kTiers = 6;  // enumerator widths 1, 2, 4, 8, 16, 32 words (out-degree <= 1024)

// Device-side status bits (one uint32 per context, OR-ed by kernels).
constexpr uint32_t kStBadGraph = 1u << 0;   // invalid id, unsorted row, self-loop, asymmetry
constexpr uint32_t kStTimeout = 1u << 1;    // a bounded wait gave up
constexpr uint32_t kStUnsupported = 1u << 2;
constexpr uint32_t kStOverflow = 1u << 3;   // an internal capacity was exceeded

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

__device__ __forceinline__ uint32_t warp_min_u32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

// SplitMix64 output function (Steele, Lea & Flood 2014), the clique hash's mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid-wide barrier for a cooperative launch (all blocks co-resident).
// Generation-counter sense; a block that waits longer than `limit_ns`
// nanoseconds sets kStTimeout in *err and returns.  Returns false once any
// block has reported a timeout, so every block leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, volatile unsigned int* gen, unsigned int nblocks,
                                             unsigned long long limit_ns, unsigned int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int g = *gen;
    __threadfence();
    unsigned int arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((unsigned int*)gen, 1u);
    } else {
      unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (global_ns() - t0 > limit_ns) {
          atomicOr(err, kStTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*((volatile unsigned int*)err) & kStTimeout) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------- host records
struct DevGraph {
  uint32_t n = 0;
  uint64_t m = 0;             // undirected edges
  uint32_t degeneracy = 0;
  uint32_t max_out = 0;
  uint32_t peel_rounds = 0;
  uint32_t* core = nullptr;   // [n]
  uint32_t* rank = nullptr;   // [n] rank of each original id
  uint32_t* vert = nullptr;   // [n] original id of each rank
  uint64_t* orow = nullptr;   // [n+1] DAG CSR in rank space
  uint32_t* ocol = nullptr;   // [m]
  uint32_t tier_roots[kTiers] = {};  // vertices per bitmap-width tier (out-degree 1..32, 33..64, ...)
};

struct Scratch {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Server;  // the serving loop (kc_serve.cu)

// Launch settings chosen by the autotuner (kc_tune.cu); a zero field keeps
// the default.
struct Tuning {
  uint32_t split = 0;       // kc_opts.split_threshold encoding
  uint32_t wpb_small = 0;   // warps per block, tiers of 1-4 words (default 8)
  uint32_t wpb_large = 0;   // warps per block, tiers of 8-32 words (default 4)
  uint64_t memo_bytes = 0;  // memo budget (default kc_opts.memo_bytes, else 1 GiB)
};

}  // namespace kc

struct kc_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  cudaStream_t own_stream = nullptr;
  kc_opts opts{};
  uint32_t next_handle = 1;
  std::unordered_map<uint32_t, kc::DevGraph> graphs;
  std::vector<kc::Scratch> scratch;       // reusable device work buffers, by slot
  uint64_t scratch_bytes = 0;             // bytes held by them now, and at most so far
  uint64_t scratch_peak = 0;
  uint64_t gstate_budget = 0;             // bytes for per-warp state in global memory per tier (0: 1 GiB)
  cudaStream_t cur_stream = nullptr;      // stream of the running call (orders scratch allocations)
  uint32_t* d_status = nullptr;           // device status bits
  unsigned long long* d_acc = nullptr;    // device accumulators (count, checksum, written, stats ...)
  unsigned long long* h_acc = nullptr;    // pinned host mirror
  unsigned long long* d_binom = nullptr;  // C(n, j) mod 2^64 for n <= KC_MAX_OUTDEG, j <= KC_MAX_K (2-plex counts)
  cudaEvent_t ev[16] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kc::kTiers] = {};
  cudaEvent_t ev_tier0[kc::kTiers] = {};
  cudaEvent_t ev_tier1[kc::kTiers] = {};
  cudaStream_t tier_stream[kc::kTiers] = {};
  kc_stats last{};
  kc_upload_stats last_up{};
  std::string last_error;
  kc::Server* server = nullptr;           // kc_serve_* state, if serving was ever started
  kc::Tuning tuning;                      // launch settings in force (autotuner)
  std::unordered_map<std::string, kc::Tuning> tune_table;  // tuned settings by class key
  std::string tune_path;                  // file of tuned settings ("" : memory only)
  std::string gpu_name;
};

namespace kc {

// Accumulator slots in ctx->d_acc.
enum AccSlot : int {
  kAccCount = 0,
  kAccChecksum,
  kAccWritten,
  kAccRootsTotal,
  kAccRootsPruned,
  kAccRootsHeavy,
  kAccBuildWords,
  kAccMemoHits,
  kAccMemoInserts,
  kAccMemoFull,
  kAccMemoFrames,
  kAccTasks,
  kAccWordOps,
  kAccBuildNs,     // warp-nanoseconds spent building root bit-matrices (a5)
  kAccBusyNs,      // warp-nanoseconds spent on roots and tasks in all
  kAccMemoPeak,    // most trie entries stored for one root
  kAccPlex,        // frames counted by the 2-plex closed form
  kAccQueue0,      // root-queue counters (one per width tier)
  kAccArena0 = kAccQueue0 + kTiers,     // split path: arena units used, per tier
  kAccTaskUsed0 = kAccArena0 + kTiers,  // split path: tasks queued, per tier
  kAccTaskHead0 = kAccTaskUsed0 + kTiers,  // split path: tasks taken, per tier
  kAccSlots = kAccTaskHead0 + kTiers
};

// Scratch slots.
enum ScratchSlot : int {
  kScrA = 0, kScrB, kScrC, kScrD, kScrE, kScrF, kScrG, kScrScan, kScrSort, kScrSortList, kScrEnum, kScrMemo,
  kScrRoots, kScrPeel, kScrSplit, kScrBatch,
  kScrSlots
};

// Whether a single-graph count of k-cliques uses the memo (kc_opts.memo_min_k;
// default from k = 8 with the 2-plex closed form on, from k = 3 with it off).
inline bool count_uses_memo(const kc_ctx* ctx, uint32_t k) {
  const uint32_t min_k = ctx->opts.memo_min_k ? ctx->opts.memo_min_k : (ctx->opts.no_plex ? 3u : 8u);
  return ctx->opts.no_memo == 0 && k >= min_k;
}

int scratch_get(kc_ctx* ctx, int slot, size_t bytes, void** out);
int cuda_fail(kc_ctx* ctx, cudaError_t e, const char* what);

#define KC_CUDA(call)                                        \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return ::kc::cuda_fail(ctx, _e, #call); \
  } while (0)

#define KC_TRY(call)              \
  do {                            \
    int _s = (call);              \
    if (_s != KC_OK) return _s;   \
  } while (0)

// ----------------------------------------------------------- launch helpers
// Exclusive scan of n uint32 counts into n+1 uint64 offsets (out[n] = total).
int exclusive_scan_u32_to_u64(kc_ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t s,
                              uint32_t* launches);
// Sort each row [ptr[r], ptr[r+1]) of data ascending (uint32 keys).  When
// ucount != nullptr also moves each row's distinct keys to the row front and
// writes their number to ucount[r].
int segmented_sort(kc_ctx* ctx, uint32_t* data, const uint64_t* ptr, uint32_t rows, uint64_t total, uint32_t max_row,
                   uint32_t* ucount, cudaStream_t s, uint32_t* launches);

// Serving (kc_serve.cu): stop the loop and free its state (kc_destroy).
void serve_release(kc_ctx* ctx);

// Upload pipeline (kc_prep.cu).
int prep_graph(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr, const uint32_t* col, uint32_t flags,
               DevGraph* g, cudaStream_t s);

// Enumeration (kc_enum.cu).  mode 0: count, mode 1: list.
struct EnumArgs {
  uint32_t k = 0;
  int mode = 0;
  uint32_t root_lo = 0, root_hi = 0;
  uint32_t* d_buf = nullptr;
  uint64_t cap = 0;
  bool memo = true;
  bool prune = true;
};
int run_enum(kc_ctx* ctx, const DevGraph& g, const EnumArgs& a, cudaStream_t s);

// Batched counting (kc_enum.cu): one query per (graph, k); every query with
// n > 0 and k >= 3 is counted in one set of tier launches into counts[q].
// With checksums != nullptr the queries are listed instead (no tuples kept;
// every query with n > 0 and k >= 2): counts[q] and checksums[q] are
// kc_list's total and checksum.
struct BatchQuery {
  const uint64_t* orow;  // the query graph's DAG (rank space)
  const uint32_t* ocol;
  const uint32_t* vert;
  uint32_t n;            // 0: nothing to enumerate (answered on the host)
  uint32_t k;
};
int run_batch(kc_ctx* ctx, const BatchQuery* hq, uint32_t nq, bool memo, bool prune, uint64_t* counts,
              cudaStream_t s, uint64_t* checksums = nullptr);

// Autotuning (kc_tune.cu): load the cache file (kc_create); apply the tuned
// settings of a batch's class, probing first when the class is new
// (tier_roots: the batch's roots per width tier, summed over its graphs).
void tune_load(kc_ctx* ctx);
int tune_for_batch(kc_ctx* ctx, const BatchQuery* hq, uint32_t nq, const uint64_t* tier_roots, cudaStream_t s,
                   kc_tune_result* out);
int tune_for_graph(kc_ctx* ctx, const DevGraph& g, uint32_t k, cudaStream_t s);

}  // namespace kc
