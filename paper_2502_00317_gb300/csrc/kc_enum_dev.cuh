// kc_enum_dev.cuh -- device code of the per-root enumeration of libkc.so
// (one warp per root of the DAG), shared by the per-width translation units.
//
// For a root u with d out-neighbours the warp
//   1. builds the DAG induced by N(u) (Algorithm 2: the subgraph G_u) as a
//      d x d bit-matrix in root-local indices 0..d-1 (out-neighbours sorted by
//      rank, so row i holds only columns j > i);
//   2. runs Algorithm 5 on G[N(u) ∪ {u}] (Sec. V): r_i for every local vertex
//      and r(u) for the root, capped at k; the root is dropped when r(u) < k
//      (Lemma 1).  Below the root the same r_i bound a pick: vertex v can be
//      the minimum of an l-clique inside any subgraph of G_u only if r_v >= l;
//   3. lists or counts the (k-1)-cliques of G_u by depth-first search over
//      candidate bitmaps (Algorithm 1/2 recursion, intersections are AND of
//      bitmap rows, sizes are popcounts):
//        - count mode stops two levels early: the 2-cliques of a candidate set
//          S are the edges sum_{v in S} popc(S & row(v));
//        - list mode emits each clique at the last level;
//        - the memo variant (count mode) is the device form of the Induced
//          Subgraph Trie (Sec. IV, Algorithms 3 and 4): f(S, l), the number of
//          l-cliques in G[S], is stored in a per-warp hash table keyed by
//          (S, l).  A frame walks S from its largest vertex down (the order of
//          the identifying string) and after each vertex v stores the count
//          of the prefix subgraph S ∩ [v, ∞) -- the trie path node t_i with
//          Marked[l] set.  A frame starts from its longest stored prefix
//          (binary search over the prefix lengths), and an (S, l) that is
//          stored whole is a retrieval (ListingIST) instead of a search.  The
//          Eq. (1) density test decides where this starts; below a dense
//          frame every frame is memoised, as Algorithm 3 recurses into itself.
#pragma once

#include <algorithm>
#include <type_traits>

#include "kc_internal.cuh"

namespace kc {

constexpr int KMAX = KC_MAX_K;  // stack depth bound (k - 1 <= KMAX - 1)

struct EnumKArgs {
  const uint64_t* orow;
  const uint32_t* ocol;
  const uint32_t* vert;
  const uint32_t* roots;
  uint32_t nroots;
  unsigned int* qctr;
  uint32_t k;
  int prune;
  int memo;
  int plex;                   // count 2-plex candidate sets by their closed form (Sec. VII-A)
  const unsigned long long* binom;  // C(n, j) mod 2^64, rows of KC_MAX_K + 1 (with plex)
  uint32_t* out;
  unsigned long long cap;
  unsigned long long* acc;
  uint8_t* gstate;            // per-warp state in global memory (heavy tiers)
  unsigned long long gstride; // bytes per warp
  uint32_t* memo_tags;        // per-warp tables: cap entries each
  uint32_t* memo_keys;
  unsigned long long* memo_vals;
  uint32_t memo_cap;          // entries per warp (power of two)
  uint32_t memo_cap2;         // entries per warp for its narrow subproblems (after those; 0: none)
  uint8_t* larena;            // listing with the trie: per-warp arenas of stored l-clique lists
  uint32_t larena_bytes;      // bytes per warp
  uint32_t* status;
  // split path (heavy roots): arena of published roots and a task queue
  uint32_t split_wedges;      // 0: never split
  int split_min_d;
  int edge_all;               // EdgeParallel decomposition: every root's first-level branches are tasks
  uint8_t* arena;
  unsigned long long arena_units;  // 16-byte units
  unsigned long long* arena_used;
  unsigned long long* tasks;
  unsigned long long task_cap;
  unsigned long long* task_used;
  unsigned long long* task_head;
  // batched counting: per-query graph and k, the query of each root, counts
  const BatchQuery* bq;         // nullptr: one graph (the fields above)
  const uint32_t* roots_q;      // [nroots] query of each root
  unsigned long long* bcount;   // [queries] counts
  unsigned long long* bsum;     // [queries] listing checksums (list mode)
  uint32_t query;               // query bound to this copy of the arguments
  // layout of the per-warp state
  uint32_t depth;               // D: stack depth of every state (k + 1, the batch's largest k + 1)
  uint32_t sstride;             // shared-memory bytes per warp
  uint32_t coff;                // offset of the narrow branch state in the warp's shared memory
  uint32_t soff_stats;          // offset of the warp's per-root counters
};

// Bytes of one warp's working state at width W with stacks of depth D (the
// layout of WarpState::carve; D = k + 1 covers every depth of a k-clique search).
__host__ __device__ constexpr size_t warp_state_raw(int W, int D) {
  return (size_t)D * 8 + 32 * 4 + (size_t)32 * W * 4 * 2 + (size_t)32 * W * W * 4 + (size_t)D * W * 4 * 2 +
         (size_t)D * 4 * 2 + (size_t)(D + 1) * 4 + (size_t)32 * W * 2 + D + 32 * W + D + D;
}

// Per-warp stride of that state (16-byte aligned).
__host__ __device__ constexpr size_t warp_state_stride(int W, int D) { return (warp_state_raw(W, D) + 15) & ~(size_t)15; }

// Threads per block of the width-W kernels (8 warps up to 4 words, 4 beyond)
// and the blocks per SM their register budget is sized for: the searches are
// latency-bound, so the kernels keep to 64 registers (W <= 2), about 85
// (W = 4) or 128 (W >= 8), for 32, 24 and 16 resident warps per SM.
__host__ __device__ constexpr int kc_block_threads(int W) { return W <= 4 ? 256 : 128; }
__host__ __device__ constexpr int kc_min_blocks(int W) { return W <= 2 ? 4 : (W <= 4 ? 3 : 4); }

// Width of the narrow bit-matrix a branch of a width-W root is re-indexed
// into when its candidate set is small (0: none).  The narrow state lives in
// shared memory after the root's own.
__host__ __device__ constexpr int compact_width(int W) { return W >= 16 ? 8 : W / 2; }

// Shared-memory bytes per warp of a width-W kernel: the root's state (widths
// up to 8; wider ones keep it in global memory) and the narrow branch state.
__host__ __device__ constexpr size_t warp_smem_bytes(int W, int D) {
  return (W <= 8 ? warp_state_stride(W, D) : 0) + (compact_width(W) ? warp_state_stride(compact_width(W), D) : 0) +
         64;  // the warp's per-root counters (WarpStat)
}

// Per-warp working state, carved from shared or global memory.
template <int W>
struct WarpState {
  uint32_t* nbr;              // [32W] ranks of N+(u), ascending
  uint32_t* oid;              // [32W] original ids of those vertices (listing with the trie)
  uint32_t* rows;             // [32W*W] bit-matrix rows
  uint32_t* masks;            // [D*W] masks[l*W+w]: local vertices with r >= l
  uint32_t* cand;             // [D*W] candidate set per depth
  unsigned long long* sum;    // [D] frame partial counts (memo variant)
  int32_t* pos;               // [D] next pick position (descending), -1 when done
  int32_t* cur;               // [D] vertex whose child frame is open
  uint32_t* sid;              // [D+1] sorted original ids of the open clique prefix
  uint16_t* pidx;             // [32W] narrow state: the wider state's index of each vertex
  uint8_t* sins;              // [D] insertion index of each pick in sid
  uint8_t* rr;                // [32W] r values (Algorithm 5), capped at k
  uint8_t* dense;             // [D] frame uses the memo
  uint8_t* fullins;           // [D] frame's whole set already stored
  uint32_t* crow;             // [32] rows of a candidate set re-indexed to 0..31 (count_compact)
  uint8_t* cbase;             // this warp's narrow branch state (shared memory), or nullptr
  unsigned long long* stats;  // [kWsCount] this warp's per-root counters (shared memory; lane 0)
  __device__ void carve(uint8_t* base, int D) {
    uint8_t* p = base;
    sum = (unsigned long long*)p; p += (size_t)D * 8;
    crow = (uint32_t*)p; p += 32 * 4;
    nbr = (uint32_t*)p; p += (size_t)32 * W * 4;
    oid = (uint32_t*)p; p += (size_t)32 * W * 4;
    rows = (uint32_t*)p; p += (size_t)32 * W * W * 4;
    masks = (uint32_t*)p; p += (size_t)D * W * 4;
    cand = (uint32_t*)p; p += (size_t)D * W * 4;
    pos = (int32_t*)p; p += (size_t)D * 4;
    cur = (int32_t*)p; p += (size_t)D * 4;
    sid = (uint32_t*)p; p += (size_t)(D + 1) * 4;
    pidx = (uint16_t*)p; p += (size_t)32 * W * 2;
    sins = p; p += D;
    rr = p; p += 32 * W;
    dense = p; p += D;
    fullins = p;
    cbase = nullptr;
    stats = nullptr;
  }
};

// ------------------------------------------------------------ bit helpers
// Largest set bit of (S & M) at index <= from, or -1.
template <int W>
__device__ __forceinline__ int next_desc(const uint32_t* S, const uint32_t* M, int from) {
  if (from < 0) return -1;
  int w = from >> 5;
  uint32_t x = S[w] & M[w] & (0xFFFFFFFFu >> (31 - (from & 31)));
  while (true) {
    if (x) return (w << 5) + 31 - __clz(x);
    if (--w < 0) return -1;
    x = S[w] & M[w];
  }
}

template <int W>
__device__ __forceinline__ int top_bit(const uint32_t (&c)[W]) {
#pragma unroll
  for (int w = W - 1; w >= 0; w--)
    if (c[w]) return (w << 5) + 31 - __clz(c[w]);
  return -1;
}

// c[i] without a dynamic register-array index.
template <int W>
__device__ __forceinline__ uint32_t word_at(const uint32_t (&c)[W], uint32_t i) {
  uint32_t r = 0;
#pragma unroll
  for (int w = 0; w < W; w++) r = ((uint32_t)w == i) ? c[w] : r;
  return r;
}

// Number of edges of G[S] (the 2-cliques of S); lane-partial.  `ops` counts
// the candidate words intersected (AND + POPC), the enumerator's work unit.
template <int W>
__device__ __forceinline__ uint32_t edges_partial(const uint32_t (&S)[W], const uint32_t* rows, uint32_t& ops) {
  const uint32_t lane = lane_id();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < W; w++) {
    if ((S[w] >> lane) & 1u) {
      const uint32_t* rv = rows + (size_t)((w << 5) + lane) * W;
      ops += W - w;
#pragma unroll
      for (int w2 = w; w2 < W; w2++) c += __popc(S[w2] & rv[w2]);
    }
  }
  return c;
}

// ------------------------------------------------------------------- memo
struct Memo {
  uint32_t* tags;
  uint32_t* keys;
  unsigned long long* vals;
  uint32_t cap;
  uint32_t tagbase;  // epoch << 7
  uint8_t* lar;      // listing with the trie: this warp's arena of stored clique lists
  uint32_t lcap;     // its bytes
  uint32_t* ltop;    // bytes the current root has used (lives in the kernel)
};

// MODE 1 lists plainly, MODE 3 lists with the trie (both report cliques).
__host__ __device__ constexpr bool is_list(int mode) { return mode == 1 || mode == 3; }
// MODE 2 counts with the trie, MODE 3 lists with it.
__host__ __device__ constexpr bool uses_trie(int mode) { return mode == 2 || mode == 3; }

template <int W>
__device__ __forceinline__ uint32_t memo_hash(const uint32_t (&key)[W], uint32_t l) {
  uint32_t h = 0x9E3779B9u * (l + 1u);
#pragma unroll
  for (int w = 0; w < W; w++) {
    h ^= key[w] + 0x7F4A7C15u + (h << 6) + (h >> 2);
    h *= 0x85EBCA6Bu;
  }
  h ^= h >> 15;
  h *= 0xC2B2AE35u;
  h ^= h >> 13;
  return h;
}

// Warp-wide probe of a 32-slot window; returns the matching slot or -1, and
// (by reference) the first free slot of the window or -1.
template <int W>
__device__ __forceinline__ int memo_probe(const Memo& m, const uint32_t (&key)[W], uint32_t l, uint32_t h,
                                          int* free_slot) {
  const uint32_t lane = lane_id();
  uint32_t slot = (h + lane) & (m.cap - 1);
  uint32_t t = m.tags[slot];
  uint32_t want = m.tagbase | l;
  bool match = false;
  if (t == want) {
    match = true;
#pragma unroll
    for (int w = 0; w < W; w++) match &= (m.keys[(size_t)slot * W + w] == key[w]);
  }
  uint32_t bm = __ballot_sync(0xFFFFFFFFu, match);
  uint32_t be = __ballot_sync(0xFFFFFFFFu, (t & ~0x7Fu) != m.tagbase);
  *free_slot = be ? (int)((h + __ffs(be) - 1) & (m.cap - 1)) : -1;
  return bm ? (int)((h + __ffs(bm) - 1) & (m.cap - 1)) : -1;
}

template <int W>
__device__ __forceinline__ bool memo_find(const Memo& m, const uint32_t (&key)[W], uint32_t l,
                                          unsigned long long* val) {
  int fs;
  int s = memo_probe<W>(m, key, l, memo_hash<W>(key, l), &fs);
  if (s < 0) return false;
  *val = m.vals[s];
  return true;
}

// Store (key, l) -> val; returns 1 if stored, 0 if the window was full.
template <int W>
__device__ __forceinline__ int memo_store(const Memo& m, const uint32_t (&key)[W], uint32_t l, unsigned long long val) {
  const uint32_t h = memo_hash<W>(key, l);
  int fs;
  int s = memo_probe<W>(m, key, l, h, &fs);
  if (s < 0) s = fs;
  if (s < 0) return 0;
  const uint32_t lane = lane_id();
  if (lane < W) m.keys[(size_t)s * W + lane] = word_at<W>(key, lane);
  if (lane == 0) {
    m.vals[s] = val;
    m.tags[s] = m.tagbase | l;
  }
  __syncwarp();
  return 1;
}

// A new trie for the next root: every entry of an older epoch is stale.
__device__ __forceinline__ void next_epoch(Memo& memo, uint32_t* epoch) {
  if (++*epoch >= (1u << 25)) {
    for (uint32_t i = lane_id(); i < memo.cap; i += 32) memo.tags[i] = 0u;
    __syncwarp();
    *epoch = 1;
  }
  memo.tagbase = *epoch << 7;
}

// Bits of c at index >= v.
template <int W>
__device__ __forceinline__ void suffix_of(const uint32_t (&c)[W], int v, uint32_t (&out)[W]) {
#pragma unroll
  for (int w = 0; w < W; w++) {
    int lo = w << 5;
    out[w] = (v <= lo) ? c[w] : (v >= lo + 32 ? 0u : (c[w] & (0xFFFFFFFFu << (v - lo))));
  }
}

// Position of the j-th set bit (0-based, ascending) of c.
template <int W>
__device__ __forceinline__ int select_bit(const uint32_t (&c)[W], int j) {
#pragma unroll
  for (int w = 0; w < W; w++) {
    int p = __popc(c[w]);
    if (j < p) {
      uint32_t x = c[w];
      for (int i = 0; i < j; i++) x &= x - 1;
      return (w << 5) + __ffs(x) - 1;
    }
    j -= p;
  }
  return -1;
}

// Triangles of G[S] (the 3-cliques of S), lane-partial: lanes take the
// vertices v of S that can start a 3-clique (r_v >= 3) and each counts the
// edges of S ∩ row(v) on its own.
template <int W>
__device__ __forceinline__ uint32_t tri_partial_body(const uint32_t (&S)[W], const uint32_t* rows, const uint32_t* m3,
                                                    uint32_t& ops) {
  const uint32_t lane = lane_id();
  uint32_t acc = 0;
#pragma unroll
  for (int w = 0; w < W; w++) {
    if (((S[w] & m3[w]) >> lane) & 1u) {
      const uint32_t* rv = rows + (size_t)((w << 5) + lane) * W;
      ops += W - w;
      uint32_t T[W];
#pragma unroll
      for (int q = 0; q < W; q++) T[q] = (q < w) ? 0u : (S[q] & rv[q]);
#pragma unroll
      for (int q = w; q < W; q++) {
        uint32_t y = T[q];
        while (y) {
          const int b = __ffs(y) - 1;
          y &= y - 1;
          const uint32_t* rw = rows + (size_t)((q << 5) + b) * W;
          ops += W - q;
#pragma unroll
          for (int q2 = q; q2 < W; q2++) acc += __popc(T[q2] & rw[q2]);
        }
      }
    }
  }
  return acc;
}

// Widths of 8 words and more count triangles out of line (its unrolled
// W x W body is large and is reached from several call sites).
template <int W>
__device__ __noinline__ uint32_t tri_partial_outlined(const uint32_t (&S_in)[W], const uint32_t* rows,
                                                      const uint32_t* m3, uint32_t& ops_in) {
  uint32_t S[W];
#pragma unroll
  for (int w = 0; w < W; w++) S[w] = S_in[w];
  uint32_t ops = 0;
  const uint32_t r = tri_partial_body<W>(S, rows, m3, ops);
  ops_in += ops;
  return r;
}

template <int W>
__device__ __forceinline__ uint32_t tri_partial(const uint32_t (&S)[W], const uint32_t* rows, const uint32_t* m3,
                                               uint32_t& ops) {
  if constexpr (W >= 8) return tri_partial_outlined<W>(S, rows, m3, ops);
  else return tri_partial_body<W>(S, rows, m3, ops);
}

// Cliques of size need + 1 whose smallest vertex is the caller's, given its
// candidate word c0 in a graph of at most 32 vertices with one 32-bit row of
// larger neighbours per vertex (R): a depth-first search of this lane alone,
// each step one AND + POPC on a single word; the last two picks are counted
// as the edges of the candidate set.  need >= 1.
__device__ __forceinline__ uint32_t lane_count(const uint32_t* R, uint32_t c0, uint32_t need, uint32_t& ops) {
  if (need == 1) return __popc(c0);
  uint32_t stk[KMAX];
  uint32_t cnt = 0;
  int d = 0;
  stk[0] = c0;
  while (d >= 0) {
    uint32_t c = stk[d];
    const uint32_t rem = need - (uint32_t)d;  // vertices still to pick from c
    if (rem == 2) {
      uint32_t x = c;
      while (x) {
        const int j = __ffs(x) - 1;
        x &= x - 1;
        cnt += __popc(x & R[j]);
        ops++;
      }
      d--;
      continue;
    }
    if ((uint32_t)__popc(c) < rem) {
      d--;
      continue;
    }
    const int j = __ffs(c) - 1;
    c &= c - 1;
    stk[d] = c;
    const uint32_t nc = c & R[j];
    ops++;
    if ((uint32_t)__popc(nc) >= rem - 1) stk[++d] = nc;
  }
  return cnt;
}

struct Acc {
  unsigned long long cnt = 0, sum = 0;
  uint32_t ops = 0;          // candidate words intersected since the last fold into ops64
  uint32_t plex = 0;         // frames counted by the 2-plex closed form
  unsigned long long ops64 = 0;
  unsigned long long hits = 0, ins = 0, full = 0, frames = 0;
};

// Counters updated once per root or task, kept by lane 0 in the warp's
// shared memory instead of registers.
enum WarpStat : int {
  kWsPruned = 0,  // roots dropped by the soft-embedding test
  kWsWords,       // DAG words read by the builds
  kWsHeavy,       // roots published to the split path
  kWsTasks,       // tasks queued
  kWsBuildNs,     // nanoseconds in builds
  kWsBusyNs,      // nanoseconds on roots and tasks
  kWsInsMark,     // trie inserts when the current root started
  kWsInsPeak,     // most trie inserts of one root
  kWsCount
};

// Chunks of 16 bytes each lane keeps in flight while gathering rows (fewer
// at widths 1 and 2, whose kernels keep to 64 registers).
__host__ __device__ constexpr int build_unroll(int W) { return W <= 2 ? 2 : 4; }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
  const uint32_t lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)v, src);
  const uint32_t hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), src);
  return ((uint64_t)hi << 32) | lo;
}

// Step 1 for root u: the rows of G_u.  Row i holds bit j (j > i) when nbr[j]
// is in N+(nbr[i]).  The warp takes the rows 32 at a time: lane t reads the
// extent [b, e) of row g + t's out-list, the 16-byte chunks covering all 32
// lists are numbered consecutively (a warp scan of the chunk counts), and
// every lane then loads build_unroll(W) chunks at once, finding each chunk's row
// by a binary search over the lanes' chunk offsets.  A chunk is the aligned
// 16-byte block holding the entries, so it never leaves the block of a valid
// entry; entries outside [b, e) are masked.  Each entry w <= nbr[d - 1] is
// looked up in nbr (ascending: by shuffles at width 1, in shared memory
// beyond) and sets its bit.  Returns this lane's count of DAG words read.
template <int W>
__device__ __forceinline__ uint32_t build_rows(WarpState<W>& st, const EnumKArgs& a, int d) {
  const uint32_t lane = lane_id();
  const uint32_t last = st.nbr[d - 1];
  const uintptr_t addr = (uintptr_t)a.ocol;
  const uint4* base4 = (const uint4*)(addr & ~(uintptr_t)15);
  const uint32_t dl = (uint32_t)((addr & 15u) >> 2);  // entry p is word p + dl of base4
  const uint32_t nb = (W == 1 && (int)lane < d) ? st.nbr[lane] : 0xFFFFFFFFu;
  int span = 1;  // largest power of two <= d (shared-memory search)
  while (2 * span <= d) span *= 2;
  constexpr int kBuildUnroll = build_unroll(W);
  uint32_t words = 0;
  for (int g = 0; g < d - 1; g += 32) {
    const int i = g + (int)lane;
    uint64_t c0 = 0;    // first chunk of row i's out-list
    uint32_t meta = 0;  // its first entry's word in that chunk (bits 0..1) and its length (bits 2..)
    uint32_t nch = 0;   // its chunks
    if (i < d - 1) {
      const uint32_t v = st.nbr[i];
      const uint64_t b = a.orow[v], e = a.orow[v + 1];
      const uint32_t len = (uint32_t)(e - b);
      c0 = (b + dl) >> 2;
      const uint32_t boff = (uint32_t)((b + dl) & 3u);
      meta = boff | (len << 2);
      nch = len ? (boff + len + 3) >> 2 : 0u;  // an empty list reads nothing
      words += len;
    }
    uint32_t pre = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, pre, o);
      if ((int)lane >= o) pre += t;
    }
    const uint32_t excl = pre - nch;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, pre, 31);
    for (uint32_t f0 = 0; f0 < total; f0 += 32 * kBuildUnroll) {
      uint4 val[kBuildUnroll];
      uint32_t tag[kBuildUnroll];  // row (bits 0..15) and valid entries (bits 16..19)
#pragma unroll
      for (int q = 0; q < kBuildUnroll; q++) {
        const uint32_t f = f0 + (uint32_t)(q * 32) + lane;
        int r = 0;  // the largest lane whose first chunk number is <= f
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1)
          if (__shfl_sync(0xFFFFFFFFu, excl, r + s) <= f) r += s;
        const uint32_t ci = f - __shfl_sync(0xFFFFFFFFu, excl, r);  // chunk of the row
        const uint64_t cr = shfl_u64(c0, r);
        const uint32_t mr = __shfl_sync(0xFFFFFFFFu, meta, r);
        tag[q] = 0;
        val[q] = make_uint4(0u, 0u, 0u, 0u);
        if (f < total) {
          val[q] = __ldg(base4 + cr + ci);
          // words 4 ci + x of the row's chunks hold entries when boff <= 4 ci + x < boff + len
          const uint32_t boff = mr & 3u, len = mr >> 2;
          uint32_t vm = 0;
#pragma unroll
          for (int x = 0; x < 4; x++) vm |= (4 * ci + x >= boff && 4 * ci + x < boff + len) ? (1u << x) : 0u;
          tag[q] = (uint32_t)(g + r) | (vm << 16);
        }
      }
#pragma unroll
      for (int q = 0; q < kBuildUnroll; q++) {
        const int row = (int)(tag[q] & 0xFFFFu);
#pragma unroll
        for (int x = 0; x < 4; x++) {
          const uint32_t w = x == 0 ? val[q].x : (x == 1 ? val[q].y : (x == 2 ? val[q].z : val[q].w));
          const bool live = ((tag[q] >> (16 + x)) & 1u) && w <= last;
          if (W == 1) {
            int j = 0;  // entries of nbr below w (lanes hold nbr, padded with the largest value)
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1)
              if (__shfl_sync(0xFFFFFFFFu, nb, j + s - 1) < w) j += s;
            const bool hit = __shfl_sync(0xFFFFFFFFu, nb, j) == w;
            if (live && hit) atomicOr(&st.rows[row], 1u << j);
          } else if (live) {
            int j = 0;
            for (int s = span; s >= 1; s >>= 1)
              if (j + s <= d && st.nbr[j + s - 1] < w) j += s;
            if (j < d && st.nbr[j] == w) atomicOr(&st.rows[(size_t)row * W + (j >> 5)], 1u << (j & 31));
          }
        }
      }
    }
  }
  return words;
}

// Largest j < p whose bit is set in B (and in A, when A is not null), or -1.
template <int W>
__device__ __forceinline__ int top_below(const uint32_t* A, const uint32_t* B, int p) {
  if (p <= 0) return -1;
  uint32_t lim = (p & 31) ? ((1u << (p & 31)) - 1u) : 0xFFFFFFFFu;
  for (int w = (p - 1) >> 5; w >= 0; w--) {
    uint32_t x = B[w] & lim;
    if (A) x &= A[w];
    if (x) return (w << 5) + 31 - __clz(x);
    lim = 0xFFFFFFFFu;
  }
  return -1;
}

// Algorithm 5 (soft embeddings, Sec. V) over the root's d local vertices,
// r capped at rcap; writes st.rr[0..d) and returns r of the root itself.
// Algorithm 5 walks a vertex's out-neighbours from the largest down with a
// counter c = 1 and increments c at each neighbour whose r is at least c.
// The neighbour where c reaches t + 1 is therefore the largest neighbour
// below the one where c reached t whose r is at least t.  Writing B_t for the
// vertices with r >= t, B_{t+1} follows from B_t alone: a vertex is in B_{t+1}
// when its row, restricted to B_t and below its previous increment point p,
// is not empty, and its new p is that set's top bit.  So all rows advance
// together, one round per t (lane = row), instead of one vertex after
// another; the root's own walk is the same over all d vertices.  B_t is kept
// in st.masks[t] (the masks of the search, which it equals for t < k) and
// each row's p in st.pidx (unused by a root's own state).  Same values as
// the vertex-by-vertex form: rows only hold larger vertices, and each B_t is
// complete before round t reads it.
template <int W>
__device__ uint32_t soft_embedding(WarpState<W>& st, int d, uint32_t rcap) {
  const uint32_t lane = lane_id();
  if (lane < W) {
    const int lo = (int)lane << 5;
    st.masks[W + lane] = d >= lo + 32 ? 0xFFFFFFFFu : (d > lo ? ((1u << (d - lo)) - 1u) : 0u);
  }
  for (int i = (int)lane; i < d; i += 32) {
    st.pidx[i] = (uint16_t)d;  // no increment point yet: the whole row
    st.rr[i] = 1;
  }
  __syncwarp();
  int q = d;  // the root's walk (the same on every lane)
  uint32_t root_r = 1;
  for (uint32_t t = 1; t < rcap; t++) {
    const uint32_t* B = st.masks + (size_t)t * W;  // B_t
    if (q >= 0) {
      q = top_below<W>(nullptr, B, q);
      if (q >= 0) root_r = t + 1;
    }
    bool any = false;
    for (int w = 0; w < W; w++) {
      const int i = (w << 5) + (int)lane;
      bool has = false;
      if (i < d) {
        const int np = top_below<W>(st.rows + (size_t)i * W, B, (int)st.pidx[i]);
        has = np >= 0;
        st.pidx[i] = (uint16_t)(has ? np : 0);  // 0: no further round can succeed
        if (has) st.rr[i] = (uint8_t)(t + 1);
      }
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, has);
      if (lane == 0 && t + 1 < rcap) st.masks[(size_t)(t + 1) * W + w] = bal;
      any |= bal != 0u;
    }
    __syncwarp();
    if (!any && q < 0) break;
  }
  __syncwarp();
  return root_r;
}

// Steps 1 and 2 for root u: bitmap rows, Algorithm 5, masks.  Returns false
// when the soft-embedding test drops the root.
template <int W>
__device__ bool build_root(WarpState<W>& st, const EnumKArgs& a, uint32_t u, int d, Acc& acc) {
  const uint32_t lane = lane_id();
  const uint32_t k = a.k, need = k - 1;
  const uint64_t ob = a.orow[u];
  for (int i = lane; i < d; i += 32) st.nbr[i] = a.ocol[ob + i];
  for (int i = lane; i < d * W; i += 32) st.rows[i] = 0u;
  __syncwarp();
  uint32_t words = build_rows<W>(st, a, d);
  __syncwarp();
  words = warp_sum(words);
  if (lane == 0) st.stats[kWsWords] += words;
  __syncwarp();
  // Algorithm 5 on G[N(u) ∪ {u}], r capped at k
  const uint32_t rcap = k;
  if (a.prune) {
    const uint32_t root_r = soft_embedding<W>(st, d, rcap);
    if (root_r < k) {
      if (lane == 0) st.stats[kWsPruned]++;
      return false;
    }
  } else {
    for (int i = lane; i < d; i += 32) st.rr[i] = (uint8_t)rcap;
    __syncwarp();
  }
  // masks[l] = local vertices with r >= l, for l in [1, k-1]
  for (uint32_t l = 1; l <= need; l++) {
#pragma unroll
    for (int w = 0; w < W; w++) {
      int i = (w << 5) + lane;
      bool b = i < d && st.rr[i] >= l;
      uint32_t m = __ballot_sync(0xFFFFFFFFu, b);
      if (lane == 0) st.masks[l * W + w] = m;
    }
  }
  __syncwarp();
  return true;
}

// Number of l-cliques (l >= 2) of G[S] for |S| = m <= 32, lane-partial (the
// lanes' values add up to it).  S is re-indexed to 0..m-1 in ascending order
// with one 32-bit row each, built by one ballot per vertex (lane j answers
// whether the vertex's row holds vertex j); lane i then counts the cliques
// whose smallest vertex is its vertex i on its own (lane_count).  At width 1
// the root-local indices already fit one word and only the mask by S is
// needed.  Called by the whole warp.
// Largest clique size counted by count_compact.  Its lane-local search has no
// memo, so its work grows like C(m, l - 1) on a dense set; up to 4 that stays
// below C(31, 3) steps per lane, and larger sizes go through the warp-level
// search (and the memo, where Eq. (1) calls for it) until they shrink to 4.
constexpr uint32_t kCompactMaxL = 4;

template <int W>
__device__ uint32_t count_compact(const WarpState<W>& st, const uint32_t (&S)[W], uint32_t m, uint32_t l,
                                  uint32_t& ops) {
  const uint32_t lane = lane_id();
  uint32_t myrow = 0;
  bool start;
  if (W == 1) {
    start = (S[0] >> lane) & 1u;
    if (start) myrow = st.rows[lane] & S[0];
  } else {
    start = lane < m;
    const int sv = start ? select_bit<W>(S, (int)lane) : 0;
    for (uint32_t i = 0; i + 1 < m; i++) {
      const int si = __shfl_sync(0xFFFFFFFFu, sv, (int)i);
      const bool bit = start && lane > i && ((st.rows[(size_t)si * W + (sv >> 5)] >> (sv & 31)) & 1u);
      const uint32_t b = __ballot_sync(0xFFFFFFFFu, bit);
      if (lane == i) myrow = b;
    }
  }
  st.crow[lane] = myrow;
  __syncwarp();
  const uint32_t c = start ? lane_count(st.crow, myrow, l - 1, ops) : 0u;
  __syncwarp();  // crow is rewritten by the next call
  return c;
}

template <int W>
__device__ __forceinline__ void all_bits(int d, uint32_t (&S)[W]) {
#pragma unroll
  for (int w = 0; w < W; w++) {
    int lo = w << 5;
    S[w] = d >= lo + 32 ? 0xFFFFFFFFu : (d <= lo ? 0u : (0xFFFFFFFFu >> (lo + 32 - d)));
  }
}

// Count of the cl-cliques of G[c] for cl <= 3, summed over the warp.
template <int W>
__device__ __forceinline__ unsigned long long small_count(const WarpState<W>& st, const uint32_t (&c)[W], uint32_t cl,
                                                          Acc& acc) {
  if (cl == 1) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < W; w++) s += __popc(c[w]);
    return s;
  }
  if (cl == 2) return warp_sum(edges_partial<W>(c, st.rows, acc.ops));
  return warp_sum(tri_partial<W>(c, st.rows, st.masks + 3 * W, acc.ops));
}

// Open a memoised frame for (c, cl): a stored whole key is a retrieval (returns
// true, value in *start_sum); otherwise *start_sum/*start_pos resume after the
// longest stored prefix of c (Sec. IV: the sibling link first, else a binary
// search over prefix lengths).
template <int W>
__device__ bool memo_open(const Memo& memo, const uint32_t (&c)[W], uint32_t cl, unsigned long long* start_sum,
                          int* start_pos, Acc& acc) {
  unsigned long long v;
  if (memo_find<W>(memo, c, cl, &v)) {
    *start_sum = v;
    acc.hits++;
    return true;
  }
  int m = 0;
#pragma unroll
  for (int w = 0; w < W; w++) m += __popc(c[w]);
  const int pmin = select_bit<W>(c, 0);
  uint32_t T1[W];
  suffix_of<W>(c, pmin + 1, T1);
  unsigned long long hv = 0;
  int hi = m;
  if (m > 1 && memo_find<W>(memo, T1, cl, &hv)) {
    hi = 1;
  } else {
    int lo = 2;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      uint32_t T[W];
      suffix_of<W>(c, select_bit<W>(c, mid), T);
      unsigned long long tv;
      if (memo_find<W>(memo, T, cl, &tv)) {
        hi = mid;
        hv = tv;
      } else {
        lo = mid + 1;
      }
    }
  }
  *start_sum = 0;
  *start_pos = top_bit<W>(c);
  if (hi < m) {
    *start_sum = hv;
    *start_pos = select_bit<W>(c, hi) - 1;
    acc.hits++;
  }
  acc.frames++;
  return false;
}

// Eq. (1) for a candidate set of sz vertices and e edges needing cl-cliques:
// 2 cl |E| > (cl - 1) |V|^2.
__device__ __forceinline__ bool eq1_holds(uint32_t cl, uint32_t sz, uint32_t e) {
  return 2ull * cl * e > (unsigned long long)(cl - 1) * sz * sz;
}

template <int W>
__device__ __forceinline__ bool eq1_dense(const WarpState<W>& st, const uint32_t (&c)[W], uint32_t cl, uint32_t sz,
                                          Acc& acc) {
  return eq1_holds(cl, sz, warp_sum(edges_partial<W>(c, st.rows, acc.ops)));
}

// The 2-plex early termination DIST applies for large k (Sec. VII-A), for
// counting.  G[S] is a 2-plex when every vertex of S is non-adjacent to at
// most one other vertex of S: its p = C(|S|, 2) - e non-edges then form a
// matching, and an l-clique of G[S] takes from each non-adjacent pair none or
// one of its two vertices, so G[S] has
//     sum over j of C(p, j) 2^j C(|S| - 2p, l - j)
// l-cliques (mod 2^64, with the binomials mod 2^64).  e = |E(S)|.  Returns
// false when G[S] is not a 2-plex.  The test: no vertex v has two missing
// vertices above it (M_v = S ∩ (v, ∞) minus row v has at most one member), and
// the vertices that touch a non-edge -- those with a non-empty M_v and the
// members of every M_v -- are 2p distinct vertices.  `scratch` holds W words
// (the sources' bitmap).  Called by the whole warp.
template <int W>
__device__ __forceinline__ bool plex2_tail(const WarpState<W>& st, const uint32_t (&S)[W], uint32_t sz, uint32_t l,
                                       uint32_t p, const unsigned long long* binom, uint32_t* scratch,
                                       unsigned long long* out) {
  if (p > 0) {
    const uint32_t lane = lane_id();
    bool bad = false;
    for (int w = 0; w < W; w++) {  // sources: lane's vertex (w, lane)
      uint32_t cnt = 0;
      if ((S[w] >> lane) & 1u) {
        const uint32_t* rv = st.rows + (size_t)((w << 5) + lane) * W;
        for (int w2 = w; w2 < W; w2++) {
          const uint32_t above = w2 > w ? 0xFFFFFFFFu : (lane == 31 ? 0u : (0xFFFFFFFFu << (lane + 1)));
          cnt += __popc(S[w2] & above & ~rv[w2]);
        }
      }
      bad |= cnt > 1;
      const uint32_t src = __ballot_sync(0xFFFFFFFFu, cnt == 1);
      if (lane == 0) scratch[w] = src;
    }
    if (__any_sync(0xFFFFFFFFu, bad)) return false;
    __syncwarp();
    uint32_t touched = 0;  // |sources ∪ members of the M_v|
    for (int w2 = 0; w2 < W; w2++) {
      uint32_t m = 0;
      for (int w = 0; w <= w2; w++) {
        if ((S[w] >> lane) & 1u) {
          const uint32_t above = w2 > w ? 0xFFFFFFFFu : (lane == 31 ? 0u : (0xFFFFFFFFu << (lane + 1)));
          m |= S[w2] & above & ~st.rows[(size_t)((w << 5) + lane) * W + w2];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m |= __shfl_xor_sync(0xFFFFFFFFu, m, o);
      touched += __popc(m | scratch[w2]);
    }
    __syncwarp();
    if (touched != 2 * p) return false;
  }
  constexpr int kCols = KC_MAX_K + 1;
  const uint32_t free_v = sz - 2 * p;
  unsigned long long t = 0;
  for (uint32_t j = 0; j <= p && j <= l; j++) {
    if (l - j > free_v) continue;
    t += binom[(size_t)p * kCols + j] * (1ull << j) * binom[(size_t)free_v * kCols + (l - j)];
  }
  *out = t;
  return true;
}

// The quick part of the test first: a 2-plex has at most |S| / 2 non-edges.
template <int W>
__device__ __forceinline__ bool plex2_count(const WarpState<W>& st, const uint32_t (&S)[W], uint32_t sz, uint32_t l,
                                            uint32_t e, const unsigned long long* binom, uint32_t* scratch,
                                            unsigned long long* out) {
  if (sz < l || sz < 2) return false;
  const unsigned long long pairs = (unsigned long long)sz * (sz - 1) / 2;
  if (e > pairs || 2 * (pairs - e) > sz) return false;
  return plex2_tail<W>(st, S, sz, l, (uint32_t)(pairs - e), binom, scratch, out);
}

// Plain depth-first search (MODE 0 count, MODE 1 list) below the frame at
// depth `base`, which the caller has set up (cand, pos and, for listing, the
// sorted prefix sid of length base + 1).
template <int W, int MODE>
__device__ void dfs_plain(WarpState<W>& st, const EnumKArgs& a, int base, Acc& acc) {
  const uint32_t lane = lane_id();
  const uint32_t k = a.k, need = k - 1;
  int depth = base;
  while (depth >= base) {
    const uint32_t l = need - depth;  // vertices still to pick from cand[depth]
    const uint32_t* S = st.cand + depth * W;
    if (MODE == 0 && l >= 3 && l <= kCompactMaxL) {
      uint32_t s[W], m = 0;
#pragma unroll
      for (int w = 0; w < W; w++) {
        s[w] = S[w];
        m += __popc(s[w]);
      }
      if (m <= 32) {
        acc.cnt += count_compact<W>(st, s, m, l, acc.ops);
        depth--;
        continue;
      }
    }
    if (MODE == 0 && l <= 3) {
      uint32_t s[W];
#pragma unroll
      for (int w = 0; w < W; w++) s[w] = S[w];
      if (l == 3) acc.cnt += tri_partial<W>(s, st.rows, st.masks + 3 * W, acc.ops);
      else if (l == 2) acc.cnt += edges_partial<W>(s, st.rows, acc.ops);
      else if (lane == 0) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < W; w++) c += __popc(s[w]);
        acc.cnt += c;
      }
      __syncwarp();
      depth--;
      continue;
    }
    if (MODE == 1 && l == 1) {
      // emit C ∪ {x} for each x in S: ids sorted, hashed, written
      const int plen = depth + 1;  // root + picks
#pragma unroll 1
      for (int w = 0; w < W; w++) {
        uint32_t x = S[w];
        if (!x) continue;
        bool mine = (x >> lane) & 1u;
        unsigned long long base_slot = 0;
        if (a.cap) {  // cap 0: total and checksum only, no slots
          if (lane == 0) base_slot = atomicAdd(&a.acc[kAccWritten], (unsigned long long)__popc(x));
          base_slot = __shfl_sync(0xFFFFFFFFu, base_slot, 0);
        }
        if (mine) {
          uint32_t id = a.vert[st.nbr[(w << 5) + lane]];
          unsigned long long slot = base_slot + __popc(x & lanemask_lt());
          bool wr = slot < a.cap;
          uint32_t* o = a.out + slot * (unsigned long long)k;
          uint64_t h = mix64(0x9E3779B97F4A7C15ull ^ (uint64_t)k);
          int j = 0;
          bool placed = false;
          for (int q = 0; q < plen; q++) {
            uint32_t y = st.sid[q];
            if (!placed && id < y) {
              h = mix64(h ^ (uint64_t)id);
              if (wr) o[j] = id;
              j++;
              placed = true;
            }
            h = mix64(h ^ (uint64_t)y);
            if (wr) o[j] = y;
            j++;
          }
          if (!placed) {
            h = mix64(h ^ (uint64_t)id);
            if (wr) o[j] = id;
          }
          acc.sum += h;
          acc.cnt += 1;
        }
      }
      __syncwarp();
      depth--;
      if (depth >= base) {
        if (lane == 0) {
          int plen2 = depth + 2;
          for (int q = st.sins[depth]; q + 1 < plen2; q++) st.sid[q] = st.sid[q + 1];
        }
        __syncwarp();
      }
      continue;
    }
    int v = next_desc<W>(S, st.masks + l * W, st.pos[depth]);
    if (v < 0) {
      __syncwarp();
      depth--;
      if (MODE == 1 && depth >= base) {
        if (lane == 0) {
          int plen2 = depth + 2;
          for (int q = st.sins[depth]; q + 1 < plen2; q++) st.sid[q] = st.sid[q + 1];
        }
        __syncwarp();
      }
      continue;
    }
    uint32_t c[W];
    uint32_t sz = 0, anym = 0;
    const uint32_t* rv = st.rows + (size_t)v * W;
    const uint32_t* mk = st.masks + (l - 1) * W;
#pragma unroll
    for (int w = 0; w < W; w++) {
      c[w] = S[w] & rv[w];
      sz += __popc(c[w]);
      anym |= c[w] & mk[w];
    }
    if (lane == 0) acc.ops += W;
    __syncwarp();
    if (lane == 0) st.pos[depth] = v - 1;
    if (MODE == 0 && a.plex && l - 1 >= 4 && sz >= l - 1 && anym) {
      // a child set that is a 2-plex is counted in closed form (Sec. VII-A)
      const uint32_t e = warp_sum(edges_partial<W>(c, st.rows, acc.ops));
      unsigned long long pv = 0;
      if (plex2_count<W>(st, c, sz, l - 1, e, a.binom, st.crow, &pv)) {
        if (lane == 0) {
          acc.cnt += pv;
          acc.plex++;
        }
        __syncwarp();
        continue;
      }
    }
    if (sz >= l - 1 && anym) {
      if (lane < W) st.cand[(depth + 1) * W + lane] = word_at<W>(c, lane);
      if (lane == 0) {
        st.pos[depth + 1] = top_bit<W>(c);
        if (MODE == 1) {
          uint32_t id = a.vert[st.nbr[v]];
          int plen = depth + 1;
          int q = plen;
          while (q > 0 && st.sid[q - 1] > id) {
            st.sid[q] = st.sid[q - 1];
            q--;
          }
          st.sid[q] = id;
          st.sins[depth] = (uint8_t)q;
        }
      }
      depth++;
    }
    __syncwarp();
  }
}

// Memoised count below the frame at depth `base` (set up by the caller: cand,
// pos, sum, dense, fullins); returns that frame's value, the same on every lane.
template <int W>
__device__ unsigned long long dfs_memo(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, int base, Acc& acc) {
  const uint32_t lane = lane_id();
  const uint32_t need = a.k - 1;
  int depth = base;
  unsigned long long result = 0;
  while (true) {
    const uint32_t l = need - depth;
    uint32_t S[W];
#pragma unroll
    for (int w = 0; w < W; w++) S[w] = st.cand[depth * W + w];
    const bool fd = st.dense[depth];
    int v = next_desc<W>(st.cand + depth * W, st.masks + l * W, st.pos[depth]);
    if (v < 0) {
      unsigned long long val = st.sum[depth];
      if (fd && !st.fullins[depth]) {
        int okk = memo_store<W>(memo, S, l, val);
        acc.ins += okk;
        acc.full += 1 - okk;
      }
      if (depth == base) {
        result = val;
        break;
      }
      depth--;
      const uint32_t lp = need - depth;
      uint32_t P[W];
#pragma unroll
      for (int w = 0; w < W; w++) P[w] = st.cand[depth * W + w];
      unsigned long long ps = st.sum[depth] + val;
      const int pv = st.cur[depth];
      const bool pd = st.dense[depth];
      __syncwarp();
      if (lane == 0) st.sum[depth] = ps;
      if (pd) {
        uint32_t T[W];
        suffix_of<W>(P, pv, T);
        int okk = memo_store<W>(memo, T, lp, ps);
        acc.ins += okk;
        acc.full += 1 - okk;
        bool whole = true;
#pragma unroll
        for (int w = 0; w < W; w++) whole &= (T[w] == P[w]);
        if (lane == 0 && whole) st.fullins[depth] = 1;
      }
      __syncwarp();
      continue;
    }
    __syncwarp();
    if (lane == 0) st.pos[depth] = v - 1;
    uint32_t c[W];
    uint32_t sz = 0;
    const uint32_t* rv = st.rows + (size_t)v * W;
#pragma unroll
    for (int w = 0; w < W; w++) {
      c[w] = S[w] & rv[w];
      sz += __popc(c[w]);
    }
    if (lane == 0) acc.ops += W;
    const uint32_t cl = l - 1;
    unsigned long long val = 0;
    bool resolved = true;
    bool cd = false;
    unsigned long long start_sum = 0;
    int start_pos = -1;
    if (cl <= 3) {
      if (sz < cl) val = 0;
      else if (cl == 3 && sz <= 32) val = warp_sum(count_compact<W>(st, c, sz, cl, acc.ops));
      else val = small_count<W>(st, c, cl, acc);
    } else {
      uint32_t anym = 0;
      const uint32_t* mk = st.masks + cl * W;
#pragma unroll
      for (int w = 0; w < W; w++) anym |= c[w] & mk[w];
      if (sz >= cl && anym) {
        // |E(c)| for the 2-plex test and Eq. (1) (below a dense frame Eq. (1) is not needed)
        const uint32_t e = (a.plex || (a.memo && !fd)) ? warp_sum(edges_partial<W>(c, st.rows, acc.ops)) : 0u;
        if (a.plex && plex2_count<W>(st, c, sz, cl, e, a.binom, st.crow, &val)) {
          if (lane == 0) acc.plex++;
        } else {
          cd = fd || (a.memo && eq1_holds(cl, sz, e));
          if (!cd && sz <= 32 && cl <= kCompactMaxL) {
            val = warp_sum(count_compact<W>(st, c, sz, cl, acc.ops));
          } else if (cd) {
            if (memo_open<W>(memo, c, cl, &start_sum, &start_pos, acc)) val = start_sum;
            else resolved = false;
          } else {
            resolved = false;
            start_pos = top_bit<W>(c);
          }
        }
      }
    }
    if (resolved) {
      unsigned long long ns = st.sum[depth] + val;
      __syncwarp();
      if (lane == 0) st.sum[depth] = ns;
      if (fd) {
        uint32_t T[W];
        suffix_of<W>(S, v, T);
        int okk = memo_store<W>(memo, T, l, ns);
        acc.ins += okk;
        acc.full += 1 - okk;
        bool whole = true;
#pragma unroll
        for (int w = 0; w < W; w++) whole &= (T[w] == S[w]);
        if (lane == 0 && whole) st.fullins[depth] = 1;
      }
      __syncwarp();
      continue;
    }
    // open the child frame
    if (lane < W) st.cand[(depth + 1) * W + lane] = word_at<W>(c, lane);
    if (lane == 0) {
      st.cur[depth] = v;
      st.pos[depth + 1] = start_pos;
      st.sum[depth + 1] = cd ? start_sum : 0ull;
      st.dense[depth + 1] = cd;
      st.fullins[depth + 1] = 0;
    }
    __syncwarp();
    depth++;
  }
  return result;
}

// ----------------------------------------------- listing with the trie
// MODE 3 lists like MODE 1 and reuses repeated sub-searches the way the
// Induced Subgraph Trie does for listing (Sec. IV, Algorithms 3 and 4): in a
// dense region (Eq. (1); below a dense frame every frame, as Algorithm 3
// recurses into itself) the l-cliques of a frame's set S are stored once --
// as tuples of local indices in this warp's arena, keyed by (S, l) in the
// warp's hash table -- and a later frame with the same (S, l) under another
// clique prefix replays them (ListingIST) instead of searching: each stored
// tuple joined with the prefix is emitted, lanes taking one tuple each.  A
// frame is recorded only while no ancestor is recording and when its C(|S|,
// l) upper bound fits the arena; the arena and table start empty for every
// root.  Replays and searches emit exactly the same cliques.

// C(m, l) saturated at 2^32 - 1: an upper bound on the l-cliques of an m-set.
__device__ __forceinline__ uint32_t binom_sat(uint32_t m, uint32_t l) {
  if (l > m) return 0;
  unsigned long long c = 1;
  for (uint32_t i = 1; i <= l; i++) {
    c = c * (m - l + i) / i;  // C(m - l + i, i), exact at every step
    if (c > 0xFFFFFFFFull) return 0xFFFFFFFFu;
  }
  return (uint32_t)c;
}

// Local-index type of stored tuples: one byte while a root has at most 256
// out-neighbours (widths up to 8 words), two beyond.
template <int W>
using LIdx = typename std::conditional<(W <= 8), uint8_t, uint16_t>::type;

// Emits prefix ∪ t for every stored tuple t (cnt tuples of lt local indices):
// ids sorted, hashed, written, one tuple per lane.
template <int W>
__device__ void list_replay(const WarpState<W>& st, const EnumKArgs& a, const LIdx<W>* ent, uint32_t cnt,
                            uint32_t lt, int plen, Acc& acc) {
  const uint32_t lane = lane_id();
  const uint32_t k = a.k;
  for (uint32_t t0 = 0; t0 < cnt; t0 += 32) {
    const uint32_t nb = min(32u, cnt - t0);
    unsigned long long base_slot = 0;
    if (a.cap) {
      if (lane == 0) base_slot = atomicAdd(&a.acc[kAccWritten], (unsigned long long)nb);
      base_slot = __shfl_sync(0xFFFFFFFFu, base_slot, 0);
    }
    if (lane < nb) {
      const LIdx<W>* tp = ent + (size_t)(t0 + lane) * lt;
      uint32_t ids[KMAX];
      for (uint32_t j = 0; j < lt; j++) {  // insertion sort by original id
        const uint32_t id = st.oid[tp[j]];
        uint32_t q = j;
        while (q > 0 && ids[q - 1] > id) {
          ids[q] = ids[q - 1];
          q--;
        }
        ids[q] = id;
      }
      const unsigned long long slot = base_slot + lane;
      const bool wr = slot < a.cap;
      uint32_t* o = a.out + slot * (unsigned long long)k;
      uint64_t h = mix64(0x9E3779B97F4A7C15ull ^ (uint64_t)k);
      int i = 0, q = 0;
      uint32_t j = 0;
      while (i < plen || j < lt) {
        uint32_t y;
        if (j >= lt || (i < plen && st.sid[i] < ids[j])) y = st.sid[i++];
        else y = ids[j++];
        h = mix64(h ^ (uint64_t)y);
        if (wr) o[q] = y;
        q++;
      }
      acc.sum += h;
      acc.cnt += 1;
    }
  }
  __syncwarp();
}

// Listing below the frame at depth `base` (set up by the caller: cand, pos,
// the sorted prefix sid of length base + 1, dense[base]).  lar / lcap / *ltop:
// this warp's arena, its size and the bytes this root has used.
template <int W>
__device__ void dfs_list_memo(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, uint8_t* lar, uint32_t lcap,
                              uint32_t* ltop, int base, Acc& acc) {
  using T = LIdx<W>;
  const uint32_t lane = lane_id();
  const uint32_t k = a.k, need = k - 1;
  int depth = base;
  int rec = -1;  // depth of the frame being recorded
  uint32_t rec_off = 0, rec_cnt = 0, rec_l = 0;
  bool rec_ok = true;
  // the base frame itself: a retrieval, or the start of a recording
  {
    const uint32_t l = need - base;
    if (st.dense[base] && l >= 2 && memo.cap) {
      uint32_t S[W], m = 0;
#pragma unroll
      for (int w = 0; w < W; w++) {
        S[w] = st.cand[base * W + w];
        m += __popc(S[w]);
      }
      unsigned long long v;
      if (memo_find<W>(memo, S, l, &v)) {
        acc.hits++;
        list_replay<W>(st, a, (const T*)(lar + (v >> 24)), (uint32_t)(v & 0xFFFFFFull), l, base + 1, acc);
        return;
      }
      const unsigned long long bound = (unsigned long long)binom_sat(m, l) * l * sizeof(T);
      if (*ltop + bound <= lcap) {
        rec = base;
        rec_off = *ltop;
        rec_cnt = 0;
        rec_l = l;
        rec_ok = true;
      }
    }
  }
  while (depth >= base) {
    const uint32_t l = need - depth;  // vertices still to pick from cand[depth]
    const uint32_t* S = st.cand + depth * W;
    if (l == 1) {
      // emit C ∪ {x} for each x in S: ids sorted, hashed, written; recorded
      // as tuples (picks from the recorded frame down, then x) when recording
      const int plen = depth + 1;
#pragma unroll 1
      for (int w = 0; w < W; w++) {
        uint32_t x = S[w];
        if (!x) continue;
        const bool mine = (x >> lane) & 1u;
        unsigned long long base_slot = 0;
        if (a.cap) {
          if (lane == 0) base_slot = atomicAdd(&a.acc[kAccWritten], (unsigned long long)__popc(x));
          base_slot = __shfl_sync(0xFFFFFFFFu, base_slot, 0);
        }
        const uint32_t rank_in = __popc(x & lanemask_lt());
        if (rec >= 0 && rec_ok) {
          if ((unsigned long long)rec_off + (unsigned long long)(rec_cnt + __popc(x)) * rec_l * sizeof(T) > lcap) {
            rec_ok = false;
          } else if (mine) {
            T* dst = (T*)(lar + rec_off) + (size_t)(rec_cnt + rank_in) * rec_l;
            for (uint32_t j = 0; j + 1 < rec_l; j++) dst[j] = (T)st.cur[rec + j];
            dst[rec_l - 1] = (T)((w << 5) + lane);
          }
          rec_cnt += __popc(x);
        }
        if (mine) {
          const uint32_t id = st.oid[(w << 5) + lane];
          const unsigned long long slot = base_slot + rank_in;
          const bool wr = slot < a.cap;
          uint32_t* o = a.out + slot * (unsigned long long)k;
          uint64_t h = mix64(0x9E3779B97F4A7C15ull ^ (uint64_t)k);
          int j = 0;
          bool placed = false;
          for (int q = 0; q < plen; q++) {
            const uint32_t y = st.sid[q];
            if (!placed && id < y) {
              h = mix64(h ^ (uint64_t)id);
              if (wr) o[j] = id;
              j++;
              placed = true;
            }
            h = mix64(h ^ (uint64_t)y);
            if (wr) o[j] = y;
            j++;
          }
          if (!placed) {
            h = mix64(h ^ (uint64_t)id);
            if (wr) o[j] = id;
          }
          acc.sum += h;
          acc.cnt += 1;
        }
      }
      __syncwarp();
      depth--;
      if (depth >= base) {
        if (lane == 0)
          for (int q = st.sins[depth]; q + 1 < depth + 2; q++) st.sid[q] = st.sid[q + 1];
        __syncwarp();
      }
      continue;
    }
    const int v = next_desc<W>(S, st.masks + l * W, st.pos[depth]);
    if (v < 0) {
      if (depth == rec) {  // the recorded frame is complete: store its l-cliques
        if (rec_ok) {
          uint32_t key[W];
#pragma unroll
          for (int w = 0; w < W; w++) key[w] = S[w];
          const int okk = memo_store<W>(memo, key, rec_l, ((unsigned long long)rec_off << 24) | rec_cnt);
          acc.ins += okk;
          acc.full += 1 - okk;
          if (okk) *ltop = rec_off + ((rec_cnt * rec_l * (uint32_t)sizeof(T) + 3u) & ~3u);
        }
        rec = -1;
      }
      __syncwarp();
      depth--;
      if (depth >= base) {
        if (lane == 0)
          for (int q = st.sins[depth]; q + 1 < depth + 2; q++) st.sid[q] = st.sid[q + 1];
        __syncwarp();
      }
      continue;
    }
    uint32_t c[W];
    uint32_t sz = 0, anym = 0;
    const uint32_t* rv = st.rows + (size_t)v * W;
    const uint32_t* mk = st.masks + (l - 1) * W;
#pragma unroll
    for (int w = 0; w < W; w++) {
      c[w] = S[w] & rv[w];
      sz += __popc(c[w]);
      anym |= c[w] & mk[w];
    }
    if (lane == 0) acc.ops += W;
    __syncwarp();
    if (lane == 0) st.pos[depth] = v - 1;
    if (sz >= l - 1 && anym) {
      const uint32_t cl = l - 1;
      const bool cd = st.dense[depth] || (a.memo && cl > 3 && eq1_dense<W>(st, c, cl, sz, acc));
      if (lane < W) st.cand[(depth + 1) * W + lane] = word_at<W>(c, lane);
      if (lane == 0) {
        st.pos[depth + 1] = top_bit<W>(c);
        st.cur[depth] = v;
        st.dense[depth + 1] = cd ? 1 : 0;
        const uint32_t id = st.oid[v];
        int q = depth + 1;
        while (q > 0 && st.sid[q - 1] > id) {
          st.sid[q] = st.sid[q - 1];
          q--;
        }
        st.sid[q] = id;
        st.sins[depth] = (uint8_t)q;
      }
      __syncwarp();
      bool replayed = false;
      if (cd && rec < 0 && cl >= 2 && memo.cap) {
        unsigned long long ev;
        if (memo_find<W>(memo, c, cl, &ev)) {
          acc.hits++;
          list_replay<W>(st, a, (const T*)(lar + (ev >> 24)), (uint32_t)(ev & 0xFFFFFFull), cl, depth + 2, acc);
          replayed = true;
        } else {
          const unsigned long long bound = (unsigned long long)binom_sat(sz, cl) * cl * sizeof(T);
          if (*ltop + bound <= lcap) {
            rec = depth + 1;
            rec_off = *ltop;
            rec_cnt = 0;
            rec_l = cl;
            rec_ok = true;
          }
        }
      }
      if (replayed) {  // the child is resolved: take its pick back out of the prefix
        if (lane == 0)
          for (int q = st.sins[depth]; q + 1 < depth + 2; q++) st.sid[q] = st.sid[q + 1];
        __syncwarp();
        continue;
      }
      depth++;
    }
    __syncwarp();
  }
}

// The searches are compiled once per width, in that width's translation
// unit (kc_enum_w*.cu, relocatable device code), and called out of line from
// every kernel: a width-W kernel also runs the narrow searches of smaller
// widths, and inlining them all would multiply the build time.  A call per
// root or branch costs little next to the search behind it.
template <int W, int MODE>
__device__ void dfs_plain_call(WarpState<W>& st, const EnumKArgs& a, int base, Acc& acc);
template <int W>
__device__ unsigned long long dfs_memo_call(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, int base,
                                            Acc& acc);
template <int W>
__device__ void dfs_list_memo_call(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, uint8_t* lar,
                                   uint32_t lcap, uint32_t* ltop, int base, Acc& acc);

#define KC_DFS_DECL(W)                                                                                    \
  template <>                                                                                             \
  __device__ void dfs_plain_call<W, 0>(WarpState<W> & st, const EnumKArgs& a, int base, Acc& acc);       \
  template <>                                                                                             \
  __device__ void dfs_plain_call<W, 1>(WarpState<W> & st, const EnumKArgs& a, int base, Acc& acc);       \
  template <>                                                                                             \
  __device__ unsigned long long dfs_memo_call<W>(WarpState<W> & st, const EnumKArgs& a, const Memo& memo, \
                                                 int base, Acc& acc);                                     \
  template <>                                                                                             \
  __device__ void dfs_list_memo_call<W>(WarpState<W> & st, const EnumKArgs& a, const Memo& memo,         \
                                        uint8_t* lar, uint32_t lcap, uint32_t* ltop, int base, Acc& acc);
KC_DFS_DECL(1)
KC_DFS_DECL(2)
KC_DFS_DECL(4)
KC_DFS_DECL(8)
KC_DFS_DECL(16)
KC_DFS_DECL(32)

// Adds the counters a search updates to the caller's accumulators.
__device__ __forceinline__ void acc_add(Acc& to, const Acc& from) {
  to.cnt += from.cnt;
  to.sum += from.sum;
  to.ops += from.ops;
  to.hits += from.hits;
  to.ins += from.ins;
  to.full += from.full;
  to.frames += from.frames;
  to.plex += from.plex;
}

// The definitions, for the width's own translation unit.  A search reached
// out of line (a narrow subproblem of a wider root, or a wide width) works on
// fresh counters, added to the caller's at the end, so that inside the
// search they live in registers.
#define KC_DFS_DEF(W)                                                                                            \
  template <>                                                                                                    \
  __device__ __noinline__ void dfs_plain_call<W, 0>(WarpState<W> & st_in, const EnumKArgs& a, int base,         \
                                                    Acc& acc_in) {                                               \
    Acc acc{};                                                                                                   \
    dfs_plain<W, 0>(st_in, a, base, acc);                                                                           \
    acc_add(acc_in, acc);                                                                                        \
  }                                                                                                              \
  template <>                                                                                                    \
  __device__ __noinline__ void dfs_plain_call<W, 1>(WarpState<W> & st_in, const EnumKArgs& a, int base,         \
                                                    Acc& acc_in) {                                               \
    Acc acc{};                                                                                                   \
    dfs_plain<W, 1>(st_in, a, base, acc);                                                                           \
    acc_add(acc_in, acc);                                                                                        \
  }                                                                                                              \
  template <>                                                                                                    \
  __device__ __noinline__ unsigned long long dfs_memo_call<W>(WarpState<W> & st_in, const EnumKArgs& a,         \
                                                              const Memo& memo_in, int base, Acc& acc_in) {      \
    Acc acc{};                                                                                                   \
    const unsigned long long v = dfs_memo<W>(st_in, a, memo_in, base, acc);                                            \
    acc_add(acc_in, acc);                                                                                        \
    return v;                                                                                                    \
  }                                                                                                              \
  template <>                                                                                                    \
  __device__ __noinline__ void dfs_list_memo_call<W>(WarpState<W> & st_in, const EnumKArgs& a,                  \
                                                     const Memo& memo_in, uint8_t* lar, uint32_t lcap,           \
                                                     uint32_t* ltop, int base, Acc& acc_in) {                    \
    Acc acc{};                                                                                                   \
    uint32_t top = *ltop;                                                                                        \
    dfs_list_memo<W>(st_in, a, memo_in, lar, lcap, &top, base, acc);                                                   \
    *ltop = top;                                                                                                 \
    acc_add(acc_in, acc);                                                                                        \
  }

// The kernel's own width: inlined below 16 words (as one unit with the
// kernel, the state and counters stay in registers); the wide widths go
// out of line, where the unrolled 16- and 32-word loops would otherwise be
// copied into every call site.
template <int W, int MODE>
__device__ __forceinline__ void dfs_plain_at(WarpState<W>& st, const EnumKArgs& a, int base, Acc& acc) {
  if constexpr (W >= 16) dfs_plain_call<W, MODE>(st, a, base, acc);
  else dfs_plain<W, MODE>(st, a, base, acc);
}

template <int W>
__device__ __forceinline__ unsigned long long dfs_memo_at(WarpState<W>& st, const EnumKArgs& a, const Memo& memo,
                                                          int base, Acc& acc) {
  if constexpr (W >= 16) return dfs_memo_call<W>(st, a, memo, base, acc);
  else return dfs_memo<W>(st, a, memo, base, acc);
}

template <int W>
__device__ __forceinline__ void dfs_list_memo_at(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, uint8_t* lar,
                                                 uint32_t lcap, uint32_t* ltop, int base, Acc& acc) {
  if constexpr (W >= 16) dfs_list_memo_call<W>(st, a, memo, lar, lcap, ltop, base, acc);
  else dfs_list_memo<W>(st, a, memo, lar, lcap, ltop, base, acc);
}

// The narrow state of a branch whose candidate set c (m vertices, in the
// root's width W) fits in W2 words: vertex j of the narrow state is the j-th
// smallest member of c, row j holds its larger neighbours inside c (one
// ballot per row and word: lane t answers whether row s_j of the wide matrix
// holds member t), and it keeps its rank, its r value and the masks by r.
template <int W, int W2>
__device__ void build_compact(const WarpState<W>& st, WarpState<W2>& cs, const uint32_t (&c)[W], int m, uint32_t need,
                              Acc& acc) {
  const uint32_t lane = lane_id();
  int base = 0;
#pragma unroll
  for (int w = 0; w < W; w++) {
    const uint32_t x = c[w];
    if ((x >> lane) & 1u) cs.pidx[base + __popc(x & lanemask_lt())] = (uint16_t)((w << 5) + lane);
    base += __popc(x);
  }
  __syncwarp();
  for (int j = lane; j < m; j += 32) {
    const int sp = cs.pidx[j];
    cs.nbr[j] = st.nbr[sp];
    cs.rr[j] = st.rr[sp];
  }
  for (int i = lane; i < m * W2; i += 32) cs.rows[i] = 0u;
  __syncwarp();
#pragma unroll 1
  for (int q = 0; q < W2; q++) {
    const int t = (q << 5) + (int)lane;  // this lane's narrow column
    const bool have = t < m;
    const int sp = have ? cs.pidx[t] : 0;
    const int sw = sp >> 5;
    const uint32_t sb = 1u << (sp & 31);
    const int iend = min(m, (q << 5) + 31);  // rows i < t of this word
#pragma unroll 1
    for (int i0 = 0; i0 < iend; i0 += 32) {
      const int cnt = min(32, iend - i0);
      uint32_t mine = 0;
#pragma unroll 1
      for (int ii = 0; ii < cnt; ii++) {
        const int i = i0 + ii;
        const int si = cs.pidx[i];
        const bool bit = have && t > i && (st.rows[(size_t)si * W + sw] & sb);
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, bit);
        if ((int)lane == ii) mine = b;
      }
      if ((int)lane < cnt) cs.rows[(size_t)(i0 + lane) * W2 + q] = mine;
    }
  }
  for (uint32_t l = 1; l <= need; l++) {
#pragma unroll
    for (int q = 0; q < W2; q++) {
      const int t = (q << 5) + (int)lane;
      const uint32_t mk = __ballot_sync(0xFFFFFFFFu, t < m && cs.rr[t] >= l);
      if (lane == 0) cs.masks[l * W2 + q] = mk;
    }
  }
  if (lane == 0) acc.ops += (uint32_t)(m * W2);  // one word produced per row and narrow word
  __syncwarp();
}

// A branch searched in its narrow state: the frame at depth 1 holds every
// narrow vertex; the clique prefix (root and v1) comes from the wide state.
template <int W, int W2, int MODE>
__device__ void run_narrow(WarpState<W>& st, const EnumKArgs& a, Memo& memo2, uint32_t* epoch2,
                           const uint32_t (&c)[W], int m, bool dense, Acc& acc) {
  const uint32_t lane = lane_id();
  WarpState<W2> cs;
  cs.carve(st.cbase, (int)a.depth);
  build_compact<W, W2>(st, cs, c, m, a.k - 1, acc);
  uint32_t S[W2];
  all_bits<W2>(m, S);
  if (lane < W2) cs.cand[W2 + lane] = word_at<W2>(S, lane);
  if (lane == 0) {
    cs.pos[1] = m - 1;
    if (MODE == 1) {
      cs.sid[0] = st.sid[0];
      cs.sid[1] = st.sid[1];
    }
    cs.sum[1] = 0;
    cs.dense[1] = dense ? 1 : 0;  // a dense frame memoises from the start (Algorithm 3)
    cs.fullins[1] = 0;
  }
  __syncwarp();
  if (MODE == 2) {
    next_epoch(memo2, epoch2);
    const unsigned long long v = dfs_memo_call<W2>(cs, a, memo2, 1, acc);
    if (lane == 0) acc.cnt += v;
  } else {
    dfs_plain_call<W2, MODE>(cs, a, 1, acc);
  }
}

template <int W, int MODE>
__device__ void narrow_dispatch(WarpState<W>& st, const EnumKArgs& a, Memo& memo2, uint32_t* epoch2,
                                const uint32_t (&c)[W], int m, int W2, bool dense, Acc& acc) {
  if (W2 == 1) {
    run_narrow<W, 1, MODE>(st, a, memo2, epoch2, c, m, dense, acc);
    return;
  }
  if constexpr (compact_width(W) >= 2) {
    if (W2 == 2) {
      run_narrow<W, 2, MODE>(st, a, memo2, epoch2, c, m, dense, acc);
      return;
    }
  }
  if constexpr (compact_width(W) >= 4) {
    if (W2 == 4) {
      run_narrow<W, 4, MODE>(st, a, memo2, epoch2, c, m, dense, acc);
      return;
    }
  }
  if constexpr (compact_width(W) >= 8) {
    if (W2 == 8) run_narrow<W, 8, MODE>(st, a, memo2, epoch2, c, m, dense, acc);
  }
}

// Everything below one first-level branch v1 of a built root (a branch of
// the root's own loop, or a task of the split path): the (k-2)-cliques of
// G_u ∩ N(v1).  A branch that is not dense by Eq. (1) and whose candidate set
// fits a bit-matrix at most half as wide is searched in that narrow state.
template <int W, int MODE>
__device__ __forceinline__ void run_branch_body(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, Memo& memo2,
                                                uint32_t* epoch2, uint32_t u, int d, int v1, Acc& acc,
                                                bool parent_dense) {
  const uint32_t lane = lane_id();
  const uint32_t need = a.k - 1;
  uint32_t S0[W], c[W];
  all_bits<W>(d, S0);
  uint32_t sz = 0;
  const uint32_t* rv = st.rows + (size_t)v1 * W;
#pragma unroll
  for (int w = 0; w < W; w++) {
    c[w] = S0[w] & rv[w];
    sz += __popc(c[w]);
  }
  if (lane == 0) acc.ops += W;
  const uint32_t cl = need - 1;
  if (sz < cl) return;
  if (cl >= 2) {
    // Lemma 1: a cl-clique inside c starts at a vertex with r >= cl
    uint32_t anym = 0;
    const uint32_t* mk = st.masks + cl * W;
#pragma unroll
    for (int w = 0; w < W; w++) anym |= c[w] & mk[w];
    if (!anym) return;
  }
  // a branch whose set is a 2-plex is counted in closed form (Sec. VII-A)
  uint32_t e = 0;
  bool have_e = false;
  if (!is_list(MODE) && a.plex && cl >= 4) {
    e = warp_sum(edges_partial<W>(c, st.rows, acc.ops));
    have_e = true;
    unsigned long long pv = 0;
    if (plex2_count<W>(st, c, sz, cl, e, a.binom, st.crow, &pv)) {
      if (lane == 0) {
        acc.cnt += pv;
        acc.plex++;
      }
      return;
    }
  }
  // Eq. (1) for the branch's frame; below a dense frame every frame is
  // memoised (Algorithm 3 recurses into itself)
  const bool cd = uses_trie(MODE) && cl > 3 &&
                  (parent_dense || (a.memo && (have_e ? eq1_holds(cl, sz, e) : eq1_dense<W>(st, c, cl, sz, acc))));
  if (!is_list(MODE) && cl >= 3 && cl <= kCompactMaxL && sz <= 32 && !cd) {
    acc.cnt += count_compact<W>(st, c, sz, cl, acc.ops);
    return;
  }
  if (is_list(MODE) && lane == 0) {
    uint32_t iu = a.vert[u], iv = a.vert[st.nbr[v1]];
    st.sid[0] = min(iu, iv);
    st.sid[1] = max(iu, iv);
  }
  if constexpr (compact_width(W) > 0) {
    // a dense branch of a root of 16 or 32 words is narrowed too, with its
    // trie in the narrow index space: the branch's own frames still share
    // their entries, and every intersection shrinks to a few words
    const bool narrow_dense = cd && W >= 16 && MODE == 2 && memo2.cap != 0;
    if ((!cd || narrow_dense) && (is_list(MODE) ? cl >= 2 : cl >= 3)) {
      // the narrowest width that holds the set: W2 words hold 32 * W2 vertices
      const int W2 = sz <= 32 ? 1 : (sz <= 64 ? 2 : (sz <= 128 ? 4 : (sz <= 256 ? 8 : 16)));
      if (2 * W2 <= W && W2 <= compact_width(W) && (int)sz <= 32 * W2) {
        __syncwarp();
        if (is_list(MODE)) narrow_dispatch<W, 1>(st, a, memo2, epoch2, c, (int)sz, W2, false, acc);
        else if (MODE == 2 && memo2.cap == 0) narrow_dispatch<W, 0>(st, a, memo2, epoch2, c, (int)sz, W2, false, acc);
        else narrow_dispatch<W, MODE>(st, a, memo2, epoch2, c, (int)sz, W2, cd, acc);
        return;
      }
    }
  }
  if (!is_list(MODE) && cl <= 3) {
    unsigned long long v = small_count<W>(st, c, cl, acc);
    if (lane == 0) acc.cnt += v;
    return;
  }
  if (lane < W) st.cand[W + lane] = word_at<W>(c, lane);
  if (MODE == 1 || (MODE == 3 && !cd)) {
    if (lane == 0) st.pos[1] = top_bit<W>(c);
    __syncwarp();
    dfs_plain_at<W, 1>(st, a, 1, acc);
    return;
  }
  if (MODE == 3) {  // a dense branch: listed through the trie
    if (lane == 0) {
      st.pos[1] = top_bit<W>(c);
      st.dense[1] = 1;
    }
    __syncwarp();
    dfs_list_memo_at<W>(st, a, memo, memo.lar, memo.lcap, memo.ltop, 1, acc);
    return;
  }
  if (MODE == 0) {
    if (lane == 0) st.pos[1] = top_bit<W>(c);
    __syncwarp();
    dfs_plain_at<W, 0>(st, a, 1, acc);
    return;
  }
  // MODE 2
  unsigned long long ssum = 0;
  int spos = top_bit<W>(c);
  if (cd && memo_open<W>(memo, c, cl, &ssum, &spos, acc)) {
    if (lane == 0) acc.cnt += ssum;
    return;
  }
  if (lane == 0) {
    st.pos[1] = spos;
    st.sum[1] = cd ? ssum : 0ull;
    st.dense[1] = cd;
    st.fullins[1] = 0;
  }
  __syncwarp();
  unsigned long long v = dfs_memo_at<W>(st, a, memo, 1, acc);
  if (lane == 0) acc.cnt += v;
}

// One branch: inlined below 16 words; out of line beyond, on fresh
// counters (see the search wrappers).
template <int W, int MODE>
__device__ __noinline__ void run_branch_outlined(WarpState<W>& st_in, const EnumKArgs& a, const Memo& memo_in,
                                                 Memo& memo2, uint32_t* epoch2, uint32_t u, int d, int v1,
                                                 Acc& acc_in, bool parent_dense) {
  Acc acc{};
  run_branch_body<W, MODE>(st_in, a, memo_in, memo2, epoch2, u, d, v1, acc, parent_dense);
  acc_add(acc_in, acc);
}

template <int W, int MODE>
__device__ __forceinline__ void run_branch(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, Memo& memo2,
                                           uint32_t* epoch2, uint32_t u, int d, int v1, Acc& acc, bool parent_dense) {
  if constexpr (W >= 16) run_branch_outlined<W, MODE>(st, a, memo, memo2, epoch2, u, d, v1, acc, parent_dense);
  else run_branch_body<W, MODE>(st, a, memo, memo2, epoch2, u, d, v1, acc, parent_dense);
}

// Heavy root: copy its built state to the arena and queue one task per
// first-level branch v1 < limit (the branches this warp has not done).
// Returns false when the arena is full (keep it local).
template <int W, int MODE>
__device__ bool publish_root(WarpState<W>& st, const EnumKArgs& a, uint32_t u, int d, Acc& acc, int limit,
                             bool dense) {
  const uint32_t lane = lane_id();
  const uint32_t need = a.k - 1;
  const uint64_t units = (16 + (uint64_t)d * 4 + (uint64_t)d * W * 4 + (uint64_t)d + 15) / 16;
  unsigned long long off = 0;
  if (lane == 0) off = atomicAdd(a.arena_used, units);
  off = __shfl_sync(0xFFFFFFFFu, off, 0);
  if (off + units > a.arena_units) return false;
  uint8_t* base = a.arena + off * 16;
  uint32_t* hdr = (uint32_t*)base;
  uint32_t* nbr = hdr + 4;
  uint32_t* rows = nbr + d;
  uint8_t* rr = (uint8_t*)(rows + (size_t)d * W);
  if (lane == 0) {
    hdr[0] = u;
    hdr[1] = (uint32_t)d;
    hdr[2] = a.query;
    hdr[3] = dense ? 1u : 0u;
  }
  for (int i = lane; i < d; i += 32) {
    nbr[i] = st.nbr[i];
    rr[i] = st.rr[i];
  }
  for (int i = lane; i < d * W; i += 32) rows[i] = st.rows[i];
  // one task per v1 < limit with r_v1 >= k-1
  uint32_t S0[W];
  all_bits<W>(limit, S0);
  const uint32_t* mk = st.masks + need * W;
  uint32_t nt = 0;
#pragma unroll
  for (int w = 0; w < W; w++) nt += __popc(S0[w] & mk[w]);
  unsigned long long t0 = 0;
  if (lane == 0) t0 = atomicAdd(a.task_used, (unsigned long long)nt);
  t0 = __shfl_sync(0xFFFFFFFFu, t0, 0);
  uint32_t done = 0;
#pragma unroll 1
  for (int w = 0; w < W; w++) {
    uint32_t x = S0[w] & mk[w];
    if ((x >> lane) & 1u) {
      unsigned long long slot = t0 + done + __popc(x & lanemask_lt());
      if (slot < a.task_cap) a.tasks[slot] = (off << 32) | (unsigned long long)((w << 5) + lane);
    }
    done += __popc(x);
  }
  __threadfence();
  if (lane == 0) {
    st.stats[kWsHeavy]++;
    st.stats[kWsTasks] += nt;
  }
  // branches past the queue's capacity stay with this warp
  if (t0 + nt > a.task_cap) {
    Memo none{}, none2{};
    uint32_t ep2 = 0;
    uint32_t skip = t0 < a.task_cap ? (uint32_t)(a.task_cap - t0) : 0u;
    uint32_t idx = 0;
    for (int w = 0; w < W; w++) {
      uint32_t x = S0[w] & mk[w];
      while (x) {
        int b = __ffs(x) - 1;
        x &= x - 1;
        if (idx++ >= skip) run_branch<W, is_list(MODE) ? 1 : 0>(st, a, none, none2, &ep2, u, d, (w << 5) + b, acc,
                                                                   false);
      }
    }
  }
  return true;
}

template <int W>
__device__ void flush_acc(const EnumKArgs& a, Acc& acc, const unsigned long long* ws) {
  const uint32_t lane = lane_id();
  unsigned long long cnt = warp_sum(acc.cnt);
  unsigned long long sum = warp_sum(acc.sum);
  unsigned long long ops = warp_sum(acc.ops64 + acc.ops);
  const unsigned long long plex = warp_sum((unsigned long long)acc.plex);
  if (lane == 0) {
    if (ops) atomicAdd(&a.acc[kAccWordOps], ops);
    if (cnt) atomicAdd(&a.acc[kAccCount], cnt);
    if (sum) atomicAdd(&a.acc[kAccChecksum], sum);
    if (ws[kWsPruned]) atomicAdd(&a.acc[kAccRootsPruned], ws[kWsPruned]);
    if (ws[kWsWords]) atomicAdd(&a.acc[kAccBuildWords], ws[kWsWords]);
    if (acc.hits) atomicAdd(&a.acc[kAccMemoHits], acc.hits);
    if (acc.ins) atomicAdd(&a.acc[kAccMemoInserts], acc.ins);
    if (acc.full) atomicAdd(&a.acc[kAccMemoFull], acc.full);
    if (acc.frames) atomicAdd(&a.acc[kAccMemoFrames], acc.frames);
    if (plex) atomicAdd(&a.acc[kAccPlex], plex);
    if (ws[kWsHeavy]) atomicAdd(&a.acc[kAccRootsHeavy], ws[kWsHeavy]);
    if (ws[kWsTasks]) atomicAdd(&a.acc[kAccTasks], ws[kWsTasks]);
    if (ws[kWsBuildNs]) atomicAdd(&a.acc[kAccBuildNs], ws[kWsBuildNs]);
    if (ws[kWsBusyNs]) atomicAdd(&a.acc[kAccBusyNs], ws[kWsBusyNs]);
    const unsigned long long peak = max(ws[kWsInsPeak], acc.ins - ws[kWsInsMark]);
    if (peak) atomicMax(&a.acc[kAccMemoPeak], peak);
  }
}

template <int W>
__device__ __forceinline__ void carve_state(WarpState<W>& st, const EnumKArgs& a, uint8_t* smem) {
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint8_t* mine = smem + (size_t)(threadIdx.x >> 5) * a.sstride;
  if (a.gstate) st.carve(a.gstate + gwarp * a.gstride, (int)a.depth);
  else st.carve(mine, (int)a.depth);
  if (compact_width(W)) st.cbase = mine + a.coff;
  st.stats = (unsigned long long*)(mine + a.soff_stats);
  if (lane_id() < kWsCount) st.stats[lane_id()] = 0ull;
  __syncwarp();
}

// This warp's memo tables: the root's index space, then (where the width has
// a narrow branch state) a quarter-size table for the narrow subproblems,
// each of which starts its own epoch there.
template <int W>
__device__ __forceinline__ void warp_memo(const EnumKArgs& a, Memo* m, Memo* m2) {
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  *m = Memo{};
  *m2 = Memo{};
  if (a.larena) {
    m->lar = a.larena + gwarp * a.larena_bytes;
    m->lcap = a.larena_bytes;
  }
  if (!a.memo_cap) return;
  const uint64_t stride = (uint64_t)a.memo_cap + a.memo_cap2;
  m->tags = a.memo_tags + gwarp * stride;
  m->keys = a.memo_keys + gwarp * stride * W;
  m->vals = a.memo_vals + gwarp * stride;
  m->cap = a.memo_cap;
  if (a.memo_cap2) {
    m2->tags = m->tags + a.memo_cap;
    m2->keys = m->keys + (size_t)a.memo_cap * W;  // the narrow keys (width <= W/2) fit in the same stride
    m2->vals = m->vals + a.memo_cap;
    m2->cap = a.memo_cap2;
  }
}

// Phase 1: one warp per root, roots taken from the tier's list.
// MODE 0: count (plain), 1: list, 2: count with memo, 3: list with memo.
// Everything for one root u of the graph in `a`: build, prune, then split,
// count or list.  Counts accumulate in acc.cnt (lane-partial).
template <int W, int MODE>
__device__ void root_body(WarpState<W>& st, const EnumKArgs& a, Memo& memo, uint32_t* epoch, Memo& memo2,
                          uint32_t* epoch2, uint32_t u, Acc& acc, bool timed) {
  const uint32_t lane = lane_id();
  const uint32_t need = a.k - 1;
  const int d = (int)(a.orow[u + 1] - a.orow[u]);
  const unsigned long long tb = timed ? global_ns() : 0ull;
  const bool kept = build_root<W>(st, a, u, d, acc);
  if (timed && lane == 0) st.stats[kWsBuildNs] += global_ns() - tb;
  if (!kept) return;
  uint32_t S0[W];
  all_bits<W>(d, S0);
  if (uses_trie(MODE)) {
    next_epoch(memo, epoch);
    if (lane == 0) {
      st.stats[kWsInsPeak] = max(st.stats[kWsInsPeak], acc.ins - st.stats[kWsInsMark]);
      st.stats[kWsInsMark] = acc.ins;
    }
    if (MODE == 3) {
      if (memo.ltop) *memo.ltop = 0;  // the arena holds this root's lists only
      for (int i = lane; i < d; i += 32) st.oid[i] = a.vert[st.nbr[i]];
      __syncwarp();
    }
  }
  // Eq. (1) on G_u for the root frame; a root whose G_u is a 2-plex is
  // counted in closed form (Sec. VII-A)
  bool dense0 = false;
  if ((uses_trie(MODE) && a.memo && need > 3) || (!is_list(MODE) && a.plex && need >= 4)) {
    uint32_t er = 0;
    for (int i = lane; i < d * W; i += 32) er += __popc(st.rows[i]);
    er = warp_sum(er);
    if (!is_list(MODE) && a.plex && need >= 4) {
      unsigned long long pv = 0;
      if (plex2_count<W>(st, S0, (uint32_t)d, need, er, a.binom, st.crow, &pv)) {
        if (lane == 0) {
          acc.cnt += pv;
          acc.plex++;
        }
        return;
      }
    }
    dense0 = uses_trie(MODE) && a.memo && need > 3 && eq1_holds(need, (uint32_t)d, er);
  }
  // EdgeParallel (Sec. VII-D) as the whole decomposition: every root's
  // first-level branches (u, v1) are tasks of the second phase
  if (a.edge_all && need >= 2 && publish_root<W, MODE>(st, a, u, d, acc, d, dense0)) return;
  // heavy roots go to the split path: one task per first-level branch
  // dense roots keep their memo whole unless they are wide (more than 64 out-neighbours)
  if (a.split_wedges && d > a.split_min_d && (!dense0 || W >= 4) && need >= 4) {
    uint32_t wg = 0;
    for (int i = lane; i < d; i += 32) {
      uint32_t p = 0;
#pragma unroll
      for (int w = 0; w < W; w++) p += __popc(st.rows[(size_t)i * W + w]);
      wg += p * (p - 1) / 2;
    }
    wg = warp_sum(wg);
    // a wide dense root's search grows with k: its threshold halves for every k above 5
    const uint32_t thr = dense0 ? (a.split_wedges >> min(need - 4u, 12u)) : a.split_wedges;
    if (wg > thr && publish_root<W, MODE>(st, a, u, d, acc, d, dense0)) return;
  }
  if (W >= 16 && (need >= 4 || (is_list(MODE) && need >= 2))) {
    // the root frame of a wide root (16 or 32 words): one branch after
    // another, from the largest vertex down (the order of the identifying
    // strings, so that a dense branch resumes from its sibling's stored set),
    // each searched in a narrow state where its candidate set allows.
    // Narrower roots search from the root frame itself: at 2 to 8 words a
    // branch's re-indexing costs about what it saves.
    if (lane < W) st.cand[lane] = word_at<W>(S0, lane);
    __syncwarp();
    const uint32_t* m1 = st.masks + need * W;
    for (int v1 = next_desc<W>(st.cand, m1, d - 1); v1 >= 0; v1 = next_desc<W>(st.cand, m1, v1 - 1))
      run_branch<W, MODE>(st, a, memo, memo2, epoch2, u, d, v1, acc, dense0);
  } else if (!is_list(MODE) && need >= 2 && need <= kCompactMaxL && d <= 32 && !dense0) {
    // the whole root at once: one word per row, lanes take the smallest vertex
    acc.cnt += count_compact<W>(st, S0, (uint32_t)d, need, acc.ops);
  } else if (MODE == 0 || MODE == 1 || (MODE == 3 && need < 2)) {
    if (lane < W) st.cand[lane] = word_at<W>(S0, lane);
    if (lane == 0) {
      st.pos[0] = d - 1;
      if (is_list(MODE)) st.sid[0] = a.vert[u];
    }
    __syncwarp();
    dfs_plain_at<W, is_list(MODE) ? 1 : 0>(st, a, 0, acc);
  } else if (MODE == 3) {
    if (lane < W) st.cand[lane] = word_at<W>(S0, lane);
    if (lane == 0) {
      st.pos[0] = d - 1;
      st.sid[0] = a.vert[u];
      st.dense[0] = dense0 ? 1 : 0;
    }
    __syncwarp();
    dfs_list_memo_at<W>(st, a, memo, memo.lar, memo.lcap, memo.ltop, 0, acc);
  } else {
    if (need <= 3) {
      unsigned long long v = small_count<W>(st, S0, need, acc);
      if (lane == 0) acc.cnt += v;
    } else {
      if (lane < W) st.cand[lane] = word_at<W>(S0, lane);
      if (lane == 0) {
        st.pos[0] = d - 1;
        st.sum[0] = 0;
        st.dense[0] = dense0;
        st.fullins[0] = 0;
      }
      __syncwarp();
      unsigned long long v = dfs_memo_at<W>(st, a, memo, 0, acc);
      if (lane == 0) acc.cnt += v;
    }
  }
}

// The graph and k of batch query q (batched counting).
__device__ __forceinline__ void bind_query(EnumKArgs& b, const EnumKArgs& a, uint32_t q) {
  const BatchQuery bq = a.bq[q];
  b.orow = bq.orow;
  b.ocol = bq.ocol;
  b.vert = bq.vert;
  b.k = bq.k;
  b.query = q;
}

// A batch query's count (and, listing, checksum) so far, moved from the
// lanes' partials to its slots.
template <int MODE>
__device__ __forceinline__ void flush_query(const EnumKArgs& a, uint32_t q, Acc& acc) {
  const unsigned long long c = warp_sum(acc.cnt);
  acc.cnt = 0;
  if (lane_id() == 0 && c) atomicAdd(&a.bcount[q], c);
  if (is_list(MODE)) {
    const unsigned long long h = warp_sum(acc.sum);
    acc.sum = 0;
    if (lane_id() == 0 && h) atomicAdd(&a.bsum[q], h);
  }
}

// Phase 1: one warp per root, roots taken from the tier's list.  With a batch
// (a.bq set) each list entry also names its query.
// MODE 0: count (plain), 1: list, 2: count with memo, 3: list with memo.
template <int W, int MODE>
__global__ void __launch_bounds__(kc_block_threads(W), kc_min_blocks(W)) k_enum(const __grid_constant__ EnumKArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = lane_id();
  WarpState<W> st;
  carve_state<W>(st, a, smem);
  Acc acc;
  Memo memo, memo2;
  warp_memo<W>(a, &memo, &memo2);
  uint32_t ltop = 0;
  memo.ltop = &ltop;
  uint32_t epoch = 0, epoch2 = 0;
  while (true) {
    uint32_t qi = 0;
    if (lane == 0) qi = atomicAdd(a.qctr, 1u);
    qi = __shfl_sync(0xFFFFFFFFu, qi, 0);
    if (qi >= a.nroots) break;
    const uint32_t u = a.roots[qi];
    // one root in 16 of each warp is timed (the clock read is not free): the
    // build's share of warp time is estimated on those
    const bool timed = (qi & 15u) == 0;
    const unsigned long long t0 = timed ? global_ns() : 0ull;
    if (a.bq) {
      const uint32_t q = a.roots_q[qi];
      EnumKArgs b = a;
      bind_query(b, a, q);
      root_body<W, MODE>(st, b, memo, &epoch, memo2, &epoch2, u, acc, timed);
      flush_query<MODE>(a, q, acc);
    } else {
      root_body<W, MODE>(st, a, memo, &epoch, memo2, &epoch2, u, acc, timed);
    }
    if (timed && lane == 0) st.stats[kWsBusyNs] += global_ns() - t0;
    acc.ops64 += acc.ops;
    acc.ops = 0;
    __syncwarp();
  }
  flush_acc<W>(a, acc, st.stats);
}

// Phase 2: the split path.  Every warp takes (root, v1) tasks; a root's built
// state is loaded from the arena when the task's root changes.
template <int W, int MODE>
__global__ void __launch_bounds__(kc_block_threads(W), kc_min_blocks(W)) k_tasks(const __grid_constant__ EnumKArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = lane_id();
  WarpState<W> st;
  carve_state<W>(st, a, smem);
  EnumKArgs b = a;  // bound to the current root's query in a batch
  uint32_t need = a.k - 1;
  Acc acc;
  Memo memo, memo2;
  warp_memo<W>(a, &memo, &memo2);
  uint32_t ltop = 0;
  memo.ltop = &ltop;
  uint32_t epoch = 1u << 24, epoch2 = 1u << 24;  // above every epoch of phase 1
  const unsigned long long ntasks = min(*(volatile unsigned long long*)a.task_used, a.task_cap);
  unsigned long long cur = ~0ull;
  uint32_t u = 0;
  int d = 0;
  bool dense = false;
  while (true) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.task_head, 1ull);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= ntasks) break;
    const bool timed = (t & 15ull) == 0;
    const unsigned long long t0 = timed ? global_ns() : 0ull;
    const unsigned long long task = a.tasks[t];
    const unsigned long long off = task >> 32;
    const int v1 = (int)(task & 0xFFFFFFFFull);
    if (off != cur) {
      const uint8_t* base = a.arena + off * 16;
      const uint32_t* hdr = (const uint32_t*)base;
      u = hdr[0];
      d = (int)hdr[1];
      dense = hdr[3] != 0;
      if (a.bq) {
        bind_query(b, a, hdr[2]);
        need = b.k - 1;
      }
      const uint32_t* nbr = hdr + 4;
      const uint32_t* rows = nbr + d;
      const uint8_t* rr = (const uint8_t*)(rows + (size_t)d * W);
      for (int i = lane; i < d; i += 32) {
        st.nbr[i] = nbr[i];
        st.rr[i] = rr[i];
      }
      for (int i = lane; i < d * W; i += 32) st.rows[i] = rows[i];
      __syncwarp();
      for (uint32_t l = 1; l <= need; l++) {
#pragma unroll
        for (int w = 0; w < W; w++) {
          int i = (w << 5) + lane;
          bool b = i < d && st.rr[i] >= l;
          uint32_t m = __ballot_sync(0xFFFFFFFFu, b);
          if (lane == 0) st.masks[l * W + w] = m;
        }
      }
      __syncwarp();
      cur = off;
      if (uses_trie(MODE)) {
        next_epoch(memo, &epoch);
        if (lane == 0) {
          st.stats[kWsInsPeak] = max(st.stats[kWsInsPeak], acc.ins - st.stats[kWsInsMark]);
          st.stats[kWsInsMark] = acc.ins;
        }
      }
      if (MODE == 3) {
        ltop = 0;
        const uint32_t* vmap = a.bq ? b.vert : a.vert;
        for (int i = lane; i < d; i += 32) st.oid[i] = vmap[st.nbr[i]];
        __syncwarp();
      }
    }
    // the kernel's own arguments are read in place; only a batch binds a copy
    run_branch<W, MODE>(st, a.bq ? b : a, memo, memo2, &epoch2, u, d, v1, acc, dense);
    if (a.bq) flush_query<MODE>(a, b.query, acc);
    if (timed && lane == 0) st.stats[kWsBusyNs] += global_ns() - t0;
    acc.ops64 += acc.ops;
    acc.ops = 0;
    __syncwarp();
  }
  flush_acc<W>(a, acc, st.stats);
}

// Bitmap words of width tier t: 1, 2, 4, ..., 32 words.
__host__ __device__ constexpr int tier_words(int t) { return 1 << t; }

// Kernel entry points of one width, for mode 0 (count), 1 (list), 2 (count
// with the memo), 3 (list with the memo); each kc_enum_w*.cu instantiates one
// width with this.  With MEMO 0 mode 2 would fall back to the count without
// the memo.
#define KC_TIER_KERNELS(W, MEMO)                                                 \
  void tier_kernels_w##W(int mode, const void** fe, const void** ft) {          \
    if (mode == 1) {                                                             \
      *fe = (const void*)k_enum<W, 1>;                                           \
      *ft = (const void*)k_tasks<W, 1>;                                          \
    } else if (mode == 3) {                                                      \
      *fe = (const void*)k_enum<W, 3>;                                           \
      *ft = (const void*)k_tasks<W, 3>;                                          \
    } else if (mode == 2 && MEMO) {                                              \
      *fe = (const void*)k_enum<W, (MEMO ? 2 : 0)>;                              \
      *ft = (const void*)k_tasks<W, (MEMO ? 2 : 0)>;                             \
    } else {                                                                     \
      *fe = (const void*)k_enum<W, 0>;                                           \
      *ft = (const void*)k_tasks<W, 0>;                                          \
    }                                                                            \
  }

void tier_kernels_w1(int mode, const void** fe, const void** ft);
void tier_kernels_w2(int mode, const void** fe, const void** ft);
void tier_kernels_w4(int mode, const void** fe, const void** ft);
void tier_kernels_w8(int mode, const void** fe, const void** ft);
void tier_kernels_w16(int mode, const void** fe, const void** ft);
void tier_kernels_w32(int mode, const void** fe, const void** ft);

}  // namespace kc
