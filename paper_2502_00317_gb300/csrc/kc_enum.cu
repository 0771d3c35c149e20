// kc_enum.cu -- per-root enumeration of libkc.so (one warp per root of the DAG).
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
#include <algorithm>
#include <mutex>
#include <vector>

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
  uint32_t* out;
  unsigned long long cap;
  unsigned long long* acc;
  uint8_t* gstate;            // per-warp state in global memory (heavy tiers)
  unsigned long long gstride; // bytes per warp
  uint32_t* memo_tags;        // per-warp tables: cap entries each
  uint32_t* memo_keys;
  unsigned long long* memo_vals;
  uint32_t memo_cap;          // entries per warp (power of two)
  uint32_t* status;
  // split path (heavy roots): arena of published roots and a task queue
  uint32_t split_wedges;      // 0: never split
  int split_min_d;
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
  uint32_t query;               // query bound to this copy of the arguments
};


// Per-warp working state, carved from shared or global memory.
template <int W>
struct WarpState {
  uint32_t* nbr;              // [32W] ranks of N+(u), ascending
  uint32_t* rows;             // [32W*W] bit-matrix rows
  uint32_t* masks;            // [KMAX*W] masks[l*W+w]: local vertices with r >= l
  uint32_t* cand;             // [KMAX*W] candidate set per depth
  unsigned long long* sum;    // [KMAX] frame partial counts (memo variant)
  int32_t* pos;               // [KMAX] next pick position (descending), -1 when done
  int32_t* cur;               // [KMAX] vertex whose child frame is open
  uint32_t* sid;              // [KMAX+1] sorted original ids of the open clique prefix
  uint8_t* sins;              // [KMAX] insertion index of each pick in sid
  uint8_t* rr;                // [32W] r values (Algorithm 5), capped at k
  uint8_t* dense;             // [KMAX] frame uses the memo
  uint8_t* fullins;           // [KMAX] frame's whole set already stored
  uint32_t* crow;             // [32] rows of a candidate set re-indexed to 0..31 (count_compact)
  __host__ __device__ static constexpr size_t bytes() {
    return (size_t)32 * W * 4 + (size_t)32 * W * W * 4 + (size_t)KMAX * W * 4 * 2 + (size_t)KMAX * 8 +
           (size_t)KMAX * 4 * 2 + (size_t)(KMAX + 1) * 4 + KMAX + 32 * W + KMAX * 2 + 16 + 32 * 4;
  }
  __device__ void carve(uint8_t* base) {
    uint8_t* p = base;
    sum = (unsigned long long*)p; p += (size_t)KMAX * 8;
    crow = (uint32_t*)p; p += 32 * 4;
    nbr = (uint32_t*)p; p += (size_t)32 * W * 4;
    rows = (uint32_t*)p; p += (size_t)32 * W * W * 4;
    masks = (uint32_t*)p; p += (size_t)KMAX * W * 4;
    cand = (uint32_t*)p; p += (size_t)KMAX * W * 4;
    pos = (int32_t*)p; p += (size_t)KMAX * 4;
    cur = (int32_t*)p; p += (size_t)KMAX * 4;
    sid = (uint32_t*)p; p += (size_t)(KMAX + 1) * 4;
    sins = p; p += KMAX;
    rr = p; p += 32 * W;
    dense = p; p += KMAX;
    fullins = p;
  }
};

template <int W>
__host__ __device__ constexpr size_t warp_state_bytes() {
  return (WarpState<W>::bytes() + 15) & ~(size_t)15;
}

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
};

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
__device__ __forceinline__ int memo_probe(const Memo& m, const uint32_t (&key)[W], uint32_t l, int* free_slot) {
  const uint32_t lane = lane_id();
  uint32_t h = memo_hash<W>(key, l);
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
  int s = memo_probe<W>(m, key, l, &fs);
  if (s < 0) return false;
  *val = m.vals[s];
  return true;
}

// Store (key, l) -> val; returns 1 if stored, 0 if the window was full.
template <int W>
__device__ __forceinline__ int memo_store(const Memo& m, const uint32_t (&key)[W], uint32_t l, unsigned long long val) {
  int fs;
  int s = memo_probe<W>(m, key, l, &fs);
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
__device__ __forceinline__ uint32_t tri_partial(const uint32_t (&S)[W], const uint32_t* rows, const uint32_t* m3,
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
  unsigned long long ops64 = 0;
  unsigned long long pruned = 0, words = 0, hits = 0, ins = 0, full = 0, frames = 0, heavy = 0, tasks = 0;
};

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
  const uint32_t last = st.nbr[d - 1];
  uint32_t words = 0;
  if (W == 1) {
    // at most 31 rows: the warp reads each out-list 32 entries at a time and
    // places each entry by a binary search in nbr (ranks above the row)
    for (int i = 0; i < d - 1; i++) {
      const uint32_t v = st.nbr[i];
      const uint64_t b = a.orow[v], e = a.orow[v + 1];
      for (uint64_t p0 = b; p0 < e; p0 += 32) {
        const uint64_t p = p0 + lane;
        const uint32_t w = p < e ? __ldg(&a.ocol[p]) : 0xFFFFFFFFu;
        words += (p < e);
        if (w <= last) {
          int lo = i + 1, hi = d;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (st.nbr[mid] < w) lo = mid + 1;
            else hi = mid;
          }
          if (lo < d && st.nbr[lo] == w) atomicOr(&st.rows[(size_t)i * W + (lo >> 5)], 1u << (lo & 31));
        }
        if (__all_sync(0xFFFFFFFFu, w > last)) break;
      }
    }
  } else {
    // one lane per row: row i holds the positions j > i with nbr[j] in
    // N+(nbr[i]), found by merging the two ascending lists; 32 rows at once
    for (int i = lane; i < d - 1; i += 32) {
      const uint32_t v = st.nbr[i];
      const uint64_t b = a.orow[v], e = a.orow[v + 1];
      uint32_t* row = st.rows + (size_t)i * W;
      int j = i + 1;
      uint64_t p = b;
      while (p < e && j < d) {
        const uint32_t w = __ldg(&a.ocol[p]);
        if (w > last) break;
        while (j < d && st.nbr[j] < w) j++;
        if (j < d && st.nbr[j] == w) {
          row[j >> 5] |= 1u << (j & 31);
          j++;
        }
        p++;
      }
      words += (uint32_t)(p - b);
    }
  }
  acc.words += words;
  __syncwarp();
  // Algorithm 5 on G[N(u) ∪ {u}], r capped at k
  const uint32_t rcap = k;
  if (a.prune) {
    uint32_t root_r = rcap;
    if (lane == 0) {
      for (int i = d - 1; i >= 0; i--) {
        uint32_t c = 1;
        const uint32_t* row = st.rows + (size_t)i * W;
        for (int w = W - 1; w >= 0 && c < rcap; w--) {
          uint32_t x = row[w];
          while (x && c < rcap) {
            int b = 31 - __clz(x);
            x &= ~(1u << b);
            if (c <= st.rr[(w << 5) + b]) c++;
          }
        }
        st.rr[i] = (uint8_t)c;
      }
      uint32_t c = 1;
      for (int j = d - 1; j >= 0 && c < rcap; j--)
        if (c <= st.rr[j]) c++;
      root_r = c;
    }
    root_r = __shfl_sync(0xFFFFFFFFu, root_r, 0);
    __syncwarp();
    if (root_r < k) {
      acc.pruned++;
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

// Eq. (1) for a candidate set c needing cl-cliques: 2 cl |E| > (cl - 1) |V|^2.
template <int W>
__device__ __forceinline__ bool eq1_dense(const WarpState<W>& st, const uint32_t (&c)[W], uint32_t cl, uint32_t sz,
                                          Acc& acc) {
  uint32_t e = warp_sum(edges_partial<W>(c, st.rows, acc.ops));
  return 2ull * cl * e > (unsigned long long)(cl - 1) * sz * sz;
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
        if (lane == 0) base_slot = atomicAdd(&a.acc[kAccWritten], (unsigned long long)__popc(x));
        base_slot = __shfl_sync(0xFFFFFFFFu, base_slot, 0);
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
        cd = fd || (a.memo && eq1_dense<W>(st, c, cl, sz, acc));
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

// Everything below one first-level branch v1 of a built root (a task of the
// split path, or a branch kept local): the (k-2)-cliques of G_u ∩ N(v1).
template <int W, int MODE>
__device__ void run_branch(WarpState<W>& st, const EnumKArgs& a, const Memo& memo, uint32_t u, int d, int v1,
                           Acc& acc) {
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
  if (MODE != 1 && cl >= 3 && cl <= kCompactMaxL && sz <= 32 &&
      (MODE == 0 || !(a.memo && cl > 3 && eq1_dense<W>(st, c, cl, sz, acc)))) {
    acc.cnt += count_compact<W>(st, c, sz, cl, acc.ops);
    return;
  }
  if (MODE != 1 && cl <= 3) {
    unsigned long long v = small_count<W>(st, c, cl, acc);
    if (lane == 0) acc.cnt += v;
    return;
  }
  if (lane < W) st.cand[W + lane] = word_at<W>(c, lane);
  if (MODE == 1) {
    if (lane == 0) {
      uint32_t iu = a.vert[u], iv = a.vert[st.nbr[v1]];
      st.sid[0] = min(iu, iv);
      st.sid[1] = max(iu, iv);
      st.pos[1] = top_bit<W>(c);
    }
    __syncwarp();
    dfs_plain<W, 1>(st, a, 1, acc);
    return;
  }
  if (MODE == 0) {
    if (lane == 0) st.pos[1] = top_bit<W>(c);
    __syncwarp();
    dfs_plain<W, 0>(st, a, 1, acc);
    return;
  }
  // MODE 2
  bool cd = a.memo && eq1_dense<W>(st, c, cl, sz, acc);
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
  unsigned long long v = dfs_memo<W>(st, a, memo, 1, acc);
  if (lane == 0) acc.cnt += v;
}

// Heavy root: copy its built state to the arena and queue one task per
// first-level branch.  Returns false when the arena is full (keep it local).
template <int W, int MODE>
__device__ bool publish_root(WarpState<W>& st, const EnumKArgs& a, uint32_t u, int d, Acc& acc) {
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
  }
  for (int i = lane; i < d; i += 32) {
    nbr[i] = st.nbr[i];
    rr[i] = st.rr[i];
  }
  for (int i = lane; i < d * W; i += 32) rows[i] = st.rows[i];
  // one task per v1 with r_v1 >= k-1
  uint32_t S0[W];
  all_bits<W>(d, S0);
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
  acc.heavy++;
  acc.tasks += nt;
  // branches past the queue's capacity stay with this warp
  if (t0 + nt > a.task_cap) {
    Memo none{};
    uint32_t skip = t0 < a.task_cap ? (uint32_t)(a.task_cap - t0) : 0u;
    uint32_t idx = 0;
    for (int w = 0; w < W; w++) {
      uint32_t x = S0[w] & mk[w];
      while (x) {
        int b = __ffs(x) - 1;
        x &= x - 1;
        if (idx++ >= skip) run_branch<W, MODE == 1 ? 1 : 0>(st, a, none, u, d, (w << 5) + b, acc);
      }
    }
  }
  return true;
}

template <int W>
__device__ void flush_acc(const EnumKArgs& a, Acc& acc) {
  const uint32_t lane = lane_id();
  unsigned long long cnt = warp_sum(acc.cnt);
  unsigned long long sum = warp_sum(acc.sum);
  unsigned long long words = warp_sum(acc.words);
  unsigned long long ops = warp_sum(acc.ops64 + acc.ops);
  if (lane == 0) {
    if (ops) atomicAdd(&a.acc[kAccWordOps], ops);
    if (cnt) atomicAdd(&a.acc[kAccCount], cnt);
    if (sum) atomicAdd(&a.acc[kAccChecksum], sum);
    if (acc.pruned) atomicAdd(&a.acc[kAccRootsPruned], acc.pruned);
    if (words) atomicAdd(&a.acc[kAccBuildWords], words);
    if (acc.hits) atomicAdd(&a.acc[kAccMemoHits], acc.hits);
    if (acc.ins) atomicAdd(&a.acc[kAccMemoInserts], acc.ins);
    if (acc.full) atomicAdd(&a.acc[kAccMemoFull], acc.full);
    if (acc.frames) atomicAdd(&a.acc[kAccMemoFrames], acc.frames);
    if (acc.heavy) atomicAdd(&a.acc[kAccRootsHeavy], acc.heavy);
    if (acc.tasks) atomicAdd(&a.acc[kAccTasks], acc.tasks);
  }
}

template <int W>
__device__ __forceinline__ void carve_state(WarpState<W>& st, const EnumKArgs& a, uint8_t* smem) {
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (a.gstate) st.carve(a.gstate + gwarp * a.gstride);
  else st.carve(smem + (size_t)(threadIdx.x >> 5) * warp_state_bytes<W>());
}

template <int W>
__device__ __forceinline__ Memo warp_memo(const EnumKArgs& a) {
  const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  Memo m{};
  if (a.memo_cap) {
    m.tags = a.memo_tags + gwarp * a.memo_cap;
    m.keys = a.memo_keys + gwarp * a.memo_cap * W;
    m.vals = a.memo_vals + gwarp * a.memo_cap;
    m.cap = a.memo_cap;
  }
  return m;
}

__device__ __forceinline__ void next_epoch(Memo& memo, uint32_t* epoch) {
  if (++*epoch >= (1u << 25)) {
    for (uint32_t i = lane_id(); i < memo.cap; i += 32) memo.tags[i] = 0u;
    __syncwarp();
    *epoch = 1;
  }
  memo.tagbase = *epoch << 7;
}

// Phase 1: one warp per root, roots taken from the tier's list.
// MODE 0: count (plain), 1: list, 2: count with memo.
// Everything for one root u of the graph in `a`: build, prune, then split,
// count or list.  Counts accumulate in acc.cnt (lane-partial).
template <int W, int MODE>
__device__ void root_body(WarpState<W>& st, const EnumKArgs& a, Memo& memo, uint32_t* epoch, uint32_t u, Acc& acc) {
  const uint32_t lane = lane_id();
  const uint32_t need = a.k - 1;
  const int d = (int)(a.orow[u + 1] - a.orow[u]);
  if (!build_root<W>(st, a, u, d, acc)) return;
  uint32_t S0[W];
  all_bits<W>(d, S0);
  if (MODE == 2) next_epoch(memo, epoch);
  // Eq. (1) on G_u for the root frame
  bool dense0 = false;
  if (MODE == 2 && a.memo && need > 3) {
    uint32_t er = 0;
    for (int i = lane; i < d * W; i += 32) er += __popc(st.rows[i]);
    er = warp_sum(er);
    dense0 = 2ull * need * er > (unsigned long long)(need - 1) * d * d;
  }
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
    if (wg > thr && publish_root<W, MODE>(st, a, u, d, acc)) return;
  }
  if (MODE != 1 && need >= 2 && need <= kCompactMaxL && d <= 32 && !dense0) {
    // the whole root at once: one word per row, lanes take the smallest vertex
    acc.cnt += count_compact<W>(st, S0, (uint32_t)d, need, acc.ops);
  } else if (MODE == 0 || MODE == 1) {
    if (lane < W) st.cand[lane] = word_at<W>(S0, lane);
    if (lane == 0) {
      st.pos[0] = d - 1;
      if (MODE == 1) st.sid[0] = a.vert[u];
    }
    __syncwarp();
    dfs_plain<W, MODE>(st, a, 0, acc);
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
      unsigned long long v = dfs_memo<W>(st, a, memo, 0, acc);
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

// A batch query's count so far, moved from the lanes' partials to its slot.
__device__ __forceinline__ void flush_query(const EnumKArgs& a, uint32_t q, Acc& acc) {
  const unsigned long long c = warp_sum(acc.cnt);
  acc.cnt = 0;
  if (lane_id() == 0 && c) atomicAdd(&a.bcount[q], c);
}

// Phase 1: one warp per root, roots taken from the tier's list.  With a batch
// (a.bq set) each list entry also names its query.
// MODE 0: count (plain), 1: list, 2: count with memo.
template <int W, int MODE>
__global__ void __launch_bounds__(256) k_enum(EnumKArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = lane_id();
  WarpState<W> st;
  carve_state<W>(st, a, smem);
  Acc acc;
  Memo memo = warp_memo<W>(a);
  uint32_t epoch = 0;
  while (true) {
    uint32_t qi = 0;
    if (lane == 0) qi = atomicAdd(a.qctr, 1u);
    qi = __shfl_sync(0xFFFFFFFFu, qi, 0);
    if (qi >= a.nroots) break;
    const uint32_t u = a.roots[qi];
    if (MODE != 1 && a.bq) {
      const uint32_t q = a.roots_q[qi];
      EnumKArgs b = a;
      bind_query(b, a, q);
      root_body<W, MODE>(st, b, memo, &epoch, u, acc);
      flush_query(a, q, acc);
    } else {
      root_body<W, MODE>(st, a, memo, &epoch, u, acc);
    }
    acc.ops64 += acc.ops;
    acc.ops = 0;
    __syncwarp();
  }
  flush_acc<W>(a, acc);
}

// Phase 2: the split path.  Every warp takes (root, v1) tasks; a root's built
// state is loaded from the arena when the task's root changes.
template <int W, int MODE>
__global__ void __launch_bounds__(256) k_tasks(EnumKArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t lane = lane_id();
  WarpState<W> st;
  carve_state<W>(st, a, smem);
  EnumKArgs b = a;  // bound to the current root's query in a batch
  uint32_t need = a.k - 1;
  Acc acc;
  Memo memo = warp_memo<W>(a);
  uint32_t epoch = 1u << 24;  // above every epoch of phase 1
  const unsigned long long ntasks = min(*(volatile unsigned long long*)a.task_used, a.task_cap);
  unsigned long long cur = ~0ull;
  uint32_t u = 0;
  int d = 0;
  while (true) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.task_head, 1ull);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= ntasks) break;
    const unsigned long long task = a.tasks[t];
    const unsigned long long off = task >> 32;
    const int v1 = (int)(task & 0xFFFFFFFFull);
    if (off != cur) {
      const uint8_t* base = a.arena + off * 16;
      const uint32_t* hdr = (const uint32_t*)base;
      u = hdr[0];
      d = (int)hdr[1];
      if (MODE != 1 && a.bq) {
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
      if (MODE == 2) next_epoch(memo, &epoch);
    }
    run_branch<W, MODE>(st, b, memo, u, d, v1, acc);
    if (MODE != 1 && a.bq) flush_query(a, b.query, acc);
    acc.ops64 += acc.ops;
    acc.ops = 0;
    __syncwarp();
  }
  flush_acc<W>(a, acc);
}

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
__host__ __device__ constexpr int tier_words(int t) { return 1 << t; }  // 1, 2, 4, ..., 32 words

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
  uint32_t memo_cap = 0;       // entries per warp (0: no memo)
  uint64_t memo_bytes = 0;
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

template <int W, int MODE>
static int plan_tier(kc_ctx* ctx, uint32_t nroots, bool split, TierPlan* tp) {
  constexpr size_t wbytes = warp_state_bytes<W>();
  const bool in_smem = W <= 8;
  tp->W = W;
  tp->mode = MODE;
  tp->nroots = nroots;
  tp->fn = (const void*)k_enum<W, MODE>;
  tp->fn_tasks = (const void*)k_tasks<W, MODE>;
  if (nroots == 0) return KC_OK;
  tp->warps_per_block = W <= 4 ? 8 : 4;
  tp->smem = in_smem ? wbytes * tp->warps_per_block : 0;
  if (tp->smem > 48 * 1024) {
    KC_CUDA(cudaFuncSetAttribute(k_enum<W, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp->smem));
    KC_CUDA(cudaFuncSetAttribute(k_tasks<W, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp->smem));
  }
  int per_sm = 0;
  KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enum<W, MODE>, tp->warps_per_block * 32, tp->smem));
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
    uint64_t max_warps = std::max<uint64_t>(4, (1ull << 30) / wbytes);
    blocks = std::max<uint64_t>(1, std::min<uint64_t>(blocks, max_warps / tp->warps_per_block));
    tp->gstate_bytes = wbytes;
  }
  tp->blocks = blocks;
  if (MODE == 2) {
    uint64_t warps = blocks * tp->warps_per_block;
    uint32_t cap = 1u << 12;
    uint64_t budget = ctx->opts.memo_bytes ? ctx->opts.memo_bytes : (1ull << 30);
    uint64_t per_entry = 4 + 4ull * W + 8;
    while (cap > 256 && warps * cap * per_entry > budget / kTiers) cap >>= 1;
    tp->memo_cap = cap;
    tp->memo_bytes = warps * cap * per_entry;
  }
  return KC_OK;
}

template <int MODE>
static int plan_all(kc_ctx* ctx, const uint32_t* hcnt, bool split, TierPlan* plans) {
  // tiers wider than 8 words keep their state in global memory and count without the memo
  constexpr int M16 = (MODE == 2) ? 0 : MODE;
  KC_TRY((plan_tier<1, MODE>(ctx, hcnt[0], false, &plans[0])));
  KC_TRY((plan_tier<2, MODE>(ctx, hcnt[1], split, &plans[1])));
  KC_TRY((plan_tier<4, MODE>(ctx, hcnt[2], split, &plans[2])));
  KC_TRY((plan_tier<8, MODE>(ctx, hcnt[3], split, &plans[3])));
  KC_TRY((plan_tier<16, M16>(ctx, hcnt[4], split, &plans[4])));
  KC_TRY((plan_tier<32, M16>(ctx, hcnt[5], split, &plans[5])));
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
  const uint32_t split_wedges =
      ctx->opts.split_threshold == 0 ? kDefaultSplitWedges
      : (ctx->opts.split_threshold == 0xFFFFFFFFu ? 0u : ctx->opts.split_threshold);
  // the split path needs at least two levels below the first branch (k >= 5)
  const bool split = split_wedges != 0 && split_ok;
  TierPlan plans[kTiers];
  if (mode == 1) KC_TRY(plan_all<1>(ctx, hcnt, split, plans));
  else if (mode == 2) KC_TRY(plan_all<2>(ctx, hcnt, split, plans));
  else KC_TRY(plan_all<0>(ctx, hcnt, split, plans));
  // one scratch region for every tier's global state, memo tables, arena and task queue
  uint64_t total = 0;
  uint64_t goff[kTiers], moff[kTiers], aoff[kTiers], toff[kTiers];
  for (int t = 0; t < kTiers; t++) {
    goff[t] = total;
    total += (plans[t].gstate_bytes * plans[t].blocks * std::max(plans[t].warps_per_block, 1) + 255) & ~255ull;
    moff[t] = total;
    total += (plans[t].memo_bytes + 255) & ~255ull;
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
      x.memo_vals = (unsigned long long*)mb;
      x.memo_tags = (uint32_t*)(mb + warps * tp.memo_cap * 8);
      x.memo_keys = (uint32_t*)(mb + warps * tp.memo_cap * 12);
      x.memo_cap = tp.memo_cap;
      KC_CUDA(cudaMemsetAsync(x.memo_tags, 0, warps * tp.memo_cap * 4, ts));
    }
    if (tp.split) {
      x.split_wedges = split_wedges;
      x.split_min_d = 32;
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
    const int mode = ea.mode == 1 ? 1 : ((ea.memo && k >= 3) ? 2 : 0);
    EnumKArgs args{};
    args.orow = g.orow;
    args.ocol = g.ocol;
    args.vert = g.vert;
    args.k = k;
    args.prune = ea.prune ? 1 : 0;
    args.memo = ea.memo ? 1 : 0;
    args.out = ea.d_buf;
    args.cap = ea.cap;
    args.acc = ctx->d_acc;
    args.status = ctx->d_status;
    uint32_t* troots[kTiers];
    for (int t = 0; t < kTiers; t++) troots[t] = lists + (size_t)t * lcap;
    KC_TRY(launch_tiers(ctx, args, hcnt, troots, nullptr, mode, k >= 5, s, &launches, &enum_launches));
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
      if (bq.k >= 3 && d >= bq.k - 1) {
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
              cudaStream_t s) {
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
  KC_TRY(scratch_get(ctx, kScrBatch, qbytes + obytes + cbytes + 256, &meta));
  BatchQuery* d_q = (BatchQuery*)meta;
  uint64_t* d_off = (uint64_t*)((uint8_t*)meta + qbytes);
  unsigned long long* d_cnt = (unsigned long long*)((uint8_t*)meta + qbytes + obytes);
  uint32_t* d_tc = (uint32_t*)((uint8_t*)meta + qbytes + obytes + cbytes);
  KC_CUDA(cudaMemcpyAsync(d_q, hq, (size_t)nq * sizeof(BatchQuery), cudaMemcpyHostToDevice, s));
  KC_CUDA(cudaMemcpyAsync(d_off, qoff.data(), ((size_t)nq + 1) * 8, cudaMemcpyHostToDevice, s));
  KC_CUDA(cudaMemsetAsync(d_cnt, 0, (size_t)nq * 8, s));
  KC_CUDA(cudaMemsetAsync(d_tc, 0, 256, s));
  BinBatchArgs ba{};
  ba.bq = d_q;
  ba.qoff = d_off;
  ba.nq = nq;
  ba.total = total;
  ba.cnts = d_tc;
  ba.acc = ctx->d_acc;
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
    args.prune = prune ? 1 : 0;
    args.memo = memo ? 1 : 0;
    args.acc = ctx->d_acc;
    args.status = ctx->d_status;
    args.bq = d_q;
    args.bcount = d_cnt;
    uint32_t* troots[kTiers];
    uint32_t* troots_q[kTiers];
    for (int t = 0; t < kTiers; t++) {
      troots[t] = ba.roots + ba.tier_off[t];
      troots_q[t] = ba.roots_q + ba.tier_off[t];
    }
    KC_TRY(launch_tiers(ctx, args, hcnt, troots, troots_q, memo ? 2 : 0, any5, s, &launches, &enum_launches));
  }
  KC_CUDA(cudaEventRecord(ev[7], s));
  KC_CUDA(cudaMemcpyAsync(counts, d_cnt, (size_t)nq * 8, cudaMemcpyDeviceToHost, s));
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

template <int W>
int static_tier(int num_sms, const EnumKArgs& x, cudaStream_t s) {
  kc_ctx* ctx = nullptr;  // for KC_CUDA: errors carry no context
  const int wpb = W <= 4 ? 8 : 4;
  const size_t smem = warp_state_bytes<W>() * wpb;
  if (smem > 48 * 1024)
    KC_CUDA(cudaFuncSetAttribute(k_enum<W, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enum<W, 0>, wpb * 32, smem));
  uint64_t blocks = (uint64_t)num_sms * std::max(per_sm, 1);
  blocks = std::max<uint64_t>(1, std::min<uint64_t>(blocks, (x.nroots + wpb - 1) / wpb));
  k_enum<W, 0><<<(unsigned)blocks, wpb * 32, smem, s>>>(x);
  KC_CUDA(cudaGetLastError());
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
  // the count kernel stores vert[root] without using it; the row offsets,
  // read as 2n+2 words, are a readable stand-in for that n-word array
  x.vert = (const uint32_t*)d_orow;
  x.k = k;
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
      if (t == 0) KC_TRY(static_tier<1>(num_sms, y, s));
      if (t == 1) KC_TRY(static_tier<2>(num_sms, y, s));
      if (t == 2) KC_TRY(static_tier<4>(num_sms, y, s));
      if (t == 3) KC_TRY(static_tier<8>(num_sms, y, s));
    }
  }
  unsigned long long total = 0;
  KC_CUDA(cudaMemcpyAsync(&total, &acc[kAccCount], sizeof(total), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  *count = total;
  return KC_OK;
}
