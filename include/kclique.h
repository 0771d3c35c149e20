/*
 * kclique.h -- C ABI of libkc.so: exact k-clique counting and listing on one
 * GB300 (sm_103a), after DIST (Nam, Jang, Park, Yang, Long; arXiv 2502.00317).
 *
 * Problem (Sec. II-A, Definition 1): given a simple undirected graph G and an
 * integer k, list all k-cliques of G.  A clique is a vertex SET (Sec. II-A),
 * so a listed clique has no order; this library writes each one as its k
 * original vertex ids sorted ascending.
 *
 * Conventions for every call:
 *   - every call returns an int status: KC_OK (0) or one of KC_E_*;
 *     kc_strerror() names it; no C++ exception crosses this boundary;
 *   - pointers documented "host" are read or written by the CPU, pointers
 *     documented "device" must be device memory of the context's GPU;
 *   - `stream` is a cudaStream_t passed as void* (NULL: the context's own
 *     stream).  Calls that return host results synchronise that stream;
 *   - a kc_ctx is not thread-safe: one thread at a time per context.
 */
#ifndef KCLIQUE_H
#define KCLIQUE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
#define KC_OK 0
#define KC_E_INVALID_ARG 1     /* NULL pointer, k == 0, bad flag, bad range */
#define KC_E_INVALID_GRAPH 2   /* CSR not simple/symmetric/sorted (without KC_CANONICALIZE) or id >= n */
#define KC_E_OOM 3             /* a device or host allocation failed */
#define KC_E_CAPACITY 4        /* listing: more cliques than the output buffer holds */
#define KC_E_DEVICE_TIMEOUT 5  /* a bounded device-side wait ran out (the context stays usable) */
#define KC_E_CUDA 6            /* a CUDA runtime call failed */
#define KC_E_BUSY 7            /* the resource is in use */
#define KC_E_UNSUPPORTED 8     /* outside the compiled limits (k > KC_MAX_K, out-degree > KC_MAX_OUTDEG) */
#define KC_E_NOT_FOUND 9       /* unknown graph handle or ticket */

#define KC_MAX_K 64            /* largest k the device enumerator accepts */
#define KC_MAX_OUTDEG 1024     /* largest out-degree in the degeneracy DAG (bounded by the degeneracy) */

/* ----------------------------------------------------------- upload flags */
#define KC_HOST_PTRS 0x1u      /* rowptr/col are host pointers (copied to the device) */
#define KC_DEVICE_PTRS 0x2u    /* rowptr/col are device pointers (copied device-to-device) */
#define KC_CANONICALIZE 0x4u   /* drop self-loops and repeats, add missing reverse entries, sort rows */

typedef struct kc_ctx kc_ctx;
typedef uint32_t kc_graph; /* handle of a graph resident on the device, 0 is never valid */

/* Options of a context.  Zero-initialise, set struct_size = sizeof(kc_opts),
 * then change what you need; a zero field takes its default. */
typedef struct kc_opts {
  uint32_t struct_size;
  uint32_t no_memo;        /* 1: never use the device form of the Induced Subgraph Trie (Sec. IV) */
  uint32_t no_prune;       /* 1: never prune by soft embeddings (Sec. V, Algorithm 5) */
  uint32_t split_threshold;/* a root of width > 32 whose G_u has more wedges (sum of C(out-degree, 2)) than
                              this is split into one task per first-level branch (Sec. VII-D);
                              0: default 16384 for k >= 6; 0xFFFFFFFF: never split; a value set here
                              (or by the autotuner) applies for k >= 5 */
  uint64_t memo_bytes;     /* device bytes for the memo tables (0: default 1 GiB); the tau of Sec. VI */
  uint64_t spin_limit;     /* nanoseconds before a device-side wait gives up with KC_E_DEVICE_TIMEOUT
                              (0: default 2 s) */
  uint32_t decomposition;  /* how roots become GPU work items (Sec. VII-D): KC_NODE_PARALLEL (0, default):
                              one warp per root, heavy roots split as above; KC_EDGE_PARALLEL: every
                              root's first-level branches (u, v) are separate tasks, for any k >= 3 */
  uint32_t autotune;       /* 1: kc_count and kc_count_batched pick their launch settings (see kc_tune) per
                              class of input, probing once per class and caching the choice */
  const char* tune_cache;  /* file that keeps the tuned choices across processes (NULL: the environment
                              variable KC_TUNE_CACHE, else memory only); read at kc_create, appended to */
  uint32_t no_plex;        /* 1: never count a 2-plex subgraph by its closed form (the 2-plex early
                              termination of Sec. VII-A); counting only, listing never uses it */
  uint32_t memo_min_k;     /* kc_count uses the memo (unless no_memo) for k >= this; 0: the default, 8 with
                              the 2-plex closed form on and 3 with it off (with the closed form taking the
                              dense cliques, the memo's bookkeeping costs more than it saves below k = 8);
                              listing and kc_count_batched are not affected */
} kc_opts;

#define KC_NODE_PARALLEL 0u
#define KC_EDGE_PARALLEL 1u

/* Graph facts after upload. */
typedef struct kc_graph_info {
  uint32_t n;              /* vertices */
  uint32_t degeneracy;     /* delta(G): the largest core number (Sec. II-A) */
  uint64_t m;              /* undirected edges after canonicalisation */
  uint32_t max_out_degree; /* of the degeneracy DAG; <= degeneracy */
  uint32_t peel_rounds;    /* grid-wide peeling sub-rounds (barriers) used */
} kc_graph_info;

/* Telemetry of the last kc_count / kc_list call on a context (device times
 * from CUDA events on the launching stream; counters from the kernels). */
typedef struct kc_stats {
  float ms_bin;            /* root filter and binning (a4) */
  float ms_enum;           /* build + prune + enumerate/memo kernels (a5-a10) */
  float ms_total;          /* whole call */
  uint32_t enum_launches;  /* enumerator kernel launches in the call */
  uint32_t total_launches; /* every kernel launch in the call */
  uint64_t roots_total;    /* roots with out-degree >= k-1 */
  uint64_t roots_pruned;   /* of those, dropped by the soft-embedding test on the root */
  uint64_t roots_heavy;    /* roots handled by the split (heavy) path */
  uint64_t build_words;    /* 32-bit words read from the DAG while building root bitmaps */
  uint64_t memo_hits;      /* device trie hits */
  uint64_t memo_inserts;   /* device trie insertions */
  uint64_t memo_full;      /* insertions refused because a table was full */
  uint64_t memo_frames;    /* memoised frames opened (device trie walks) */
  float ms_tier[6];        /* device time of each width tier (1, 2, 4, 8, 16, 32 words) */
  uint32_t roots_tier[6];  /* roots in each width tier */
  uint64_t word_ops;       /* 32-bit candidate words intersected (AND + POPC) by the enumerator, plus the
                              words of the narrow bit-matrices built for branches */
  uint64_t warp_ns_build;  /* summed over warps: nanoseconds spent building root bit-matrices (a5) */
  uint64_t warp_ns_busy;   /* summed over warps: nanoseconds spent on roots and tasks in all */
  uint64_t memo_peak;      /* most trie entries stored for one root (the size the paper bounds by tau) */
  uint64_t plex_frames;    /* frames counted by the 2-plex closed form (Sec. VII-A) instead of a search */
} kc_stats;

/* Per-stage device times of the last kc_upload (CUDA events). */
typedef struct kc_upload_stats {
  float ms_copy;           /* H2D or D2D copy of the CSR */
  float ms_canon;          /* validation or canonicalisation (a1) */
  float ms_peel;           /* k-core peeling (a2) */
  float ms_orient;         /* DAG orientation and relabelling (a3) */
  float ms_total;
  uint32_t launches;
} kc_upload_stats;

/* Create a context on CUDA device `device`.  opts may be NULL.  *out receives
 * the context, which owns every device buffer it allocates. */
int kc_create(kc_ctx** out, int device, const kc_opts* opts);

/* Destroy a context and every graph still resident in it. */
int kc_destroy(kc_ctx* ctx);

/*
 * Upload a graph given as CSR with n vertices (ids 0..n-1): rowptr has n+1
 * uint64 entries, col has rowptr[n] uint32 entries.  flags must contain
 * exactly one of KC_HOST_PTRS / KC_DEVICE_PTRS.  The arrays stay owned by the
 * caller; they are copied.  Without KC_CANONICALIZE the CSR must already be
 * simple (Sec. II-A): no self-loop, no repeat, every entry's reverse present,
 * rows sorted ascending, else KC_E_INVALID_GRAPH.  With KC_CANONICALIZE any
 * entries with ids < n are accepted and cleaned on the device.
 *
 * The upload then computes on the device, with no host round trip per round:
 *   - the degeneracy order (Sec. II-A) by parallel k-core peeling, level by
 *     level: order key (core number, position of removal within its level;
 *     the second part depends on timing, no count does);
 *   - the DAG based on it (Sec. II-A), relabelled to rank space, each out-list
 *     sorted ascending (Algorithm 2, first line).
 * *out receives the handle.  Synchronises the stream.
 */
int kc_upload(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr, const uint32_t* col, uint32_t flags,
              kc_graph* out, void* stream);

/* Release a graph's device memory. */
int kc_free_graph(kc_ctx* ctx, kc_graph g);

/* Facts about an uploaded graph (host struct). */
int kc_graph_info_get(kc_ctx* ctx, kc_graph g, kc_graph_info* info);

/*
 * Copy the upload's results to caller-owned host arrays (any may be NULL):
 * core[n] core numbers, rank[n] position of each vertex in the order,
 * orow[n+1] and ocol[m] the DAG in rank space (out-list of rank r is
 * ocol[orow[r] .. orow[r+1]), ranks ascending).  For tests and tooling.
 */
int kc_export_dag(kc_ctx* ctx, kc_graph g, uint32_t* core, uint32_t* rank, uint64_t* orow, uint32_t* ocol);

/*
 * Count the k-cliques of an uploaded graph (Definition 1) into *count (host).
 * k = 1 gives n, k = 2 gives m.  Work per root u of the DAG: the (k-1)-cliques
 * of the subgraph induced by N(u) (Algorithm 2), pruned by soft embeddings
 * (Sec. V), with candidate sets that are 2-plexes counted in closed form
 * (Sec. VII-A) and, for dense subgraphs by Eq. (1) and k >= memo_min_k,
 * repeated sub-counts reused through a device form of the Induced Subgraph
 * Trie (Sec. IV, Algorithms 3-4).  Synchronises the stream.
 */
int kc_count(kc_ctx* ctx, kc_graph g, uint32_t k, uint64_t* count, void* stream);

/*
 * List every k-clique into d_buf (device, caller-owned, room for cap tuples
 * of k uint32 ids): tuple i occupies d_buf[i*k .. i*k+k-1], ids ascending;
 * the order of tuples is unspecified.  *written (host) = tuples written =
 * min(total, cap); *total = all k-cliques; *checksum = sum mod 2^64 over all
 * k-cliques of the SplitMix64-chained hash of its sorted id tuple (h =
 * mix(0x9E3779B97F4A7C15 ^ k), then h = mix(h ^ id) for each id ascending).
 * total and checksum always cover every clique; when total > cap the call
 * still fills d_buf with an unspecified subset and returns KC_E_CAPACITY.
 * cap may be 0 (d_buf may then be NULL) to get total and checksum only;
 * that call returns KC_OK.
 * Synchronises the stream.
 */
int kc_list(kc_ctx* ctx, kc_graph g, uint32_t k, uint32_t* d_buf, uint64_t cap, uint64_t* written,
            uint64_t* total, uint64_t* checksum, void* stream);

/*
 * As kc_list, restricted to the k-cliques whose first vertex in the
 * degeneracy order has rank in [root_lo, root_hi) (one NodeParallel subtask
 * per root, Sec. VII-D).  Disjoint ranges partition the cliques, so their
 * totals add and their checksums wrap-add to the full listing's.
 */
int kc_list_range(kc_ctx* ctx, kc_graph g, uint32_t k, uint32_t root_lo, uint32_t root_hi, uint32_t* d_buf,
                  uint64_t cap, uint64_t* written, uint64_t* total, uint64_t* checksum, void* stream);

/*
 * Batched counting: counts[i] (host) = the number of ks[i]-cliques of the
 * resident graph graphs[i], for i < nq.  Graphs may repeat, with the same or
 * different k.  The roots of every query (one NodeParallel subtask per root,
 * Sec. VII-D) are binned together by bitmap width and enumerated by one set
 * of tier launches -- the same kernels as kc_count, each warp binding the
 * query of the root it takes -- instead of one set of launches per graph.
 * Results equal nq separate kc_count calls.  Errors: KC_E_INVALID_ARG (NULL
 * array with nq > 0, a k of 0), KC_E_NOT_FOUND (unknown graph),
 * KC_E_UNSUPPORTED (k > KC_MAX_K).  Synchronises the stream.
 */
int kc_count_batched(kc_ctx* ctx, const kc_graph* graphs, const uint32_t* ks, uint32_t nq, uint64_t* counts,
                     void* stream);

/*
 * Count the k-cliques of a DAG that is already in device memory, without
 * allocating any memory.  The paper has no counterpart: this entry point is
 * for callers that cannot call cudaMalloc (or any allocator) when they
 * count: a process whose own pool allocator already holds the device's free
 * memory (a serving framework, a deep-learning runtime), where a further
 * cudaMalloc fails or fragments that pool; a latency-bound loop that cannot
 * afford cudaMalloc/cudaFree, which can synchronise the whole device; code
 * that must not fail for lack of memory once it has started.  Such callers
 * cannot create a kc_ctx either (kc_create and kc_upload allocate), so this
 * call takes no context.
 *
 * Input (device memory of the current device, caller-owned, read only):
 *   d_orow[n+1] uint64 row offsets, d_orow[0] = 0, non-decreasing;
 *   d_ocol[d_orow[n]] uint32 out-neighbours: row r lists ranks strictly
 *   ascending, each in (r, n) -- an oriented DAG in rank space such as
 *   kc_export_dag returns (any total order gives the same count).
 * Output: *count (host) = the number of k-cliques; k = 1 gives n, k = 2 the
 * number of DAG edges.  The work is the plain count of kc_count (one warp per
 * root, the same pruning as kc_count) without the memo and without the
 * heavy-root split.
 *
 * Scratch lives in one fixed device array of 3 MiB + 768 B inside the
 * library, which every GPU that loads libkc.so holds until the process
 * exits.  Its limits: every out-degree at most 256 (else KC_E_UNSUPPORTED,
 * nothing counted); roots are binned 131,072 at a time, so n is not
 * otherwise bounded.  The array keeps the last call's contents; each call
 * clears what must start at zero.  All calls on a device share the one
 * array, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race and give wrong counts: serialise them.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Errors: KC_E_INVALID_ARG (NULL d_orow or
 * count, NULL d_ocol with edges, k = 0), KC_E_UNSUPPORTED (k > KC_MAX_K,
 * out-degree > 256), KC_E_INVALID_GRAPH (the DAG breaks the layout above;
 * checked on the device before any other kernel reads it), KC_E_CUDA.
 * Synchronises `stream` (NULL: the legacy default stream) several times.
 */
int kc_count_dag_noalloc(uint32_t n, const uint64_t* d_orow, const uint32_t* d_ocol, uint32_t k, uint64_t* count,
                         void* stream);

/* ---------------------------------------------------------------- serving
 * A request loop inside the library (no counterpart in the paper, which
 * runs one listing at a time): requests (a resident graph or an inline CSR,
 * k, and a mode: count, or list without keeping the tuples -- count and
 * checksum) are queued by kc_serve_submit and taken by `lanes` worker
 * threads.  Each lane owns its own device scratch and streams.  Whenever a
 * lane is free it takes every queued request that fits -- at most max_batch,
 * and only while the memory cap allows -- and enumerates them together (the
 * kc_count_batched path: the batch's counts in one set of tier launches, its
 * listings in another).  Requests that arrive while a batch runs wait for
 * the next free lane, so with two or more lanes batches overlap on the GPU.
 * A request's result is the same alone and in any mix.
 *
 * Device memory: mem_cap_bytes bounds what serving allocates (the resident
 * graphs are the caller's and are not counted).  Admitted, unfinished
 * requests may reserve half of it: a request's bytes bound what a batch
 * allocates for it (root lists, heavy-root arena and task queue of its width
 * tiers, an inline graph's upload).  The lanes' own scratch (memo tables and
 * per-warp state, planned within cap / (2 lanes) each, at least one block of
 * per-warp state per width tier) takes the other half; a lane that holds
 * more than its share after a batch releases its scratch.  A request whose
 * bytes exceed half the cap completes alone with KC_E_OOM.
 *
 * While serving, the context's resident graphs are read-only: do not call
 * kc_upload, kc_free_graph, kc_count, kc_list or kc_count_batched on it until
 * kc_serve_stop returns.  The kc_serve_* calls themselves may come from any
 * number of host threads.
 */
typedef struct kc_serve_opts {
  uint32_t struct_size;    /* sizeof(kc_serve_opts) */
  uint32_t lanes;          /* worker lanes (0: 2) */
  uint32_t max_batch;      /* requests per batch at most (0: 4096) */
  uint32_t reserved;
  uint64_t mem_cap_bytes;  /* cap on the device bytes serving allocates (0: 64 GiB) */
} kc_serve_opts;

#define KC_SERVE_COUNT 0u      /* mode: count the k-cliques (kc_count) */
#define KC_SERVE_LIST 1u       /* mode: list the k-cliques without keeping them: count and checksum
                                  (kc_list with cap = 0) */

typedef struct kc_serve_result {
  uint64_t count;          /* k-cliques (when status == KC_OK) */
  int32_t status;          /* KC_OK, or the error of this request */
  uint32_t batch_size;     /* requests in the batch that served it */
  uint64_t t_submit_ns;    /* steady-clock times: submission, batch start, completion */
  uint64_t t_start_ns;
  uint64_t t_done_ns;
  uint64_t checksum;       /* KC_SERVE_LIST: kc_list's checksum of the k-cliques; KC_SERVE_COUNT: 0 */
  uint32_t mode;           /* the request's mode */
  uint32_t enumerated;     /* 1 if the GPU enumerated it, 0 if it was answered at submission */
} kc_serve_result;

typedef struct kc_serve_stats {
  uint64_t submitted;
  uint64_t completed;
  uint64_t failed;         /* completed with a status other than KC_OK */
  uint64_t batches;
  double p50_ms;           /* latency (submission to completion) percentiles of completed requests */
  double p99_ms;
  double mean_batch;       /* requests per batch */
  double req_per_s;        /* completed / (last completion - first submission) */
  double cliques_per_s;
  uint64_t peak_reserved_bytes; /* most device bytes reserved at once: admitted requests plus the lanes'
                              scratch budgets (at most mem_cap_bytes) */
  double p50_enum_ms;      /* latency percentiles of the requests the GPU enumerated (answered-at- */
  double p99_enum_ms;      /* submission requests left out) */
  uint64_t lane_scratch_bytes; /* device scratch the lanes hold now */
} kc_serve_stats;

/* Start serving on ctx (opts may be NULL).  KC_E_BUSY if already serving. */
int kc_serve_start(kc_ctx* ctx, const kc_serve_opts* opts);

/* Queue a request on resident graph g: mode KC_SERVE_COUNT counts the
 * k-cliques (kc_count), KC_SERVE_LIST lists them without keeping the tuples
 * (kc_list with cap = 0: count and checksum).  *ticket receives the
 * request's id.  Errors of the request itself (k = 0, another mode,
 * k > KC_MAX_K, unknown graph) are returned here. */
int kc_serve_submit(kc_ctx* ctx, kc_graph g, uint32_t k, uint32_t mode, uint64_t* ticket);

/* As kc_serve_submit for a graph given inline as a host CSR (same layout and
 * flags as kc_upload, KC_HOST_PTRS implied); the arrays are copied before
 * the call returns.  The lane uploads it, enumerates it and frees it; its
 * device bytes count against the cap until then.  A graph whose footprint
 * alone exceeds half the cap completes with status KC_E_OOM. */
int kc_serve_submit_csr(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr, const uint32_t* col, uint32_t flags,
                        uint32_t k, uint32_t mode, uint64_t* ticket);

/* Result of a request: KC_OK and *out filled once it is complete (the
 * request is then forgotten), KC_E_BUSY while it is queued or running,
 * KC_E_NOT_FOUND for an unknown or already collected ticket.  kc_serve_wait
 * blocks up to timeout_ms (negative: no limit) for it. */
int kc_serve_poll(kc_ctx* ctx, uint64_t ticket, kc_serve_result* out);
int kc_serve_wait(kc_ctx* ctx, uint64_t ticket, int64_t timeout_ms, kc_serve_result* out);

/* Counters and latency percentiles since kc_serve_start. */
int kc_serve_stats_get(kc_ctx* ctx, kc_serve_stats* out);

/* Stop serving: requests not yet taken by a lane complete with status
 * KC_E_BUSY, running batches finish, the lanes are released. */
int kc_serve_stop(kc_ctx* ctx);

/* ------------------------------------------------------------ autotuning
 * Launch settings with no counterpart in the paper: warps per block of the
 * narrow (up to 4 words) and wide width tiers, the heavy-root split
 * threshold, and the memo budget.  kc_tune times the batched count of the
 * given queries (graphs[i], ks[i]) under candidate settings -- the split
 * threshold first, then each warps-per-block choice, then the memo budget,
 * keeping each change that is faster -- and applies the fastest to the
 * context (every later call uses it).  The result is the same count under
 * every setting; only the time differs.  *out (may be NULL) reports the
 * choice, the probe times, and the class key under which the choice is
 * cached (graph sizes, width tiers and k of the queries, and the GPU).
 * Errors: those of kc_count_batched.  Synchronises the context's stream. */
typedef struct kc_tune_result {
  uint32_t split_threshold;  /* chosen (kc_opts encoding: 0xFFFFFFFF never) */
  uint32_t warps_small;      /* warps per block, tiers of 1-4 words */
  uint32_t warps_large;      /* warps per block, tiers of 8-32 words */
  uint32_t probes;           /* timed batched counts run */
  uint64_t memo_bytes;       /* chosen memo budget */
  float ms_default;          /* the probe under the default settings */
  float ms_tuned;            /* the probe under the chosen settings */
  uint32_t cached;           /* 1: taken from the cache, no probe run */
  char key[116];             /* class key, NUL-terminated */
} kc_tune_result;

int kc_tune(kc_ctx* ctx, const kc_graph* graphs, const uint32_t* ks, uint32_t nq, kc_tune_result* out);

/* Telemetry of the last count/list call, and of the last upload. */
int kc_last_stats(kc_ctx* ctx, kc_stats* out);
int kc_last_upload_stats(kc_ctx* ctx, kc_upload_stats* out);

/* Name of a status code (static string). */
const char* kc_strerror(int status);

/* Text of the last CUDA error seen by the context (static per context). */
const char* kc_last_error(kc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* KCLIQUE_H */
