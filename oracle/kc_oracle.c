/*
 * kc_oracle.c -- THE ORACLE.  Test infrastructure only.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header, table or helper with
 * the CUDA path, and the CUDA path never calls it.
 *
 * What it computes is the plain definition (Sec. II-A): the set of all
 * k-vertex subsets of V in which every pair of distinct vertices is adjacent
 * (clique definition; Definition 1, k-clique listing), in a simple
 * undirected graph (Sec. II-A, "graph").  It uses the ordering framework of
 * Algorithm 1 (Danisch et al.): orient G by a total order into a DAG, then
 * for every vertex u recursively list the (l-1)-cliques among the common
 * out-neighbours, with the base case reached when one vertex is left.
 * Intersections are linear merges of sorted out-lists.  There is no trie,
 * no pruning, no bitmap and no blocking: one root after another.
 *
 * Steps, each a plain restatement:
 *   1. canonicalise the input CSR: drop self-loops and repeated entries,
 *      add the reverse of every entry (the graph is simple, Sec. II-A);
 *   2. degeneracy order (Sec. II-A): repeatedly remove a vertex of minimum
 *      current degree; among equal degrees the smallest id goes first;
 *      core[v] = the largest minimum degree seen up to v's removal;
 *   3. DAG of G based on that order (Sec. II-A): keep (u, v) iff u comes
 *      before v; out-lists are kept in rank space, sorted ascending;
 *   4. Algorithm 1 recursion per root, threads taking roots dynamically.
 *      Count mode may add |cand ∩ N(v)| at the next-to-last level instead of
 *      visiting each last vertex: the same set, counted.
 *   5. every reported clique is mapped to original ids, sorted ascending and
 *      hashed with a SplitMix64-finaliser chain; the hashes are summed mod
 *      2^64 (an order-independent checksum in which a duplicate shows).
 *
 * The SplitMix64 finaliser is Steele, Lea and Flood's mixing function
 * (OOPSLA 2014; constants as in Vigna's public-domain splitmix64.c).
 */
#include <errno.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define KCO_OK 0
#define KCO_E_ARG -1
#define KCO_E_GRAPH -2
#define KCO_E_OOM -3

typedef struct kco_graph {
  uint32_t n;
  uint64_t m;          /* undirected edges after canonicalisation */
  uint64_t *adj_ptr;   /* canonical undirected CSR, rows sorted */
  uint32_t *adj;
  uint32_t *rank;      /* rank[v]: position of v in the degeneracy order */
  uint32_t *vert;      /* vert[r]: vertex at position r */
  uint32_t *core;      /* core number of each vertex */
  uint32_t degeneracy; /* max core number */
  uint64_t *out_ptr;   /* DAG out-lists in rank space */
  uint32_t *out;
  uint32_t max_out;
} kco_graph;

/* ------------------------------------------------------------------ hash */
static uint64_t kco_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The finaliser alone, exported so that the tests can pin it to published
 * SplitMix64 outputs. */
uint64_t kco_mix64_value(uint64_t z) { return kco_mix64(z); }

uint64_t kco_clique_hash(const uint32_t *ids_sorted, uint32_t k) {
  uint64_t h = kco_mix64(0x9E3779B97F4A7C15ULL ^ (uint64_t)k);
  for (uint32_t i = 0; i < k; i++) h = kco_mix64(h ^ (uint64_t)ids_sorted[i]);
  return h;
}

/* ------------------------------------------------------------- canonical */
static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

static int canonicalise(kco_graph *g, uint32_t n, const uint64_t *rowptr, const uint32_t *col) {
  uint64_t *deg = calloc((size_t)n + 1, sizeof(uint64_t));
  if (!deg) return KCO_E_OOM;
  for (uint32_t u = 0; u < n; u++) {
    if (rowptr[u + 1] < rowptr[u]) { free(deg); return KCO_E_GRAPH; }
    for (uint64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
      uint32_t v = col[e];
      if (v >= n) { free(deg); return KCO_E_GRAPH; }
      if (v == u) continue;
      deg[u]++;
      deg[v]++;
    }
  }
  uint64_t *ptr = malloc(((size_t)n + 1) * sizeof(uint64_t));
  uint64_t *fill = malloc(((size_t)n + 1) * sizeof(uint64_t));
  uint64_t tot = 0;
  for (uint32_t u = 0; u < n; u++) tot += deg[u];
  uint32_t *tmp = malloc((tot ? tot : 1) * sizeof(uint32_t));
  if (!ptr || !fill || !tmp) { free(deg); free(ptr); free(fill); free(tmp); return KCO_E_OOM; }
  ptr[0] = 0;
  for (uint32_t u = 0; u < n; u++) ptr[u + 1] = ptr[u] + deg[u];
  memcpy(fill, ptr, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint32_t u = 0; u < n; u++)
    for (uint64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
      uint32_t v = col[e];
      if (v == u) continue;
      tmp[fill[u]++] = v;
      tmp[fill[v]++] = u;
    }
  /* sort each row, drop repeats, compact in place */
  uint64_t w = 0;
  for (uint32_t u = 0; u < n; u++) {
    uint64_t b = ptr[u], e = ptr[u + 1];
    qsort(tmp + b, e - b, sizeof(uint32_t), cmp_u32);
    uint64_t start = w;
    for (uint64_t i = b; i < e; i++)
      if (i == b || tmp[i] != tmp[i - 1]) tmp[w++] = tmp[i];
    fill[u] = start; /* reuse as new row start */
  }
  fill[n] = w;
  free(ptr);
  free(deg);
  g->adj_ptr = fill;
  {
    uint32_t *shrunk = realloc(tmp, (w ? w : 1) * sizeof(uint32_t));
    g->adj = shrunk ? shrunk : tmp;
  }
  g->m = w / 2;
  return KCO_OK;
}

/* ------------------------------------------------------- degeneracy order */
/* Binary min-heap of keys (degree << 32 | id) with lazy deletion: a popped key
 * whose degree is stale is skipped.  The minimum key is the vertex of minimum
 * current degree with the smallest id. */
typedef struct { uint64_t *a; uint64_t size, cap; } heap_t;

static int heap_push(heap_t *h, uint64_t key) {
  if (h->size == h->cap) {
    uint64_t nc = h->cap ? 2 * h->cap : 1024;
    uint64_t *na = realloc(h->a, nc * sizeof(uint64_t));
    if (!na) return KCO_E_OOM;
    h->a = na;
    h->cap = nc;
  }
  uint64_t i = h->size++;
  while (i > 0) {
    uint64_t p = (i - 1) / 2;
    if (h->a[p] <= key) break;
    h->a[i] = h->a[p];
    i = p;
  }
  h->a[i] = key;
  return KCO_OK;
}

static uint64_t heap_pop(heap_t *h) {
  uint64_t top = h->a[0];
  uint64_t last = h->a[--h->size];
  uint64_t i = 0;
  for (;;) {
    uint64_t l = 2 * i + 1, r = l + 1, s = i;
    uint64_t sv = last;
    if (l < h->size && h->a[l] < sv) { s = l; sv = h->a[l]; }
    if (r < h->size && h->a[r] < sv) { s = r; sv = h->a[r]; }
    if (s == i) break;
    h->a[i] = h->a[s];
    i = s;
  }
  if (h->size) h->a[i] = last;
  return top;
}

static int degeneracy_order(kco_graph *g) {
  uint32_t n = g->n;
  uint32_t *deg = malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  uint8_t *gone = calloc(n ? n : 1, 1);
  g->rank = malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  g->vert = malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  g->core = malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  heap_t h = {0};
  if (!deg || !gone || !g->rank || !g->vert || !g->core) { free(deg); free(gone); return KCO_E_OOM; }
  for (uint32_t v = 0; v < n; v++) {
    deg[v] = (uint32_t)(g->adj_ptr[v + 1] - g->adj_ptr[v]);
    if (heap_push(&h, ((uint64_t)deg[v] << 32) | v)) { free(deg); free(gone); free(h.a); return KCO_E_OOM; }
  }
  uint32_t r = 0, kmax = 0;
  while (r < n) {
    uint64_t key = heap_pop(&h);
    uint32_t v = (uint32_t)key, d = (uint32_t)(key >> 32);
    if (gone[v] || d != deg[v]) continue; /* stale entry */
    gone[v] = 1;
    if (d > kmax) kmax = d;
    g->core[v] = kmax;
    g->rank[v] = r;
    g->vert[r] = v;
    r++;
    for (uint64_t e = g->adj_ptr[v]; e < g->adj_ptr[v + 1]; e++) {
      uint32_t w = g->adj[e];
      if (!gone[w]) {
        deg[w]--;
        if (heap_push(&h, ((uint64_t)deg[w] << 32) | w)) { free(deg); free(gone); free(h.a); return KCO_E_OOM; }
      }
    }
  }
  g->degeneracy = kmax;
  free(h.a);
  free(deg);
  free(gone);
  return KCO_OK;
}

/* ----------------------------------------------------------------- orient */
static int orient(kco_graph *g) {
  uint32_t n = g->n;
  g->out_ptr = malloc(((size_t)n + 1) * sizeof(uint64_t));
  g->out = malloc((g->m ? g->m : 1) * sizeof(uint32_t));
  if (!g->out_ptr || !g->out) return KCO_E_OOM;
  uint64_t w = 0;
  g->max_out = 0;
  for (uint32_t r = 0; r < n; r++) {
    uint32_t v = g->vert[r];
    g->out_ptr[r] = w;
    for (uint64_t e = g->adj_ptr[v]; e < g->adj_ptr[v + 1]; e++) {
      uint32_t rw = g->rank[g->adj[e]];
      if (rw > r) g->out[w++] = rw;
    }
    qsort(g->out + g->out_ptr[r], w - g->out_ptr[r], sizeof(uint32_t), cmp_u32);
    if (w - g->out_ptr[r] > g->max_out) g->max_out = (uint32_t)(w - g->out_ptr[r]);
  }
  g->out_ptr[n] = w;
  return KCO_OK;
}

void kco_free(kco_graph *g) {
  if (!g) return;
  free(g->adj_ptr); free(g->adj); free(g->rank); free(g->vert); free(g->core);
  free(g->out_ptr); free(g->out);
  free(g);
}

/* Build the oracle's graph: canonicalise, order, orient.  status gets KCO_*. */
kco_graph *kco_build(uint32_t n, const uint64_t *rowptr, const uint32_t *col, int *status) {
  kco_graph *g = calloc(1, sizeof(kco_graph));
  int st = g ? KCO_OK : KCO_E_OOM;
  if (st == KCO_OK) { g->n = n; st = canonicalise(g, n, rowptr, col); }
  if (st == KCO_OK) st = degeneracy_order(g);
  if (st == KCO_OK) st = orient(g);
  if (status) *status = st;
  if (st != KCO_OK) { kco_free(g); return NULL; }
  return g;
}

uint32_t kco_n(const kco_graph *g) { return g->n; }
uint64_t kco_m(const kco_graph *g) { return g->m; }
uint32_t kco_degeneracy(const kco_graph *g) { return g->degeneracy; }
uint32_t kco_max_out(const kco_graph *g) { return g->max_out; }
void kco_get_core(const kco_graph *g, uint32_t *out) { memcpy(out, g->core, (size_t)g->n * sizeof(uint32_t)); }
void kco_get_rank(const kco_graph *g, uint32_t *out) { memcpy(out, g->rank, (size_t)g->n * sizeof(uint32_t)); }
void kco_get_adj(const kco_graph *g, uint64_t *ptr, uint32_t *adj) {
  memcpy(ptr, g->adj_ptr, ((size_t)g->n + 1) * sizeof(uint64_t));
  memcpy(adj, g->adj, (size_t)g->adj_ptr[g->n] * sizeof(uint32_t));
}
/* out-lists with ORIGINAL ids of both endpoints: src[e] -> dst[e] for the m DAG edges */
void kco_get_dag_edges(const kco_graph *g, uint32_t *src, uint32_t *dst) {
  for (uint32_t r = 0; r < g->n; r++)
    for (uint64_t e = g->out_ptr[r]; e < g->out_ptr[r + 1]; e++) {
      src[e] = g->vert[r];
      dst[e] = g->vert[g->out[e]];
    }
}

/* ---------------------------------------------------------------- listing */
typedef struct {
  const kco_graph *g;
  uint32_t k;
  int mode;            /* 0: count (fast last level), 1: every clique (checksum, per-vertex, output) */
  uint32_t root_lo, root_hi;
  uint32_t *next_root; /* shared dynamic counter */
  uint32_t *out_buf;   /* optional tuple output (single thread only) */
  uint64_t out_cap;
  uint64_t out_written;
  /* per thread */
  uint64_t count, checksum;
  uint64_t *per_vertex; /* optional, length n */
  uint32_t *cand;       /* (k+1) * (max_out+1) */
  uint32_t *clique;     /* k ranks */
  int status;
} job_t;

static uint64_t intersect(const uint32_t *a, uint64_t na, const uint32_t *b, uint64_t nb, uint32_t *out) {
  uint64_t i = 0, j = 0, w = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else { out[w++] = a[i]; i++; j++; }
  }
  return w;
}

static uint64_t intersect_size(const uint32_t *a, uint64_t na, const uint32_t *b, uint64_t nb) {
  uint64_t i = 0, j = 0, w = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else { w++; i++; j++; }
  }
  return w;
}

static void report(job_t *J, uint32_t t) {
  const kco_graph *g = J->g;
  uint32_t ids[64] = {0};
  for (uint32_t i = 0; i < t; i++) {
    /* insertion sort of original ids */
    uint32_t x = g->vert[J->clique[i]];
    uint32_t p = i;
    while (p > 0 && ids[p - 1] > x) { ids[p] = ids[p - 1]; p--; }
    ids[p] = x;
  }
  J->count++;
  J->checksum += kco_clique_hash(ids, t);
  if (J->per_vertex)
    for (uint32_t i = 0; i < t; i++) J->per_vertex[ids[i]]++;
  if (J->out_buf) {
    if (J->out_written < J->out_cap) memcpy(J->out_buf + J->out_written * t, ids, t * sizeof(uint32_t));
    J->out_written++;
  }
}

/* C = clique[0..t-1] (ranks), cand = common out-neighbours of C, sorted. */
static void rec(job_t *J, uint32_t t, const uint32_t *cand, uint64_t nc) {
  const kco_graph *g = J->g;
  uint32_t k = J->k;
  if (t == k) { report(J, t); return; }
  if (nc < k - t) return; /* not enough vertices left: nothing to report */
  if (J->mode == 0 && t + 2 == k) {
    for (uint64_t i = 0; i < nc; i++) {
      uint32_t v = cand[i];
      J->count += intersect_size(cand + i + 1, nc - i - 1, g->out + g->out_ptr[v], g->out_ptr[v + 1] - g->out_ptr[v]);
    }
    return;
  }
  uint32_t *next = J->cand + (uint64_t)(t + 1) * (g->max_out + 1);
  for (uint64_t i = 0; i < nc; i++) {
    uint32_t v = cand[i];
    J->clique[t] = v;
    if (t + 1 == k) { report(J, k); continue; }
    uint64_t nn = intersect(cand + i + 1, nc - i - 1, g->out + g->out_ptr[v], g->out_ptr[v + 1] - g->out_ptr[v], next);
    rec(J, t + 1, next, nn);
  }
}

static void run_root(job_t *J, uint32_t r) {
  const kco_graph *g = J->g;
  J->clique[0] = r;
  if (J->k == 1) { report(J, 1); return; }
  rec(J, 1, g->out + g->out_ptr[r], g->out_ptr[r + 1] - g->out_ptr[r]);
}

static void *worker(void *arg) {
  job_t *J = arg;
  const uint32_t chunk = 64;
  for (;;) {
    uint32_t s = __atomic_fetch_add(J->next_root, chunk, __ATOMIC_RELAXED);
    if (s >= J->root_hi) break;
    uint32_t e = s + chunk < J->root_hi ? s + chunk : J->root_hi;
    for (uint32_t r = s; r < e; r++) run_root(J, r);
  }
  return NULL;
}

/*
 * Count (mode 0) or enumerate (mode 1) the k-cliques whose minimum vertex in
 * the oracle's order has rank in [root_lo, root_hi).  Mode 1 also gives the
 * checksum and, when per_vertex != NULL (length n), per-vertex counts.
 * nthreads = 0 uses every online CPU.  *threads_used gets the thread count.
 */
int kco_run(const kco_graph *g, uint32_t k, int mode, uint32_t root_lo, uint32_t root_hi, int nthreads,
            uint64_t *count, uint64_t *checksum, uint64_t *per_vertex, int *threads_used) {
  if (!g || k == 0 || k > 64 || (mode != 0 && mode != 1)) return KCO_E_ARG;
  if (root_hi > g->n) root_hi = g->n;
  if (root_lo > root_hi) root_lo = root_hi;
  if (nthreads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    nthreads = c > 0 ? (int)c : 1;
  }
  if (per_vertex) nthreads = 1; /* keep per-vertex accumulation simple */
  uint32_t next = root_lo;
  job_t *jobs = calloc((size_t)nthreads, sizeof(job_t));
  pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return KCO_E_OOM; }
  int st = KCO_OK;
  for (int i = 0; i < nthreads; i++) {
    job_t *J = &jobs[i];
    J->g = g; J->k = k; J->mode = (mode == 0 && k >= 3 && !per_vertex) ? 0 : 1;
    J->root_lo = root_lo; J->root_hi = root_hi; J->next_root = &next;
    J->per_vertex = per_vertex;
    J->cand = malloc((size_t)(k + 1) * (g->max_out + 1) * sizeof(uint32_t));
    J->clique = malloc((size_t)(k + 1) * sizeof(uint32_t));
    if (!J->cand || !J->clique) st = KCO_E_OOM;
  }
  int started = 0;
  if (st == KCO_OK) {
    for (int i = 0; i < nthreads; i++) {
      if (nthreads == 1) { worker(&jobs[0]); started = 0; break; }
      if (pthread_create(&th[i], NULL, worker, &jobs[i]) != 0) break;
      started++;
    }
    for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
  }
  uint64_t c = 0, s = 0;
  for (int i = 0; i < nthreads; i++) {
    c += jobs[i].count;
    s += jobs[i].checksum;
    free(jobs[i].cand);
    free(jobs[i].clique);
  }
  free(jobs);
  free(th);
  if (count) *count = c;
  if (checksum) *checksum = s;
  if (threads_used) *threads_used = nthreads;
  return st;
}

/* Single-threaded listing of every k-clique as a sorted original-id tuple into
 * out (cap tuples of k ids); *total gets the number of cliques. */
int kco_list(const kco_graph *g, uint32_t k, uint32_t *out, uint64_t cap, uint64_t *total, uint64_t *checksum) {
  if (!g || k == 0 || k > 64) return KCO_E_ARG;
  uint32_t next = 0;
  job_t J;
  memset(&J, 0, sizeof(J));
  J.g = g; J.k = k; J.mode = 1; J.root_lo = 0; J.root_hi = g->n; J.next_root = &next;
  J.out_buf = out; J.out_cap = cap;
  J.cand = malloc((size_t)(k + 1) * (g->max_out + 1) * sizeof(uint32_t));
  J.clique = malloc((size_t)(k + 1) * sizeof(uint32_t));
  if (!J.cand || !J.clique) { free(J.cand); free(J.clique); return KCO_E_OOM; }
  worker(&J);
  free(J.cand);
  free(J.clique);
  if (total) *total = J.count;
  if (checksum) *checksum = J.checksum;
  return KCO_OK;
}
