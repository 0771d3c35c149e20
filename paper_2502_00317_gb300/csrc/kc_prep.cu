// kc_prep.cu -- upload pipeline of libkc.so: copy, validate or canonicalise
// the CSR (the graph must be simple, Sec. II-A), k-core peeling for the
// degeneracy order (Sec. II-A), and the DAG based on it in rank space
// (Algorithm 2, first line).
#include <cooperative_groups.h>

#include <algorithm>

#include "kc_internal.cuh"

namespace kc {

// ============================================================== block scan
// Exclusive scan of one value per thread across a block (blockDim multiple of 32).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? s_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  T warp_off = wid ? s_warp[wid - 1] : T(0);
  if (total) *total = s_warp[nw - 1];
  T r = warp_off + x - v;
  __syncthreads();
  return r;
}

// ==================================================================== scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const Tin* __restrict__ in, uint64_t n,
                                                              uint64_t* __restrict__ bsum) {
  __shared__ uint64_t s_warp[32];
  uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
  for (uint32_t i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    uint64_t idx = base + i;
    if (idx < n) s += (uint64_t)in[idx];
  }
  uint64_t tot;
  block_exclusive_scan<uint64_t>(s, s_warp, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const Tin* __restrict__ in, uint64_t n,
                                                            const uint64_t* __restrict__ boff,
                                                            uint64_t* __restrict__ out) {
  __shared__ uint64_t s_warp[32];
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    uint64_t idx = base + j;
    v[j] = idx < n ? (uint64_t)in[idx] : 0;
    s += v[j];
  }
  uint64_t tot;
  uint64_t off = block_exclusive_scan<uint64_t>(s, s_warp, &tot);
  uint64_t b = boff ? boff[blockIdx.x] : 0;
  off += b;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    uint64_t idx = base + j;
    if (idx < n) out[idx] = off;
    off += v[j];
  }
  uint64_t last_block = n ? (n - 1) / kScanTile : 0;
  if (blockIdx.x == last_block && threadIdx.x == 0) out[n] = b + tot;
}

static uint64_t scan_scratch_words(uint64_t n) {
  uint64_t words = 0;
  while (n > kScanTile) {
    uint64_t nb = (n + kScanTile - 1) / kScanTile;
    words += 2 * nb + 1;
    n = nb;
  }
  return words;
}

template <typename Tin>
static int scan_level(kc_ctx* ctx, const Tin* in, uint64_t* out, uint64_t n, uint64_t* scr, cudaStream_t s,
                      uint32_t* launches) {
  uint64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= 1) {
    k_scan_down<Tin><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    KC_CUDA(cudaGetLastError());
    (*launches)++;
    return KC_OK;
  }
  uint64_t* bsum = scr;
  uint64_t* boff = scr + nb;
  k_scan_reduce<Tin><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum);
  KC_CUDA(cudaGetLastError());
  (*launches)++;
  KC_TRY(scan_level<uint64_t>(ctx, bsum, boff, nb, scr + 2 * nb + 1, s, launches));
  k_scan_down<Tin><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, boff, out);
  KC_CUDA(cudaGetLastError());
  (*launches)++;
  return KC_OK;
}

int exclusive_scan_u32_to_u64(kc_ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t s,
                              uint32_t* launches) {
  void* scr = nullptr;
  uint64_t words = scan_scratch_words(n) + 1;
  KC_TRY(scratch_get(ctx, kScrScan, words * sizeof(uint64_t), &scr));
  return scan_level<uint32_t>(ctx, in, out, n, (uint64_t*)scr, s, launches);
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// ========================================================= segmented sort
constexpr int kSortBlock = 256;
constexpr uint32_t kSortSmem = 4096;  // keys a block sorts in shared memory

// Rows of <= 32 keys: one warp, bitonic network over lanes.
__global__ void k_segsort_warp(uint32_t* __restrict__ data, const uint64_t* __restrict__ ptr, uint32_t rows,
                               uint32_t* __restrict__ ucount, uint32_t* __restrict__ mid_list,
                               uint32_t* __restrict__ big_list, uint32_t* __restrict__ list_cnt) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = gw; r < rows; r += nw) {
    uint64_t b = ptr[r], e = ptr[r + 1];
    uint64_t len = e - b;
    if (len > 32) {
      if (lane == 0) {
        if (len <= kSortSmem) mid_list[atomicAdd(&list_cnt[0], 1u)] = (uint32_t)r;
        else big_list[atomicAdd(&list_cnt[1], 1u)] = (uint32_t)r;
      }
      continue;
    }
    uint32_t x = lane < len ? data[b + lane] : 0xFFFFFFFFu;
    // bitonic sort of 32 lanes
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, stride);
        bool up = ((lane & size) == 0);
        bool lower = ((lane & stride) == 0);
        uint32_t mn = min(x, y), mx = max(x, y);
        x = (lower == up) ? mn : mx;
      }
    }
    if (ucount) {
      uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, x, 1);
      bool keep = lane < len && (lane == 0 || prev != x);
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) data[b + __popc(bal & lanemask_lt())] = x;
      if (lane == 0) ucount[r] = __popc(bal);
    } else if (lane < len) {
      data[b + lane] = x;
    }
  }
}

__device__ void smem_bitonic(uint32_t* a, uint32_t n2) {
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < n2 / 2; i += blockDim.x) {
        uint32_t lo = 2 * stride * (i / stride) + (i % stride);
        uint32_t hi = lo + stride;
        bool up = ((lo & size) == 0);
        uint32_t x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
    }
  }
  __syncthreads();
}

// Move the distinct keys of a sorted row to its front (block-wide); returns their count.
__device__ uint32_t block_unique_inplace(uint32_t* row, uint32_t len, const uint32_t* src_sorted, uint32_t* s_warp) {
    uint32_t written = 0;
  for (uint32_t t0 = 0; t0 < len; t0 += blockDim.x) {
    uint32_t i = t0 + threadIdx.x;
    uint32_t x = 0, p = 0;
    bool keep = false;
    if (i < len) {
      x = src_sorted[i];
      p = i ? src_sorted[i - 1] : 0;
      keep = (i == 0) || (p != x);
    }
    uint32_t tot;
    uint32_t off = block_exclusive_scan<uint32_t>(keep ? 1u : 0u, s_warp, &tot);
    if (keep) row[written + off] = x;
    written += tot;
    __syncthreads();
  }
  return written;
}

// Rows of 33..4096 keys: one block, bitonic sort in shared memory.
__global__ void __launch_bounds__(kSortBlock) k_segsort_block(uint32_t* __restrict__ data,
                                                              const uint64_t* __restrict__ ptr,
                                                              const uint32_t* __restrict__ list,
                                                              const uint32_t* __restrict__ list_cnt,
                                                              uint32_t* __restrict__ ucount) {
  __shared__ uint32_t a[kSortSmem];
  __shared__ uint32_t s_warp[32];
  uint32_t cnt = list_cnt[0];
  for (uint32_t li = blockIdx.x; li < cnt; li += gridDim.x) {
    uint32_t r = list[li];
    uint64_t b = ptr[r];
    uint32_t len = (uint32_t)(ptr[r + 1] - b);
    uint32_t n2 = 64;
    while (n2 < len) n2 <<= 1;
    for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) a[i] = i < len ? data[b + i] : 0xFFFFFFFFu;
    smem_bitonic(a, n2);
    if (ucount) {
      uint32_t u = block_unique_inplace(data + b, len, a, s_warp);
      if (threadIdx.x == 0) ucount[r] = u;
    } else {
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) data[b + i] = a[i];
    }
    __syncthreads();
  }
}

// Rows of > 4096 keys: one block; sort 4096-key chunks in shared memory, then
// merge runs pairwise through `aux` (merge-path split per thread).
__global__ void __launch_bounds__(kSortBlock) k_segsort_big(uint32_t* __restrict__ data,
                                                            uint32_t* __restrict__ aux,
                                                            const uint64_t* __restrict__ ptr,
                                                            const uint32_t* __restrict__ list,
                                                            const uint32_t* __restrict__ list_cnt,
                                                            uint32_t* __restrict__ ucount) {
  __shared__ uint32_t a[kSortSmem];
  __shared__ uint32_t s_warp[32];
  uint32_t cnt = list_cnt[1];
  for (uint32_t li = blockIdx.x; li < cnt; li += gridDim.x) {
    uint32_t r = list[li];
    uint64_t b = ptr[r];
    uint64_t len = ptr[r + 1] - b;
    uint32_t* src = data + b;
    uint32_t* dst = aux + b;
    for (uint64_t c0 = 0; c0 < len; c0 += kSortSmem) {
      uint32_t cl = (uint32_t)umin64(kSortSmem, len - c0);
      for (uint32_t i = threadIdx.x; i < kSortSmem; i += blockDim.x) a[i] = i < cl ? src[c0 + i] : 0xFFFFFFFFu;
      smem_bitonic(a, kSortSmem);
      for (uint32_t i = threadIdx.x; i < cl; i += blockDim.x) src[c0 + i] = a[i];
      __syncthreads();
    }
    for (uint64_t w = kSortSmem; w < len; w <<= 1) {
      for (uint64_t p0 = 0; p0 < len; p0 += 2 * w) {
        const uint32_t* A = src + p0;
        uint64_t la = umin64(w, len - p0);
        const uint32_t* B = A + la;
        uint64_t lb = (p0 + la < len) ? umin64(w, len - p0 - la) : 0;
        uint64_t L = la + lb;
        uint64_t per = (L + blockDim.x - 1) / blockDim.x;
        uint64_t d0 = umin64(L, per * threadIdx.x);
        uint64_t d1 = umin64(L, d0 + per);
        // merge path: i elements from A, d0 - i from B
        uint64_t lo = d0 > lb ? d0 - lb : 0, hi = umin64(d0, la);
        while (lo < hi) {
          uint64_t mid = (lo + hi) >> 1;
          if (A[mid] <= B[d0 - mid - 1]) lo = mid + 1;
          else hi = mid;
        }
        uint64_t i = lo, j = d0 - lo;
        for (uint64_t d = d0; d < d1; d++) {
          bool takeA = (j >= lb) || (i < la && A[i] <= B[j]);
          dst[p0 + d] = takeA ? A[i++] : B[j++];
        }
      }
      __syncthreads();
      uint32_t* t = src;
      src = dst;
      dst = t;
    }
    if (src != data + b) {
      for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) data[b + i] = src[i];
      __syncthreads();
    }
    if (ucount) {
      // distinct keys to the front, tile by tile; each tile is staged in shared
      // memory before any write, and the previous tile's last key is kept aside
      uint32_t written = 0;
      uint32_t* row = data + b;
      __shared__ uint32_t s_last;
      for (uint64_t t0 = 0; t0 < len; t0 += blockDim.x) {
        uint64_t i = t0 + threadIdx.x;
        uint32_t x = i < len ? row[i] : 0u;
        a[threadIdx.x] = x;
        __syncthreads();
        bool keep = false;
        if (i < len) {
          uint32_t p = threadIdx.x ? a[threadIdx.x - 1] : s_last;
          keep = (i == 0) || (p != x);
        }
        uint32_t tot;
        uint32_t off = block_exclusive_scan<uint32_t>(keep ? 1u : 0u, s_warp, &tot);
        if (keep) row[written + off] = x;
        written += tot;
        if (threadIdx.x == 0) s_last = a[blockDim.x - 1];
        __syncthreads();
      }
      if (threadIdx.x == 0) ucount[r] = written;
    }
    __syncthreads();
  }
}

int segmented_sort(kc_ctx* ctx, uint32_t* data, const uint64_t* ptr, uint32_t rows, uint64_t total, uint32_t max_row,
                   uint32_t* ucount, cudaStream_t s, uint32_t* launches) {
  if (rows == 0) return KC_OK;
  void* lists = nullptr;
  KC_TRY(scratch_get(ctx, kScrSortList, (2ull * rows + 4) * sizeof(uint32_t), &lists));
  uint32_t* mid_list = (uint32_t*)lists;
  uint32_t* big_list = mid_list + rows;
  uint32_t* list_cnt = big_list + rows;
  KC_CUDA(cudaMemsetAsync(list_cnt, 0, 4 * sizeof(uint32_t), s));
  unsigned blocks = (unsigned)std::min<uint64_t>((rows + 7) / 8, (uint64_t)ctx->num_sms * 16);
  k_segsort_warp<<<std::max(blocks, 1u), 256, 0, s>>>(data, ptr, rows, ucount, mid_list, big_list, list_cnt);
  KC_CUDA(cudaGetLastError());
  (*launches)++;
  if (max_row > 32) {
    k_segsort_block<<<ctx->num_sms * 4, kSortBlock, 0, s>>>(data, ptr, mid_list, list_cnt, ucount);
    KC_CUDA(cudaGetLastError());
    (*launches)++;
  }
  if (max_row > kSortSmem) {
    void* aux = nullptr;
    KC_TRY(scratch_get(ctx, kScrSort, total * sizeof(uint32_t), &aux));
    k_segsort_big<<<ctx->num_sms, kSortBlock, 0, s>>>(data, (uint32_t*)aux, ptr, big_list, list_cnt, ucount);
    KC_CUDA(cudaGetLastError());
    (*launches)++;
  }
  return KC_OK;
}

// ============================================================ validation
// The CSR must be simple and symmetric with sorted rows (Sec. II-A).  One warp
// per row; any violation sets kStBadGraph.  Also records the max row length.
__global__ void k_validate(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t n,
                           uint32_t* __restrict__ deg, uint32_t* __restrict__ status,
                           uint32_t* __restrict__ max_deg) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t nnz = rowptr[n];
  for (uint64_t u = gw; u < n; u += nw) {
    uint64_t b = rowptr[u], e = rowptr[u + 1];
    bool bad = (e < b) || (e > nnz);
    if (!bad) {
      for (uint64_t idx = b + lane; idx < e; idx += 32) {
        uint32_t v = col[idx];
        if (v >= n || v == u || (idx > b && col[idx - 1] >= v)) {
          bad = true;
          continue;
        }
        uint64_t lo = rowptr[v], hi = rowptr[v + 1];
        if (hi < lo || hi > nnz) {
          bad = true;
          continue;
        }
        while (lo < hi) {
          uint64_t mid = (lo + hi) >> 1;
          if (col[mid] < u) lo = mid + 1;
          else hi = mid;
        }
        if (lo >= rowptr[v + 1] || col[lo] != (uint32_t)u) bad = true;
      }
    }
    if (__any_sync(0xFFFFFFFFu, bad)) {
      if (lane == 0) atomicOr(status, kStBadGraph);
    }
    if (lane == 0) {
      uint32_t d = bad ? 0u : (uint32_t)(e - b);
      deg[u] = d;
      atomicMax(max_deg, d);
    }
  }
}

// ======================================================= canonicalisation
// Pass 1: count both directions of every non-loop entry; ids >= n are errors.
__global__ void k_canon_count(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t n,
                              uint64_t nnz, uint32_t* __restrict__ cnt, uint32_t* __restrict__ status) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = gw; u < n; u += nw) {
    uint64_t b = rowptr[u], e = rowptr[u + 1];
    if (e < b || e > nnz) {
      if (lane == 0) atomicOr(status, kStBadGraph);
      continue;
    }
    uint32_t own = 0;
    for (uint64_t idx = b + lane; idx < e; idx += 32) {
      uint32_t v = col[idx];
      if (v >= n) {
        atomicOr(status, kStBadGraph);
        continue;
      }
      if (v == u) continue;
      own++;
      atomicAdd(&cnt[v], 1u);
    }
    own = warp_sum(own);
    if (lane == 0 && own) atomicAdd(&cnt[u], own);
  }
}

// Pass 2: scatter both directions into per-row slots.
__global__ void k_canon_scatter(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t n,
                                uint64_t nnz, uint64_t* __restrict__ fill, uint32_t* __restrict__ tmp) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = gw; u < n; u += nw) {
    uint64_t b = rowptr[u], e = rowptr[u + 1];
    if (e < b || e > nnz) continue;
    for (uint64_t idx = b + lane; idx < e; idx += 32) {
      uint32_t v = col[idx];
      if (v >= n || v == u) continue;
      unsigned long long p = atomicAdd((unsigned long long*)&fill[u], 1ull);
      tmp[p] = v;
      p = atomicAdd((unsigned long long*)&fill[v], 1ull);
      tmp[p] = (uint32_t)u;
    }
  }
}

// Pass 3 (after per-row sort+unique): copy distinct keys to the final CSR.
__global__ void k_canon_compact(const uint64_t* __restrict__ ptr, const uint32_t* __restrict__ tmp,
                                const uint64_t* __restrict__ rowptr, uint32_t* __restrict__ col, uint32_t n,
                                uint32_t* __restrict__ deg, uint32_t* __restrict__ max_deg) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = gw; u < n; u += nw) {
    uint64_t src = ptr[u], dst = rowptr[u];
    uint32_t len = (uint32_t)(rowptr[u + 1] - dst);
    for (uint32_t i = lane; i < len; i += 32) col[dst + i] = tmp[src + i];
    if (lane == 0) {
      deg[u] = len;
      atomicMax(max_deg, len);
    }
  }
}

// =================================================================== peel
// k-core peeling in one cooperative launch, one level k at a time (Sec. II-A:
// repeatedly remove a vertex of minimum degree; removing every vertex of
// degree <= k before any of degree > k gives the same core numbers).
//
// Level k: every block scans its slice of the vertices and claims (CAS on
// core[]) the live ones of degree <= k into a shared-memory wave buffer.  A
// block then removes its wave -- consecutive ranks from one atomic per wave,
// and one degree decrement for every live neighbour of degree > k.  A
// neighbour whose degree falls from k+1 to k is claimed and joins the block's
// next wave at once, so cascades inside a level need no grid-wide barrier.
// Waves that outgrow the buffer spill to a global list, which every block
// shares out after a barrier.  A level ends when no block has work and the
// spill list is empty (one barrier per level when nothing spills).
//
// A vertex removed at level k keeps at most k live neighbours, so every
// out-degree of the resulting DAG is at most the degeneracy.  The order key
// is (core number, position of removal within the level); the second part
// depends on timing, which changes no count (any total order gives the same
// cliques, Sec. II-A).
struct PeelArgs {
  const uint64_t* rowptr;
  const uint32_t* col;
  uint32_t n;
  uint32_t* deg;
  uint32_t* core;
  uint32_t* rank;
  uint32_t* vert;
  uint32_t* spill0;   // [n] spill lists of even / odd sub-rounds
  uint32_t* spill1;
  uint32_t* ctr;      // [0..2] spill counts, [4..6] removals, per sub-round (rotating); [3] ranks given
  uint32_t* bar;      // [2] count, generation
  uint32_t* status;
  uint32_t* result;   // [0] degeneracy, [1] grid-wide sub-rounds
  unsigned long long spin_limit;  // ns
};

constexpr int kPeelThreads = 512;
constexpr uint32_t kPeelWave = 2048;  // shared-memory wave buffer entries
constexpr uint32_t kPeelBig = 512;    // vertices of higher degree are removed by the whole block
constexpr uint32_t kPeelBigMax = 64;  // big vertices per wave handled block-wide (the rest: one warp each)

__device__ __forceinline__ void peel_push(uint32_t* buf, uint32_t* cnt, uint32_t v, uint32_t* spill,
                                          uint32_t* spill_cnt) {
  const uint32_t p = atomicAdd(cnt, 1u);
  if (p < kPeelWave) {
    buf[p] = v;
  } else {
    spill[atomicAdd(spill_cnt, 1u)] = v;
  }
}

// Removal of v's edges [b, e) by the threads t = first, first + stride, ...:
// every live neighbour of degree > k loses one; one falling to k is claimed
// and queued.  Four neighbours per trip, loads issued before the atomics.
__device__ __forceinline__ void peel_edges(const PeelArgs& a, uint64_t b, uint64_t e, uint32_t first, uint32_t stride,
                                           uint32_t k, uint32_t* q, uint32_t* qn, uint32_t* spill,
                                           uint32_t* spill_cnt) {
  for (uint64_t i0 = b + first; i0 < e; i0 += 4ull * stride) {
    uint32_t u[4], dg[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint64_t p = i0 + (uint64_t)j * stride;
      u[j] = p < e ? __ldg(&a.col[p]) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) dg[j] = u[j] != 0xFFFFFFFFu ? __ldcg(&a.deg[u[j]]) : 0u;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      if (dg[j] <= k) continue;  // past the row end, removed, or already claimed at this level
      const uint32_t old = atomicSub(&a.deg[u[j]], 1u);
      if (old == k + 1) {
        if (atomicCAS(&a.core[u[j]], kAlive, k) == kAlive) peel_push(q, qn, u[j], spill, spill_cnt);
      } else if (old <= k) {
        atomicAdd(&a.deg[u[j]], 1u);  // lost a race with another decrement: undo
      }
    }
  }
}

__global__ void __launch_bounds__(kPeelThreads) k_peel(PeelArgs a) {
  __shared__ uint32_t s_q[2][kPeelWave];
  __shared__ uint32_t s_qn[2];
  __shared__ uint32_t s_base;
  __shared__ uint32_t s_big[kPeelBigMax];
  __shared__ uint32_t s_nbig;
  const uint32_t nb = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const uint32_t lane = tid & 31u, warp = tid >> 5, nwarps = blockDim.x >> 5;
  volatile uint32_t* vctr = a.ctr;
  // Every decision below is taken on values that no block can change until
  // all blocks have read them (per-sub-round slots, rotated over three), so
  // all blocks take the same branches and meet at the same barriers.
  uint32_t k = 0, sub = 0, degen = 0, removed = 0;
  int cur = 0;
  while (true) {
    if (removed >= a.n) break;
    const uint32_t removed0 = removed;
    bool first = true;
    while (true) {
      // ---- sub-round `sub`: spills go to list sub % 2, counted in ctr[sub % 3];
      // removals are counted in ctr[4 + sub % 3]
      uint32_t* spill = (sub & 1u) ? a.spill1 : a.spill0;
      uint32_t* spill_cnt = &a.ctr[sub % 3];
      if (bid == 0 && tid == 0) {
        // the slots of sub-round sub + 1 were last read right after barrier sub - 2
        a.ctr[(sub + 1) % 3] = 0;
        a.ctr[4 + (sub + 1) % 3] = 0;
      }
      __syncthreads();
      if (tid == 0) s_qn[cur] = 0;
      __syncthreads();
      if (first) {
        for (uint64_t v = (uint64_t)bid * blockDim.x + tid; v < a.n; v += (uint64_t)nb * blockDim.x) {
          if (__ldcg(&a.core[v]) == kAlive && __ldcg(&a.deg[v]) <= k && atomicCAS(&a.core[v], kAlive, k) == kAlive)
            peel_push(s_q[cur], &s_qn[cur], (uint32_t)v, spill, spill_cnt);
        }
      } else {
        // the previous sub-round's spill list, shared out by block
        const uint32_t prev = sub - 1;
        const uint32_t cnt = vctr[prev % 3];
        const uint32_t* list = (prev & 1u) ? a.spill1 : a.spill0;
        const uint32_t per = (cnt + nb - 1) / nb;
        const uint32_t lo = min(cnt, bid * per), hi = min(cnt, lo + per);
        for (uint32_t i = lo + tid; i < hi; i += blockDim.x) peel_push(s_q[cur], &s_qn[cur], __ldcg(&list[i]), spill, spill_cnt);
      }
      // ---- waves inside this block
      while (true) {
        __syncthreads();
        const uint32_t cnt = min(s_qn[cur], kPeelWave);
        if (cnt == 0) break;
        __syncthreads();
        if (tid == 0) {
          s_base = atomicAdd(&a.ctr[3], cnt);
          atomicAdd(&a.ctr[4 + sub % 3], cnt);
          s_qn[cur ^ 1] = 0;
          s_nbig = 0;
        }
        __syncthreads();
        const uint32_t base = s_base;
        uint32_t* nq = s_q[cur ^ 1];
        uint32_t* nqn = &s_qn[cur ^ 1];
        for (uint32_t i = warp; i < cnt; i += nwarps) {
          const uint32_t v = s_q[cur][i];
          if (lane == 0) {
            a.rank[v] = base + i;
            a.vert[base + i] = v;
          }
          const uint64_t b = a.rowptr[v], e = a.rowptr[v + 1];
          if (e - b > kPeelBig) {
            uint32_t slot = 0;
            if (lane == 0) slot = atomicAdd(&s_nbig, 1u);
            slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
            if (slot < kPeelBigMax) {
              if (lane == 0) s_big[slot] = v;
              continue;
            }
          }
          peel_edges(a, b, e, lane, 32, k, nq, nqn, spill, spill_cnt);
        }
        __syncthreads();
        // high-degree vertices of this wave: the whole block strides over each edge list
        const uint32_t nbig = min(s_nbig, kPeelBigMax);
        for (uint32_t j = 0; j < nbig; j++) {
          const uint32_t v = s_big[j];
          peel_edges(a, a.rowptr[v], a.rowptr[v + 1], tid, blockDim.x, k, nq, nqn, spill, spill_cnt);
        }
        cur ^= 1;
      }
      if (!grid_barrier(&a.bar[0], &a.bar[1], nb, a.spin_limit, a.status)) return;
      const uint32_t spilled = vctr[sub % 3];
      removed += vctr[4 + sub % 3];
      sub++;
      first = false;
      if (spilled == 0) break;
    }
    if (removed > removed0) degen = k;
    k++;
  }
  if (bid == 0 && tid == 0) {
    a.result[0] = degen;
    a.result[1] = sub;
  }
}

// ================================================================= orient
// DAG based on the order (Sec. II-A): keep (u, v) iff rank(u) < rank(v).
// Also counts the vertices of each bitmap-width tier (out-degree 1..32,
// 33..64, ..., 513..1024; wider ones in tier_hist[kTiers]), which bound the
// scratch a count of the graph can need.
__global__ void k_orient_count(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t n,
                               const uint32_t* __restrict__ rank, uint32_t* __restrict__ outdeg,
                               uint32_t* __restrict__ max_out, uint32_t* __restrict__ tier_hist) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t hist = 0;  // lane t < kTiers + 1 counts tier t
  for (uint64_t v = gw; v < n; v += nw) {
    uint32_t rv = rank[v];
    uint32_t c = 0;
    for (uint64_t idx = rowptr[v] + lane; idx < rowptr[v + 1]; idx += 32) c += rank[col[idx]] > rv;
    c = warp_sum(c);
    if (lane == 0) {
      outdeg[rv] = c;
      atomicMax(max_out, c);
    }
    if (c) {
      const uint32_t words = (c + 31) >> 5;
      uint32_t t = 0;
      while (t < (uint32_t)kTiers && (1u << t) < words) t++;
      hist += (lane == t);
    }
  }
  if (lane <= (uint32_t)kTiers && hist) atomicAdd(&tier_hist[lane], hist);
}

__global__ void k_orient_fill(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t n,
                              const uint32_t* __restrict__ rank, const uint64_t* __restrict__ orow,
                              uint32_t* __restrict__ ocol) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = gw; v < n; v += nw) {
    uint32_t rv = rank[v];
    uint64_t base = orow[rv];
    uint64_t b = rowptr[v], e = rowptr[v + 1];
    for (uint64_t i0 = b; i0 < e; i0 += 32) {
      uint64_t idx = i0 + lane;
      uint32_t rw = idx < e ? rank[col[idx]] : 0u;
      bool keep = idx < e && rw > rv;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) ocol[base + __popc(bal & lanemask_lt())] = rw;
      base += __popc(bal);
    }
  }
}

__global__ void k_max_u32(const uint32_t* __restrict__ a, uint32_t n, uint32_t* __restrict__ out) {
  uint32_t m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, a[i]);
  m = warp_max_u32(m);
  if (lane_id() == 0 && m) atomicMax(out, m);
}

// ================================================================ driver
static unsigned grid_for_warps(kc_ctx* ctx, uint64_t warps, int threads) {
  uint64_t blocks = (warps * 32 + threads - 1) / threads;
  uint64_t cap = (uint64_t)ctx->num_sms * 16;
  return (unsigned)std::max<uint64_t>(1, std::min(blocks, cap));
}

int prep_graph(kc_ctx* ctx, uint32_t n, const uint64_t* rowptr_in, const uint32_t* col_in, uint32_t flags,
               DevGraph* g, cudaStream_t s) {
  ctx->cur_stream = s;
  kc_upload_stats st{};
  uint32_t launches = 0;
  cudaEvent_t* ev = ctx->ev;
  KC_CUDA(cudaEventRecord(ev[0], s));
  const bool host = (flags & KC_HOST_PTRS) != 0;
  // ---- copy the caller's CSR
  uint64_t nnz = 0;
  if (host) {
    nnz = rowptr_in[n];
  } else {
    KC_CUDA(cudaMemcpyAsync(&nnz, rowptr_in + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
  }
  void *p_rowptr = nullptr, *p_col = nullptr;
  KC_TRY(scratch_get(ctx, kScrA, (n + 1ull) * sizeof(uint64_t), &p_rowptr));
  KC_TRY(scratch_get(ctx, kScrB, std::max<uint64_t>(nnz, 1) * sizeof(uint32_t), &p_col));
  cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  KC_CUDA(cudaMemcpyAsync(p_rowptr, rowptr_in, (n + 1ull) * sizeof(uint64_t), kind, s));
  if (nnz) KC_CUDA(cudaMemcpyAsync(p_col, col_in, nnz * sizeof(uint32_t), kind, s));
  KC_CUDA(cudaEventRecord(ev[1], s));

  uint32_t* d_small = nullptr;  // [0] status, [1] max_deg, [2] max_out, [3..4] peel result, [8..14] tier counts
  KC_TRY(scratch_get(ctx, kScrC, 64, (void**)&d_small));
  KC_CUDA(cudaMemsetAsync(d_small, 0, 64, s));
  uint32_t* d_status = d_small;
  uint32_t* d_maxdeg = d_small + 1;
  uint32_t* d_maxout = d_small + 2;
  uint32_t* d_peelres = d_small + 3;

  const uint64_t* rowptr = (const uint64_t*)p_rowptr;
  const uint32_t* col = (const uint32_t*)p_col;
  uint32_t* deg = nullptr;
  KC_TRY(scratch_get(ctx, kScrD, std::max<uint64_t>(n, 1) * sizeof(uint32_t) * 4, (void**)&deg));
  // deg | alive0 | alive1 | frontier share one buffer
  uint32_t* alive0 = deg + n;
  uint32_t* alive1 = alive0 + n;
  uint32_t* frontier = alive1 + n;
  unsigned wgrid = grid_for_warps(ctx, n, 256);

  if (flags & KC_CANONICALIZE) {
    uint32_t* cnt = nullptr;
    uint64_t *ptr = nullptr, *newptr = nullptr;
    uint32_t *tmp = nullptr, *ncol = nullptr;
    KC_TRY(scratch_get(ctx, kScrE, (n + 1ull) * sizeof(uint64_t) * 3 + std::max<uint64_t>(n, 1) * 4, (void**)&ptr));
    uint64_t* fill = ptr + (n + 1);
    newptr = fill + (n + 1);
    cnt = (uint32_t*)(newptr + (n + 1));
    KC_TRY(scratch_get(ctx, kScrF, std::max<uint64_t>(2 * nnz, 1) * sizeof(uint32_t), (void**)&tmp));
    KC_CUDA(cudaMemsetAsync(cnt, 0, std::max<uint64_t>(n, 1) * 4, s));
    k_canon_count<<<wgrid, 256, 0, s>>>(rowptr, col, n, nnz, cnt, d_status);
    KC_CUDA(cudaGetLastError());
    launches++;
    KC_TRY(exclusive_scan_u32_to_u64(ctx, cnt, ptr, n, s, &launches));
    KC_CUDA(cudaMemcpyAsync(fill, ptr, (n + 1ull) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    k_canon_scatter<<<wgrid, 256, 0, s>>>(rowptr, col, n, nnz, fill, tmp);
    KC_CUDA(cudaGetLastError());
    launches++;
    // longest row before dedup picks the sort tiers
    uint64_t tot2 = 0;
    KC_CUDA(cudaMemcpyAsync(&tot2, ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    k_max_u32<<<wgrid, 256, 0, s>>>(cnt, n, d_small + 8);
    KC_CUDA(cudaGetLastError());
    launches++;
    uint32_t h_rowmax[1] = {0};
    KC_CUDA(cudaMemcpyAsync(h_rowmax, d_small + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    uint32_t bound = h_rowmax[0];
    KC_TRY(segmented_sort(ctx, tmp, ptr, n, tot2, bound, cnt, s, &launches));
    KC_TRY(exclusive_scan_u32_to_u64(ctx, cnt, newptr, n, s, &launches));
    uint64_t nnz2 = 0;
    KC_CUDA(cudaMemcpyAsync(&nnz2, newptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    KC_TRY(scratch_get(ctx, kScrG, std::max<uint64_t>(nnz2, 1) * sizeof(uint32_t), (void**)&ncol));
    k_canon_compact<<<wgrid, 256, 0, s>>>(ptr, tmp, newptr, ncol, n, deg, d_maxdeg);
    KC_CUDA(cudaGetLastError());
    launches++;
    rowptr = newptr;
    col = ncol;
    nnz = nnz2;
  } else {
    k_validate<<<wgrid, 256, 0, s>>>(rowptr, col, n, deg, d_status, d_maxdeg);
    KC_CUDA(cudaGetLastError());
    launches++;
  }
  KC_CUDA(cudaEventRecord(ev[2], s));
  uint32_t h_small[16] = {0};
  KC_CUDA(cudaMemcpyAsync(h_small, d_small, sizeof(h_small), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  if (h_small[0] & kStBadGraph) return KC_E_INVALID_GRAPH;
  if (nnz & 1ull) return KC_E_INVALID_GRAPH;

  // ---- allocate the graph's own arrays
  g->n = n;
  g->m = nnz / 2;
  KC_CUDA(cudaMallocAsync(&g->core, std::max<uint64_t>(n, 1) * sizeof(uint32_t), s));
  KC_CUDA(cudaMallocAsync(&g->rank, std::max<uint64_t>(n, 1) * sizeof(uint32_t), s));
  KC_CUDA(cudaMallocAsync(&g->vert, std::max<uint64_t>(n, 1) * sizeof(uint32_t), s));
  KC_CUDA(cudaMallocAsync(&g->orow, (n + 1ull) * sizeof(uint64_t), s));
  KC_CUDA(cudaMallocAsync(&g->ocol, std::max<uint64_t>(g->m, 1) * sizeof(uint32_t), s));

  // ---- peel (one cooperative launch)
  if (n > 0) {
    KC_CUDA(cudaMemsetAsync(g->core, 0xFF, (uint64_t)n * sizeof(uint32_t), s));
    int per_sm = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel, kPeelThreads, 0));
    per_sm = std::max(1, std::min(per_sm, 2));
    unsigned nb = (unsigned)(ctx->num_sms * per_sm);
    uint64_t need_blocks = ((uint64_t)n + kPeelThreads - 1) / kPeelThreads;
    nb = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(nb, need_blocks));
    uint32_t* pw = nullptr;
    KC_TRY(scratch_get(ctx, kScrPeel, 16 * sizeof(uint32_t), (void**)&pw));
    KC_CUDA(cudaMemsetAsync(pw, 0, 16 * sizeof(uint32_t), s));
    PeelArgs pa;
    pa.rowptr = rowptr;
    pa.col = col;
    pa.n = n;
    pa.deg = deg;
    pa.core = g->core;
    pa.rank = g->rank;
    pa.vert = g->vert;
    pa.spill0 = alive0;
    pa.spill1 = alive1;
    pa.ctr = pw;
    pa.bar = pw + 8;
    pa.status = d_status;
    pa.result = d_peelres;
    pa.spin_limit = ctx->opts.spin_limit;
    void* args[] = {&pa};
    KC_CUDA(cudaLaunchCooperativeKernel((const void*)k_peel, dim3(nb), dim3(kPeelThreads), args, 0, s));
    launches++;
    // a peel that gave up at a bounded wait leaves ranks unset: stop before anything indexes with them
    uint32_t h_status = 0;
    KC_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h_status & kStTimeout) return KC_E_DEVICE_TIMEOUT;
  }
  KC_CUDA(cudaEventRecord(ev[3], s));
  // ---- orient
  uint32_t* outdeg = frontier;  // reuse (peel is done with it)
  // the tier counts (canonicalisation used the same words for its longest row)
  KC_CUDA(cudaMemsetAsync(d_small + 8, 0, (kTiers + 1) * sizeof(uint32_t), s));
  if (n > 0) {
    k_orient_count<<<wgrid, 256, 0, s>>>(rowptr, col, n, g->rank, outdeg, d_maxout, d_small + 8);
    KC_CUDA(cudaGetLastError());
    launches++;
  }
  KC_TRY(exclusive_scan_u32_to_u64(ctx, outdeg, g->orow, n, s, &launches));
  if (n > 0) {
    k_orient_fill<<<wgrid, 256, 0, s>>>(rowptr, col, n, g->rank, g->orow, g->ocol);
    KC_CUDA(cudaGetLastError());
    launches++;
  }
  KC_CUDA(cudaMemcpyAsync(h_small, d_small, sizeof(h_small), cudaMemcpyDeviceToHost, s));
  KC_CUDA(cudaStreamSynchronize(s));
  if (h_small[0] & kStTimeout) return KC_E_DEVICE_TIMEOUT;
  g->max_out = h_small[2];
  g->degeneracy = h_small[3];
  g->peel_rounds = h_small[4];
  for (int t = 0; t < kTiers; t++) g->tier_roots[t] = h_small[8 + t];
  KC_TRY(segmented_sort(ctx, g->ocol, g->orow, n, g->m, g->max_out, nullptr, s, &launches));
  KC_CUDA(cudaEventRecord(ev[4], s));
  KC_CUDA(cudaEventSynchronize(ev[4]));
  cudaEventElapsedTime(&st.ms_copy, ev[0], ev[1]);
  cudaEventElapsedTime(&st.ms_canon, ev[1], ev[2]);
  cudaEventElapsedTime(&st.ms_peel, ev[2], ev[3]);
  cudaEventElapsedTime(&st.ms_orient, ev[3], ev[4]);
  cudaEventElapsedTime(&st.ms_total, ev[0], ev[4]);
  st.launches = launches;
  ctx->last_up = st;
  return KC_OK;
}

}  // namespace kc
