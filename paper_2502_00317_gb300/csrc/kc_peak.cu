// kc_peak.cu -- integer-pipe peak of this GPU for the enumerator's work unit
// (libkc_peak.so, used by the benchmark for the roofline denominator).
//
// The enumerator's unit is a word-op: one 32-bit AND of two candidate words
// followed by a POPC of the result and its accumulation.  This kernel issues
// nothing but word-ops, in 8 independent chains per thread at full
// occupancy, so it runs at the rate of the slowest pipe the unit uses
// (POPC).  The chain's data change every step so nothing is hoisted.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_word_ops(uint32_t seed, int iters, unsigned long long* sink) {
  uint32_t x[kChains], s[kChains];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kChains; j++) {
    x[j] = (seed ^ t) * (2654435761u + 2u * j) + j;
    s[j] = 0;
  }
  const uint32_t y = seed * 40503u + t;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < kUnroll; r++) {
#pragma unroll
      for (int j = 0; j < kChains; j++) {
        s[j] += __popc(x[j] & y);
        x[j] ^= s[j];
      }
    }
  }
  uint32_t tot = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) tot += s[j] ^ x[j];
  if (tot == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps the work live; practically never taken
}

}  // namespace

// Measures word-ops per second on the current device: best of `reps` timed
// launches of `iters` loop trips each (after one warm-up launch).  Returns 0 on
// success, else the CUDA error code.  *ops_per_launch receives the word-ops
// of one launch, *best_ms its best time.
extern "C" int kc_peak_word_ops(int iters, int reps, double* ops_per_s, double* ops_per_launch, float* best_ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_word_ops, 256, 0);
  if (e != cudaSuccess) return (int)e;
  const unsigned blocks = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  unsigned long long* sink = nullptr;
  if ((e = cudaMalloc(&sink, sizeof(unsigned long long))) != cudaSuccess) return (int)e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  k_word_ops<<<blocks, 256>>>(1u, iters, sink);
  float best = 1e30f;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(a);
    k_word_ops<<<blocks, 256>>>(2u + r, iters, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return (int)e;
  const double ops = (double)blocks * 256.0 * iters * kUnroll * kChains;
  *ops_per_launch = ops;
  *best_ms = best;
  *ops_per_s = ops / (best * 1e-3);
  return 0;
}
