// rescore.cu -- candidate selection of the elite re-scoring: the n best
// chromosomes of a reduced-precision fitness vector, by (fitness, index) with
// NaN as +infinity (the ranking elitism uses, paper Section 3). Their fitness
// is then re-evaluated in FP64 by the Gram form (gram.cu) and replaces the
// reduced value, so elitism (Section 3; 2 elites, Section 5) and the
// tournaments rank the best candidates by accurate values.
//
// select_top_kernel, one CTA: each thread keeps the top 16 of its strided
// elements in registers, each warp merges its lanes' lists, warp 0 merges the
// 8 warps'. Fitness values are compared through order-preserving integer
// keys (integer compares instead of the FP64 pipe).
#include <math_constants.h>

#include "game_internal.cuh"

namespace game {

namespace {

constexpr int kSelThreads = 256;

// Fitness as an order-preserving unsigned key (NaN as +infinity, -0 as +0),
// so the ranking runs on integer compares instead of the slow FP64 pipe.
__device__ __forceinline__ uint64_t fit_key(double f) {
  if (isnan(f)) f = CUDART_INF;
  if (f == 0.0) f = 0.0;
  const uint64_t u = (uint64_t)__double_as_longlong(f);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
constexpr uint64_t kNoKey = ~0ull;

__device__ __forceinline__ bool key_before(uint64_t fa, int a, uint64_t fb, int b) {
  return fa < fb || (fa == fb && a < b);
}

// Warp-wide arg-min of (key, index); every lane receives the winner.
__device__ __forceinline__ void warp_argmin(uint64_t& k, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t ok = __shfl_xor_sync(0xffffffffu, k, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (key_before(ok, oi, k, i)) {
      k = ok;
      i = oi;
    }
  }
}

// Sorted list of kMaxRescore (key, index) pairs held in registers.
struct TopList {
  uint64_t k[kMaxRescore];
  int i[kMaxRescore];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int j = 0; j < kMaxRescore; ++j) {
      k[j] = kNoKey;
      i[j] = 0x7fffffff;
    }
  }
  __device__ __forceinline__ void insert(uint64_t key, int idx) {
    if (!key_before(key, idx, k[kMaxRescore - 1], i[kMaxRescore - 1])) return;
    k[kMaxRescore - 1] = key;
    i[kMaxRescore - 1] = idx;
#pragma unroll
    for (int j = kMaxRescore - 1; j > 0; --j) {
      if (key_before(k[j], i[j], k[j - 1], i[j - 1])) {
        const uint64_t tk = k[j];
        const int ti = i[j];
        k[j] = k[j - 1];
        i[j] = i[j - 1];
        k[j - 1] = tk;
        i[j - 1] = ti;
      }
    }
  }
  __device__ __forceinline__ void pop_front() {
#pragma unroll
    for (int j = 0; j < kMaxRescore - 1; ++j) {
      k[j] = k[j + 1];
      i[j] = i[j + 1];
    }
    k[kMaxRescore - 1] = kNoKey;
    i[kMaxRescore - 1] = 0x7fffffff;
  }
};

__global__ void __launch_bounds__(kSelThreads)
select_top_kernel(const double* __restrict__ fit, int P, int n, int* __restrict__ cand) {
  __shared__ uint64_t wk[kSelThreads / 32][kMaxRescore];
  __shared__ int wi[kSelThreads / 32][kMaxRescore];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TopList L;
  L.clear();
  for (int p = tid; p < P; p += kSelThreads) L.insert(fit_key(fit[p]), p);
  // each warp: n rounds of arg-min over its lanes' list heads
  for (int r = 0; r < n; ++r) {
    uint64_t k = L.k[0];
    int i = L.i[0];
    warp_argmin(k, i);
    if (L.i[0] == i && i != 0x7fffffff) L.pop_front();
    if (lane == 0) {
      wk[warp][r] = k;
      wi[warp][r] = i;
    }
  }
  __syncthreads();
  if (warp != 0) return;
  L.clear();
#pragma unroll
  for (int j = 0; j < kMaxRescore; ++j)
    if (j < n && lane < kSelThreads / 32) {
      L.k[j] = wk[lane][j];
      L.i[j] = wi[lane][j];
    }
  for (int r = 0; r < n; ++r) {
    uint64_t k = L.k[0];
    int i = L.i[0];
    warp_argmin(k, i);
    if (L.i[0] == i && i != 0x7fffffff) L.pop_front();
    if (lane == 0) cand[r] = i;
  }
}

}  // namespace

cudaError_t launch_select_top(const double* fit, int P, int n, int* cand, cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  if (n > kMaxRescore || n > P) return cudaErrorInvalidValue;
  select_top_kernel<<<1, kSelThreads, 0, st>>>(fit, P, n, cand);
  return cudaGetLastError();
}

}  // namespace game
