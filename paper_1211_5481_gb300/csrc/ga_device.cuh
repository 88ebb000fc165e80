// ga_device.cuh -- the GA operators as device functions, shared by the
// single-problem kernels (ga_ops.cu) and the batched ones (batch.cu). The
// definitions (ranking key, parent selection, crossover, mutation,
// immigrants) are documented in ga_ops.cu.
#pragma once
#include <math_constants.h>

#include "game_internal.cuh"
#include "philox.cuh"

namespace game {
namespace ga {

constexpr int kPlanThreads = 1024;
constexpr int kMaxElites = 256;

// Ranking key of a fitness value as an unsigned integer whose order is the
// order of the values (NaN as +infinity, -0 as +0, so equal values tie as in
// FP64 comparison): the GPU ranks with integer compares instead of the slow
// FP64 pipe.
__device__ __forceinline__ uint64_t rank_key(double f) {
  if (isnan(f)) f = CUDART_INF;
  if (f == 0.0) f = 0.0;
  const uint64_t u = (uint64_t)__double_as_longlong(f);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
constexpr uint64_t kKeyMax = ~0ull;   // above every rank_key

// (ka, a) ranks before (kb, b)
__device__ __forceinline__ bool ranks_before(uint64_t ka, int a, uint64_t kb, int b) {
  return ka < kb || (ka == kb && a < b);
}

// Gene e = p K + k of the initial population (uniform in [-1, 1)).
__device__ __forceinline__ float init_gene(uint64_t seed, int K, int64_t e) {
  const uint32_t p = (uint32_t)(e / K), k = (uint32_t)(e % K);
  return uniform_gene(philox4x32_10(seed, 0u, p, k, kTagInit).x);
}

// Roulette weight of a fitness value: floor(2^32 RN(1 / RN(1 + f))), 0 for
// a NaN, negative or infinite f (all operations IEEE round-to-nearest).
__device__ __forceinline__ uint64_t roulette_weight(double f) {
  if (!(f >= 0.0) || isinf(f)) return 0;
  const double w = __ddiv_rn(1.0, __dadd_rn(1.0, f));
  return __double2ull_rz(__dmul_rn(w, 4294967296.0));
}

// Parent r (0 or 1) of pair q, drawn from the ga.P current chromosomes.
// Every mode takes its words from Philox(seed; g, q, r, TOUR | call << 8).
__device__ __forceinline__ int select_parent(const GaDev& ga, const double* __restrict__ fit,
                                             uint64_t seed, uint32_t g, uint32_t q, uint32_t r) {
  if (ga.sel == GAME_SEL_RANKING) {
    // u uniform on [0, P (P + 1) / 2); rank k covers C(k) <= u < C(k + 1),
    // C(k) = sum_{j<k} (P - j) = k P - k (k - 1) / 2
    const uint32_t x = philox4x32_10(seed, g, q, r, kTagTour).x;
    const uint64_t P = (uint64_t)ga.P;
    const uint64_t u = ((uint64_t)x * (P * (P + 1) / 2)) >> 32;
    int lo = 0, hi = ga.P - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      const uint64_t c = (uint64_t)mid * P - (uint64_t)mid * (uint64_t)(mid - 1) / 2;
      if (c <= u) lo = mid;
      else hi = mid - 1;
    }
    return ga.order[lo];
  }
  if (ga.sel == GAME_SEL_ROULETTE) {
    // u uniform on [0, W) from 64 bits; chromosome p covers [cum[p], cum[p + 1])
    const uint4 w = philox4x32_10(seed, g, q, r, kTagTour);
    const uint64_t W = ga.cum[ga.P];
    if (W == 0) return (int)(((uint64_t)w.x * (uint64_t)ga.P) >> 32);
    const uint64_t u = __umul64hi(((uint64_t)w.x << 32) | w.y, W);
    int lo = 0, hi = ga.P - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (u < ga.cum[mid + 1]) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  }
  // tournament: the best of T uniform candidates
  int win = -1;
  uint64_t wk = 0;
  uint4 w = make_uint4(0, 0, 0, 0);
  for (int s = 0; s < ga.T; ++s) {
    if ((s & 3) == 0) w = philox4x32_10(seed, g, q, r, kTagTour | ((uint32_t)(s >> 2) << 8));
    const uint32_t word = (s & 3) == 0 ? w.x : (s & 3) == 1 ? w.y : (s & 3) == 2 ? w.z : w.w;
    const int c = (int)(((uint64_t)word * (uint64_t)ga.P) >> 32);
    const uint64_t ck = rank_key(fit[c]);
    if (win < 0 || ranks_before(ck, c, wk, win)) {
      win = c;
      wk = ck;
    }
  }
  return win;
}

// One CTA of kPlanThreads threads: elites, parent selection and crossover plan of
// one problem (plan[s] = {head parent, tail parent, cut, elite flag}) for
// ga.Nout output slots; tournaments draw from the ga.P current chromosomes.
__device__ __forceinline__ void plan_body(const GaDev& ga, const double* __restrict__ fit,
                                          uint64_t seed, uint32_t g, int4* __restrict__ plan) {
  __shared__ int elite[kMaxElites];
  __shared__ uint64_t wkey[kPlanThreads / 32];
  __shared__ int widx[kPlanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // 1. elites, one block-wide arg-min per elite
  for (int e = 0; e < ga.E; ++e) {
    uint64_t bk = kKeyMax;
    int bi = 0x7fffffff;
    for (int p = tid; p < ga.P; p += kPlanThreads) {
      bool taken = false;
      for (int j = 0; j < e; ++j) taken |= (elite[j] == p);
      if (taken) continue;
      const uint64_t k = rank_key(fit[p]);
      if (ranks_before(k, p, bk, bi)) {
        bk = k;
        bi = p;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ranks_before(ok, oi, bk, bi)) {
        bk = ok;
        bi = oi;
      }
    }
    if (lane == 0) {
      wkey[wid] = bk;
      widx[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {
      bk = wkey[lane];
      bi = widx[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ranks_before(ok, oi, bk, bi)) {
          bk = ok;
          bi = oi;
        }
      }
      if (lane == 0) elite[e] = bi;
    }
    __syncthreads();
  }
  for (int e = tid; e < ga.E; e += kPlanThreads) plan[e] = make_int4(elite[e], elite[e], ga.K, 1);

  // 2.-3. pairs: parent selection and crossover decision
  const int npairs = (ga.Nout - ga.E + 1) / 2;
  for (int q = tid; q < npairs; q += kPlanThreads) {
    int parent[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
      parent[r] = select_parent(ga, fit, seed, g, (uint32_t)q, (uint32_t)r);
    const uint4 wx = philox4x32_10(seed, g, (uint32_t)q, 0u, kTagCross);
    int cut = ga.K;
    if ((wx.x >> 8) < ga.thr_pc)
      cut = 1 + (int)(((uint64_t)wx.y * (uint64_t)(ga.K - 1)) >> 32);
    const int s0 = ga.E + 2 * q;
    plan[s0] = make_int4(parent[0], parent[1], cut, 0);
    if (s0 + 1 < ga.Nout) plan[s0 + 1] = make_int4(parent[1], parent[0], cut, 0);
  }
}

// Gene e = s K + k of the next population.
__device__ __forceinline__ float breed_gene(const GaDev& ga, const float* __restrict__ pop,
                                            const int4* __restrict__ plan, uint64_t seed,
                                            uint32_t g, int64_t e) {
  const int s = (int)(e / ga.K), k = (int)(e % ga.K);
  float v;
  if (s >= ga.Nout - ga.I) {
    v = uniform_gene(philox4x32_10(seed, g, (uint32_t)s, (uint32_t)k, kTagImmigrant).x);
  } else {
    const int4 pl = plan[s];
    v = pop[(int64_t)(k < pl.z ? pl.x : pl.y) * ga.K + k];
    if (s >= ga.E) {
      const uint4 w = philox4x32_10(seed, g, (uint32_t)s, (uint32_t)k, kTagMut);
      if ((w.x >> 8) < ga.thr_pm) {
        const float z = irwin_hall12(seed, g, (uint32_t)s, (uint32_t)k);
        v = __fadd_rn(v, __fmul_rn(ga.sigma, z));
        if (v < -1.0f) v = -1.0f;
        if (v > 1.0f) v = 1.0f;
      }
    }
  }
  return v;
}

}  // namespace ga
}  // namespace game
