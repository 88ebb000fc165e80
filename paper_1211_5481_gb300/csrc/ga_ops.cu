// ga_ops.cu -- GA operators on the device: initialisation, elitism,
// tournament selection, one-point crossover, Gaussian mutation, clamping and
// immigrants (paper Section 3 names crossover, mutation and elitism, with
// genes in [-1, 1]; Section 5 gives the rates and 2 elites; Section 4 the
// random replacement of older individuals).
//
// Definitions (identical on the CPU oracle, so results are bit-exact):
//  * ranking key (fit, index), NaN fitness as +infinity, lower is better;
//  * elites: slots 0..E-1 receive the E best chromosomes unchanged;
//  * pair q: two tournaments of T candidates c = floor(w * P / 2^32), words w
//    from Philox(seed; g, q, r, TOUR | call << 8); crossover iff the top 24
//    bits of Philox(seed; g, q, 0, CROSS).x are below floor(pc * 2^24), at
//    cut = 1 + floor(.y * (K-1) / 2^32); children to slots E+2q, E+2q+1;
//  * mutation of gene k of slot s >= E iff Philox(seed; g, s, k, MUT).x >> 8
//    is below floor(pm * 2^24): gene = clamp(gene + sigma * z, -1, 1), z an
//    Irwin-Hall-12 normal, both operations rounded to FP32 without FMA;
//  * immigrants: the last I slots get fresh uniform genes.
// ga_plan_kernel (one CTA) decides, per slot, the head parent, the tail
// parent and the cut; ga_breed_kernel then builds every gene in parallel.
#include "game_internal.cuh"
#include "philox.cuh"

#include <math_constants.h>

namespace game {

namespace {

constexpr int kPlanThreads = 1024;
constexpr int kMaxElites = 256;

__device__ __forceinline__ double rank_key(double f) { return isnan(f) ? CUDART_INF : f; }

// (fa, a) ranks before (fb, b)
__device__ __forceinline__ bool ranks_before(double fa, int a, double fb, int b) {
  return fa < fb || (fa == fb && a < b);
}

__global__ void init_population_kernel(uint64_t seed, int P, int K, float* __restrict__ pop) {
  const int64_t n = (int64_t)P * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = (uint32_t)(e / K), k = (uint32_t)(e % K);
    pop[e] = uniform_gene(philox4x32_10(seed, 0u, p, k, kTagInit).x);
  }
}

__global__ void __launch_bounds__(kPlanThreads)
ga_plan_kernel(GaDev ga, const double* __restrict__ fit, uint64_t seed, uint32_t g,
               int4* __restrict__ plan) {
  __shared__ int elite[kMaxElites];
  __shared__ double wkey[kPlanThreads / 32];
  __shared__ int widx[kPlanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  // 1. elites, one block-wide arg-min per elite
  for (int e = 0; e < ga.E; ++e) {
    double bk = CUDART_INF;
    int bi = 0x7fffffff;
    for (int p = tid; p < ga.P; p += kPlanThreads) {
      bool taken = false;
      for (int j = 0; j < e; ++j) taken |= (elite[j] == p);
      if (taken) continue;
      const double k = rank_key(fit[p]);
      if (ranks_before(k, p, bk, bi)) {
        bk = k;
        bi = p;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ok = __shfl_xor_sync(0xffffffffu, bk, o);
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
        const double ok = __shfl_xor_sync(0xffffffffu, bk, o);
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

  // 2.-3. pairs: tournaments and crossover decision
  const int npairs = (ga.P - ga.E + 1) / 2;
  for (int q = tid; q < npairs; q += kPlanThreads) {
    int parent[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int win = -1;
      double wk = 0.0;
      uint4 w = make_uint4(0, 0, 0, 0);
      for (int s = 0; s < ga.T; ++s) {
        if ((s & 3) == 0) w = philox4x32_10(seed, g, (uint32_t)q, (uint32_t)r,
                                            kTagTour | ((uint32_t)(s >> 2) << 8));
        const uint32_t word = (s & 3) == 0 ? w.x : (s & 3) == 1 ? w.y : (s & 3) == 2 ? w.z : w.w;
        const int c = (int)(((uint64_t)word * (uint64_t)ga.P) >> 32);
        const double ck = rank_key(fit[c]);
        if (win < 0 || ranks_before(ck, c, wk, win)) {
          win = c;
          wk = ck;
        }
      }
      parent[r] = win;
    }
    const uint4 wx = philox4x32_10(seed, g, (uint32_t)q, 0u, kTagCross);
    int cut = ga.K;
    if ((wx.x >> 8) < ga.thr_pc)
      cut = 1 + (int)(((uint64_t)wx.y * (uint64_t)(ga.K - 1)) >> 32);
    const int s0 = ga.E + 2 * q;
    plan[s0] = make_int4(parent[0], parent[1], cut, 0);
    if (s0 + 1 < ga.P) plan[s0 + 1] = make_int4(parent[1], parent[0], cut, 0);
  }
}

__global__ void ga_breed_kernel(GaDev ga, const float* __restrict__ pop,
                                const int4* __restrict__ plan, uint64_t seed, uint32_t g,
                                float* __restrict__ next) {
  const int64_t n = (int64_t)ga.P * ga.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ga.K), k = (int)(e % ga.K);
    float v;
    if (s >= ga.P - ga.I) {
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
    next[e] = v;
  }
}

int blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

}  // namespace

cudaError_t launch_init_population(uint64_t seed, int P, int K, float* pop, cudaStream_t st) {
  init_population_kernel<<<blocks_for((int64_t)P * K, 256), 256, 0, st>>>(seed, P, K, pop);
  return cudaGetLastError();
}

cudaError_t launch_generation(const GaDev& ga, const float* pop, const double* fit,
                              uint64_t seed, uint32_t g, int4* plan, float* next,
                              cudaStream_t st) {
  if (ga.E > kMaxElites) return cudaErrorInvalidValue;
  ga_plan_kernel<<<1, kPlanThreads, 0, st>>>(ga, fit, seed, g, plan);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ga_breed_kernel<<<blocks_for((int64_t)ga.P * ga.K, 256), 256, 0, st>>>(ga, pop, plan, seed,
                                                                        g, next);
  return cudaGetLastError();
}

}  // namespace game
