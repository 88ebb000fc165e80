// ga_ops.cu -- GA operators on the device: initialisation, elitism,
// tournament selection, one-point crossover, Gaussian mutation, clamping and
// immigrants (paper Section 3 names crossover, mutation and elitism, with
// genes in [-1, 1]; Section 5 gives the rates and 2 elites; Section 4 the
// random replacement of older individuals).
//
// Definitions (identical on the CPU oracle, so results are bit-exact):
//  * ranking key (fit, index), NaN fitness as +infinity, lower is better;
//  * elites: slots 0..E-1 receive the E best chromosomes unchanged;
//  * pair q, parent r in {0, 1}: selected from the P chromosomes by
//    - tournament: the best of T candidates c = floor(w * P / 2^32), words w
//      from Philox(seed; g, q, r, TOUR | call << 8);
//    - ranking (linear): x = Philox(seed; g, q, r, TOUR).x,
//      u = floor(x W / 2^32) with W = P (P + 1) / 2, and the chromosome of
//      rank k (0 = best by the ranking key) where
//      k P - k (k - 1) / 2 <= u < (k + 1) P - (k + 1) k / 2 (weight P - k);
//    - roulette: weights w_p = floor(2^32 RN(1 / RN(1 + fit_p))) (0 for
//      NaN or infinite fit), W = sum w_p, u = floor((x 2^32 + y) W / 2^64)
//      from the same call's words x, y, and the p with
//      sum_{j<p} w_j <= u < sum_{j<=p} w_j (W = 0: p = floor(x P / 2^32));
//    crossover iff the top 24
//    bits of Philox(seed; g, q, 0, CROSS).x are below floor(pc * 2^24), at
//    cut = 1 + floor(.y * (K-1) / 2^32); children to slots E+2q, E+2q+1;
//  * mutation of gene k of slot s >= E iff Philox(seed; g, s, k, MUT).x >> 8
//    is below floor(pm * 2^24): gene = clamp(gene + sigma * z, -1, 1), z an
//    Irwin-Hall-12 normal, both operations rounded to FP32 without FMA;
//  * immigrants: the last I slots get fresh uniform genes.
// ranking_order_kernel (one CTA, bitonic sort in shared memory) or
// roulette_cum_kernel (one CTA, exact integer scan) prepares the selection
// table; ga_plan_kernel (one CTA) decides, per slot, the head parent, the
// tail parent and the cut; ga_breed_kernel then builds every gene in
// parallel.
#include "ga_device.cuh"

namespace game {

namespace {

using ga::kMaxElites;
using ga::kPlanThreads;

__global__ void init_population_kernel(uint64_t seed, int P, int K, float* __restrict__ pop) {
  const int64_t n = (int64_t)P * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    pop[e] = ga::init_gene(seed, K, e);
}

__host__ __device__ inline int pow2_at_least(int P) {
  int n2 = 1;
  while (n2 < P) n2 <<= 1;
  return n2;
}

// order[r] = the chromosome of rank r (order may be NULL: the result stays in
// sidx): a bitonic sort of (rank key, index) over the next power of two
// >= P, padded with keys above every chromosome; skey [n2] and sidx [n2] in
// shared memory.
__device__ void ranking_sort_body(int P, const double* __restrict__ fit, uint64_t* skey,
                                  int* sidx, int* __restrict__ order) {
  const int n2 = pow2_at_least(P);
  for (int i = threadIdx.x; i < n2; i += kPlanThreads) {
    skey[i] = i < P ? ga::rank_key(fit[i]) : ga::kKeyMax;
    sidx[i] = i < P ? i : 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kPlanThreads) {
        const int l = i ^ j;
        if (l <= i) continue;
        const bool up = (i & k) == 0;   // ascending run
        const bool swap = up ? ga::ranks_before(skey[l], sidx[l], skey[i], sidx[i])
                             : ga::ranks_before(skey[i], sidx[i], skey[l], sidx[l]);
        if (swap) {
          const uint64_t tk = skey[i];
          skey[i] = skey[l];
          skey[l] = tk;
          const int ti = sidx[i];
          sidx[i] = sidx[l];
          sidx[l] = ti;
        }
      }
      __syncthreads();
    }
  if (order)
    for (int i = threadIdx.x; i < P; i += kPlanThreads) order[i] = sidx[i];
}

__global__ void __launch_bounds__(kPlanThreads)
ranking_order_kernel(int P, const double* __restrict__ fit, int* __restrict__ order) {
  extern __shared__ __align__(16) uint64_t skey[];
  ranking_sort_body(P, fit, skey, reinterpret_cast<int*>(skey + pow2_at_least(P)), order);
}

// cum[p + 1] = sum_{j<=p} roulette_weight(fit[j]), cum[0] = 0: each thread
// sums a contiguous chunk, an exclusive scan of the chunk sums gives its
// offset (integers, so the result does not depend on the order).
__device__ void roulette_cum_body(int P, const double* __restrict__ fit, uint64_t* cum) {
  __shared__ uint64_t wsum[kPlanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int chunk = (P + kPlanThreads - 1) / kPlanThreads;
  const int lo = min(P, tid * chunk), hi = min(P, lo + chunk);
  uint64_t s = 0;
  for (int p = lo; p < hi; ++p) s += ga::roulette_weight(fit[p]);
  uint64_t inc = s;   // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint64_t t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t v = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += v;
    }
    wsum[lane] = t;   // inclusive over warps
  }
  __syncthreads();
  uint64_t run = (wid > 0 ? wsum[wid - 1] : 0) + inc - s;
  for (int p = lo; p < hi; ++p) {
    run += ga::roulette_weight(fit[p]);
    cum[p + 1] = run;
  }
  if (tid == 0) cum[0] = 0;
}

__global__ void __launch_bounds__(kPlanThreads)
roulette_cum_kernel(int P, const double* __restrict__ fit, uint64_t* __restrict__ cum) {
  roulette_cum_body(P, fit, cum);
}

__global__ void __launch_bounds__(kPlanThreads)
ga_plan_kernel(GaDev g_, const double* __restrict__ fit, uint64_t seed, uint32_t g,
               int4* __restrict__ plan) {
  ga::plan_body(g_, fit, seed, g, plan);
}

__global__ void ga_breed_kernel(GaDev g_, const float* __restrict__ pop,
                                const int4* __restrict__ plan, uint64_t seed, uint32_t g,
                                float* __restrict__ next) {
  const int64_t n = (int64_t)g_.Nout * g_.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    next[e] = ga::breed_gene(g_, pop, plan, seed, g, e);
}

// Small populations (P, Nout <= kFusedMax, Nout K <= kFusedGenes): the
// selection table, the plan and every gene of the next population in one CTA
// and one launch instead of three or four, with the table and the plan in
// shared memory; the same device functions, so the same result bit for bit.
constexpr int kFusedMax = 1024;
constexpr int64_t kFusedGenes = 65536;

__host__ __device__ inline int fused_table_bytes(const GaDev& ga) {
  return ga.sel == GAME_SEL_RANKING    ? pow2_at_least(ga.P) * 12
         : ga.sel == GAME_SEL_ROULETTE ? (ga.P + 1) * 8
                                       : 0;
}

__global__ void __launch_bounds__(kPlanThreads)
ga_fused_kernel(GaDev g_, const float* __restrict__ pop, const double* __restrict__ fit,
                uint64_t seed, uint32_t g, float* __restrict__ next) {
  extern __shared__ __align__(16) uint64_t fsm[];
  GaDev ga = g_;
  const int tb = (fused_table_bytes(g_) + 15) & ~15;
  int4* plan = reinterpret_cast<int4*>(reinterpret_cast<char*>(fsm) + tb);
  if (ga.sel == GAME_SEL_RANKING) {
    int* sidx = reinterpret_cast<int*>(fsm + pow2_at_least(ga.P));
    ranking_sort_body(ga.P, fit, fsm, sidx, nullptr);
    ga.order = sidx;
  } else if (ga.sel == GAME_SEL_ROULETTE) {
    roulette_cum_body(ga.P, fit, fsm);
    ga.cum = fsm;
  }
  __syncthreads();
  ga::plan_body(ga, fit, seed, g, plan);
  __syncthreads();
  const int64_t n = (int64_t)ga.Nout * ga.K;
  for (int64_t e = threadIdx.x; e < n; e += kPlanThreads)
    next[e] = ga::breed_gene(ga, pop, plan, seed, g, e);
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

static int ranking_smem_bytes(int P) {
  int n2 = 1;
  while (n2 < P) n2 <<= 1;
  return n2 * (int)(sizeof(uint64_t) + sizeof(int));
}

cudaError_t launch_generation(const GaDev& ga, const float* pop, const double* fit,
                              uint64_t seed, uint32_t g, int4* plan, float* next,
                              cudaStream_t st) {
  if (ga.E > kMaxElites) return cudaErrorInvalidValue;
  if (ga.P <= kFusedMax && ga.Nout <= kFusedMax && (int64_t)ga.Nout * ga.K <= kFusedGenes) {
    const int smem = ((fused_table_bytes(ga) + 15) & ~15) + ga.Nout * (int)sizeof(int4);
    ga_fused_kernel<<<1, kPlanThreads, smem, st>>>(ga, pop, fit, seed, g, next);
    return cudaGetLastError();
  }
  if (ga.sel == GAME_SEL_RANKING) {
    if (ga.P > kMaxRankingP || !ga.order) return cudaErrorInvalidValue;
    const int smem = ranking_smem_bytes(ga.P);
    if (smem > 48 * 1024) {
      const cudaError_t e =
          cudaFuncSetAttribute(ranking_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    ranking_order_kernel<<<1, kPlanThreads, smem, st>>>(ga.P, fit, ga.order);
  } else if (ga.sel == GAME_SEL_ROULETTE) {
    if (!ga.cum) return cudaErrorInvalidValue;
    roulette_cum_kernel<<<1, kPlanThreads, 0, st>>>(ga.P, fit, ga.cum);
  }
  ga_plan_kernel<<<1, kPlanThreads, 0, st>>>(ga, fit, seed, g, plan);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ga_breed_kernel<<<blocks_for((int64_t)ga.Nout * ga.K, 256), 256, 0, st>>>(ga, pop, plan, seed,
                                                                        g, next);
  return cudaGetLastError();
}

}  // namespace game
