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
  ga_breed_kernel<<<blocks_for((int64_t)ga.Nout * ga.K, 256), 256, 0, st>>>(ga, pop, plan, seed,
                                                                        g, next);
  return cudaGetLastError();
}

}  // namespace game
