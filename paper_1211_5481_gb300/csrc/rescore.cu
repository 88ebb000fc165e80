// rescore.cu -- elite re-scoring: the n best chromosomes of a reduced-precision
// fitness vector are evaluated again with FP32 products and an FP64 sum of
// squared residuals, and their entries of the vector are replaced, so that
// elitism and the tournaments rank the best candidates by accurate values.
//
// Fitness is the MSE of Eq. 3 (paper Section 3; Section 5 fixes MSE):
//   fit_p = (1/M) sum_m (y_m - a_{p,0} - sum_c a_{p,c+1} phi_c(x_m))^2.
// Per pattern the expansion phi is stepped by the same FP32 recurrences as
// the CUDA-core form (T_{j+1} = 2x T_j - T_{j-1}; cos/sin of jx from one
// sincosf and the angle recurrence), the gene sums are FP32 FMAs in gene
// order and the residual is FP32; each thread adds the squares of its 4
// patterns of a step in FP32 and accumulates those sums in FP64.
//
// Candidates: the n best by (fit, index), NaN as +infinity (select_top_kernel,
// one CTA: each thread keeps the top 16 of its strided elements in registers,
// each warp merges its lanes' lists, warp 0 merges the 8 warps'). Evaluation:
// groups of 8 candidates (blockIdx.y) over pattern slices (blockIdx.x); each
// thread computes an 8-candidate x 4-pattern block of outputs, the genes of
// each column broadcast from shared memory and the expansion of its 4
// patterns stepped in registers. The CTA's FP64 sums go to part[group][blockIdx.x][8];
// the last CTA of a group to finish (an atomic ticket) adds the rows in a fixed
// order and writes fit[cand] = sum / M, so the result does not depend on the
// order in which CTAs finish.
#include <math_constants.h>

#include "game_internal.cuh"

namespace game {

namespace {

constexpr int kSelThreads = 256;
constexpr int kGroup = 8;       // candidates per evaluation group
constexpr int kEvalThreads = 256;

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

// acc[k][q] += g_q * phi[k] for one contraction column: the 8 candidates'
// genes (two broadcast 16-byte shared-memory loads) times the thread's kPT
// expansion values.
template <int kPT>
__device__ __forceinline__ void column8(float (&acc)[kPT][kGroup], const float4* gp,
                                        const float (&phi)[kPT]) {
  const float4 ga = gp[0], gb = gp[1];
  const float g[kGroup] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
#pragma unroll
  for (int k = 0; k < kPT; ++k)
#pragma unroll
    for (int q = 0; q < kGroup; ++q) acc[k][q] = fmaf(g[q], phi[k], acc[k][q]);
}

// kPT patterns per thread per step (the launcher picks kPT so that the
// steps fill whole waves of resident CTAs).
template <int kPT>
__global__ void __launch_bounds__(kEvalThreads, 3)
rescore_kernel(int64_t M, int N, int d, int basis, int Kp, const float* __restrict__ Xt,
               const float* __restrict__ y, const float* __restrict__ pop, int K,
               const int* __restrict__ cand, int n, double* __restrict__ part,
               unsigned int* __restrict__ tickets, double* __restrict__ fit) {
  extern __shared__ __align__(16) float gs[];     // [Kp][8] genes 1..K-1 of the group
  __shared__ float a0s[kGroup];
  __shared__ double ssum[kGroup][kEvalThreads];   // per-thread FP64 sums
  __shared__ double wsum[kEvalThreads / 32][kGroup];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = blockIdx.y;
  const int nin = min(kGroup, n - grp * kGroup);

  for (int e = tid; e < Kp * kGroup; e += kEvalThreads) {
    const int c = e / kGroup, q = e % kGroup;
    gs[e] = q < nin ? pop[(int64_t)cand[grp * kGroup + q] * K + 1 + c] : 0.f;
  }
  if (tid < kGroup) a0s[tid] = tid < nin ? pop[(int64_t)cand[grp * kGroup + tid] * K] : 0.f;
#pragma unroll
  for (int q = 0; q < kGroup; ++q) ssum[q][tid] = 0.0;
  __syncthreads();

  // A step covers kPT * 256 patterns: thread tid takes base + k*256 + tid.
  // base is a multiple of 256, so the thread's patterns sit at the same row
  // of X blocks 2k apart.
  const int64_t span = (int64_t)kPT * kEvalThreads;
  const int64_t stride = (int64_t)gridDim.x * span;
  const int64_t blk = (int64_t)N * kPatBlock;   // floats per block of 128 patterns
  const float4* g4 = reinterpret_cast<const float4*>(gs);
  for (int64_t base = (int64_t)blockIdx.x * span; base < M; base += stride) {
    const int64_t m0 = base + tid;
    const float* xp = Xt + ((uint64_t)m0 / kPatBlock) * blk + ((uint64_t)m0 % kPatBlock);
    bool ok[kPT];
    float yk[kPT], xn[kPT];
#pragma unroll
    for (int k = 0; k < kPT; ++k) {
      ok[k] = m0 + k * kEvalThreads < M;
      yk[k] = ok[k] ? __ldg(y + m0 + k * kEvalThreads) : 0.f;
      xn[k] = ok[k] ? __ldg(xp + 2 * k * blk) : 0.f;
    }
    float acc[kPT][kGroup];
#pragma unroll
    for (int k = 0; k < kPT; ++k)
#pragma unroll
      for (int q = 0; q < kGroup; ++q) acc[k][q] = 0.f;

    const float4* gp = g4;
    for (int i = 0; i < N; ++i) {
      float x[kPT];
#pragma unroll
      for (int k = 0; k < kPT; ++k) {
        x[k] = xn[k];
        // the next feature's values, one feature ahead
        if (i + 1 < N) xn[k] = ok[k] ? __ldg(xp + 2 * k * blk + (i + 1) * kPatBlock) : 0.f;
      }
      if (basis == GAME_BASIS_CHEB) {
        // T_{j+1} = 2x T_j - T_{j-1}; two degrees per trip, the two state
        // registers taking turns as T_j and T_{j-1}
        float u[kPT], v[kPT], x2[kPT];   // u = T_{j-1}, v = T_j on entry
#pragma unroll
        for (int k = 0; k < kPT; ++k) {
          u[k] = 1.f;
          v[k] = x[k];
          x2[k] = x[k] + x[k];
        }
        int j = 1;
        for (; j < d; j += 2, gp += 4) {
          column8(acc, gp, v);
#pragma unroll
          for (int k = 0; k < kPT; ++k) u[k] = fmaf(x2[k], v[k], -u[k]);
          column8(acc, gp + 2, u);
#pragma unroll
          for (int k = 0; k < kPT; ++k) v[k] = fmaf(x2[k], u[k], -v[k]);
        }
        if (j == d) {
          column8(acc, gp, v);
          gp += 2;
        }
      } else {
        // cos(jx) and sin(jx) by f_{j+1} = 2 cos(x) f_j - f_{j-1}
        float sx[kPT], cx[kPT], c2[kPT];
#pragma unroll
        for (int k = 0; k < kPT; ++k) {
          sincosf(x[k], &sx[k], &cx[k]);
          c2[k] = cx[k] + cx[k];
        }
#pragma unroll 1
        for (int b = 0; b < 2; ++b) {
          float u[kPT], v[kPT];
#pragma unroll
          for (int k = 0; k < kPT; ++k) {
            u[k] = b ? 0.f : 1.f;
            v[k] = b ? sx[k] : cx[k];
          }
          int j = 1;
          for (; j < d; j += 2, gp += 4) {
            column8(acc, gp, v);
#pragma unroll
            for (int k = 0; k < kPT; ++k) u[k] = fmaf(c2[k], v[k], -u[k]);
            column8(acc, gp + 2, u);
#pragma unroll
            for (int k = 0; k < kPT; ++k) v[k] = fmaf(c2[k], u[k], -v[k]);
          }
          if (j == d) {
            column8(acc, gp, v);
            gp += 2;
          }
        }
      }
    }
    // residuals in FP32, the step's squares summed in FP32 (4 patterns per
    // chromosome), then accumulated in FP64
#pragma unroll
    for (int q = 0; q < kGroup; ++q) {
      const float a0 = a0s[q];
      float sq = 0.f;
#pragma unroll
      for (int k = 0; k < kPT; ++k) {
        const float r = ok[k] ? (yk[k] - a0) - acc[k][q] : 0.f;
        sq = fmaf(r, r, sq);
      }
      ssum[q][tid] += (double)sq;
    }
  }
  double sse[kGroup];
#pragma unroll
  for (int q = 0; q < kGroup; ++q) sse[q] = ssum[q][tid];
  (void)Kp;

  // CTA sum in a fixed order: lanes by xor-butterfly, then warps in order
#pragma unroll
  for (int q = 0; q < kGroup; ++q) {
    double s = sse[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[warp][q] = s;
  }
  __syncthreads();
  double* prow = part + ((int64_t)grp * gridDim.x + blockIdx.x) * kGroup;
  if (tid < kGroup) {
    double s = 0.0;
    for (int w = 0; w < kEvalThreads / 32; ++w) s += wsum[w][tid];
    prow[tid] = s;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned int t = atomicAdd(&tickets[grp], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  if (tid < nin) {
    __threadfence();
    const double* col0 = part + (int64_t)grp * gridDim.x * kGroup + tid;
    double s = 0.0;
    for (unsigned int r = 0; r < gridDim.x; ++r) s += __ldcg(col0 + (int64_t)r * kGroup);
    fit[cand[grp * kGroup + tid]] = s / (double)M;
  }
  if (tid == 0) tickets[grp] = 0u;   // ready for the next launch
}

}  // namespace

typedef void (*RescoreFn)(int64_t, int, int, int, int, const float*, const float*,
                          const float*, int, const int*, int, double*, unsigned int*, double*);
constexpr int kNumPT = 4;
const RescoreFn kRescoreFns[kNumPT] = {rescore_kernel<1>, rescore_kernel<2>, rescore_kernel<3>,
                                       rescore_kernel<4>};

// Resident CTAs per SM of the kPT variant for this shape; also lets it take
// the genes of the longest chromosome in dynamic shared memory.
static int rescore_per_sm(int pt, const Shape& s) {
  int per_sm = 0;
  const RescoreFn fn = kRescoreFns[pt - 1];
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kMaxK * kGroup * sizeof(float))) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEvalThreads,
                                                    rescore_smem_bytes(s)) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm;
}

// Patterns per thread and grid: every CTA is resident at once; the fewest
// waves of steps win, then the largest kPT. (Measured on the 10^6-pattern
// classification set: a step's time hardly depends on kPT; kPT = 4 and
// kPT = 3 both take 3 waves there, and kPT = 4 was the faster.)
RescorePlan plan_rescore(const Shape& s, int num_sms) {
  RescorePlan best{4, 1};
  double best_cost = 1e300;
  for (int pt = kNumPT; pt >= 1; --pt) {
    const int64_t slots = (int64_t)rescore_per_sm(pt, s) * num_sms;
    const int64_t steps = (s.M + (int64_t)pt * kEvalThreads - 1) / ((int64_t)pt * kEvalThreads);
    const int64_t grid = steps < slots ? steps : slots;
    const int64_t waves = (steps + grid - 1) / grid;
    const double cost = (double)waves;
    if (cost < best_cost) {
      best_cost = cost;
      best = {pt, (int)grid};
    }
  }
  return best;
}

size_t rescore_smem_bytes(const Shape& s) { return (size_t)s.Kp * kGroup * sizeof(float); }




cudaError_t launch_rescore(const RescorePlan& pl, const Shape& s, const float* Xt,
                           const float* y,
                           const float* pop, int P, int n, double* fit, int* cand,
                           double* part, unsigned int* tickets, cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  if (n > kMaxRescore || n > P) return cudaErrorInvalidValue;
  select_top_kernel<<<1, kSelThreads, 0, st>>>(fit, P, n, cand);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (pl.pt < 1 || pl.pt > kNumPT) return cudaErrorInvalidValue;
  dim3 grid(pl.grid, (n + kGroup - 1) / kGroup);
  kRescoreFns[pl.pt - 1]<<<grid, kEvalThreads, rescore_smem_bytes(s), st>>>(
      s.M, s.N, s.d, s.basis, s.Kp, Xt, y, pop, s.K, cand, n, part, tickets, fit);
  return cudaGetLastError();
}

}  // namespace game
