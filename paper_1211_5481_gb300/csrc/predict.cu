// predict.cu -- outputs of one chromosome (Eq. 2) on a set of patterns in
// FP64, and the binary classification counts behind the accuracy,
// completeness and contamination that Section 5 reports.
//
// One thread per pattern, grid-strided: the expansion by the FP64
// recurrences (Chebyshev T_{j+1} = 2 x T_j - T_{j-1}; trigonometric
// cos / sin (j x) by the angle-addition recurrence from sincos(x)), the
// genes held in shared memory as FP64, the sum taken in gene order. With
// shared genes (tied) every feature reads genes 1 + b d + (j - 1).
// Classification: positive target when y > threshold, positive prediction
// when Out > threshold; per-thread counts, a warp sum, then one 64-bit
// integer atomic per warp and count (integer sums: the result does not
// depend on the order).
#include "game_internal.cuh"

namespace game {

namespace {

constexpr int kThreads = 256;

template <bool TILED>
__device__ __forceinline__ double feature(const float* __restrict__ X, int64_t m, int N, int i) {
  return TILED ? (double)X[(m / kPatBlock) * (int64_t)N * kPatBlock + (int64_t)i * kPatBlock +
                           m % kPatBlock]
               : (double)X[m * N + i];
}

template <bool TILED>
__global__ void __launch_bounds__(kThreads)
predict_kernel(int64_t M, int N, int d, int basis, int tied, int Kg,
               const float* __restrict__ X, const float* __restrict__ chrom,
               const float* __restrict__ y, double threshold, double* __restrict__ out,
               unsigned long long* __restrict__ counts) {
  extern __shared__ double ga[];   // [Kg] genes
  for (int k = threadIdx.x; k < Kg; k += kThreads) ga[k] = (double)chrom[k];
  __syncthreads();
  const int B = basis == GAME_BASIS_TRIG ? 2 : 1;
  unsigned long long c[4] = {0, 0, 0, 0};   // TP, FP, TN, FN
  for (int64_t m = blockIdx.x * (int64_t)kThreads + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * kThreads) {
    double o = ga[0];
    for (int i = 0; i < N; ++i) {
      const double x = feature<TILED>(X, m, N, i);
      const double* g = ga + 1 + (tied ? 0 : i * B * d);
      if (basis == GAME_BASIS_CHEB) {
        double tm = 1.0, t = x;
        for (int j = 1; j <= d; ++j) {
          o = fma(g[j - 1], t, o);
          const double tn = 2.0 * x * t - tm;
          tm = t;
          t = tn;
        }
      } else {
        double s1, c1;
        sincos(x, &s1, &c1);
        double cj = c1, sj = s1;   // cos(j x), sin(j x)
        for (int j = 1; j <= d; ++j) {
          o = fma(g[j - 1], cj, o);
          o = fma(g[d + j - 1], sj, o);
          const double cn = cj * c1 - sj * s1, sn = sj * c1 + cj * s1;
          cj = cn;
          sj = sn;
        }
      }
    }
    if (out) out[m] = o;
    if (counts) {
      const bool act = (double)y[m] > threshold, pred = o > threshold;
      c[pred ? (act ? 0 : 1) : (act ? 3 : 2)] += 1;
    }
  }
  if (counts) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned long long v = c[q];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(counts + q, v);
    }
  }
}

}  // namespace

cudaError_t launch_predict(const Shape& s, int tied, int Kg, const float* X, bool tiled,
                           int64_t M, const float* chrom, const float* y, double threshold,
                           double* out, unsigned long long* counts, int num_sms,
                           cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  int64_t blocks = (M + kThreads - 1) / kThreads;
  if (blocks > 8 * (int64_t)num_sms) blocks = 8 * (int64_t)num_sms;
  const size_t smem = (size_t)Kg * sizeof(double);   // <= 32 KB (Kg <= 4097)
  if (tiled)
    predict_kernel<true><<<(int)blocks, kThreads, smem, st>>>(M, s.N, s.d, s.basis, tied, Kg, X,
                                                               chrom, y, threshold, out, counts);
  else
    predict_kernel<false><<<(int)blocks, kThreads, smem, st>>>(M, s.N, s.d, s.basis, tied, Kg,
                                                                X, chrom, y, threshold, out,
                                                                counts);
  return cudaGetLastError();
}

}  // namespace game
