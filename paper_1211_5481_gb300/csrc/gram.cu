// gram.cu -- the Gram form of the MSE fitness (FP64).
//
// With phi~(x) = (1, phi_1(x), ..., phi_{K-1}(x)) the expansion of Eq. 1 /
// Eq. 6 with a leading 1 for the bias gene, the output of Eq. 2 is
// Out_p(m) = a_p . phi~(x_m), so the MSE of Eq. 3 is a quadratic form:
//   fit_p = (yy - 2 a_p . b + a_p^T G a_p) / M,
//   G = sum_m phi~(x_m) phi~(x_m)^T [K][K], b = sum_m y_m phi~(x_m), yy = sum_m y_m^2.
// G, b and yy depend only on the training set: they are accumulated once per
// handle (FP64 expansion -- the Chebyshev recurrence, or sin / cos of x and
// the angle recurrence -- and FP64 sums), after which a generation costs
// P K^2 FP64 multiply-adds instead of M P K. The subtraction cancels when the
// fit is good (fit << yy / M), which is why everything here is FP64.
//
// Shared genes (Eq. 2 as printed): the expansion is
// psi~(x) = (1, psi_1(x), ..., psi_{B d}(x)) with psi_{b,j}(x) =
// sum_i phi_{b,j}(x_i) (features in order), written by expand_tied_kernel;
// everything else is the same with K = B d + 1.
// The MSE is clamped at 0 against cancellation; RMSE is its square root.
//
// Accumulation: the patterns are taken in chunks of up to kChunk; a chunk's
// design matrix Phi [mc][K] (FP64) is written by expand_kernel, then
// gram_accum_kernel forms Phi^T Phi on the upper triangle (64 x 64 tiles,
// each thread a 4 x 4 block) over up to 32 row ranges of the chunk, each in
// row order, and gram_add_kernel adds the ranges' sums to G in range order;
// vec_accum_kernel / vec_add_kernel do the same for Phi^T y and y^T y over 64
// row ranges. Every sum runs in a fixed order (chunks in sequence, ranges
// in order, rows in order within a range), so G is reproducible.
// The quadratic forms: quad_kernel, one CTA per 8 chromosomes, thread t owns
// rows t, t + 256, ... of G a_p and reads G column-wise (G is symmetric, so
// G[k2][k1] over k2 is a coalesced column read), then a fixed-order CTA sum.
#include <math_constants.h>

#include "game_internal.cuh"

namespace game {

namespace {

constexpr int kGT = 64;        // G tile
constexpr int kQuadGroup = 8;  // chromosomes per quad CTA at most
constexpr int kVecSplits = 64; // row splits of a chunk's b and y.y sums

// Phi[r][k] for patterns m0 + r (r < mc), FP64; column 0 is 1.
__global__ void expand_kernel(int64_t m0, int mc, int N, int d, int basis, int K,
                              const float* __restrict__ Xt, double* __restrict__ Phi) {
  const int B = basis == GAME_BASIS_TRIG ? 2 : 1;
  const int64_t n = (int64_t)mc * N;   // one thread per (pattern, feature)
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / N), i = (int)(e % N);
    const int64_t m = m0 + r;
    const double x =
        (double)Xt[(m / kPatBlock) * (int64_t)N * kPatBlock + (int64_t)i * kPatBlock + m % kPatBlock];
    double* row = Phi + (int64_t)r * K;
    if (i == 0) row[0] = 1.0;
    const int64_t base = 1 + (int64_t)i * B * d;
    if (basis == GAME_BASIS_CHEB) {
      double tm = 1.0, t = x;
      for (int j = 1; j <= d; ++j) {
        row[base + j - 1] = t;
        const double tn = 2.0 * x * t - tm;
        tm = t;
        t = tn;
      }
    } else {
      double s1, c1;
      sincos(x, &s1, &c1);
      for (int bb = 0; bb < 2; ++bb) {
        double fm = bb ? 0.0 : 1.0, f = bb ? s1 : c1;
        for (int j = 1; j <= d; ++j) {
          row[base + bb * d + j - 1] = f;
          const double fn = 2.0 * c1 * f - fm;
          fm = f;
          f = fn;
        }
      }
    }
  }
}

// Psi[r][c] for patterns m0 + r with shared genes: column 0 is 1, column
// 1 + b d + (j - 1) the sum over features i = 0..N-1, in order, of
// phi_{b,j}(x_i); K = B d + 1.
__global__ void expand_tied_kernel(int64_t m0, int mc, int N, int d, int basis, int K,
                                   const float* __restrict__ Xt, double* __restrict__ Phi) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < mc; r += gridDim.x * blockDim.x) {
    const int64_t m = m0 + r;
    double* row = Phi + (int64_t)r * K;
    row[0] = 1.0;
    for (int c = 1; c < K; ++c) row[c] = 0.0;
    for (int i = 0; i < N; ++i) {
      const double x = (double)Xt[(m / kPatBlock) * (int64_t)N * kPatBlock +
                                  (int64_t)i * kPatBlock + m % kPatBlock];
      if (basis == GAME_BASIS_CHEB) {
        double tm = 1.0, t = x;
        for (int j = 1; j <= d; ++j) {
          row[j] += t;
          const double tn = 2.0 * x * t - tm;
          tm = t;
          t = tn;
        }
      } else {
        double s1, c1;
        sincos(x, &s1, &c1);
        for (int bb = 0; bb < 2; ++bb) {
          double fm = bb ? 0.0 : 1.0, f = bb ? s1 : c1;
          for (int j = 1; j <= d; ++j) {
            row[1 + bb * d + j - 1] += f;
            const double fn = 2.0 * c1 * f - fm;
            fm = f;
            f = fn;
          }
        }
      }
    }
  }
}

// The fitness from the Gram-form MSE, clamped at 0 (cancellation can leave
// an exact fit a few ulps below zero): itself, or its square root for
// GAME_ERR_RMSE.
__device__ __forceinline__ double finish_error(double mse, int err) {
  const double m = fmax(mse, 0.0);
  return err == GAME_ERR_RMSE ? sqrt(m) : m;
}

// part[z][k1][k2] = sum over rows r of split z of Phi[r][k1] Phi[r][k2], for
// the tile (blockIdx.y, blockIdx.x) of the upper triangle (tiles with
// ti > tj skip); split z = blockIdx.z takes rows [z rs, (z + 1) rs).
__global__ void __launch_bounds__(256)
gram_accum_kernel(int mc, int rs, int K, const double* __restrict__ Phi,
                  double* __restrict__ part) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  const int rlo = blockIdx.z * rs, rhi = min(mc, rlo + rs);
  __shared__ double Ps[16][2 * kGT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k10 = ti * kGT, k20 = tj * kGT;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int r0 = rlo; r0 < rhi; r0 += 16) {
    for (int e = threadIdx.x; e < 16 * 2 * kGT; e += 256) {
      const int rr = e / (2 * kGT), c = e % (2 * kGT);
      const int k = c < kGT ? k10 + c : k20 + (c - kGT);
      Ps[rr][c] = (r0 + rr < rhi && k < K) ? Phi[(int64_t)(r0 + rr) * K + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 16; ++rr) {
      double a[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ps[rr][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = Ps[rr][kGT + tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* Pz = part + (int64_t)blockIdx.z * K * K;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int k1 = k10 + ty + 16 * u, k2 = k20 + tx + 16 * v;
      if (k1 < K && k2 < K && k1 <= k2) Pz[(int64_t)k1 * K + k2] = acc[u][v];
    }
}

// G[k1][k2] += sum over the splits, in order, of part[z][k1][k2] (upper triangle).
__global__ void gram_add_kernel(int K, int splits, const double* __restrict__ part,
                                double* __restrict__ G) {
  const int64_t n = (int64_t)K * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(e / K), k2 = (int)(e % K);
    if (k1 > k2) continue;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[z * n + e];
    G[e] += s;
  }
}

// vpart[z][k] = sum over the rows r of split z (in order) of Phi[r][k] y[m0 + r]
// for k < K, and vpart[z][K] = sum of y[m0 + r]^2; split z = blockIdx.y
// takes rows [z rs, (z + 1) rs). Threads of a block read consecutive
// columns of a row (coalesced).
__global__ void vec_accum_kernel(int64_t m0, int mc, int rs, int K, const double* __restrict__ Phi,
                                 const float* __restrict__ y, double* __restrict__ vpart) {
  const int rlo = blockIdx.y * rs, rhi = min(mc, rlo + rs);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    if (k < K) {
      for (int r = rlo; r < rhi; ++r) s = fma(Phi[(int64_t)r * K + k], (double)y[m0 + r], s);
    } else {
      for (int r = rlo; r < rhi; ++r) {
        const double v = y[m0 + r];
        s = fma(v, v, s);
      }
    }
    vpart[(int64_t)blockIdx.y * (K + 1) + k] = s;
  }
}

// b[k] += sum over the splits, in order, of vpart[z][k]; yy likewise from column K.
__global__ void vec_add_kernel(int K, int splits, const double* __restrict__ vpart,
                               double* __restrict__ b, double* __restrict__ yy) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += vpart[(int64_t)z * (K + 1) + k];
  if (k < K) b[k] += s;
  else *yy += s;
}

// Lower triangle from the upper one.
__global__ void mirror_kernel(int K, double* __restrict__ G) {
  const int64_t n = (int64_t)K * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(e / K), k2 = (int)(e % K);
    if (k1 > k2) G[e] = G[(int64_t)k2 * K + k1];
  }
}

// fit_p = (yy - 2 a_p . b + a_p^T G a_p) / M for grp <= 8 chromosomes per CTA;
// with idx, entry p is chromosome idx[p] (read from pop row idx[p], written to
// fit[idx[p]]).
__global__ void __launch_bounds__(256)
quad_kernel(int P, int K, int64_t M, int grp, int err, const float* __restrict__ pop,
            const int* __restrict__ idx, const double* __restrict__ G,
            const double* __restrict__ b, const double* __restrict__ yy,
            double* __restrict__ fit) {
  extern __shared__ double as[];   // [8][K] genes of the group, FP64 (rows >= grp zero)
  __shared__ double red[kQuadGroup][8];
  const int p0 = blockIdx.x * grp;
  const int ng = min(grp, P - p0);
  for (int e = threadIdx.x; e < grp * K; e += 256) {
    const int q = e / K, k = e % K;
    const int64_t row = q < ng ? (idx ? idx[p0 + q] : p0 + q) : 0;
    as[e] = q < ng ? (double)pop[row * K + k] : 0.0;
  }
  __syncthreads();
  double quad[kQuadGroup], lin[kQuadGroup];
#pragma unroll
  for (int q = 0; q < kQuadGroup; ++q) {
    quad[q] = 0.0;
    lin[q] = 0.0;
  }
  for (int k1 = threadIdx.x; k1 < K; k1 += 256) {
    double ga[kQuadGroup];
#pragma unroll
    for (int q = 0; q < kQuadGroup; ++q) ga[q] = 0.0;
    for (int k2 = 0; k2 < K; ++k2) {
      const double g = G[(int64_t)k2 * K + k1];   // = G[k1][k2]
#pragma unroll
      for (int q = 0; q < kQuadGroup; ++q)
        if (q < grp) ga[q] = fma(g, as[q * K + k2], ga[q]);
    }
    const double bk = b[k1];
#pragma unroll
    for (int q = 0; q < kQuadGroup; ++q)
      if (q < grp) {
        quad[q] = fma(as[q * K + k1], ga[q], quad[q]);
        lin[q] = fma(as[q * K + k1], bk, lin[q]);
      }
  }
  // fixed-order CTA sums: lanes by xor-butterfly, then the 8 warps in order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kQuadGroup; ++q) {
    double v = quad[q] - 2.0 * lin[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < ng) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    const int p = p0 + threadIdx.x;
    fit[idx ? idx[p] : p] = finish_error((*yy + s) / (double)M, err);
  }
}

// Few chromosomes (n <= kMaxRescore; the elite re-scoring): the K x K
// products are spread over the whole GPU. CTA (bx, by) owns rows
// k1 in [128 bx, 128 bx + 128) (one per thread) and the k2-range
// [by ks, (by + 1) ks) of sum_k2 G[k1][k2] a_q[k2] (G read column-wise, as
// G[k2][k1]); each thread forms a_q[k1] h_q (and, in split 0,
// -2 a_q[k1] b[k1]); the CTA's sum per candidate (lanes by xor-butterfly,
// warps in order) goes to part[by][bx][q]. quad_small_finish adds the parts
// in order and writes fit[idx[q]] = (yy + sum) / M.
constexpr int kSmallRows = 128;
__global__ void __launch_bounds__(kSmallRows)
quad_small_kernel(int n, int K, int ks, const float* __restrict__ pop, const int* __restrict__ idx,
                  const double* __restrict__ G, const double* __restrict__ b,
                  double* __restrict__ part) {
  extern __shared__ double av[];   // [n][ks] genes of the k2-range
  __shared__ double red[kMaxRescore][kSmallRows / 32];
  const int k1 = blockIdx.x * kSmallRows + threadIdx.x;
  const int k2lo = blockIdx.y * ks, k2hi = min(K, k2lo + ks);
  const int len = k2hi - k2lo;
  for (int e = threadIdx.x; e < n * ks; e += kSmallRows) {
    const int q = e / ks, c = e % ks;
    av[e] = c < len ? (double)pop[(int64_t)idx[q] * K + k2lo + c] : 0.0;
  }
  __syncthreads();
  double h[kMaxRescore];
#pragma unroll
  for (int q = 0; q < kMaxRescore; ++q) h[q] = 0.0;
  if (k1 < K) {
    for (int c = 0; c < len; ++c) {
      const double g = G[(int64_t)(k2lo + c) * K + k1];
#pragma unroll
      for (int q = 0; q < kMaxRescore; ++q)
        if (q < n) h[q] = fma(g, av[q * ks + c], h[q]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kMaxRescore; ++q) {
    if (q >= n) break;
    double v = 0.0;
    if (k1 < K) {
      const double ak = pop[(int64_t)idx[q] * K + k1];
      v = ak * h[q];
      if (blockIdx.y == 0) v -= 2.0 * ak * b[k1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double sum = 0.0;
    for (int w = 0; w < kSmallRows / 32; ++w) sum += red[threadIdx.x][w];
    part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * n + threadIdx.x] = sum;
  }
}

// One warp per candidate q: lane l adds parts l, l + 32, ... in order, then
// a fixed xor-butterfly.
__global__ void quad_small_finish(int n, int nparts, int64_t M, int err,
                                  const int* __restrict__ idx,
                                  const double* __restrict__ part, const double* __restrict__ yy,
                                  double* __restrict__ fit) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= n) return;
  double s = 0.0;
  for (int j = lane; j < nparts; j += 32) s += part[(int64_t)j * n + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) fit[idx[q]] = finish_error((*yy + s) / (double)M, err);
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 16384) b = 16384;
  return (int)b;
}

}  // namespace

// Row splits of a chunk's G accumulation: about three CTAs per SM over the
// upper-triangle tiles, at most 32, and at most 1 GB of partial sums.
int gram_splits(const Shape& s, int num_sms) {
  const int KT = (s.K + kGT - 1) / kGT;
  const int tiles = KT * (KT + 1) / 2;
  int z = (3 * num_sms + tiles - 1) / tiles;
  const int64_t cap = ((int64_t)1 << 30) / ((int64_t)s.K * s.K * 8);
  if (z > cap) z = (int)cap;
  if (z > 32) z = 32;
  if (z < 1) z = 1;
  return z;
}

int64_t gram_part_doubles(const Shape& s, int num_sms) {
  const int64_t g = (int64_t)gram_splits(s, num_sms) * s.K * s.K;
  const int64_t v = (int64_t)kVecSplits * (s.K + 1);
  return g > v ? g : v;
}

int64_t gram_chunk_rows(const Shape& s) {
  // Phi chunk of at most 64k patterns and at most 256 MB
  int64_t rows = (int64_t)(256ll * 1024 * 1024) / ((int64_t)s.K * 8);
  if (rows > 65536) rows = 65536;
  if (rows < 16) rows = 16;
  return rows;
}

cudaError_t launch_gram_build(const Shape& s, const float* Xt, const float* y, double* G,
                              double* b, double* yy, double* phi_chunk, double* part,
                              int num_sms, cudaStream_t st) {
  const int K = s.K;
  cudaError_t e = cudaMemsetAsync(G, 0, (size_t)K * K * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, (size_t)K * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(yy, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int64_t CH = gram_chunk_rows(s);
  const int KT = (K + kGT - 1) / kGT;
  for (int64_t m0 = 0; m0 < s.M; m0 += CH) {
    const int mc = (int)(s.M - m0 < CH ? s.M - m0 : CH);
    if (s.tied)
      expand_tied_kernel<<<blocks_for(mc), 256, 0, st>>>(m0, mc, s.N, s.d, s.basis, K, Xt,
                                                         phi_chunk);
    else
      expand_kernel<<<blocks_for((int64_t)mc * s.N), 256, 0, st>>>(m0, mc, s.N, s.d, s.basis,
                                                                  K, Xt, phi_chunk);
    const int zs = gram_splits(s, num_sms);
    const int rs = (mc + zs - 1) / zs;
    gram_accum_kernel<<<dim3(KT, KT, zs), 256, 0, st>>>(mc, rs, K, phi_chunk, part);
    gram_add_kernel<<<blocks_for((int64_t)K * K), 256, 0, st>>>(K, zs, part, G);
    const int vrs = (mc + kVecSplits - 1) / kVecSplits;
    vec_accum_kernel<<<dim3((K + 256) / 256, kVecSplits), 256, 0, st>>>(m0, mc, vrs, K, phi_chunk,
                                                                         y, part);
    vec_add_kernel<<<(K + 256) / 256, 256, 0, st>>>(K, kVecSplits, part, b, yy);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  mirror_kernel<<<blocks_for((int64_t)K * K), 256, 0, st>>>(K, G);
  return cudaGetLastError();
}

int gram_small_parts(const Shape& s) {
  const int bx = (s.K + kSmallRows - 1) / kSmallRows;
  int by = (304 + bx - 1) / bx;   // about two CTAs per SM over the grid
  if (by > s.K) by = s.K;
  return bx * by;
}

cudaError_t launch_gram_rescore(const Shape& s, const float* pop, int n, const int* idx,
                                const double* G, const double* b, const double* yy,
                                double* part, double* fit, int err, cudaStream_t st) {
  if (n < 1 || n > kMaxRescore) return cudaErrorInvalidValue;
  const int bx = (s.K + kSmallRows - 1) / kSmallRows;
  const int by = gram_small_parts(s) / bx;
  const int ks = (s.K + by - 1) / by;
  const size_t smem = (size_t)n * ks * sizeof(double);   // <= 16 x 410 x 8 at K = 4097
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        quad_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  quad_small_kernel<<<dim3(bx, by), kSmallRows, smem, st>>>(n, s.K, ks, pop, idx, G, b, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  quad_small_finish<<<1, 32 * n, 0, st>>>(n, bx * by, s.M, err, idx, part, yy, fit);
  return cudaGetLastError();
}

cudaError_t launch_gram_fitness(const Shape& s, const float* pop, int P, const int* idx,
                                const double* G, const double* b, const double* yy,
                                double* fit, int err, cudaStream_t st) {
  // as many chromosomes per CTA (<= 8) as fit in 200 KB of FP64 genes
  int grp = (int)((200 * 1024) / ((size_t)s.K * sizeof(double)));
  if (grp > kQuadGroup) grp = kQuadGroup;
  if (grp < 1) grp = 1;
  const size_t smem = (size_t)grp * s.K * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(quad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e != cudaSuccess) return e;
  quad_kernel<<<(P + grp - 1) / grp, 256, smem, st>>>(P, s.K, s.M, grp, err, pop, idx, G, b,
                                                       yy, fit);
  return cudaGetLastError();
}

}  // namespace game
