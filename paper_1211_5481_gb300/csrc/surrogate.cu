// surrogate.cu -- a small MLP that predicts a chromosome's fitness, trained
// online on the (chromosome, exact fitness) pairs the GA produces, and used to
// screen oversampled offspring so that only the most promising get the exact
// fitness of paper Section 3 (Eq. 2, Eq. 3).
//
// Network: x in R^K (the genes) -> 256 -> 256 -> 1. Layers 1 and 2 take BF16
// operands (inputs, weights and the layer-1 activations rounded to BF16) with
// FP32 accumulation; the output layer is FP32. Activation: GELU in its tanh
// form, g(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))), c = sqrt(2/pi). Target:
// the log-fitness l = log(max(fit, 1e-30)) standardised over the training
// batch, t = (l - mean l) / sd l (FP64 statistics; sd 0 counts as 1): the
// MSE spans orders of magnitude and only the ranking of the prediction is
// used. Loss: mean of (out - t)^2 over the batch. Optimiser: Adam (lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-8) on FP32
// master weights. Initial weights uniform in +-1/sqrt(fan_in) from
// Philox4x32-10 (key = seed, counter = (layer, index, 0, tag 9)), biases 0.
//
// Parameter vector (FP32, this order): W1 [256][K], b1 [256], W2 [256][256],
// b2 [256], w3 [256], b3 [1].
//
// Kernels: one tiled GEMM with strides (C = A B with any transposition,
// FP32 accumulation, optional BF16 rounding of either operand on load, an
// optional bias + GELU epilogue), column sums in a fixed order, the GELU
// derivative, the output layer, and Adam. Screening: a one-CTA bitonic sort
// of (prediction, slot) keys, a flag per kept slot and a prefix-sum
// compaction that assembles the next population in slot order. The exact
// fitness checks the surrogate: after each screened generation the Pearson
// correlation r of the kept children's predictions with their exact
// log-fitness is measured, and the next screening trusts the surrogate only
// if r > 0.25; otherwise it keeps the first P - E children, i.e. exactly the
// children of the unscreened generation.
#include <cuda_bf16.h>

#include "game_internal.cuh"
#include "philox.cuh"

namespace game {

namespace {

constexpr int kH = kSurrogateHidden;
constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float round_bf16(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float gelu(float z) {
  const float u = kGeluC * (z + kGeluA * z * z * z);
  return 0.5f * z * (1.f + tanhf(u));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float u = kGeluC * (z + kGeluA * z * z * z);
  const float t = tanhf(u);
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluC * (1.f + 3.f * kGeluA * z * z);
}

// C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m * am + k * ak], B(k, n) =
// B[k * bk + n * bn]; FP32 accumulation in k order per thread. 128 x 128
// tiles, 256 threads, 8 x 8 outputs per thread, k-chunks of 16 through shared
// memory; each operand tile is loaded with consecutive threads along its
// contiguous dimension (ak == 1 or am == 1, bk == 1 or bn == 1). Split-K:
// blockIdx.z takes k-range [z * kz, (z + 1) * kz) and, with splits > 1, writes
// its partial product to C + z * M * ldc (reduced in order by splitk_reduce).
// Epilogue modes (splits == 1): 0 store C; 1 store Z = C + bias[n] to C and
// g(Z) (BF16-rounded when round_out) to out2; 2 store C + bias[n].
constexpr int kTM = 128, kTN = 128, kTK = 16;
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int Kd, const float* __restrict__ A, int64_t am, int64_t ak,
            const float* __restrict__ B, int64_t bk, int64_t bn, int round_a, int round_b,
            float* __restrict__ C, int64_t ldc, int mode, const float* __restrict__ bias,
            float* __restrict__ out2, int round_out, int kz) {
  __shared__ float As[kTK][kTM + 4];
  __shared__ float Bs[kTK][kTN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int kbeg = blockIdx.z * kz;
  const int kend = min(Kd, kbeg + kz);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const bool a_kc = ak == 1, b_kc = bk == 1;
  for (int k0 = kbeg; k0 < kend; k0 += kTK) {
#pragma unroll
    for (int r = 0; r < (kTK * kTM) / 256; ++r) {
      const int e = r * 256 + threadIdx.x;
      const int kk = a_kc ? e % kTK : e / kTM;
      const int mm = a_kc ? e / kTK : e % kTM;
      const int m = m0 + mm, k = k0 + kk;
      const float v = (m < M && k < kend) ? A[(int64_t)m * am + (int64_t)k * ak] : 0.f;
      As[kk][mm] = round_a ? round_bf16(v) : v;
    }
#pragma unroll
    for (int r = 0; r < (kTK * kTN) / 256; ++r) {
      const int e = r * 256 + threadIdx.x;
      const int kk = b_kc ? e % kTK : e / kTN;
      const int nn = b_kc ? e / kTK : e % kTN;
      const int n = n0 + nn, k = k0 + kk;
      const float v = (n < N && k < kend) ? B[(int64_t)k * bk + (int64_t)n * bn] : 0.f;
      Bs[kk][nn] = round_b ? round_bf16(v) : v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      const float4 a_lo = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a_hi = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
      const float4 b_lo = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float4 b_hi = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
      const float av[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
      const float bv[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* Cz = C + (int64_t)blockIdx.z * M * ldc;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 60 + ty * 4 + i);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 60 + tx * 4 + j);
      if (n >= N) continue;
      float v = acc[i][j];
      if (mode >= 1) v += bias[n];
      Cz[(int64_t)m * ldc + n] = v;
      if (mode == 1) {
        const float gv = gelu(v);
        out2[(int64_t)m * ldc + n] = round_out ? round_bf16(gv) : gv;
      }
    }
  }
}

// C[m][n] = sum over the splits, in order, of the partial products.
__global__ void splitk_reduce_kernel(int64_t MN, int splits, const float* __restrict__ parts,
                                     float* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += parts[z * MN + e];
    C[e] = s;
  }
}

// out[b] = sum_j H2[b][j] w3[j] + b3 (one warp per row, fixed lane order)
__global__ void output_kernel(int B, const float* __restrict__ H2, const float* __restrict__ w3,
                              const float* __restrict__ b3, float* __restrict__ out) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= B) return;
  float s = 0.f;
  for (int j = lane; j < kH; j += 32) s = fmaf(H2[(int64_t)w * kH + j], w3[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = s + b3[0];
}

// Mean and standard deviation of l = log(max(fit, 1e-30)) over the batch
// (FP64, fixed order: thread-strided sums then a sequential sum of the 256
// partials).
__global__ void target_stats_kernel(int B, const double* __restrict__ fit,
                                    double* __restrict__ stats) {
  __shared__ double s1[256], s2[256];
  double a = 0.0;
  for (int b = threadIdx.x; b < B; b += 256) {
    const double f = fit[b];
    a += log(f > 1e-30 ? f : 1e-30);
  }
  s1[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 256; ++i) t += s1[i];
    s1[0] = t / B;
  }
  __syncthreads();
  const double mu = s1[0];
  double q = 0.0;
  for (int b = threadIdx.x; b < B; b += 256) {
    const double f = fit[b];
    const double d = log(f > 1e-30 ? f : 1e-30) - mu;
    q += d * d;
  }
  s2[threadIdx.x] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 256; ++i) t += s2[i];
    const double sd = sqrt(t / B);
    stats[0] = mu;
    stats[1] = sd > 0.0 ? sd : 1.0;
  }
}

// d_out[b] = 2 (out[b] - t[b]) / B with the standardised target t; also the
// loss terms (out - t)^2 / B for reporting.
__global__ void dout_kernel(int B, const float* __restrict__ out, const double* __restrict__ fit,
                            const double* __restrict__ stats, float* __restrict__ dout,
                            float* __restrict__ loss_terms) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double f = fit[b];
  const float t = (float)((log(f > 1e-30 ? f : 1e-30) - stats[0]) / stats[1]);
  const float r = out[b] - t;
  dout[b] = 2.f * r / (float)B;
  loss_terms[b] = r * r / (float)B;
}

// dH2[b][j] = dout[b] w3[j], dZ2 = dH2 * g'(Z2) (in place into dZ)
__global__ void dz2_kernel(int B, const float* __restrict__ dout, const float* __restrict__ w3,
                           const float* __restrict__ Z2, float* __restrict__ dZ) {
  const int64_t n = (int64_t)B * kH;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / kH), j = (int)(e % kH);
    dZ[e] = dout[b] * w3[j] * gelu_grad(Z2[e]);
  }
}

// dZ[e] *= g'(Z[e])
__global__ void gelu_bwd_kernel(int64_t n, const float* __restrict__ Z, float* __restrict__ dZ) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dZ[e] *= gelu_grad(Z[e]);
}

// s[j] = sum_b X[b][j] y[b] (y = NULL: plain column sum), fixed order per column
__global__ void colsum_kernel(int B, int N, const float* __restrict__ X,
                              const float* __restrict__ y, float* __restrict__ s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float acc = 0.f;
  for (int b = 0; b < B; ++b) acc = fmaf(X[(int64_t)b * N + j], y ? y[b] : 1.f, acc);
  s[j] = acc;
}

__global__ void sum_kernel(int B, const float* __restrict__ v, float* __restrict__ s) {
  if (blockIdx.x != 0) return;
  __shared__ float part[256];
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += 256) acc += v[b];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < 256; ++i) t += part[i];
    s[0] = t;
  }
}

__global__ void adam_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float mh = mi / c1, vh = vi / c2;
    w[e] -= lr * mh / (sqrtf(vh) + eps);
  }
}

__global__ void init_params_kernel(uint64_t seed, int K, float* __restrict__ w) {
  const int64_t n1 = (int64_t)kH * K, n2 = (int64_t)kH * kH;
  const int64_t total = n1 + kH + n2 + kH + kH + 1;
  const float a1 = 1.f / sqrtf((float)K), a2 = 1.f / sqrtf((float)kH);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int layer;
    int64_t idx;
    float a;
    if (e < n1) {
      layer = 1, idx = e, a = a1;
    } else if (e < n1 + kH) {
      w[e] = 0.f;
      continue;
    } else if (e < n1 + kH + n2) {
      layer = 2, idx = e - n1 - kH, a = a2;
    } else if (e < n1 + kH + n2 + kH) {
      w[e] = 0.f;
      continue;
    } else if (e < n1 + kH + n2 + 2 * kH) {
      layer = 3, idx = e - n1 - 2 * kH - n2, a = a2;
    } else {
      w[e] = 0.f;
      continue;
    }
    const uint32_t r =
        philox4x32_10(seed, (uint32_t)layer, (uint32_t)idx, 0u, kTagSurrogate).x;
    // u in [-1, 1): (r >> 8) 2^-23 - 1, exact in FP32
    const float u = (float)(r >> 8) * (1.0f / 8388608.0f) - 1.0f;
    w[e] = u * a;
  }
}

// ---- screening: keep the n_keep smallest predictions of n ----
constexpr int kSortMax = 16384;

__global__ void __launch_bounds__(1024)
select_kernel(int n, int n_keep, const float* __restrict__ pred, int* __restrict__ keep_flag,
              const int* __restrict__ trusted, int* __restrict__ used_trust) {
  extern __shared__ uint64_t keys[];   // (order-preserving float bits << 32) | slot
  const int trust = *trusted;
  if (threadIdx.x == 0) *used_trust = trust;
  if (!trust) {   // the exact evaluator stands in: the unscreened generation's children
    for (int i = threadIdx.x; i < n; i += blockDim.x) keep_flag[i] = i < n_keep ? 1 : 0;
    return;
  }
  int npow = 1;
  while (npow < n) npow <<= 1;
  for (int i = threadIdx.x; i < npow; i += blockDim.x) {
    uint64_t k = ~0ull;
    if (i < n) {
      float p = pred[i];
      if (isnan(p)) p = __int_as_float(0x7f800000);   // NaN ranks last (+inf)
      uint32_t u = __float_as_uint(p);
      u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // float order as unsigned
      k = ((uint64_t)u << 32) | (uint32_t)i;
    }
    keys[i] = k;
  }
  __syncthreads();
  for (int size = 2; size <= npow; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const uint64_t a = keys[i], b = keys[j];
          if ((a > b) == up) {
            keys[i] = b;
            keys[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) keep_flag[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_keep; i += blockDim.x)
    keep_flag[(int)(keys[i] & 0xffffffffu)] = 1;
}

// pos[i] = number of kept children before child i (or -1 if child i is not
// kept): one CTA, an exclusive prefix sum of the flags in slot order.
__global__ void __launch_bounds__(1024)
assemble_kernel(int n, const int* __restrict__ keep_flag, int* __restrict__ pos) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int f = i < n ? keep_flag[i] : 0;
    int x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const int excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - f;
    if (i < n) pos[i] = f ? excl : -1;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + f;
    __syncthreads();
  }
}

__global__ void gather_kernel(int n, int E, int K, const int* __restrict__ pos,
                              const float* __restrict__ off, float* __restrict__ next) {
  // rows 0..E-1: elites; row E + pos[i] <- offspring slot E + i
  const int64_t total = (int64_t)(E + n) * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / K), k = (int)(e % K);
    if (s < E) {
      next[e] = off[e];
    } else {
      const int p = pos[s - E];
      if (p >= 0) next[(int64_t)(E + p) * K + k] = off[e];
    }
  }
}

// Pearson correlation of the kept children's predictions with their exact
// log-fitness (fit_kept[pos[i]] for kept child i), FP64 sums in a fixed
// order; trusted = r > 0.25.
__global__ void trust_kernel(int n, const float* __restrict__ pred, const int* __restrict__ flag,
                             const int* __restrict__ pos, const double* __restrict__ fit_kept,
                             float* __restrict__ r_out, int* __restrict__ trusted) {
  __shared__ double sh[5][256];
  double a[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < n; i += 256) {
    if (!flag[i]) continue;
    const double x = pred[i];
    const double f = fit_kept[pos[i]];
    const double y = log(f > 1e-30 ? f : 1e-30);
    a[0] += 1.0;
    a[1] += x;
    a[2] += y;
    a[3] += x * y;
    a[4] += x * x;
  }
  double yy = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    if (!flag[i]) continue;
    const double f = fit_kept[pos[i]];
    const double y = log(f > 1e-30 ? f : 1e-30);
    yy += y * y;
  }
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  __shared__ double syy[256];
  syy[threadIdx.x] = yy;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 256; ++i) {
      for (int k = 0; k < 5; ++k) t[k] += sh[k][i];
      t[5] += syy[i];
    }
    const double c = t[0];
    double r = 0.0;
    if (c > 1.0) {
      const double cov = t[3] / c - (t[1] / c) * (t[2] / c);
      const double vx = t[4] / c - (t[1] / c) * (t[1] / c);
      const double vy = t[5] / c - (t[2] / c) * (t[2] / c);
      r = (vx > 0.0 && vy > 0.0) ? cov / sqrt(vx * vy) : 0.0;
    }
    *r_out = (float)r;
    *trusted = r > 0.25 ? 1 : 0;
  }
}

// Split-K factor of the weight-gradient GEMMs (reduction over the batch):
// about 64 rows per split, at most kMaxSplits.
int kGradSplits(int B) {
  int sp = (B + 63) / 64;
  return sp < 1 ? 1 : (sp > kMaxSplits ? kMaxSplits : sp);
}

int grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

cudaError_t gemm(int M, int N, int Kd, const float* A, int64_t am, int64_t ak, const float* B,
                 int64_t bk, int64_t bn, int ra, int rb, float* C, int64_t ldc, int mode,
                 const float* bias, float* out2, int round_out, cudaStream_t st,
                 float* split_ws = nullptr, int splits = 1) {
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM, splits);
  int kz = (Kd + splits - 1) / splits;
  kz = (kz + kTK - 1) / kTK * kTK;
  if (splits > 1) {
    // partial products into the workspace, then their sum in split order
    gemm_kernel<<<grid, 256, 0, st>>>(M, N, Kd, A, am, ak, B, bk, bn, ra, rb, split_ws, N, 0,
                                      nullptr, nullptr, 0, kz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    splitk_reduce_kernel<<<grid1d((int64_t)M * N), 256, 0, st>>>((int64_t)M * N, splits,
                                                                  split_ws, C);
    return cudaGetLastError();
  }
  gemm_kernel<<<grid, 256, 0, st>>>(M, N, Kd, A, am, ak, B, bk, bn, ra, rb, C, ldc, mode, bias,
                                    out2, round_out, kz);
  return cudaGetLastError();
}

}  // namespace

int64_t surrogate_param_count(int K) {
  return (int64_t)kH * K + kH + (int64_t)kH * kH + kH + kH + 1;
}

cudaError_t surrogate_init(const SurrogateDev& s, uint64_t seed, cudaStream_t st) {
  const int64_t n = surrogate_param_count(s.K);
  init_params_kernel<<<grid1d(n), 256, 0, st>>>(seed, s.K, s.w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.m, 0, n * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.v, 0, n * sizeof(float), st);
  return e;
}

// Forward pass of B rows X [B][K] (FP32 genes) into out [B]; keeps Z1, H1,
// Z2, H2 [B][256] in the workspace for a backward pass.
cudaError_t surrogate_forward(const SurrogateDev& s, const float* X, int B, float* out,
                              cudaStream_t st) {
  if (B > s.Bmax) return cudaErrorInvalidValue;
  const int K = s.K;
  const float* W1 = s.w;
  const float* b1 = W1 + (int64_t)kH * K;
  const float* W2 = b1 + kH;
  const float* b2 = W2 + (int64_t)kH * kH;
  const float* w3 = b2 + kH;
  const float* b3 = w3 + kH;
  // Z1 = bf(X) bf(W1)^T + b1, H1 = bf(g(Z1))
  cudaError_t e = gemm(B, kH, K, X, K, 1, W1, 1, K, 1, 1, s.Z1, kH, 1, b1, s.H1, 1, st);
  if (e != cudaSuccess) return e;
  // Z2 = H1 bf(W2)^T + b2, H2 = g(Z2)
  e = gemm(B, kH, kH, s.H1, kH, 1, W2, 1, kH, 0, 1, s.Z2, kH, 1, b2, s.H2, 0, st);
  if (e != cudaSuccess) return e;
  output_kernel<<<(int)(((int64_t)B * 32 + 255) / 256), 256, 0, st>>>(B, s.H2, w3, b3, out);
  return cudaGetLastError();
}

// Gradient of the mean squared error of log-fitness over B pairs into s.g
// (after a forward pass of the same X); loss into s.loss[0].
cudaError_t surrogate_backward(const SurrogateDev& s, const float* X, const double* fit, int B,
                               cudaStream_t st) {
  const int K = s.K;
  const float* W1 = s.w;
  const float* W2 = W1 + (int64_t)kH * K + kH;
  const float* w3 = W2 + (int64_t)kH * kH + kH;
  float* gW1 = s.g;
  float* gb1 = gW1 + (int64_t)kH * K;
  float* gW2 = gb1 + kH;
  float* gb2 = gW2 + (int64_t)kH * kH;
  float* gw3 = gb2 + kH;
  float* gb3 = gw3 + kH;
  target_stats_kernel<<<1, 256, 0, st>>>(B, fit, s.tstat);
  dout_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, s.out, fit, s.tstat, s.dout, s.lterm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_kernel<<<1, 256, 0, st>>>(B, s.lterm, s.loss);
  // output layer
  colsum_kernel<<<1, kH, 0, st>>>(B, kH, s.H2, s.dout, gw3);
  sum_kernel<<<1, 256, 0, st>>>(B, s.dout, gb3);
  // dZ2 = dout w3 g'(Z2)
  dz2_kernel<<<grid1d((int64_t)B * kH), 256, 0, st>>>(B, s.dout, w3, s.Z2, s.dZ2);
  // gW2 = dZ2^T H1, gb2 = colsum(dZ2)
  const int splits = kGradSplits(B);
  e = gemm(kH, kH, B, s.dZ2, 1, kH, s.H1, kH, 1, 0, 0, gW2, kH, 0, nullptr, nullptr, 0, st,
           s.split_ws, splits);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<1, kH, 0, st>>>(B, kH, s.dZ2, nullptr, gb2);
  // dZ1 = (dZ2 bf(W2)) g'(Z1)
  e = gemm(B, kH, kH, s.dZ2, kH, 1, W2, kH, 1, 0, 1, s.dZ1, kH, 0, nullptr, nullptr, 0, st);
  if (e != cudaSuccess) return e;
  gelu_bwd_kernel<<<grid1d((int64_t)B * kH), 256, 0, st>>>((int64_t)B * kH, s.Z1, s.dZ1);
  // gW1 = dZ1^T bf(X), gb1 = colsum(dZ1)
  e = gemm(kH, K, B, s.dZ1, 1, kH, X, K, 1, 0, 1, gW1, K, 0, nullptr, nullptr, 0, st,
           s.split_ws, splits);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<1, kH, 0, st>>>(B, kH, s.dZ1, nullptr, gb1);
  return cudaGetLastError();
}

cudaError_t surrogate_adam(SurrogateDev& s, cudaStream_t st) {
  s.step += 1;
  const float c1 = 1.f - powf(kAdamB1, (float)s.step);
  const float c2 = 1.f - powf(kAdamB2, (float)s.step);
  const int64_t n = surrogate_param_count(s.K);
  adam_kernel<<<grid1d(n), 256, 0, st>>>(n, s.w, s.g, s.m, s.v, kAdamLr, kAdamB1, kAdamB2,
                                         kAdamEps, c1, c2);
  return cudaGetLastError();
}

cudaError_t surrogate_trust_check(int n, const float* pred, const int* flag, const int* pos,
                            const double* fit_kept, float* r_out, int* trusted, cudaStream_t st) {
  trust_kernel<<<1, 256, 0, st>>>(n, pred, flag, pos, fit_kept, r_out, trusted);
  return cudaGetLastError();
}

cudaError_t surrogate_screen(int n, int n_keep, int E, int K, const float* pred, int* flag,
                             int* pos, const float* off, float* next, const int* trusted,
                             int* used_trust, cudaStream_t st) {
  if (n > kSortMax || n_keep > n) return cudaErrorInvalidValue;
  int npow = 1;
  while (npow < n) npow <<= 1;
  const size_t smem = (size_t)npow * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kSortMax * sizeof(uint64_t)));
  if (e != cudaSuccess) return e;
  select_kernel<<<1, 1024, smem, st>>>(n, n_keep, pred, flag, trusted, used_trust);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  assemble_kernel<<<1, 1024, 0, st>>>(n, flag, pos);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gather_kernel<<<grid1d((int64_t)(E + n) * K), 256, 0, st>>>(n, E, K, pos, off, next);
  return cudaGetLastError();
}

}  // namespace game
