// layout.cu -- device layouts of the training set and of the population.
//
//  * relayout_X: X [M][N] row-major -> Xt [Mpad/128][N][128] (feature-major
//    blocks of 128 patterns) and y -> y padded with zeros to Mpad, counting
//    non-finite values and, for the Chebyshev basis, |x| > 1 (its domain).
//  * pack_fp32: genes 1..K-1 transposed to popT [Kc][Ppad] plus the bias
//    genes a0 [Ppad], zero-padded (CUDA-core contraction).
//  * pack_bf16: genes 1..K-1 rounded to BF16 in the tcgen05 operand image:
//    for chromosome tile c and K-block kb, a 16 KB block of 128 rows
//    (chromosomes) x 128 bytes (64 genes), 16-byte chunk q of row r stored at
//    chunk position q ^ (r % 8) (the 128-byte swizzle), so a bulk copy into a
//    1024-byte-aligned shared buffer yields the K-major SWIZZLE_128B layout.
//  * pack_bf16x3: the same image twice per K-block, hi = bf16(a) then
//    lo = bf16(a - hi) (split products).
//  * colmax / colscales: per contraction column k, max_m |phi_k(x_m)| over the
//    training set (the FP32 basis recurrences of the kernels) and the FP8
//    scales colscale_k = max / 448, colinv_k = 448 / max.
//  * pack_fp8: per chromosome u_p = max_k |a_pk colscale_k| / 448 (1 if 0),
//    genes a_pk colscale_k / u_p rounded to E4M3 (saturating) in the image of
//    128 rows x 128 bytes (128 genes) per (chromosome tile, K-block).
#include <cuda_fp8.h>

#include "basis.cuh"
#include "game_internal.cuh"

namespace game {

namespace {

constexpr int kFeatChunk = 32;

__global__ void relayout_X_kernel(const float* __restrict__ X, const float* __restrict__ y,
                                  int64_t M, int N, int check_domain, float* __restrict__ Xt,
                                  float* __restrict__ yp, int* __restrict__ bad) {
  __shared__ float tile[kPatBlock][kFeatChunk + 1];
  const int64_t blk = blockIdx.x;
  const int64_t m0 = blk * kPatBlock;
  int nonfinite = 0, outside = 0;
  for (int i0 = 0; i0 < N; i0 += kFeatChunk) {
    const int nf = min(kFeatChunk, N - i0);
    // coalesced read of the rows' feature chunk
    for (int e = threadIdx.x; e < kPatBlock * kFeatChunk; e += blockDim.x) {
      const int r = e / kFeatChunk, c = e % kFeatChunk;
      float v = 0.f;
      if (c < nf && m0 + r < M) {
        v = X[(m0 + r) * N + i0 + c];
        if (!isfinite(v)) ++nonfinite;
        else if (check_domain && fabsf(v) > 1.0f) ++outside;
      }
      tile[r][c] = v;
    }
    __syncthreads();
    // coalesced write, feature-major
    for (int e = threadIdx.x; e < kPatBlock * nf; e += blockDim.x) {
      const int c = e / kPatBlock, r = e % kPatBlock;
      Xt[(blk * N + i0 + c) * kPatBlock + r] = tile[r][c];
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < kPatBlock; r += blockDim.x) {
    float v = 0.f;
    if (m0 + r < M) {
      v = y[m0 + r];
      if (!isfinite(v)) ++nonfinite;
    }
    yp[m0 + r] = v;
  }
  if (nonfinite) atomicAdd(&bad[0], nonfinite);
  if (outside) atomicAdd(&bad[1], outside);
}

__global__ void pack_fp32_kernel(const float* __restrict__ pop, int P, int Ppad, int K,
                                 int Kc, float* __restrict__ popT, float* __restrict__ a0) {
  const int64_t n = (int64_t)Kc * Ppad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / Ppad), p = (int)(e % Ppad);
    popT[e] = (p < P && k + 1 < K) ? pop[(int64_t)p * K + 1 + k] : 0.f;
    if (k == 0) a0[p] = p < P ? pop[(int64_t)p * K] : 0.f;
  }
}

__global__ void pack_bf16_kernel(const float* __restrict__ pop, int P, int C, int K, int KB,
                                 uint8_t* __restrict__ popA, float* __restrict__ a0) {
  // one thread per (chromosome row, K-block, 16-byte chunk)
  const int64_t n = (int64_t)C * 128 * KB * 8;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % 8);
    const int kb = (int)((e / 8) % KB);
    const int p = (int)(e / (8 * KB));
    const int c = p / 128, r = p % 128;
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float v[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int kc = kb * 64 + q * 8 + 2 * h + u;   // contraction column
        v[u] = (p < P && kc + 1 < K) ? pop[(int64_t)p * K + 1 + kc] : 0.f;
      }
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
      w[h] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    uint8_t* dst = popA + ((int64_t)(c * KB + kb) * 128 + r) * 128 + ((q ^ (r & 7)) << 4);
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    if (kb == 0 && q == 0) a0[p] = p < P ? pop[(int64_t)p * K] : 0.f;
  }
}

__global__ void pack_bf16x3_kernel(const float* __restrict__ pop, int P, int C, int K, int KB,
                                   uint8_t* __restrict__ popA, float* __restrict__ a0) {
  const int64_t n = (int64_t)C * 128 * KB * 8;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % 8);
    const int kb = (int)((e / 8) % KB);
    const int p = (int)(e / (8 * KB));
    const int c = p / 128, r = p % 128;
    uint32_t wh[4], wl[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float v[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int kc = kb * 64 + q * 8 + 2 * h + u;
        v[u] = (p < P && kc + 1 < K) ? pop[(int64_t)p * K + 1 + kc] : 0.f;
      }
      const __nv_bfloat162 hi = __floats2bfloat162_rn(v[0], v[1]);
      const float2 hf = __bfloat1622float2(hi);
      const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0] - hf.x, v[1] - hf.y);
      wh[h] = *reinterpret_cast<const uint32_t*>(&hi);
      wl[h] = *reinterpret_cast<const uint32_t*>(&lo);
    }
    uint8_t* dst = popA + ((int64_t)(c * KB + kb) * 2 * 128 + r) * 128 + ((q ^ (r & 7)) << 4);
    *reinterpret_cast<uint4*>(dst) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(dst + 128 * 128) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    if (kb == 0 && q == 0) a0[p] = p < P ? pop[(int64_t)p * K] : 0.f;
  }
}

// One warp per chromosome row (padding rows included).
__global__ void pack_fp8_kernel(const float* __restrict__ pop, int P, int C, int K, int KB,
                                const float* __restrict__ colscale, uint8_t* __restrict__ popA,
                                float* __restrict__ a0, float* __restrict__ uscale) {
  const int lane = threadIdx.x & 31;
  const int64_t nrows = (int64_t)C * 128;
  for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; p < nrows;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const bool real = p < P;
    const float* gene = pop + p * K + 1;   // genes 1..K-1 (read only when real)
    float mx = 0.f;
    if (real)
      for (int k = lane; k < K - 1; k += 32) mx = fmaxf(mx, fabsf(gene[k] * colscale[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float u = mx > 0.f ? mx / 448.f : 1.f;
    const int c = (int)(p / 128), r = (int)(p % 128);
    for (int unit = lane; unit < KB * 8; unit += 32) {
      const int kb = unit / 8, q = unit % 8;
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int k = kb * 128 + q * 16 + 4 * h + t;
          v[t] = (real && k < K - 1) ? gene[k] * colscale[k] / u : 0.f;
        }
        const uint32_t lo =
            __nv_cvt_float2_to_fp8x2(make_float2(v[0], v[1]), __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi =
            __nv_cvt_float2_to_fp8x2(make_float2(v[2], v[3]), __NV_SATFINITE, __NV_E4M3);
        w[h] = lo | (hi << 16);
      }
      uint8_t* dst = popA + ((int64_t)(c * KB + kb) * 128 + r) * 128 + ((q ^ (r & 7)) << 4);
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (lane == 0) {
      a0[p] = real ? pop[p * K] : 0.f;
      uscale[p] = u;
    }
  }
}

// max_m |phi_k(x_m)| per column, as FP32 bit patterns (order-preserving for
// non-negative values, so the integer max is the float max).
__global__ void colmax_kernel(int64_t M, int N, int d, int basis, int Kp,
                              const float* __restrict__ Xt, unsigned int* __restrict__ colmax) {
  extern __shared__ unsigned int smax[];
  for (int k = threadIdx.x; k < Kp; k += blockDim.x) smax[k] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w * 32 < M;
       w += warps) {
    const int64_t m = w * 32 + lane;
    const bool ok = m < M;
    const int64_t mm = ok ? m : 0;
    const float* xs = Xt + (mm / kPatBlock) * (int64_t)N * kPatBlock + (mm % kPatBlock);
    for (int c0 = 0; c0 < Kp; c0 += 8) {
      float v[8];
      basis_run<8>(basis, d, Kp, xs, kPatBlock, c0, v);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const unsigned int bits = ok ? __float_as_uint(fabsf(v[e])) : 0u;
        const unsigned int mx = __reduce_max_sync(0xffffffffu, bits);
        if (lane == 0 && c0 + e < Kp) atomicMax(&smax[c0 + e], mx);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < Kp; k += blockDim.x) atomicMax(&colmax[k], smax[k]);
}

__global__ void colscales_kernel(const unsigned int* __restrict__ colmax, int ncols,
                                 float* __restrict__ colscale, float* __restrict__ colinv) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncols; k += gridDim.x * blockDim.x) {
    const float mx = __uint_as_float(colmax[k]);
    colscale[k] = mx / 448.f;
    colinv[k] = mx > 0.f ? 448.f / mx : 0.f;
  }
}

// full[p][k] = pop[p][0] for k = 0, else pop[p][1 + (k - 1) mod (B d)]:
// gene 1 + i B d + b d + (j - 1) of feature i takes the shared gene
// 1 + b d + (j - 1).
__global__ void replicate_tied_kernel(const float* __restrict__ pop, int P, int K, int Bd,
                                      float* __restrict__ full) {
  const int64_t n = (int64_t)P * K;
  const int Kg = Bd + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / K), k = (int)(e % K);
    full[e] = pop[(int64_t)p * Kg + (k == 0 ? 0 : 1 + (k - 1) % Bd)];
  }
}

int grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)(b < 65535 * 16 ? (b < 1 ? 1 : b) : 65535 * 16);
}

}  // namespace

cudaError_t launch_relayout_X(const float* X, const float* y, const Shape& s, float* Xt,
                              float* yp, int* bad_counts, cudaStream_t st) {
  const int blocks = (int)(s.Mpad / kPatBlock);
  relayout_X_kernel<<<blocks, 256, 0, st>>>(X, y, s.M, s.N, s.basis == GAME_BASIS_CHEB, Xt,
                                           yp, bad_counts);
  return cudaGetLastError();
}

cudaError_t launch_pack_fp32(const float* pop, int P, int Ppad, const Shape& s, int Kc,
                             float* popT, float* a0, cudaStream_t st) {
  const int64_t n = (int64_t)Kc * Ppad;
  pack_fp32_kernel<<<grid_for(n, 256), 256, 0, st>>>(pop, P, Ppad, s.K, Kc, popT, a0);
  return cudaGetLastError();
}

cudaError_t launch_replicate_tied(const float* pop, int P, const Shape& s, float* full,
                                  cudaStream_t st) {
  const int64_t n = (int64_t)P * s.K;
  replicate_tied_kernel<<<grid_for(n, 256), 256, 0, st>>>(pop, P, s.K, s.B * s.d, full);
  return cudaGetLastError();
}

cudaError_t launch_pack_tc(int form, const float* pop, int P, int C, const Shape& s, int KB,
                           const float* colscale, uint8_t* popA, float* a0, float* uscale,
                           cudaStream_t st) {
  const int64_t n = (int64_t)C * 128 * KB * 8;
  if (form == kFormBF16) {
    pack_bf16_kernel<<<grid_for(n, 256), 256, 0, st>>>(pop, P, C, s.K, KB, popA, a0);
  } else if (form == kFormBF16x3) {
    pack_bf16x3_kernel<<<grid_for(n, 256), 256, 0, st>>>(pop, P, C, s.K, KB, popA, a0);
  } else if (form == kFormFP8) {
    if (!colscale || !uscale) return cudaErrorInvalidValue;
    pack_fp8_kernel<<<grid_for((int64_t)C * 128 * 32, 256), 256, 0, st>>>(
        pop, P, C, s.K, KB, colscale, popA, a0, uscale);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_colmax(const Shape& s, const float* Xt, unsigned int* colmax, int ncols,
                          cudaStream_t st) {
  if (ncols < s.Kp) return cudaErrorInvalidValue;
  const size_t smem = (size_t)s.Kp * sizeof(unsigned int);
  cudaError_t e = cudaFuncSetAttribute(colmax_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kMaxK * sizeof(unsigned int)));
  if (e != cudaSuccess) return e;
  int64_t blocks = (s.M + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  colmax_kernel<<<(int)blocks, 256, smem, st>>>(s.M, s.N, s.d, s.basis, s.Kp, Xt, colmax);
  return cudaGetLastError();
}

cudaError_t launch_colscales(const unsigned int* colmax, int ncols, float* colscale,
                             float* colinv, cudaStream_t st) {
  colscales_kernel<<<grid_for(ncols, 256), 256, 0, st>>>(colmax, ncols, colscale, colinv);
  return cudaGetLastError();
}

}  // namespace game
