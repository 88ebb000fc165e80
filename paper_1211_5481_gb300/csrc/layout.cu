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

cudaError_t launch_pack_bf16(const float* pop, int P, int C, const Shape& s, int KB,
                             uint8_t* popA, float* a0, cudaStream_t st) {
  const int64_t n = (int64_t)C * 128 * KB * 8;
  pack_bf16_kernel<<<grid_for(n, 256), 256, 0, st>>>(pop, P, C, s.K, KB, popA, a0);
  return cudaGetLastError();
}

}  // namespace game
