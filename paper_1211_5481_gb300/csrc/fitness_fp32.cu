// fitness_fp32.cu -- fitness of a population with the contraction on CUDA-core
// FP32 FFMA (the plain FP32 form).
//
// For chromosome p and pattern m (paper Section 3):
//   Out_p(m) = a_{p,0} + sum_c a_{p,c+1} phi_c(x_m)         (Eq. 2)
//   fit_p    = (1/M) sum_m (y_m - Out_p(m))^2               (Eq. 3, MSE)
// A CTA owns 128 chromosomes and walks pattern tiles of 128 (grid-strided
// over blockIdx.y). Per tile the 128x128 output block is a register-blocked
// product (8x8 per thread) over K-chunks of 16: the chunk of genes comes from
// popT (coalesced), the chunk of the expansion phi is generated in registers
// from the features (basis.cuh) and staged through shared memory, double
// buffered. Neither phi nor the output block ever reaches global memory: the
// epilogue forms the residuals, squares them (or, for the MAE, takes their
// absolute values) and sums them over the tile's patterns (FP32, 128 terms),
// and adds the tile sum to an FP64 accumulator
// per chromosome. Each CTA writes its FP64 sums to part[blockIdx.y][p]; the
// reduce kernel adds the rows in a fixed order.
#include "basis.cuh"
#include "game_internal.cuh"

namespace game {

namespace {

constexpr int BP = 128;   // chromosomes per CTA
constexpr int BM = 128;   // patterns per tile
constexpr int KC = 16;    // contraction columns per chunk
constexpr int kThreads = 256;

template <bool ABS>
__global__ void __launch_bounds__(kThreads, 2)
fitness_fp32_kernel(int64_t M, int N, int d, int basis, int Kp, int Kc,
                    const float* __restrict__ Xt, const float* __restrict__ y,
                    const float* __restrict__ popT, const float* __restrict__ a0, int Ppad,
                    int ntiles, double* __restrict__ part) {
  __shared__ __align__(16) float As[2][KC][BP];
  __shared__ __align__(16) float Bs[2][KC][BM];
  __shared__ double sse_s[BP];

  const int tid = threadIdx.x;
  const int tx = tid & 15;   // pattern group
  const int ty = tid >> 4;   // chromosome group
  const int cb = blockIdx.x * BP;
  const int nch = Kc / KC;

  // A-chunk loader: 16 rows x 128 floats = 512 float4, two per thread
  const int la_row0 = tid >> 5, la_col = (tid & 31) * 4;
  // phi-chunk generator: one pattern, 8 consecutive columns
  const int gp = tid & (BM - 1);
  const int ghalf = tid >> 7;

  for (int i = tid; i < BP; i += kThreads) sse_s[i] = 0.0;

  for (int t = blockIdx.y; t < ntiles; t += gridDim.y) {
    const float* xs = Xt + (int64_t)t * N * kPatBlock + gp;

    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;

    float4 ra[2];
    float rb[8];
    // chunk 0 into buffer 0
#pragma unroll
    for (int h = 0; h < 2; ++h)
      ra[h] = *reinterpret_cast<const float4*>(
          popT + (int64_t)(la_row0 + 8 * h) * Ppad + cb + la_col);
    basis_run<8>(basis, d, Kp, xs, kPatBlock, ghalf * 8, rb);
    __syncthreads();   // previous tile's epilogue is done with the buffers
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<float4*>(&As[0][la_row0 + 8 * h][la_col]) = ra[h];
#pragma unroll
    for (int v = 0; v < 8; ++v) Bs[0][ghalf * 8 + v][gp] = rb[v];
    __syncthreads();

    for (int kc = 0; kc < nch; ++kc) {
      const int buf = kc & 1;
      const bool more = kc + 1 < nch;
      if (more) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
          ra[h] = *reinterpret_cast<const float4*>(
              popT + (int64_t)((kc + 1) * KC + la_row0 + 8 * h) * Ppad + cb + la_col);
        basis_run<8>(basis, d, Kp, xs, kPatBlock, (kc + 1) * KC + ghalf * 8, rb);
      }
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const float4 a_lo = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 a_hi = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
        const float4 b_lo = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
        const float4 b_hi = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
        const float a[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
        const float b[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
      }
      if (more) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
          *reinterpret_cast<float4*>(&As[buf ^ 1][la_row0 + 8 * h][la_col]) = ra[h];
#pragma unroll
        for (int v = 0; v < 8; ++v) Bs[buf ^ 1][ghalf * 8 + v][gp] = rb[v];
      }
      __syncthreads();
    }

    // epilogue: squared residuals of this thread's 8x8 outputs
    const int64_t mbase = (int64_t)t * BM;
    const float4 y_lo = *reinterpret_cast<const float4*>(y + mbase + tx * 4);
    const float4 y_hi = *reinterpret_cast<const float4*>(y + mbase + 64 + tx * 4);
    const float yv[8] = {y_lo.x, y_lo.y, y_lo.z, y_lo.w, y_hi.x, y_hi.y, y_hi.z, y_hi.w};
    bool ok[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) ok[v] = mbase + (v < 4 ? tx * 4 + v : 60 + tx * 4 + v) < M;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int cl = u < 4 ? ty * 4 + u : 60 + ty * 4 + u;
      const float bias = a0[cb + cl];
      float s = 0.f;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const float r = (yv[v] - bias) - acc[u][v];
        s = ok[v] ? (ABS ? s + fabsf(r) : fmaf(r, r, s)) : s;
      }
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 8);
      if (tx == 0) sse_s[cl] += (double)s;
    }
  }
  __syncthreads();
  for (int i = tid; i < BP; i += kThreads)
    part[(int64_t)blockIdx.y * Ppad + cb + i] = sse_s[i];
}

}  // namespace

Fp32Plan plan_fp32(const Shape& s, int P, int num_sms) {
  Fp32Plan pl;
  pl.BP = BP;
  pl.BM = BM;
  pl.Kc = ceil_div(s.Kp, KC) * KC;
  pl.grid_x = ceil_div(P, BP);
  const int ntiles = ceil_div(s.M, BM);
  int gy = (2 * num_sms + pl.grid_x - 1) / pl.grid_x;
  if (gy < 1) gy = 1;
  if (gy > ntiles) gy = ntiles;
  pl.grid_y = gy;
  return pl;
}

cudaError_t launch_fitness_fp32(const Fp32Plan& pl, const Shape& s, const float* Xt,
                                const float* y, const float* popT, const float* a0, int P,
                                int Ppad, double* part, int err, cudaStream_t st) {
  (void)P;
  const int ntiles = ceil_div(s.M, BM);
  dim3 grid(pl.grid_x, pl.grid_y);
  auto kern = err == GAME_ERR_MAE ? fitness_fp32_kernel<true> : fitness_fp32_kernel<false>;
  kern<<<grid, kThreads, 0, st>>>(s.M, s.N, s.d, s.basis, s.Kp, pl.Kc, Xt, y, popT, a0, Ppad,
                                  ntiles, part);
  return cudaGetLastError();
}

}  // namespace game
