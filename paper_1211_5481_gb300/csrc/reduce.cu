// reduce.cu -- cross-tile FP64 error sum: fit[p] = (sum_r part[r][p]) / M
// (the MSE from squared residuals, the MAE from absolute ones), or its square
// root for the RMSE.
//
// One warp per chromosome: lane l adds rows l, l+32, ... in order, then a
// fixed xor-butterfly combines the lanes. The order depends only on the
// number of rows, so the result is bit-identical run to run (no atomics).
#include "game_internal.cuh"

namespace game {

namespace {

__global__ void reduce_rows_kernel(const double* __restrict__ part, int rows, int P, int Ppad,
                                   int err, int64_t M, double* __restrict__ fit) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= P) return;
  double s = 0.0;
  for (int r = lane; r < rows; r += 32) s += part[(int64_t)r * Ppad + warp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double mean = s / (double)M;
    fit[warp] = err == GAME_ERR_RMSE ? sqrt(mean) : mean;
  }
}

}  // namespace

cudaError_t launch_reduce(const double* part, int rows, int P, int Ppad, int64_t M, int err,
                          double* fit, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (int)(((int64_t)P * 32 + threads - 1) / threads);
  reduce_rows_kernel<<<blocks, threads, 0, st>>>(part, rows, P, Ppad, err, M, fit);
  return cudaGetLastError();
}

}  // namespace game
