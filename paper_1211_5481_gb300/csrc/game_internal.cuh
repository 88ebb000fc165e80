// game_internal.cuh -- shared definitions of the CUDA path of libgame.so.
//
// Device data layout (all owned by the handle):
//   Xt   [Mpad/128][N][128] FP32  features, tiled by blocks of 128 patterns and
//                                 feature-major inside a block, so one block is a
//                                 contiguous, 16-byte-aligned run for bulk copies
//                                 and a warp reading one feature of 32 patterns
//                                 touches 128 consecutive bytes.
//   y    [Mpad] FP32              targets, zero past M (masked in the epilogues).
//   pop  [2][P][K] FP32           GA state, ping-pong.
//   fit  [P] FP64                 fitness of the current population.
// Evaluation scratch (grown on demand):
//   popT [Kc][Ppad] FP32          genes 1..K-1 transposed (CUDA-core form).
//   popA [C][KB][128][64] BF16    genes 1..K-1 in the tcgen05 K-major SWIZZLE_128B
//                                 operand image: one 16 KB block per (chromosome
//                                 tile c, K-block kb), bulk-copied unchanged into
//                                 shared memory.
//   a0   [Ppad] FP32              bias genes.
//   part [rows][Ppad] FP64        per-CTA partial sums of squared residuals.
// Elite re-scoring (fixed size, allocated with the handle):
//   cand [16] int32               candidate indices, best first.
//   rpart [2][grid][8] FP64       per-CTA partial sums of the re-scored candidates.
//   tickets [2] uint32            finish counters of the re-scoring CTAs (self-resetting).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/game.h"

namespace game {

constexpr int kPatBlock = 128;   // patterns per stored X block
constexpr int kMaxK = 4097;      // genes per chromosome accepted
constexpr int kMaxTournament = 64;
constexpr int kMaxRescore = 16;  // elite candidates re-scored at most

// Status word written by kernels (0 = fine).
enum DevStatus : int { kDevOk = 0, kDevTimeout = 1, kDevBadShape = 2 };

struct Shape {
  int64_t M, Mpad;
  int N, d, basis, B;
  int K;      // genes, B*N*d + 1
  int Kp;     // K - 1, the contraction length
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- kernels and launchers (defined in the .cu files) ----
// layout.cu
cudaError_t launch_relayout_X(const float* X, const float* y, const Shape& s, float* Xt,
                              float* yp, int* bad_counts, cudaStream_t st);
cudaError_t launch_pack_fp32(const float* pop, int P, int Ppad, const Shape& s, int Kc,
                             float* popT, float* a0, cudaStream_t st);
cudaError_t launch_pack_bf16(const float* pop, int P, int C, const Shape& s, int KB,
                             uint8_t* popA, float* a0, cudaStream_t st);
// fitness_fp32.cu
struct Fp32Plan { int BP, BM, Kc, grid_x, grid_y; };
Fp32Plan plan_fp32(const Shape& s, int P, int num_sms);
cudaError_t launch_fitness_fp32(const Fp32Plan& pl, const Shape& s, const float* Xt,
                                const float* y, const float* popT, const float* a0, int P,
                                int Ppad, double* part, cudaStream_t st);
// fitness_tc.cu
struct TcPlan { int BN, KB, NS, C, stages, grid, smem_bytes, tmem_cols, rows; bool ok; };
TcPlan plan_tc(const Shape& s, int P, int num_sms);
cudaError_t launch_fitness_tc(const TcPlan& pl, const Shape& s, const float* Xt,
                              const float* y, const uint8_t* popA, const float* a0, int P,
                              int Ppad, double* part, int* status, cudaStream_t st);
// rescore.cu
struct RescorePlan { int pt, grid; };   // patterns per thread, CTAs per candidate group
RescorePlan plan_rescore(const Shape& s, int num_sms);
size_t rescore_smem_bytes(const Shape& s);
cudaError_t launch_rescore(const RescorePlan& pl, const Shape& s, const float* Xt,
                           const float* y, const float* pop, int P, int n, double* fit,
                           int* cand, double* part, unsigned int* tickets, cudaStream_t st);
// api.cu
void record_error(const char* msg);
// reduce.cu
cudaError_t launch_reduce(const double* part, int rows, int P, int Ppad, int64_t M,
                          double* fit, cudaStream_t st);
// ga_ops.cu
struct GaDev {
  int P, K, E, T, I;
  uint32_t thr_pc, thr_pm;
  float sigma;
};
cudaError_t launch_init_population(uint64_t seed, int P, int K, float* pop, cudaStream_t st);
cudaError_t launch_generation(const GaDev& ga, const float* pop, const double* fit,
                              uint64_t seed, uint32_t g, int4* plan, float* next,
                              cudaStream_t st);

}  // namespace game
