// game_internal.cuh -- shared definitions of the CUDA path of libgame.so.
//
// Device data layout (all owned by the handle):
//   Xt   [Mpad/128][N][128] FP32  features (Mpad a multiple of 768), tiled by blocks of 128 patterns and
//                                 feature-major inside a block, so one block is a
//                                 contiguous, 16-byte-aligned run for bulk copies
//                                 and a warp reading one feature of 32 patterns
//                                 touches 128 consecutive bytes.
//   y    [Mpad] FP32              targets, zero past M (masked in the epilogues).
//   pop  [2][P][K] FP32           GA state, ping-pong.
//   fit  [P] FP64                 fitness of the current population.
// Evaluation scratch (grown on demand):
//   popT [Kc][Ppad] FP32          genes 1..K-1 transposed (CUDA-core form).
//   popA [C][KB][na][128][128 B]  genes 1..K-1 in the tcgen05 K-major SWIZZLE_128B
//                                 operand image: na 16 KB blocks per (chromosome
//                                 tile c, K-block kb), bulk-copied unchanged into
//                                 shared memory. BF16: 64 columns per row; bf16x3:
//                                 the hi block then the lo block; FP8 E4M3: 128
//                                 columns per row, genes scaled by colscale[k]
//                                 and 1 / uscale[p].
//   uscale [Ppad] FP32            FP8: per-chromosome scale restored in the epilogue.
//   colscale, colinv [KB*128]     FP8: per-column scales of the expansion (handle-lifetime).
//   a0   [Ppad] FP32              bias genes.
//   part [rows][Ppad] FP64        per-CTA partial sums of squared residuals.
// Elite re-scoring (fixed size, allocated with the handle):
//   cand [16] int32               candidate indices, best first (re-scored by the
//                                 Gram form, gram.cu).
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
// kDevSmemBase: a kernel found its dynamic shared memory less aligned than its
// launch plan assumed and returned before using it
enum DevStatus : int { kDevOk = 0, kDevTimeout = 1, kDevBadShape = 2, kDevSmemBase = 3 };

struct Shape {
  int64_t M, Mpad;
  int N, d, basis, B;
  int K;      // genes, B*N*d + 1
  int Kp;     // K - 1, the contraction length
  int tied;   // Gram form only: 1 = shared genes, K = B*d + 1 over psi = sum_i phi(x_i)
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- test hooks (game_test_hook, api.cu) ----
// True when the device allocation about to be made is the one the
// allocation-failure hook picked (each call counts one allocation).
bool hook_alloc_fails();
// The stall (ns) the next tensor-core fitness launch is to make, 0 for
// none; taking it clears it.
uint64_t hook_take_stall_ns();

// ---- kernels and launchers (defined in the .cu files) ----
// layout.cu
cudaError_t launch_relayout_X(const float* X, const float* y, const Shape& s, float* Xt,
                              float* yp, int* bad_counts, cudaStream_t st);
cudaError_t launch_pack_fp32(const float* pop, int P, int Ppad, const Shape& s, int Kc,
                             float* popT, float* a0, cudaStream_t st);
// full [P][s.K] = the shared-gene population pop [P][B*d + 1] with its genes
// repeated for every feature: full[p][0] = pop[p][0],
// full[p][1 + i B d + c] = pop[p][1 + c]
cudaError_t launch_replicate_tied(const float* pop, int P, const Shape& s, float* full,
                                  cudaStream_t st);
// fitness_fp32.cu
struct Fp32Plan { int BP, BM, Kc, grid_x, grid_y; };
Fp32Plan plan_fp32(const Shape& s, int P, int num_sms);
// err: GAME_ERR_MAE sums absolute residuals, any other value squared ones
cudaError_t launch_fitness_fp32(const Fp32Plan& pl, const Shape& s, const float* Xt,
                                const float* y, const float* popT, const float* a0, int P,
                                int Ppad, double* part, int err, cudaStream_t st);
// fitness_tc.cu -- operand forms of the tensor-core contraction
enum TcForm : int { kFormBF16 = 0, kFormBF16x3 = 1, kFormFP8 = 2 };
// 16 KB gene blocks per (chromosome tile, K-block): hi and lo for bf16x3
__host__ __device__ constexpr int form_na(int f) { return f == kFormBF16x3 ? 2 : 1; }
// expansion images per K-block: hi and lo for bf16x3
__host__ __device__ constexpr int form_nphi(int f) { return f == kFormBF16x3 ? 2 : 1; }
// contraction columns per K-block (one 128-byte swizzled row)
__host__ __device__ constexpr int form_cols(int f) { return f == kFormFP8 ? 128 : 64; }
// NS: expansion K-block slots (KB, or more with spare slots); xstage: 1 when
// the features are staged in shared memory, 0 when read from L2
struct TcPlan {
  int form, BN, KB, NS, xstage, C, stages, grid, smem_bytes, tmem_cols, rows;
  int ystage, slack;   // targets staged in shared memory; bytes kept for base alignment
  int pair;   // 1: the paired-SM kernel (fitness_tc2.cu), C even, grid of 2-CTA clusters
  bool ok;
};
// The launch plan of a tensor-core fitness evaluation. The BF16 form with
// more than one chromosome tile takes the paired-SM kernel where its shared
// memory fits; every other case the one-SM kernel. Ppad = C * 128.
TcPlan plan_tc(const Shape& s, int P, int num_sms, int form);
// Bytes the one-SM tensor-core kernel's dynamic shared memory needs to reach a
// 1024-byte boundary: 1024 (every case) until set_smem_base_pad records what a
// probe found on the GPU; the plans keep that much slack, and the kernel checks.
void set_smem_base_pad(int pad);
int smem_base_pad();
// records a probe's result: the largest padding any probe has found so far
void note_smem_base_pad(int pad);
// test hook: plans keep `slack` bytes (1..1024) whatever the probes found; 0 off
void set_smem_slack_override(int slack);
// writes the probe's padding (0..1023) to *out (device memory) on stream st
cudaError_t launch_smem_base_probe(int* out, cudaStream_t st);
TcPlan plan_tc_pair(const Shape& s, int P, int num_sms);
cudaError_t launch_fitness_tc_pair(const TcPlan& pl, const Shape& s, const float* Xt,
                                   const float* y, const uint8_t* popA, const float* a0, int Ppad,
                                   double* part, int* status, int err, cudaStream_t st);
// err: GAME_ERR_MAE sums absolute residuals, any other value squared ones
cudaError_t launch_fitness_tc(const TcPlan& pl, const Shape& s, const float* Xt,
                              const float* y, const uint8_t* popA, const float* a0,
                              const float* uscale, const float* colinv, int P, int Ppad,
                              double* part, int* status, int err, cudaStream_t st);
// layout.cu: FP8 column scales. colmax [KB*128] receives max_m |phi_k(x_m)|
// as FP32 bit patterns (zero-initialised by the caller); scales turns it into
// colscale = colmax / 448 and colinv = 448 / colmax (0 where colmax is 0).
cudaError_t launch_colmax(const Shape& s, const float* Xt, unsigned int* colmax, int ncols,
                          cudaStream_t st);
cudaError_t launch_colscales(const unsigned int* colmax, int ncols, float* colscale,
                             float* colinv, cudaStream_t st);
cudaError_t launch_pack_tc(int form, const float* pop, int P, int C, const Shape& s, int KB,
                           const float* colscale, uint8_t* popA, float* a0, float* uscale,
                           cudaStream_t st);
// batch_tc.cu -- many problems in one persistent tensor-core launch (BF16)
struct BatchRun {           // one problem, as the batched kernels see it
  const float* Xt;          // [Mpad/128][N][128]
  const float* y;           // [Mpad]
  const uint8_t* popA;      // [C][KB][128][128 B] BF16 operand image
  const float* a0;          // [Ppad]
  int64_t M;
  int64_t part_base;        // first partial row of this problem (doubles)
  int N, d, basis, Kp, K, P, Ppad, C, KB, BN, nmma_last, ntiles;
};
// One work item (problem r, pattern tile t) as every role of the batched
// fitness kernel reads it: one 96-byte load per item, no indirection.
struct alignas(16) BatchItem {
  const float* Xt;          // the problem's features [Mpad/128][N][128]
  const float* y;           // the problem's targets [Mpad]
  const uint8_t* popA;      // the problem's BF16 operand image
  const float* a0;          // the problem's bias genes [Ppad]
  double* prow;             // this tile's partial row: part + part_base_r + t Ppad_r
  int64_t m0;               // first pattern of the tile
  int N, d, basis, Kp, KB, C, BN, nmma_last, valid;
  int CG;                   // chromosome tiles per accumulator set: min(C, 256 / BN)
  int RK;                   // expansion K-block slots: KB, or fewer, a power of two (a ring:
                            // K-block kb in slot kb & (RK - 1)) when the item's chromosome
                            // tiles form one accumulator group
  int pad1;
};
struct BatchArgs {
  const BatchItem* recs;    // the items in the order CTAs take them
  int nitems;
  int* work;                // next item to take (zeroed before each launch)
  int* status;
  int KBmax, set_cols, phi_bytes, tmem_cols;   // accumulator set s at tmem + s set_cols
};
int batch_smem_bytes(int phi_bytes, int KBmax);
// sets the kernel's dynamic shared-memory limit (call outside stream capture)
cudaError_t prepare_fitness_batch(int smem_bytes);
// launch only (capturable)
cudaError_t launch_fitness_batch(const BatchArgs& a, int grid, int smem_bytes, cudaStream_t st);

// rescore.cu: the n best of fit (by (fit, index), NaN last) into cand [n]
cudaError_t launch_select_top(const double* fit, int P, int n, int* cand, cudaStream_t st);
// surrogate.cu -- the MLP fitness surrogate (K -> 256 -> 256 -> 1)
constexpr int kSurrogateHidden = 256;
constexpr float kAdamLr = 1e-3f, kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;
constexpr int kScreenMax = 16384;   // children screened per generation at most
constexpr int kMaxSplits = 32;      // split-K of the surrogate's weight gradients
struct SurrogateDev {
  int K, Bmax;
  int64_t step;            // Adam steps taken
  float* w;                // parameters, FP32 master
  float* g;                // gradient
  float* m;                // Adam moments
  float* v;
  float *Z1, *H1, *Z2, *H2, *dZ1, *dZ2;   // [Bmax][256] workspace
  float *out, *dout, *lterm;              // [Bmax]
  float* loss;             // [1]
  double* tstat;           // [2] mean and sd of the batch's log-fitness
  double* lfit;            // [Bmax] the batch's log-fitness
  float* split_ws;         // [kMaxSplits][256][max(K, 256)] split-K partial products
  int* status;             // the handle's device status word (expired waits)
};
int64_t surrogate_param_count(int K);
cudaError_t surrogate_init(const SurrogateDev& s, uint64_t seed, cudaStream_t st);
cudaError_t surrogate_forward(const SurrogateDev& s, const float* X, int B, float* out,
                              cudaStream_t st);
cudaError_t surrogate_backward(const SurrogateDev& s, const float* X, const double* fit, int B,
                               cudaStream_t st);
cudaError_t surrogate_adam(SurrogateDev& s, cudaStream_t st);
// keeps the n_keep smallest predictions of the n children (slots E..E+n-1 of
// off [E+n][K]) and writes the elites then the kept children in slot order to
// next [E+n_keep][K]; flag [n] (1 = kept) and pos [n] are scratch / outputs.
// (the screening keeps the first n_keep children when *trusted is 0, and
// records the flag it used in *used_trust)
cudaError_t surrogate_screen(int n, int n_keep, int E, int K, const float* pred, int* flag,
                             int* pos, const float* off, float* next, const int* trusted,
                             int* used_trust, cudaStream_t st);
// r = Pearson correlation of the kept children's predictions with their exact
// log-fitness (fit_kept [n_kept] in slot order; their logs go through s.lfit);
// *trusted = r > 0.25.
cudaError_t surrogate_trust_check(const SurrogateDev& s, int n, int n_kept, const float* pred,
                                  const int* flag, const int* pos, const double* fit_kept,
                                  float* r_out, int* trusted, cudaStream_t st);

// gram.cu -- the Gram form of the MSE (FP64)
int64_t gram_chunk_rows(const Shape& s);
// doubles of the build's partial-sum scratch
int64_t gram_part_doubles(const Shape& s, int num_sms);
// G [K][K], b [K], yy [1] of the training set; phi_chunk [gram_chunk_rows][K]
// and part [gram_part_doubles] are scratch.
cudaError_t launch_gram_build(const Shape& s, const float* Xt, const float* y, double* G,
                              double* b, double* yy, double* phi_chunk, double* part,
                              int num_sms, cudaStream_t st);
// fit of the P chromosomes pop [P][K] (idx NULL), or of rows idx[0..P-1]
// written to fit[idx[p]]; err GAME_ERR_MSE or GAME_ERR_RMSE
cudaError_t launch_gram_fitness(const Shape& s, const float* pop, int P, const int* idx,
                                const double* G, const double* b, const double* yy,
                                double* fit, int err, cudaStream_t st);
// the elite re-scoring: n <= kMaxRescore chromosomes pop rows idx[q], spread
// over the GPU; part [gram_small_parts(s) * n] is scratch
int gram_small_parts(const Shape& s);
cudaError_t launch_gram_rescore(const Shape& s, const float* pop, int n, const int* idx,
                                const double* G, const double* b, const double* yy,
                                double* part, double* fit, int err, cudaStream_t st);

// predict.cu: Out(m) of chrom [Kg] in FP64 for M patterns of X (tiled: the
// handle's [Mpad/128][N][128] layout, else row-major [M][N]) into out (may be
// NULL); with counts (may be NULL) adds {TP, FP, TN, FN} against y
cudaError_t launch_predict(const Shape& s, int tied, int Kg, const float* X, bool tiled,
                           int64_t M, const float* chrom, const float* y, double threshold,
                           double* out, unsigned long long* counts, int num_sms,
                           cudaStream_t st);

// api.cu
void record_error(const char* msg);
// reduce.cu
// fit[p] = (sum of the rows) / M, or its square root for GAME_ERR_RMSE
cudaError_t launch_reduce(const double* part, int rows, int P, int Ppad, int64_t M, int err,
                          double* fit, cudaStream_t st);
// ga_ops.cu
struct GaDev {
  int P, K, E, T, I;
  int Nout;   // output slots: P for a generation, more for oversampled offspring
  uint32_t thr_pc, thr_pm;
  float sigma;
  int sel = GAME_SEL_TOURNAMENT;   // GAME_SEL_*
  int* order = nullptr;            // ranking: chromosome of rank r [P]
  uint64_t* cum = nullptr;         // roulette: inclusive weight sums, cum[0] = 0 [P + 1]
};
constexpr int kMaxRankingP = 16384;   // ranking sorts the population in shared memory
cudaError_t launch_init_population(uint64_t seed, int P, int K, float* pop, cudaStream_t st);
cudaError_t launch_generation(const GaDev& ga, const float* pop, const double* fit,
                              uint64_t seed, uint32_t g, int4* plan, float* next,
                              cudaStream_t st);

}  // namespace game
