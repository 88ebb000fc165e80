// batch.cu -- many independent GAME runs advanced together: one launch per
// stage for all runs (operators, operand pack, fused fitness, FP64 reduce),
// the stages of a generation captured once into a CUDA graph.
//
// Every run is the single-problem method of the paper (Section 3: Eq. 2
// outputs, Eq. 3 MSE fitness, elitism / tournament / crossover / mutation on
// genes in [-1, 1]) with its own training set, degree, basis, population
// size and seed; the operators and their random draws are those of
// ga_ops.cu (shared device functions in ga_device.cuh), keyed by the run's
// seed and generation, so run r of a batch follows the same trajectory as a
// single handle with that seed would given the same fitness values.
//
// The fitness of all runs is one persistent tensor-core launch over
// (run, pattern tile) items (batch_tc.cu). The tile width BN of each run is
// given by the caller, or picked per (K-block count, chromosome-tile count)
// bucket by timing the whole launch with the bucket at every feasible width
// (the autotuner), or is the largest feasible width. Fitness values depend on BN
// in their last bits (the FP32 sums inside a tile), so a run is reproducible
// for a given tile choice; game_batch_get_tiles returns the choice.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "ga_device.cuh"
#include "game_internal.cuh"

namespace game {

namespace {

constexpr int kPhiBudget = 156 * 1024;   // expansion K-blocks of one item
constexpr int kMaxSmemBatch = 232448;
constexpr int kMaxKBBatch = 32;          // per-K-block phases live in 32-bit masks

struct BatchGaRun {
  GaDev ga;
  double* fit;
  float* pop[2];
  int4* plan;
  uint64_t seed;
};

// ---------------- batched kernels (blockIdx.y = run, except plan / reduce) ----------------

__global__ void init_batch_kernel(const BatchGaRun* __restrict__ g) {
  const BatchGaRun& R = g[blockIdx.y];
  const int64_t n = (int64_t)R.ga.P * R.ga.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    R.pop[0][e] = ga::init_gene(R.seed, R.ga.K, e);
}

// Genes 1..K-1 of pop[src] to the BF16 operand image (as pack_bf16 in layout.cu).
__global__ void pack_batch_kernel(const BatchRun* __restrict__ runs,
                                  const BatchGaRun* __restrict__ g, int src) {
  const BatchRun& R = runs[blockIdx.y];
  const float* pop = g[blockIdx.y].pop[src];
  const int K = R.K, P = R.P, KB = R.KB;
  uint8_t* popA = const_cast<uint8_t*>(R.popA);
  float* a0 = const_cast<float*>(R.a0);
  const int64_t n = (int64_t)R.C * 128 * KB * 8;
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
        const int kc = kb * 64 + q * 8 + 2 * h + u;
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

__global__ void __launch_bounds__(ga::kPlanThreads)
plan_batch_kernel(const BatchGaRun* __restrict__ g, const uint32_t* __restrict__ gens) {
  const BatchGaRun& R = g[blockIdx.x];
  ga::plan_body(R.ga, R.fit, R.seed, gens[blockIdx.x], R.plan);
}

__global__ void breed_batch_kernel(const BatchGaRun* __restrict__ g,
                                   const uint32_t* __restrict__ gens, int src) {
  const BatchGaRun& R = g[blockIdx.y];
  const uint32_t gen = gens[blockIdx.y];
  const float* pop = R.pop[src];
  float* next = R.pop[src ^ 1];
  const int64_t n = (int64_t)R.ga.Nout * R.ga.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    next[e] = ga::breed_gene(R.ga, pop, R.plan, R.seed, gen, e);
}

// One warp per chromosome of all runs (chrom_begin: prefix sums of P_r):
// fit_r[p] = sum over the run's tiles, in order, / M_r. With
// inc, the run's generation counter advances (the reduce is the last stage
// of a generation).
__global__ void reduce_batch_kernel(const BatchRun* __restrict__ runs,
                                    const BatchGaRun* __restrict__ g,
                                    const int* __restrict__ chrom_begin, int R, int total,
                                    const double* __restrict__ part, uint32_t* __restrict__ gens,
                                    int inc) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= total) return;
  int lo = 0, hi = R - 1;   // last run with chrom_begin <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chrom_begin[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  const BatchRun& B = runs[lo];
  const int p = w - chrom_begin[lo];
  const double* col = part + B.part_base + p;
  double s = 0.0;
  for (int t = lane; t < B.ntiles; t += 32)
    s += col[(int64_t)t * B.Ppad];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    g[lo].fit[p] = s / (double)B.M;
    if (inc && p == 0) gens[lo] += 1u;
  }
}

int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace
}  // namespace game

using namespace game;

struct game_batch {
  int R = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;   // created here: the legacy stream cannot be captured
  int device = 0, num_sms = 0;
  game_params prm{};
  std::vector<Shape> shape;
  std::vector<int> P, C, KB, BN, Ppad;
  std::vector<uint64_t> seed;
  std::vector<int64_t> off_X, off_y, off_pop, off_fit, off_A, off_a0;
  // pooled device arrays (one allocation per kind for all runs)
  float* Xt = nullptr;
  float* y = nullptr;
  float* pop[2] = {nullptr, nullptr};
  double* fit = nullptr;
  int4* plan = nullptr;
  uint8_t* popA = nullptr;
  float* a0 = nullptr;
  uint32_t* gens = nullptr;
  int* status = nullptr;
  int* chrom_begin = nullptr;
  int total_chrom = 0;
  BatchRun* runs_d = nullptr;
  BatchGaRun* ga_d = nullptr;
  // fitness launch of the current tile choice
  BatchItem* recs = nullptr;
  int* work = nullptr;        // the fitness launch's item counter
  double* part = nullptr;
  size_t items_cap = 0, part_cap = 0;
  BatchArgs args{};
  int grid = 0, smem = 0;
  int64_t nitems = 0;
  // graphs of a generation: parity 0 (pop[0] -> pop[1]) and parity 1
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t gen = 0;
};

namespace {

thread_local std::string g_batch_err;

int bfail(int code, const std::string& msg) {
  g_batch_err = msg;
  game::record_error(msg.c_str());
  return code;
}

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(GAME_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (hook_alloc_fails()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
}
void dfree(void* p) {
  if (p) cudaFree(p);
}

bool is_dev(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Expansion K-block slots of an item with KB K-blocks, C chromosome tiles
// and tile width bn: one per K-block when they fit the budget; else a ring
// (K-block kb in slot kb & (slots - 1)) where the item's chromosome tiles
// form one accumulator group, so the MMAs release each K-block as soon as
// they have used it: 4 slots at 256 patterns (one thread per pattern row
// fills the K-blocks in order), 8 at 128 and 16 at 64 patterns (two and four
// threads per row; while the threads' ranges start within the ring's first
// pass they fill side by side, beyond it a thread waits at its first K-block
// for the MMAs of the row's earlier ones, which still beats the next
// narrower tiles); else 0 (the width does not fit).
static_assert(4 * 256 * 128 <= kPhiBudget && 8 * 128 * 128 <= kPhiBudget &&
                  16 * 64 * 128 <= kPhiBudget,
              "ring slots exceed the expansion budget");
int phi_slots(int KB, int C, int bn) {
  if (KB * bn * 128 <= kPhiBudget) return KB;
  if (bn == 256 && C == 1) return 4;
  if (bn == 128 && C <= 2) return 8;
  if (bn == 64 && C <= 4) return 16;
  return 0;
}

bool tile_fits(int KB, int C, int bn) { return phi_slots(KB, C, bn) > 0; }

int heuristic_bn(int KB, int C) {
  for (int bn : {256, 128, 64, 32})
    if (tile_fits(KB, C, bn)) return bn;
  return 0;
}

void fill_run(const game_batch* b, int r, BatchRun& R) {
  const Shape& s = b->shape[r];
  R.Xt = b->Xt + b->off_X[r];
  R.y = b->y + b->off_y[r];
  R.popA = b->popA + b->off_A[r];
  R.a0 = b->a0 + b->off_a0[r];
  R.M = s.M;
  R.part_base = 0;
  R.N = s.N;
  R.d = s.d;
  R.basis = s.basis;
  R.Kp = s.Kp;
  R.K = s.K;
  R.P = b->P[r];
  R.Ppad = b->Ppad[r];
  R.C = b->C[r];
  R.KB = b->KB[r];
  R.BN = b->BN[r];
  const int last_cols = s.Kp - 64 * (R.KB - 1);
  R.nmma_last = (last_cols + 15) / 16;
  R.ntiles = (int)((s.M + R.BN - 1) / R.BN);
}

// Builds the fitness launch for the runs in `which` at the current tile
// widths: run descriptors (with partial-row bases), the item list in
// schedule order, and the shared-memory plan. Uploads through the stream.
int build_launch(game_batch* b, const std::vector<int>& which) {
  std::vector<BatchRun> runs(b->R);
  for (int r = 0; r < b->R; ++r) fill_run(b, r, runs[r]);
  int64_t part_total = 0;
  std::vector<int2> items;
  std::vector<double> cost;
  int KBmax = 1, set_max = 32, phi_bytes = 0;
  for (int r : which) {
    BatchRun& R = runs[r];
    R.part_base = part_total;
    part_total += (int64_t)R.ntiles * R.Ppad;
    const int RK = phi_slots(R.KB, R.C, R.BN);
    if (RK < 1) return bfail(GAME_EINVAL, "tile width does not fit");
    KBmax = std::max(KBmax, RK);   // barrier pairs: one per slot
    set_max = std::max(set_max, std::min(R.C, 256 / R.BN) * R.BN);
    phi_bytes = std::max(phi_bytes, RK * R.BN * 128);
    // cycles per item, roughly: the expansion (64 BN values per K-block at
    // about 4 per cycle, sincosf once per feature for the trigonometric
    // basis), the MMAs (about 2.5 BN per K-block and chromosome tile), the
    // epilogue (about BN per chromosome tile) and a fixed cost
    const double trig = R.basis == GAME_BASIS_TRIG ? 1.0 + 2.0 / R.d : 1.0;
    const double c = (double)R.BN * R.KB * (16.0 * trig + 2.5 * R.C) + (double)R.BN * R.C +
                     3000.0;
    for (int t = 0; t < R.ntiles; ++t) {
      items.push_back(make_int2(r, t));
      cost.push_back(c);
    }
  }
  if (KBmax > kMaxKBBatch) return bfail(GAME_EINVAL, "contraction too long for the batch");
  const int smem = batch_smem_bytes(phi_bytes, KBmax);
  if (smem > kMaxSmemBatch) return bfail(GAME_EINVAL, "batch tiles exceed shared memory");
  BCK(prepare_fitness_batch(smem));   // outside any stream capture
  const int64_t n = (int64_t)items.size();
  const int grid = (int)std::min<int64_t>(b->num_sms, std::max<int64_t>(n, 1));
  // Dynamic schedule: every CTA takes the next item of one list from a
  // global counter, so an SM that runs slower (its loads travel further, for
  // one) simply takes fewer items. The list runs by tile width, widest first
  // (a change of width drains the expansion buffers, so each CTA changes
  // width at most three times), and within a width longest first.
  std::vector<int> sched(n);
  for (int64_t i = 0; i < n; ++i) sched[i] = (int)i;
  std::stable_sort(sched.begin(), sched.end(), [&](int x, int y) {
    const int bx = runs[items[x].x].BN, by = runs[items[y].x].BN;
    return bx != by ? bx > by : cost[x] > cost[y];
  });
  // device buffers (grown on demand)
  if ((size_t)std::max<int64_t>(n, 1) > b->items_cap) {
    dfree(b->recs);
    b->recs = nullptr;
    b->items_cap = 0;
    if (dalloc(&b->recs, (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) {
      cudaGetLastError();
      return bfail(GAME_ENOMEM, "batch item lists");
    }
    b->items_cap = (size_t)std::max<int64_t>(n, 1);
  }
  if ((size_t)std::max<int64_t>(part_total, 1) > b->part_cap) {
    dfree(b->part);
    b->part = nullptr;
    b->part_cap = 0;
    if (dalloc(&b->part, (size_t)std::max<int64_t>(part_total, 1)) != cudaSuccess) {
      cudaGetLastError();
      return bfail(GAME_ENOMEM, "batch partial sums");
    }
    b->part_cap = (size_t)std::max<int64_t>(part_total, 1);
  }
  // the items in CTA order, with everything each role of the kernel reads
  std::vector<BatchItem> recs(sched.size());
  for (size_t k = 0; k < sched.size(); ++k) {
    const int2 it = items[sched[k]];
    const BatchRun& R = runs[it.x];
    BatchItem& I = recs[k];
    I = BatchItem{};
    I.Xt = R.Xt;
    I.y = R.y;
    I.popA = R.popA;
    I.a0 = R.a0;
    I.prow = b->part + R.part_base + (int64_t)it.y * R.Ppad;
    I.m0 = (int64_t)it.y * R.BN;
    I.N = R.N;
    I.d = R.d;
    I.basis = R.basis;
    I.Kp = R.Kp;
    I.KB = R.KB;
    I.C = R.C;
    I.BN = R.BN;
    I.nmma_last = R.nmma_last;
    I.valid = (int)std::min<int64_t>(R.BN, R.M - I.m0);
    I.CG = std::min(R.C, 256 / R.BN);
    I.RK = phi_slots(R.KB, R.C, R.BN);
  }
  BCK(cudaMemcpyAsync(b->runs_d, runs.data(), sizeof(BatchRun) * b->R, cudaMemcpyHostToDevice,
                      b->st));
  if (n > 0)
    BCK(cudaMemcpyAsync(b->recs, recs.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice,
                        b->st));
  BCK(cudaStreamSynchronize(b->st));   // host vectors go out of scope
  BatchArgs& a = b->args;
  a.recs = b->recs;
  a.nitems = (int)n;
  a.work = b->work;
  a.status = b->status;
  a.KBmax = KBmax;
  a.phi_bytes = phi_bytes;
  int cols = 32;
  while (cols < set_max) cols <<= 1;
  a.set_cols = cols;
  a.tmem_cols = 2 * cols;
  b->grid = grid;
  b->smem = smem;
  b->nitems = n;
  return GAME_OK;
}

int launch_fitness(game_batch* b) {
  if (b->nitems == 0) return GAME_OK;
  BCK(cudaMemsetAsync(b->work, 0, sizeof(int), b->st));   // the item counter
  BCK(launch_fitness_batch(b->args, b->grid, b->smem, b->st));
  return GAME_OK;
}

int enqueue_pack(game_batch* b, int src) {
  int maxu = 1, maxg = 1;
  for (int r = 0; r < b->R; ++r) {
    maxu = std::max(maxu, b->C[r] * 128 * b->KB[r] * 8);
    maxg = std::max(maxg, b->P[r] * b->shape[r].K);
  }
  (void)maxg;
  pack_batch_kernel<<<dim3(blocks_for(maxu, 256, 4096), b->R), 256, 0, b->st>>>(b->runs_d,
                                                                                b->ga_d, src);
  BCK(cudaGetLastError());
  return GAME_OK;
}

int enqueue_reduce(game_batch* b, int inc) {
  const int threads = 256;
  const int blocks = (int)(((int64_t)b->total_chrom * 32 + threads - 1) / threads);
  reduce_batch_kernel<<<blocks, threads, 0, b->st>>>(b->runs_d, b->ga_d, b->chrom_begin, b->R,
                                                     b->total_chrom, b->part, b->gens, inc);
  BCK(cudaGetLastError());
  return GAME_OK;
}

int enqueue_operators(game_batch* b, int src) {
  int maxg = 1;
  for (int r = 0; r < b->R; ++r) maxg = std::max(maxg, b->P[r] * b->shape[r].K);
  plan_batch_kernel<<<b->R, ga::kPlanThreads, 0, b->st>>>(b->ga_d, b->gens);
  BCK(cudaGetLastError());
  breed_batch_kernel<<<dim3(blocks_for(maxg, 256, 4096), b->R), 256, 0, b->st>>>(b->ga_d,
                                                                                 b->gens, src);
  BCK(cudaGetLastError());
  return GAME_OK;
}

// Fitness of pop[src] of every run into fit (pack, fused fitness, reduce).
int enqueue_eval(game_batch* b, int src, int inc) {
  int rc = enqueue_pack(b, src);
  if (!rc) rc = launch_fitness(b);
  if (!rc) rc = enqueue_reduce(b, inc);
  return rc;
}

int check_batch_status(game_batch* b) {
  int st = 0;
  BCK(cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  if (st != kDevOk) {
    BCK(cudaMemsetAsync(b->status, 0, sizeof(int), b->st));
    BCK(cudaStreamSynchronize(b->st));
    return bfail(GAME_ETIMEOUT, "a kernel wait timed out; results are void");
  }
  return GAME_OK;
}

// Mean time of the fitness launch over reps launches (after one warm-up).
int time_fitness(game_batch* b, int reps, double* ms) {
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  int rc = launch_fitness(b);
  if (!rc) {
    cudaEventRecord(e0, b->st);
    for (int i = 0; i < reps && !rc; ++i) rc = launch_fitness(b);
    cudaEventRecord(e1, b->st);
  }
  float t = 0.f;
  if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) ==
                                                           cudaSuccess)
    *ms = t / reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) rc = check_batch_status(b);
  return rc;
}

// The autotuner: runs bucketed by (K-block count class, widest feasible
// width, chromosome tiles).
// It starts from the widest feasible width of every run and, bucket by
// bucket (most work first), times the whole launch with the bucket at each
// other width it fits, keeping a width only when the launch gets at least
// 0.5% faster. The whole launch is timed, not the bucket alone: items share
// the SMs through one work counter, so what counts is a bucket's throughput
// next to the others; alone, a small bucket underfills the GPU and narrow
// tiles win on latency. The pack of the current population comes first, so
// the operands are real.
int autotune(game_batch* b) {
  std::vector<std::vector<int>> buckets;
  std::vector<std::pair<int, int>> keys;
  std::vector<double> work;
  for (int r = 0; r < b->R; ++r) {
    int kc = 0;
    while ((1 << kc) < b->KB[r]) ++kc;
    // the widest feasible width is part of the key: one K-block class can
    // hold runs that fit 128-pattern tiles and runs that fit only 64
    const int widest = heuristic_bn(b->KB[r], b->C[r]);
    const std::pair<int, int> key(kc * 512 + widest, b->C[r]);
    size_t i = 0;
    while (i < keys.size() && keys[i] != key) ++i;
    if (i == keys.size()) {
      keys.push_back(key);
      buckets.emplace_back();
      work.push_back(0.0);
    }
    buckets[i].push_back(r);
    work[i] += (double)b->shape[r].M * b->KB[r] * b->C[r];
  }
  std::vector<int> order(buckets.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<int> all(b->R);
  for (int r = 0; r < b->R; ++r) all[r] = r;
  for (int r = 0; r < b->R; ++r) b->BN[r] = heuristic_bn(b->KB[r], b->C[r]);
  int rc = build_launch(b, all);
  if (!rc) rc = enqueue_pack(b, b->cur);
  double ms = 0.0;
  if (!rc) rc = time_fitness(b, 8, &ms);   // clocks up before anything is compared
  for (int i : order) {
    if (rc) break;
    const std::vector<int>& runs = buckets[i];
    const int cur_bn = b->BN[runs[0]];
    int best_bn = cur_bn;
    // the current widths are timed again next to each bucket's trials, so
    // a drift of the clocks between buckets is not read as a gain
    double best = 0.0;
    rc = build_launch(b, all);
    if (!rc) rc = time_fitness(b, 4, &best);
    for (int bn : {256, 128, 64, 32}) {
      if (rc) break;
      bool ok = bn != cur_bn;
      for (int r : runs) ok = ok && tile_fits(b->KB[r], b->C[r], bn);
      if (!ok) continue;
      for (int r : runs) b->BN[r] = bn;
      rc = build_launch(b, all);
      if (!rc) rc = time_fitness(b, 4, &ms);
      if (rc) break;
      if (ms < best * 0.995) {
        best = ms;
        best_bn = bn;
      }
    }
    for (int r : runs) b->BN[r] = best_bn;
  }
  return rc;
}

int capture(game_batch* b, int parity) {
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_operators(b, parity);
  if (!rc) rc = enqueue_eval(b, parity ^ 1, 1);
  cudaError_t e = cudaStreamEndCapture(b->st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bfail(GAME_ECUDA, std::string("graph capture: ") +
                                                     cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return bfail(GAME_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return GAME_OK;
}

void destroy_batch(game_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  for (int p = 0; p < 2; ++p)
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
  dfree(b->Xt);
  dfree(b->y);
  dfree(b->pop[0]);
  dfree(b->pop[1]);
  dfree(b->fit);
  dfree(b->plan);
  dfree(b->popA);
  dfree(b->a0);
  dfree(b->gens);
  dfree(b->status);
  dfree(b->chrom_begin);
  dfree(b->runs_d);
  dfree(b->ga_d);
  dfree(b->recs);
  dfree(b->work);
  dfree(b->part);
  if (b->own_stream) cudaStreamDestroy(b->st);
  delete b;
}

}  // namespace

extern "C" {

int game_batch_create(const game_run_desc* runs, int32_t R, const game_params* prm,
                      const int32_t* tiles, int32_t autotune_tiles, void* cuda_stream,
                      game_batch_t* out) {
  if (!out) return bfail(GAME_EINVAL, "out is NULL");
  *out = nullptr;
  if (!runs || R < 1 || R > 65535) return bfail(GAME_EINVAL, "need 1..65535 runs");
  game_params p;
  if (prm) p = *prm;
  else game_params_default(&p);
  if (p.elitism < 0 || p.elitism > 256 || p.tournament < 1 || p.tournament > kMaxTournament ||
      p.immigrants < 0 || !(p.pc >= 0.f && p.pc <= 1.f) || !(p.pm >= 0.f && p.pm <= 1.f) ||
      !(p.sigma >= 0.f) || !std::isfinite(p.sigma))
    return bfail(GAME_EINVAL, "bad GA settings");
  if (p.selection != GAME_SEL_TOURNAMENT || p.tied != 0 || p.error != GAME_ERR_MSE)
    return bfail(GAME_EINVAL, "batched runs use tournament selection, per-feature genes and MSE");
  game_batch* b = new (std::nothrow) game_batch();
  if (!b) return bfail(GAME_ENOMEM, "batch handle");
  auto bail = [&](int code) {
    destroy_batch(b);
    return code;
  };
  b->R = R;
  b->prm = p;
  b->st = static_cast<cudaStream_t>(cuda_stream);
  if (!b->st) {
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(bfail(GAME_ECUDA, "stream creation"));
    b->own_stream = true;
  }
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) !=
          cudaSuccess)
    return bail(bfail(GAME_ECUDA, "device query"));
  // shapes and pooled sizes
  int64_t nX = 0, ny = 0, npop = 0, nfit = 0, nA = 0, na0 = 0;
  std::vector<int> cb(R);
  for (int r = 0; r < R; ++r) {
    const game_run_desc& d = runs[r];
    if (!d.X || !d.y || d.M < 1 || d.N < 1 || d.degree < 1 ||
        (d.basis != GAME_BASIS_CHEB && d.basis != GAME_BASIS_TRIG))
      return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) + ": bad shape"));
    Shape s{};
    s.M = d.M;
    s.Mpad = ((d.M + 255) / 256) * 256;
    s.N = d.N;
    s.d = d.degree;
    s.basis = d.basis;
    s.B = d.basis == GAME_BASIS_TRIG ? 2 : 1;
    const int64_t K = (int64_t)s.B * d.N * d.degree + 1;
    const int KB = (int)((K - 1 + 63) / 64);
    if (KB > kMaxKBBatch) return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) +
                                                             ": K - 1 above 2048"));
    s.K = (int)K;
    s.Kp = s.K - 1;
    if (d.P < p.elitism + p.immigrants + 2 || d.P > (1 << 20))
      return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) + ": bad population size"));
    const int C = (d.P + 127) / 128;
    if (!tile_fits(KB, C, 32))
      return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) + ": too many features"));
    b->shape.push_back(s);
    b->P.push_back(d.P);
    b->C.push_back(C);
    b->Ppad.push_back(b->C.back() * 128);
    b->KB.push_back(KB);
    b->seed.push_back(d.seed);
    int bn = tiles ? tiles[r] : heuristic_bn(KB, C);
    if (bn != 256 && bn != 128 && bn != 64 && bn != 32)
      return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) + ": tile width not 32..256"));
    if (!tile_fits(KB, C, bn))
      return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) + ": tile too wide"));
    b->BN.push_back(bn);
    b->off_X.push_back(nX);
    b->off_y.push_back(ny);
    b->off_pop.push_back(npop);
    b->off_fit.push_back(nfit);
    b->off_A.push_back(nA);
    b->off_a0.push_back(na0);
    cb[r] = (int)nfit;
    nX += s.Mpad * s.N;
    ny += s.Mpad;
    npop += (int64_t)d.P * K;
    nfit += d.P;
    nA += (int64_t)b->C.back() * KB * 128 * 128;
    na0 += b->Ppad.back();
  }
  if (nfit > 0x7fffffff / 32) return bail(bfail(GAME_EINVAL, "too many chromosomes in total"));
  b->total_chrom = (int)nfit;
  if (dalloc(&b->Xt, nX) != cudaSuccess || dalloc(&b->y, ny) != cudaSuccess ||
      dalloc(&b->pop[0], npop) != cudaSuccess || dalloc(&b->pop[1], npop) != cudaSuccess ||
      dalloc(&b->fit, nfit) != cudaSuccess || dalloc(&b->plan, nfit) != cudaSuccess ||
      dalloc(&b->popA, nA) != cudaSuccess || dalloc(&b->a0, na0) != cudaSuccess ||
      dalloc(&b->gens, R) != cudaSuccess || dalloc(&b->status, 4) != cudaSuccess ||
      dalloc(&b->chrom_begin, R) != cudaSuccess || dalloc(&b->runs_d, R) != cudaSuccess ||
      dalloc(&b->ga_d, R) != cudaSuccess || dalloc(&b->work, 1) != cudaSuccess) {
    cudaGetLastError();
    return bail(bfail(GAME_ENOMEM, "batch device memory"));
  }
  // training sets: staged, validated, tiled
  for (int r = 0; r < R; ++r) {
    const game_run_desc& d = runs[r];
    const Shape& s = b->shape[r];
    const float* dX = d.X;
    const float* dy = d.y;
    float* tX = nullptr;
    float* ty = nullptr;
    cudaError_t e = cudaSuccess;
    if (!is_dev(d.X)) {
      if (dalloc(&tX, (size_t)s.M * s.N) != cudaSuccess) return bail(bfail(GAME_ENOMEM, "X"));
      e = cudaMemcpyAsync(tX, d.X, (size_t)s.M * s.N * 4, cudaMemcpyHostToDevice, b->st);
      dX = tX;
    }
    if (e == cudaSuccess && !is_dev(d.y)) {
      if (dalloc(&ty, (size_t)s.M) != cudaSuccess) {
        dfree(tX);
        return bail(bfail(GAME_ENOMEM, "y"));
      }
      e = cudaMemcpyAsync(ty, d.y, (size_t)s.M * 4, cudaMemcpyHostToDevice, b->st);
      dy = ty;
    }
    int bad[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, 4 * sizeof(int), b->st);
    if (e == cudaSuccess)
      e = launch_relayout_X(dX, dy, s, b->Xt + b->off_X[r], b->y + b->off_y[r], b->status, b->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bad, b->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    dfree(tX);
    dfree(ty);
    if (e != cudaSuccess) return bail(bfail(GAME_ECUDA, std::string("training-set upload: ") +
                                                         cudaGetErrorString(e)));
    if (bad[0] || bad[1]) {
      return bail(bfail(GAME_EINVAL, "run " + std::to_string(r) +
                                         (bad[0] ? ": NaN or Inf in X or y"
                                                 : ": Chebyshev basis needs features in [-1, 1]")));
    }
  }
  // GA descriptors
  std::vector<BatchGaRun> gr(R);
  for (int r = 0; r < R; ++r) {
    GaDev g;
    g.P = b->P[r];
    g.K = b->shape[r].K;
    g.E = p.elitism;
    g.T = p.tournament;
    g.I = p.immigrants;
    g.Nout = g.P;
    g.thr_pc = (uint32_t)floor((double)p.pc * 16777216.0);
    g.thr_pm = (uint32_t)floor((double)p.pm * 16777216.0);
    g.sigma = p.sigma;
    gr[r].ga = g;
    gr[r].fit = b->fit + b->off_fit[r];
    gr[r].pop[0] = b->pop[0] + b->off_pop[r];
    gr[r].pop[1] = b->pop[1] + b->off_pop[r];
    gr[r].plan = b->plan + b->off_fit[r];
    gr[r].seed = b->seed[r];
  }
  if (cudaMemcpyAsync(b->ga_d, gr.data(), sizeof(BatchGaRun) * R, cudaMemcpyHostToDevice,
                      b->st) != cudaSuccess ||
      cudaMemcpyAsync(b->chrom_begin, cb.data(), sizeof(int) * R, cudaMemcpyHostToDevice,
                      b->st) != cudaSuccess ||
      cudaMemsetAsync(b->gens, 0, sizeof(uint32_t) * R, b->st) != cudaSuccess ||
      cudaMemsetAsync(b->status, 0, 4 * sizeof(int), b->st) != cudaSuccess ||
      cudaStreamSynchronize(b->st) != cudaSuccess)
    return bail(bfail(GAME_ECUDA, "batch descriptors"));
  // generation 0
  int maxg = 1;
  for (int r = 0; r < R; ++r) maxg = std::max(maxg, b->P[r] * b->shape[r].K);
  init_batch_kernel<<<dim3(blocks_for(maxg, 256, 4096), R), 256, 0, b->st>>>(b->ga_d);
  if (cudaGetLastError() != cudaSuccess) return bail(bfail(GAME_ECUDA, "init"));
  std::vector<int> all(R);
  for (int r = 0; r < R; ++r) all[r] = r;
  // the full launch first: it uploads the run table the pack kernel reads
  int rc = build_launch(b, all);
  if (!rc && autotune_tiles && !tiles) {
    rc = autotune(b);
    if (!rc) rc = build_launch(b, all);
  }
  if (!rc) rc = enqueue_eval(b, 0, 0);
  if (!rc) rc = check_batch_status(b);
  if (!rc) rc = capture(b, 0);
  if (!rc) rc = capture(b, 1);
  if (rc) return bail(rc);
  *out = b;
  return GAME_OK;
}

int game_batch_generation(game_batch_t b) {
  if (!b) return bfail(GAME_EINVAL, "NULL batch");
  BCK(cudaGraphLaunch(b->exec[b->cur], b->st));
  b->cur ^= 1;
  b->gen += 1;
  return GAME_OK;
}

int game_batch_get_run(game_batch_t b, int32_t r, float* pop_out, double* fit_out,
                       int64_t* generation) {
  if (!b) return bfail(GAME_EINVAL, "NULL batch");
  if (r < 0 || r >= b->R) return bfail(GAME_EINVAL, "run index out of range");
  if (generation) *generation = b->gen;
  const int64_t PK = (int64_t)b->P[r] * b->shape[r].K;
  if (pop_out)
    BCK(cudaMemcpyAsync(pop_out, b->pop[b->cur] + b->off_pop[r], PK * sizeof(float),
                        cudaMemcpyDefault, b->st));
  if (fit_out)
    BCK(cudaMemcpyAsync(fit_out, b->fit + b->off_fit[r], b->P[r] * sizeof(double),
                        cudaMemcpyDefault, b->st));
  return check_batch_status(b);
}

int game_batch_get_tiles(game_batch_t b, int32_t* tiles_out) {
  if (!b || !tiles_out) return bfail(GAME_EINVAL, "NULL argument");
  for (int r = 0; r < b->R; ++r) tiles_out[r] = b->BN[r];
  return GAME_OK;
}

int game_batch_fitness_ms(game_batch_t b, int32_t reps, double* ms_out) {
  if (!b || !ms_out || reps < 1) return bfail(GAME_EINVAL, "bad argument");
  // the population of the current generation, packed (the graph leaves the
  // operand image of the current population in place as well)
  int rc = enqueue_pack(b, b->cur);
  if (rc) return rc;
  return time_fitness(b, reps, ms_out);
}

int game_batch_sync(game_batch_t b) {
  if (!b) return bfail(GAME_EINVAL, "NULL batch");
  return check_batch_status(b);
}

int game_batch_destroy(game_batch_t b) {
  destroy_batch(b);
  return GAME_OK;
}

}  // extern "C"
