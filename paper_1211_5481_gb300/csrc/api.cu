// api.cu -- the C ABI of libgame.so (declared in include/game.h): handle
// lifetime, argument validation, memory-space detection, device buffers and
// the sequencing of the kernels of one evaluation / one generation.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "game_internal.cuh"

using namespace game;

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace game {
// Sets the calling thread's game_last_error() text (used by entry points
// defined outside this file).
void record_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {
std::atomic<int64_t> g_alloc_countdown{0};   // > 0: allocations until the failing one
std::atomic<uint64_t> g_stall_ns{0};
}  // namespace

bool hook_alloc_fails() {
  int64_t n = g_alloc_countdown.load();
  while (n > 0 && !g_alloc_countdown.compare_exchange_weak(n, n - 1)) {
  }
  return n == 1;
}

uint64_t hook_take_stall_ns() { return g_stall_ns.exchange(0); }
}  // namespace game

namespace {

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return GAME_ECUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

// Device pointer test: the driver knows every allocation it made.
bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (hook_alloc_fails()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

}  // namespace

struct game_ctx {
  Shape s{};     // contraction shape: K = B*N*d + 1 expansion columns (with the bias)
  int Kg = 0;    // genes per chromosome: s.K, or B*d + 1 with shared genes
  game_params prm{};
  cudaStream_t st = nullptr;
  int device = 0;
  int num_sms = 0;
  float* Xt = nullptr;
  float* y = nullptr;
  float* pop[2] = {nullptr, nullptr};
  int cur = 0;
  double* fit = nullptr;
  bool fit_valid = false;
  int64_t gen = 0;
  int4* plan = nullptr;
  int* status = nullptr;   // device status word written by kernels
  // elite re-scoring
  int* cand = nullptr;
  // selection tables (ranking order, roulette weight sums)
  int* sel_order = nullptr;
  uint64_t* sel_cum = nullptr;
  // shared genes: the population replicated over features, [P][s.K]
  float* rpop = nullptr;
  size_t rpop_cap = 0;
  // evaluation scratch, grown on demand
  int cap_P = 0;
  float* popT = nullptr;
  uint8_t* popA = nullptr;
  float* a0 = nullptr;
  float* uscale = nullptr;     // FP8: per-chromosome scales [cap_P]
  double* part = nullptr;
  // Gram form of the MSE (built once, at the first GAME_PREC_GRAM use)
  double* G = nullptr;
  double* gb = nullptr;
  double* gyy = nullptr;
  double* gpart = nullptr;    // re-scoring partial sums
  // FP8 column scales of the expansion (computed once, at the first FP8 use)
  unsigned int* colmax = nullptr;
  float* colscale = nullptr;
  float* colinv = nullptr;
  size_t part_cap = 0;
  float* upop = nullptr;    // device copy of a host population
  double* ufit = nullptr;
  int ucap = 0;
  size_t popT_cap = 0, popA_cap = 0;
  // fitness surrogate
  SurrogateDev sd{};
  bool sd_params = false;     // parameters allocated
  float* off = nullptr;       // offspring [Nout][K]
  int4* oplan = nullptr;      // their plan [Nout]
  float* pred = nullptr;      // predictions of the children [kScreenMax]
  int* flag = nullptr;
  int* pos = nullptr;
  int last_n = 0;             // children screened by the last generation
  int* trust = nullptr;       // [2]: the trust check's verdict, the verdict the last screening used
  float* trust_r = nullptr;   // [1]: the trust check's last correlation
  float* rX[2] = {nullptr, nullptr};     // replay: the last two populations
  double* rfit[2] = {nullptr, nullptr};  // and their exact fitness
  int ring_n = 0, ring_head = 0;
  float* uX = nullptr;        // device copies of caller arrays
  double* ufitd = nullptr;
  float* upred = nullptr;
  int sur_cap = 0;
  // per-stage timing
  bool timing = false;
  struct Span {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Span> spans;
  double tot_ms[6] = {0, 0, 0, 0, 0, 0};
  int64_t count[6] = {0, 0, 0, 0, 0, 0};
};

namespace {

enum StageKind {
  kFitness = 0,
  kPack = 1,
  kReduce = 2,
  kOperators = 3,
  kRescore = 4,
  kSurrogate = 5
};

// Records the start event of a timed stage (no-op when timing is off).
cudaEvent_t stage_begin(game_ctx* h) {
  if (!h->timing) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, h->st);
  return e;
}

void harvest_spans(game_ctx* h) {
  for (auto& sp : h->spans) {
    float ms = 0.f;
    if (cudaEventSynchronize(sp.b) == cudaSuccess && cudaEventElapsedTime(&ms, sp.a, sp.b) ==
        cudaSuccess) {
      h->tot_ms[sp.kind] += ms;
      h->count[sp.kind] += 1;
    }
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  h->spans.clear();
}

void stage_end(game_ctx* h, cudaEvent_t start, int kind) {
  if (!start) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaEventDestroy(start);
    return;
  }
  cudaEventRecord(e, h->st);
  h->spans.push_back({start, e, kind});
  if (h->spans.size() > 8192) harvest_spans(h);
}

bool valid_precision(int prec) {
  return prec == GAME_PREC_FP32 || prec == GAME_PREC_BF16 || prec == GAME_PREC_BF16X3 ||
         prec == GAME_PREC_FP8 || prec == GAME_PREC_GRAM;
}

// G, b, yy of the training set (FP64), once per handle; the build's scratch
// (a chunk of the FP64 design matrix and split partial sums) is released.
// Shape of the Gram form: the chromosome's genes (the shared-gene expansion
// psi for a tied handle).
Shape gram_shape(const game_ctx* h) {
  Shape g = h->s;
  g.K = h->Kg;
  g.Kp = h->Kg - 1;
  g.tied = h->prm.tied;
  return g;
}

int ensure_gram(game_ctx* h) {
  if (h->G) return GAME_OK;
  const int K = h->Kg;
  const Shape gs = gram_shape(h);
  const int64_t rows = gram_chunk_rows(gs);
  double* phi = nullptr;
  double* part = nullptr;
  if (dev_alloc(&h->G, (size_t)K * K) != cudaSuccess || dev_alloc(&h->gb, (size_t)K) != cudaSuccess ||
      dev_alloc(&h->gyy, 1) != cudaSuccess ||
      dev_alloc(&h->gpart, (size_t)gram_small_parts(gs) * kMaxRescore) != cudaSuccess ||
      dev_alloc(&phi, (size_t)rows * K) != cudaSuccess ||
      dev_alloc(&part, (size_t)gram_part_doubles(gs, h->num_sms)) != cudaSuccess) {
    cudaGetLastError();
    dev_free(phi);
    dev_free(part);
    dev_free(h->G);
    dev_free(h->gb);
    dev_free(h->gyy);
    dev_free(h->gpart);
    h->G = nullptr;
    h->gb = h->gyy = h->gpart = nullptr;
    return fail(GAME_ENOMEM, "Gram matrix");
  }
  cudaError_t e = launch_gram_build(gs, h->Xt, h->y, h->G, h->gb, h->gyy, phi, part, h->num_sms,
                                    h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  dev_free(phi);
  dev_free(part);
  if (e != cudaSuccess) return cuda_fail(e, "Gram build");
  return GAME_OK;
}

// tensor-core operand form of a reduced-precision GAME_PREC_*
int tc_form(int prec) {
  return prec == GAME_PREC_BF16X3 ? kFormBF16x3 : prec == GAME_PREC_FP8 ? kFormFP8 : kFormBF16;
}

// FP8 per-column scales of the training set's expansion, once per handle.
int ensure_colscales(game_ctx* h) {
  if (h->colinv) return GAME_OK;
  const int ncols = ceil_div(h->s.Kp, 128) * 128;
  if (dev_alloc(&h->colmax, ncols) != cudaSuccess || dev_alloc(&h->colscale, ncols) != cudaSuccess ||
      dev_alloc(&h->colinv, ncols) != cudaSuccess) {
    cudaGetLastError();
    dev_free(h->colmax);
    dev_free(h->colscale);
    dev_free(h->colinv);
    h->colmax = nullptr;
    h->colscale = nullptr;
    h->colinv = nullptr;
    return fail(GAME_ENOMEM, "FP8 column scales");
  }
  CK(cudaMemsetAsync(h->colmax, 0, ncols * sizeof(unsigned int), h->st));
  CK(launch_colmax(h->s, h->Xt, h->colmax, ncols, h->st));
  CK(launch_colscales(h->colmax, ncols, h->colscale, h->colinv, h->st));
  return GAME_OK;
}

// Chromosome rows of the evaluation buffers (a0, partial sums): the
// tensor-core plan's chromosome tiles (paired-SM plans take them in pairs),
// else whole tiles of 128.
int padded_P(game_ctx* h, int P, int prec) {
  if (prec == GAME_PREC_FP32 || prec == GAME_PREC_GRAM) return ceil_div(P, 128) * 128;
  return plan_tc(h->s, P, h->num_sms, tc_form(prec)).C * 128;
}

int ensure_scratch(game_ctx* h, int P, int prec) {
  if (prec == GAME_PREC_GRAM) return ensure_gram(h);
  const int Ppad = padded_P(h, P, prec);
  if (Ppad > h->cap_P) {
    dev_free(h->a0);
    dev_free(h->uscale);
    h->a0 = nullptr;
    h->uscale = nullptr;
    h->cap_P = 0;
    if (dev_alloc(&h->a0, Ppad) != cudaSuccess || dev_alloc(&h->uscale, Ppad) != cudaSuccess) {
      cudaGetLastError();
      return fail(GAME_ENOMEM, "a0 allocation");
    }
    h->cap_P = Ppad;
  }
  if (prec == GAME_PREC_FP32) {
    const Fp32Plan pl = plan_fp32(h->s, P, h->num_sms);
    const size_t need = (size_t)pl.Kc * Ppad;
    if (need > h->popT_cap) {
      dev_free(h->popT);
      h->popT = nullptr;
      h->popT_cap = 0;
      if (dev_alloc(&h->popT, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(GAME_ENOMEM, "popT allocation");
      }
      h->popT_cap = need;
    }
    const size_t pneed = (size_t)pl.grid_y * Ppad;
    if (pneed > h->part_cap) {
      dev_free(h->part);
      h->part = nullptr;
      h->part_cap = 0;
      if (dev_alloc(&h->part, pneed) != cudaSuccess) {
        cudaGetLastError();
        return fail(GAME_ENOMEM, "partials");
      }
      h->part_cap = pneed;
    }
  } else {
    const TcPlan pl = plan_tc(h->s, P, h->num_sms, tc_form(prec));
    if (!pl.ok)
      return fail(GAME_EINVAL, "contraction length too large for the tensor-core path");
    if (pl.form == kFormFP8) {
      const int rc = ensure_colscales(h);
      if (rc) return rc;
    }
    const size_t need = (size_t)pl.C * pl.KB * form_na(pl.form) * 128 * 128;
    if (need > h->popA_cap) {
      dev_free(h->popA);
      h->popA = nullptr;
      h->popA_cap = 0;
      if (dev_alloc(&h->popA, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(GAME_ENOMEM, "popA allocation");
      }
      h->popA_cap = need;
    }
    const size_t pneed = (size_t)pl.rows * Ppad;
    if (pneed > h->part_cap) {
      dev_free(h->part);
      h->part = nullptr;
      h->part_cap = 0;
      if (dev_alloc(&h->part, pneed) != cudaSuccess) {
        cudaGetLastError();
        return fail(GAME_ENOMEM, "partials");
      }
      h->part_cap = pneed;
    }
  }
  return GAME_OK;
}

// The shared-gene population dpop [P][Kg] replicated over the features into
// h->rpop [P][s.K] for the direct forms.
int replicate_tied(game_ctx* h, const float* dpop, int P) {
  const size_t need = (size_t)P * h->s.K;
  if (need > h->rpop_cap) {
    dev_free(h->rpop);
    h->rpop = nullptr;
    h->rpop_cap = 0;
    if (dev_alloc(&h->rpop, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(GAME_ENOMEM, "replicated population");
    }
    h->rpop_cap = need;
  }
  cudaEvent_t t0 = stage_begin(h);
  CK(launch_replicate_tied(dpop, P, h->s, h->rpop, h->st));
  stage_end(h, t0, kPack);
  return GAME_OK;
}

// Enqueues the fitness of a device population dpop [P][Kg] into dfit [P];
// with sums, the unnormalised error sums instead (sum over the handle's
// patterns of the squared residuals, of the absolute ones for the MAE).
int eval_device(game_ctx* h, const float* dpop, int P, int prec, double* dfit,
                bool sums = false) {
  const int err = h->prm.error;
  if (prec == GAME_PREC_GRAM && err == GAME_ERR_MAE)
    return fail(GAME_EINVAL, "the MAE has no Gram form");
  if (prec == GAME_PREC_GRAM && sums)
    return fail(GAME_EINVAL, "error sums need a direct form (not GAME_PREC_GRAM)");
  // the reduce divides by rM (and takes the root for the RMSE)
  const int64_t rM = sums ? 1 : h->s.M;
  const int rerr = sums ? (err == GAME_ERR_MAE ? GAME_ERR_MAE : GAME_ERR_MSE) : err;
  int rc = ensure_scratch(h, P, prec);
  if (rc) return rc;
  const int Ppad = padded_P(h, P, prec);
  cudaEvent_t t0;
  if (prec == GAME_PREC_GRAM) {
    t0 = stage_begin(h);
    CK(launch_gram_fitness(gram_shape(h), dpop, P, nullptr, h->G, h->gb, h->gyy, dfit, err,
                           h->st));
    stage_end(h, t0, kFitness);
    return GAME_OK;
  }
  if (h->prm.tied) {
    rc = replicate_tied(h, dpop, P);
    if (rc) return rc;
    dpop = h->rpop;
  }
  if (prec == GAME_PREC_FP32) {
    const Fp32Plan pl = plan_fp32(h->s, P, h->num_sms);
    t0 = stage_begin(h);
    CK(launch_pack_fp32(dpop, P, Ppad, h->s, pl.Kc, h->popT, h->a0, h->st));
    stage_end(h, t0, kPack);
    t0 = stage_begin(h);
    CK(launch_fitness_fp32(pl, h->s, h->Xt, h->y, h->popT, h->a0, P, Ppad, h->part, err,
                           h->st));
    stage_end(h, t0, kFitness);
    t0 = stage_begin(h);
    CK(launch_reduce(h->part, pl.grid_y, P, Ppad, rM, rerr, dfit, h->st));
    stage_end(h, t0, kReduce);
  } else {
    const TcPlan pl = plan_tc(h->s, P, h->num_sms, tc_form(prec));
    t0 = stage_begin(h);
    CK(launch_pack_tc(pl.form, dpop, P, pl.C, h->s, pl.KB, h->colscale, h->popA, h->a0,
                      h->uscale, h->st));
    stage_end(h, t0, kPack);
    t0 = stage_begin(h);
    CK(launch_fitness_tc(pl, h->s, h->Xt, h->y, h->popA, h->a0, h->uscale, h->colinv, P, Ppad,
                         h->part, h->status, err, h->st));
    stage_end(h, t0, kFitness);
    t0 = stage_begin(h);
    CK(launch_reduce(h->part, pl.rows, P, Ppad, rM, rerr, dfit, h->st));
    stage_end(h, t0, kReduce);
  }
  return GAME_OK;
}

int ensure_gram(game_ctx* h);

// Enqueues the re-scoring of the n best entries of dfit (device arrays):
// the candidates' FP64 fitness by the Gram form.
int rescore_device(game_ctx* h, const float* dpop, int P, int n, double* dfit) {
  if (h->prm.error == GAME_ERR_MAE) return fail(GAME_EINVAL, "the MAE has no Gram form to re-score with");
  int rc = ensure_gram(h);
  if (rc) return rc;
  cudaEvent_t t0 = stage_begin(h);
  CK(launch_select_top(dfit, P, n, h->cand, h->st));
  CK(launch_gram_rescore(gram_shape(h), dpop, n, h->cand, h->G, h->gb, h->gyy, h->gpart, dfit,
                         h->prm.error, h->st));
  stage_end(h, t0, kRescore);
  return GAME_OK;
}

// Fitness of the GA population: the contraction in the handle's precision,
// then, for the reduced-precision forms, the re-scoring of the best
// candidates before the operators rank them.
int eval_state(game_ctx* h) {
  int rc = eval_device(h, h->pop[h->cur], h->prm.P, h->prm.precision, h->fit);
  if (rc) return rc;
  const int n = h->prm.rescore_top < h->prm.P ? h->prm.rescore_top : h->prm.P;
  if (h->prm.precision != GAME_PREC_FP32 && h->prm.precision != GAME_PREC_GRAM && n > 0)
    return rescore_device(h, h->pop[h->cur], h->prm.P, n, h->fit);
  return GAME_OK;
}

// Surrogate parameters (once) and a workspace for at least `rows` rows.
int ensure_surrogate(game_ctx* h, int rows) {
  SurrogateDev& s = h->sd;
  if (!h->sd_params) {
    const int64_t n = surrogate_param_count(h->Kg);
    s.K = h->Kg;
    if (dev_alloc(&s.w, n) != cudaSuccess || dev_alloc(&s.g, n) != cudaSuccess ||
        dev_alloc(&s.m, n) != cudaSuccess || dev_alloc(&s.v, n) != cudaSuccess ||
        dev_alloc(&s.loss, 1) != cudaSuccess || dev_alloc(&s.tstat, 2) != cudaSuccess ||
        dev_alloc(&s.split_ws, (size_t)kMaxSplits * kSurrogateHidden *
                                   (h->Kg > kSurrogateHidden ? h->Kg : kSurrogateHidden)) !=
            cudaSuccess) {
      cudaGetLastError();
      return fail(GAME_ENOMEM, "surrogate parameters");
    }
    h->sd_params = true;
    s.step = 0;
    s.status = h->status;
    CK(surrogate_init(s, h->prm.seed, h->st));
  }
  if (rows > s.Bmax) {
    float** bufs[6] = {&s.Z1, &s.H1, &s.Z2, &s.H2, &s.dZ1, &s.dZ2};
    for (float** b : bufs) {
      dev_free(*b);
      *b = nullptr;
    }
    dev_free(s.out);
    dev_free(s.dout);
    dev_free(s.lterm);
    dev_free(s.lfit);
    s.out = s.dout = s.lterm = nullptr;
    s.lfit = nullptr;
    s.Bmax = 0;
    for (float** b : bufs)
      if (dev_alloc(b, (size_t)rows * kSurrogateHidden) != cudaSuccess) {
        cudaGetLastError();
        return fail(GAME_ENOMEM, "surrogate workspace");
      }
    if (dev_alloc(&s.out, rows) != cudaSuccess || dev_alloc(&s.dout, rows) != cudaSuccess ||
        dev_alloc(&s.lterm, rows) != cudaSuccess || dev_alloc(&s.lfit, rows) != cudaSuccess) {
      cudaGetLastError();
      return fail(GAME_ENOMEM, "surrogate workspace");
    }
    s.Bmax = rows;
  }
  return GAME_OK;
}

// One Adam step of the surrogate on device pairs (X [n][K], fit [n]).
int surrogate_step(game_ctx* h, const float* X, const double* fit, int n) {
  int rc = ensure_surrogate(h, n);
  if (rc) return rc;
  CK(surrogate_forward(h->sd, X, n, h->sd.out, h->st));
  CK(surrogate_backward(h->sd, X, fit, n, h->st));
  CK(surrogate_adam(h->sd, h->st));
  return GAME_OK;
}

// Adds the current population and its exact fitness to the replay ring and
// trains surrogate_steps rounds of one step on each stored generation,
// oldest first.
int surrogate_learn(game_ctx* h) {
  const int P = h->prm.P, K = h->Kg;
  const int slot = h->ring_head;
  CK(cudaMemcpyAsync(h->rX[slot], h->pop[h->cur], (size_t)P * K * sizeof(float),
                     cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(h->rfit[slot], h->fit, (size_t)P * sizeof(double),
                     cudaMemcpyDeviceToDevice, h->st));
  h->ring_head ^= 1;
  if (h->ring_n < 2) h->ring_n += 1;
  for (int rep = 0; rep < h->prm.surrogate_steps; ++rep)
    for (int i = h->ring_n - 1; i >= 0; --i) {
      const int sl = (slot - i + 2) % 2;
      const int rc = surrogate_step(h, h->rX[sl], h->rfit[sl], P);
      if (rc) return rc;
    }
  return GAME_OK;
}

// Buffers of the screened generation; the surrogate warm-started on the
// current population (20 steps).
int setup_screening(game_ctx* h) {
  const int P = h->prm.P, K = h->Kg, E = h->prm.elitism;
  const int n = h->prm.oversample * (P - E);
  if (dev_alloc(&h->off, (size_t)(E + n) * K) != cudaSuccess ||
      dev_alloc(&h->oplan, (size_t)(E + n)) != cudaSuccess ||
      dev_alloc(&h->pred, (size_t)n) != cudaSuccess || dev_alloc(&h->flag, (size_t)n) != cudaSuccess ||
      dev_alloc(&h->pos, (size_t)n) != cudaSuccess ||
      dev_alloc(&h->rX[0], (size_t)P * K) != cudaSuccess ||
      dev_alloc(&h->rX[1], (size_t)P * K) != cudaSuccess ||
      dev_alloc(&h->rfit[0], (size_t)P) != cudaSuccess ||
      dev_alloc(&h->rfit[1], (size_t)P) != cudaSuccess || dev_alloc(&h->trust, 2) != cudaSuccess ||
      dev_alloc(&h->trust_r, 1) != cudaSuccess) {
    cudaGetLastError();
    return fail(GAME_ENOMEM, "screening buffers");
  }
  CK(cudaMemsetAsync(h->trust, 0, 2 * sizeof(int), h->st));   // untrusted until checked
  CK(cudaMemsetAsync(h->trust_r, 0, sizeof(float), h->st));
  int rc = ensure_surrogate(h, n > P ? n : P);
  for (int i = 0; i < 20 && !rc; ++i) rc = surrogate_step(h, h->pop[h->cur], h->fit, P);
  return rc;
}

int check_status(game_ctx* h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (st != kDevOk) {
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
    CK(cudaStreamSynchronize(h->st));
    if (st == kDevSmemBase)
      return fail(GAME_ECUDA, "dynamic shared memory less aligned than planned; results are void");
    return fail(GAME_ETIMEOUT, "a kernel wait timed out; results of the affected calls are void");
  }
  return GAME_OK;
}

// Device copies of a host population and its fitness, for P chromosomes.
int ensure_upload(game_ctx* h, int P) {
  if (P <= h->ucap) return GAME_OK;
  dev_free(h->upop);
  dev_free(h->ufit);
  h->upop = nullptr;
  h->ufit = nullptr;
  h->ucap = 0;
  if (dev_alloc(&h->upop, (size_t)P * h->Kg) != cudaSuccess ||
      dev_alloc(&h->ufit, (size_t)P) != cudaSuccess) {
    cudaGetLastError();
    dev_free(h->upop);
    h->upop = nullptr;
    return fail(GAME_ENOMEM, "device copy of the population");
  }
  h->ucap = P;
  return GAME_OK;
}

int validate_params(const game_params& p, const Shape& s, std::string* why) {
  for (int r : p.reserved)
    if (r != 0) {
      *why = "reserved fields must be zero";
      return 0;
    }
  if (p.elitism < 0 || p.elitism > 256) {
    *why = "elitism must be in 0..256";
    return 0;
  }
  if (p.tournament < 1 || p.tournament > kMaxTournament) {
    *why = "tournament must be in 1..64";
    return 0;
  }
  if (p.immigrants < 0) {
    *why = "immigrants must be >= 0";
    return 0;
  }
  const int64_t P = p.P == 0 ? (int64_t)s.B * s.N + 1 : p.P;
  if (P < (int64_t)p.elitism + p.immigrants + 2 || P > (1 << 24)) {
    *why = "population size must be >= elitism + immigrants + 2 (and <= 2^24)";
    return 0;
  }
  if (!(p.pc >= 0.f && p.pc <= 1.f) || !(p.pm >= 0.f && p.pm <= 1.f)) {
    *why = "rates must be in [0, 1]";
    return 0;
  }
  if (!(p.sigma >= 0.f) || !isfinite(p.sigma)) {
    *why = "sigma must be finite and >= 0";
    return 0;
  }
  if (!valid_precision(p.precision)) {
    *why = "unknown precision";
    return 0;
  }
  if (p.surrogate != 0 && p.surrogate != 1) {
    *why = "surrogate must be 0 or 1";
    return 0;
  }
  if (p.surrogate &&
      (p.oversample < 1 || (int64_t)p.oversample * ((p.P == 0 ? (int64_t)s.B * s.N + 1 : p.P) -
                                                    p.elitism) > kScreenMax)) {
    *why = "oversample must be >= 1 with oversample * (P - elitism) <= 16384";
    return 0;
  }
  if (p.rescore_top < 0 || p.rescore_top > kMaxRescore) {
    *why = "rescore_top must be in 0..16";
    return 0;
  }
  if (p.check_every < 0) {
    *why = "check_every must be >= 0";
    return 0;
  }
  if (p.selection < GAME_SEL_TOURNAMENT || p.selection > GAME_SEL_ROULETTE) {
    *why = "unknown selection";
    return 0;
  }
  if (p.selection == GAME_SEL_RANKING && P > kMaxRankingP) {
    *why = "ranking selection needs P <= 16384";
    return 0;
  }
  if (p.tied != 0 && p.tied != 1) {
    *why = "tied must be 0 or 1";
    return 0;
  }
  if (p.error < GAME_ERR_MSE || p.error > GAME_ERR_MAE) {
    *why = "unknown error function";
    return 0;
  }
  if (p.surrogate_steps < 0 || p.surrogate_steps > 64 || (p.surrogate && p.surrogate_steps < 1)) {
    *why = "surrogate_steps must be in 1..64";
    return 0;
  }
  if (p.error == GAME_ERR_MAE && (p.precision == GAME_PREC_GRAM || p.rescore_top != 0)) {
    *why = "the MAE has no Gram form: use a direct precision and rescore_top = 0";
    return 0;
  }
  return 1;
}

GaDev ga_dev(const game_ctx* h) {
  GaDev g;
  g.sel = h->prm.selection;
  g.order = h->sel_order;
  g.cum = h->sel_cum;
  g.P = h->prm.P;
  g.K = h->Kg;
  g.E = h->prm.elitism;
  g.T = h->prm.tournament;
  g.I = h->prm.immigrants;
  g.Nout = g.P;
  g.thr_pc = (uint32_t)floor((double)h->prm.pc * 16777216.0);
  g.thr_pm = (uint32_t)floor((double)h->prm.pm * 16777216.0);
  g.sigma = h->prm.sigma;
  return g;
}

void destroy_ctx(game_ctx* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  harvest_spans(h);
  dev_free(h->Xt);
  dev_free(h->y);
  dev_free(h->pop[0]);
  dev_free(h->pop[1]);
  dev_free(h->fit);
  dev_free(h->plan);
  dev_free(h->status);
  dev_free(h->cand);
  dev_free(h->sel_order);
  dev_free(h->sel_cum);
  dev_free(h->rpop);
  dev_free(h->popT);
  dev_free(h->popA);
  dev_free(h->a0);
  dev_free(h->uscale);
  dev_free(h->G);
  dev_free(h->gb);
  dev_free(h->gyy);
  dev_free(h->gpart);
  dev_free(h->colmax);
  dev_free(h->colscale);
  dev_free(h->colinv);
  dev_free(h->part);
  dev_free(h->upop);
  dev_free(h->ufit);
  SurrogateDev& s = h->sd;
  float* sb[] = {s.w, s.g, s.m, s.v, s.Z1, s.H1, s.Z2, s.H2, s.dZ1, s.dZ2, s.out, s.dout,
                 s.lterm, s.loss, s.split_ws, h->off, h->pred, h->rX[0], h->rX[1], h->uX,
                 h->upred};
  for (float* b : sb) dev_free(b);
  dev_free(h->oplan);
  dev_free(h->flag);
  dev_free(h->pos);
  dev_free(h->rfit[0]);
  dev_free(h->rfit[1]);
  dev_free(h->ufitd);
  dev_free(h->trust);
  dev_free(h->trust_r);
  dev_free(h->sd.tstat);
  dev_free(h->sd.lfit);
  delete h;
}

int copy_in(game_ctx* h, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->st));
  return GAME_OK;
}

}  // namespace

extern "C" {

const char* game_last_error(void) { return g_last_error.c_str(); }

int game_test_hook(int32_t hook, int64_t value) {
  g_last_error.clear();
  if (value < 0) return fail(GAME_EINVAL, "hook value must be >= 0");
  if (hook == GAME_HOOK_FAIL_ALLOC) {
    g_alloc_countdown.store(value);
  } else if (hook == GAME_HOOK_STALL_NS) {
    if (value > 1000000000) return fail(GAME_EINVAL, "stall limited to 1 s");
    g_stall_ns.store((uint64_t)value);
  } else if (hook == GAME_HOOK_SMEM_SLACK) {
    if (value > 1024) return fail(GAME_EINVAL, "slack limited to 1024 bytes");
    set_smem_slack_override((int)value);
  } else {
    return fail(GAME_EINVAL, "unknown hook");
  }
  return GAME_OK;
}

int game_params_default(game_params* out) {
  if (!out) return fail(GAME_EINVAL, "out is NULL");
  memset(out, 0, sizeof(*out));
  out->P = 0;
  out->elitism = 2;
  out->tournament = 3;
  out->precision = GAME_PREC_FP32;
  out->immigrants = 0;
  out->check_every = 10;
  out->pc = 0.9f;
  out->pm = 0.02f;
  out->sigma = 0.1f;
  out->mse_threshold = 0.0;
  out->seed = 1;
  out->rescore_top = 16;
  out->surrogate = 0;
  out->oversample = 8;
  out->selection = GAME_SEL_TOURNAMENT;
  out->tied = 0;
  out->error = GAME_ERR_MSE;
  out->surrogate_steps = 8;
  return GAME_OK;
}

int game_create(const float* X, const float* y, int64_t M, int32_t N, int32_t degree,
                int32_t basis, const game_params* prm, void* cuda_stream, game_t* out) {
  g_last_error.clear();
  if (!out) return fail(GAME_EINVAL, "out is NULL");
  *out = nullptr;
  if (!X || !y) return fail(GAME_EINVAL, "X and y must not be NULL");
  if (M < 1 || N < 1 || degree < 1) return fail(GAME_EINVAL, "M, N and degree must be >= 1");
  if (basis != GAME_BASIS_CHEB && basis != GAME_BASIS_TRIG)
    return fail(GAME_EINVAL, "unknown basis");
  Shape s{};
  s.M = M;
  s.Mpad = ((M + 767) / 768) * 768;   // every pattern-tile width divides 768
  s.N = N;
  s.d = degree;
  s.basis = basis;
  s.B = basis == GAME_BASIS_TRIG ? 2 : 1;
  const int64_t K = (int64_t)s.B * N * degree + 1;
  if (K > kMaxK) return fail(GAME_EINVAL, "K = B*N*d + 1 exceeds 4097 genes");
  s.K = (int)K;
  s.Kp = s.K - 1;
  if ((int64_t)N * s.Mpad > ((int64_t)1 << 36)) return fail(GAME_EINVAL, "training set too large");

  game_params p;
  if (prm) p = *prm;
  else game_params_default(&p);
  std::string why;
  if (!validate_params(p, s, &why)) return fail(GAME_EINVAL, why);
  if (p.P == 0) p.P = s.B * N + 1;   // Eq. 4
  const int Kg = p.tied ? s.B * degree + 1 : s.K;   // Eq. 5 with shared genes

  game_ctx* h = new (std::nothrow) game_ctx();
  if (!h) return fail(GAME_ENOMEM, "handle allocation");
  h->s = s;
  h->Kg = Kg;
  h->prm = p;
  h->st = static_cast<cudaStream_t>(cuda_stream);
  int rc = GAME_OK;
  auto bail = [&](int code) {
    destroy_ctx(h);
    return code;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) return bail(cuda_fail(e, "multiprocessor count"));

  if (dev_alloc(&h->Xt, (size_t)s.Mpad * N) != cudaSuccess ||
      dev_alloc(&h->y, (size_t)s.Mpad) != cudaSuccess ||
      dev_alloc(&h->pop[0], (size_t)p.P * Kg) != cudaSuccess ||
      dev_alloc(&h->pop[1], (size_t)p.P * Kg) != cudaSuccess ||
      dev_alloc(&h->fit, (size_t)p.P) != cudaSuccess ||
      dev_alloc(&h->plan, (size_t)p.P) != cudaSuccess ||
      dev_alloc(&h->status, 4) != cudaSuccess ||
      dev_alloc(&h->cand, kMaxRescore) != cudaSuccess ||
      (p.selection == GAME_SEL_RANKING && dev_alloc(&h->sel_order, (size_t)p.P) != cudaSuccess) ||
      (p.selection == GAME_SEL_ROULETTE &&
       dev_alloc(&h->sel_cum, (size_t)p.P + 1) != cudaSuccess)) {
    cudaGetLastError();
    return bail(fail(GAME_ENOMEM, "device allocation of the training set / GA state"));
  }
  // training set: device copies in the tiled layout, validated on the way
  const float* dX = X;
  const float* dy = y;
  float* tmpX = nullptr;
  float* tmpy = nullptr;
  if (!is_device_ptr(X)) {
    if (dev_alloc(&tmpX, (size_t)M * N) != cudaSuccess)
      return bail(fail(GAME_ENOMEM, "staging copy of X"));
    e = cudaMemcpyAsync(tmpX, X, (size_t)M * N * sizeof(float), cudaMemcpyHostToDevice, h->st);
    dX = tmpX;
  }
  if (e == cudaSuccess && !is_device_ptr(y)) {
    if (dev_alloc(&tmpy, (size_t)M) != cudaSuccess) {
      dev_free(tmpX);
      return bail(fail(GAME_ENOMEM, "staging copy of y"));
    }
    e = cudaMemcpyAsync(tmpy, y, (size_t)M * sizeof(float), cudaMemcpyHostToDevice, h->st);
    dy = tmpy;
  }
  int bad_h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, 4 * sizeof(int), h->st);
  if (e == cudaSuccess) e = launch_relayout_X(dX, dy, s, h->Xt, h->y, h->status, h->st);
  // where dynamic shared memory starts, for the tensor-core launch plans
  if (e == cudaSuccess) e = launch_smem_base_probe(h->status + 2, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bad_h, h->status, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, 4 * sizeof(int), h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  dev_free(tmpX);
  dev_free(tmpy);
  if (e != cudaSuccess) return bail(cuda_fail(e, "training-set upload"));
  note_smem_base_pad(bad_h[2]);
  if (bad_h[0]) return bail(fail(GAME_EINVAL, "X or y holds NaN or Inf"));
  if (bad_h[1]) return bail(fail(GAME_EINVAL, "Chebyshev basis needs features in [-1, 1]"));

  // generation 0: uniform genes, then their fitness
  e = launch_init_population(p.seed, p.P, Kg, h->pop[0], h->st);
  if (e != cudaSuccess) return bail(cuda_fail(e, "init population"));
  rc = eval_state(h);
  if (rc) return bail(rc);
  h->fit_valid = true;
  if (p.surrogate) {
    rc = setup_screening(h);
    if (rc) return bail(rc);
  }
  rc = check_status(h);
  if (rc) return bail(rc);
  h->gen = 0;
  *out = h;
  return GAME_OK;
}

int game_get_shape(game_t h, int64_t* M, int32_t* N, int32_t* K, int32_t* P) {
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  if (M) *M = h->s.M;
  if (N) *N = h->s.N;
  if (K) *K = h->Kg;
  if (P) *P = h->prm.P;
  return GAME_OK;
}

int game_plan_info(game_t h, int32_t precision, int32_t P, int32_t* info) {
  g_last_error.clear();
  if (!h || !info) return fail(GAME_EINVAL, "NULL argument");
  if (P < 1 || P > (1 << 24)) return fail(GAME_EINVAL, "P must be in 1..2^24");
  if (!valid_precision(precision)) return fail(GAME_EINVAL, "unknown precision");
  for (int i = 0; i < 8; ++i) info[i] = 0;
  if (precision == GAME_PREC_GRAM) {
    info[0] = GAME_KERNEL_GRAM;
    return GAME_OK;
  }
  if (precision == GAME_PREC_FP32) {
    const Fp32Plan pl = plan_fp32(h->s, P, h->num_sms);
    info[0] = GAME_KERNEL_FP32;
    info[1] = pl.BM;
    info[6] = pl.grid_x * pl.grid_y;
    return GAME_OK;
  }
  const TcPlan pl = plan_tc(h->s, P, h->num_sms, tc_form(precision));
  if (!pl.ok) return fail(GAME_EINVAL, "contraction length too large for the tensor-core path");
  info[0] = pl.pair ? GAME_KERNEL_TC_PAIR : GAME_KERNEL_TC;
  info[1] = pl.BN;
  info[2] = pl.KB;
  info[3] = pl.stages;
  info[4] = pl.NS;
  info[5] = pl.xstage;
  info[6] = pl.grid;
  info[7] = pl.smem_bytes;
  return GAME_OK;
}

int game_eval_fitness_prec(game_t h, const float* pop, int32_t P, int32_t precision,
                           double* fit_out) {
  g_last_error.clear();
  if (!h || !pop || !fit_out) return fail(GAME_EINVAL, "NULL argument");
  if (P < 1 || P > (1 << 24)) return fail(GAME_EINVAL, "P must be in 1..2^24");
  if (!valid_precision(precision)) return fail(GAME_EINVAL, "unknown precision");
  const bool dev_in = is_device_ptr(pop), dev_out = is_device_ptr(fit_out);
  if (dev_in != dev_out) return fail(GAME_EINVAL, "pop and fit_out must be in the same memory");
  if (dev_in) return eval_device(h, pop, P, precision, fit_out);
  int rc = ensure_upload(h, P);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->upop, pop, (size_t)P * h->Kg * sizeof(float), cudaMemcpyHostToDevice,
                     h->st));
  rc = eval_device(h, h->upop, P, precision, h->ufit);
  if (rc) return rc;
  CK(cudaMemcpyAsync(fit_out, h->ufit, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  return check_status(h);
}

int game_eval_fitness(game_t h, const float* pop, int32_t P, double* fit_out) {
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  return game_eval_fitness_prec(h, pop, P, h->prm.precision, fit_out);
}

int game_rescore_top(game_t h, const float* pop, int32_t P, double* fit, int32_t n,
                     int32_t* idx_out) {
  g_last_error.clear();
  if (!h || !pop || !fit) return fail(GAME_EINVAL, "NULL argument");
  if (P < 1 || P > (1 << 24)) return fail(GAME_EINVAL, "P must be in 1..2^24");
  if (n < 1 || n > kMaxRescore || n > P) return fail(GAME_EINVAL, "n must be in 1..min(16, P)");
  const bool dev_in = is_device_ptr(pop), dev_fit = is_device_ptr(fit);
  if (dev_in != dev_fit) return fail(GAME_EINVAL, "pop and fit must be in the same memory");
  int rc;
  if (dev_in) {
    rc = rescore_device(h, pop, P, n, fit);
  } else {
    rc = ensure_upload(h, P);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->upop, pop, (size_t)P * h->Kg * sizeof(float),
                       cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->ufit, fit, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, h->st));
    rc = rescore_device(h, h->upop, P, n, h->ufit);
    if (rc) return rc;
    CK(cudaMemcpyAsync(fit, h->ufit, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  }
  if (rc) return rc;
  if (idx_out)
    CK(cudaMemcpyAsync(idx_out, h->cand, (size_t)n * sizeof(int32_t), cudaMemcpyDefault, h->st));
  if (!dev_in || (idx_out && !is_device_ptr(idx_out))) return check_status(h);
  return GAME_OK;
}

int game_generation(game_t h, uint64_t seed) {
  g_last_error.clear();
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  if (h->gen >= 0xFFFFFFFFll) return fail(GAME_ESTATE, "generation counter exhausted");
  int rc;
  if (!h->fit_valid) {
    rc = eval_state(h);
    if (rc) return rc;
    h->fit_valid = true;
  }
  if (h->prm.surrogate) {
    // oversampled offspring, screened by the surrogate
    GaDev g = ga_dev(h);
    const int E = h->prm.elitism, P = h->prm.P, K = h->Kg;
    const int n = h->prm.oversample * (P - E);
    g.Nout = E + n;
    cudaEvent_t t0 = stage_begin(h);
    CK(launch_generation(g, h->pop[h->cur], h->fit, seed, (uint32_t)h->gen, h->oplan, h->off,
                         h->st));
    stage_end(h, t0, kOperators);
    t0 = stage_begin(h);
    rc = ensure_surrogate(h, n);
    if (rc) return rc;
    CK(surrogate_forward(h->sd, h->off + (size_t)E * K, n, h->pred, h->st));
    CK(surrogate_screen(n, P - E, E, K, h->pred, h->flag, h->pos, h->off, h->pop[h->cur ^ 1],
                        h->trust, h->trust + 1, h->st));
    stage_end(h, t0, kSurrogate);
    h->last_n = n;
    h->cur ^= 1;
    h->gen += 1;
    h->fit_valid = false;
    rc = eval_state(h);
    if (rc) return rc;
    h->fit_valid = true;
    t0 = stage_begin(h);
    CK(surrogate_trust_check(h->sd, n, P - E, h->pred, h->flag, h->pos, h->fit + E, h->trust_r,
                             h->trust, h->st));
    rc = surrogate_learn(h);
    stage_end(h, t0, kSurrogate);
    return rc;
  }
  cudaEvent_t t0 = stage_begin(h);
  CK(launch_generation(ga_dev(h), h->pop[h->cur], h->fit, seed, (uint32_t)h->gen, h->plan,
                       h->pop[h->cur ^ 1], h->st));
  stage_end(h, t0, kOperators);
  h->cur ^= 1;
  h->gen += 1;
  h->fit_valid = false;
  rc = eval_state(h);
  if (rc) return rc;
  h->fit_valid = true;
  return GAME_OK;
}

int game_train(game_t h, int32_t generations, int32_t* generations_run) {
  g_last_error.clear();
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  if (generations < 0) return fail(GAME_EINVAL, "generations must be >= 0");
  if (generations_run) *generations_run = 0;
  const int every = h->prm.check_every > 0 ? h->prm.check_every : 1;
  const bool use_stop = h->prm.mse_threshold > 0.0;
  double* fit_h = nullptr;
  if (use_stop) {
    fit_h = new (std::nothrow) double[h->prm.P];
    if (!fit_h) return fail(GAME_ENOMEM, "host fitness buffer");
  }
  int rc = GAME_OK;
  int done = 0;
  for (; done < generations; ++done) {
    if (use_stop && done % every == 0) {
      cudaError_t e = cudaMemcpyAsync(fit_h, h->fit, sizeof(double) * h->prm.P,
                                      cudaMemcpyDeviceToHost, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "stop-rule readback");
        break;
      }
      double best = INFINITY;
      for (int p = 0; p < h->prm.P; ++p)
        if (fit_h[p] < best) best = fit_h[p];
      if (best < h->prm.mse_threshold) break;
    }
    rc = game_generation(h, h->prm.seed);
    if (rc) break;
  }
  delete[] fit_h;
  if (generations_run) *generations_run = done;
  if (rc) return rc;
  return check_status(h);
}

int game_get_population(game_t h, float* pop_out, double* fit_out, int64_t* generation) {
  g_last_error.clear();
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  if (generation) *generation = h->gen;
  bool host = false;
  if (pop_out) {
    host |= !is_device_ptr(pop_out);
    CK(cudaMemcpyAsync(pop_out, h->pop[h->cur], (size_t)h->prm.P * h->Kg * sizeof(float),
                       cudaMemcpyDefault, h->st));
  }
  if (fit_out) {
    if (!h->fit_valid) {
      int rc = eval_state(h);
      if (rc) return rc;
      h->fit_valid = true;
    }
    host |= !is_device_ptr(fit_out);
    CK(cudaMemcpyAsync(fit_out, h->fit, (size_t)h->prm.P * sizeof(double), cudaMemcpyDefault,
                       h->st));
  }
  if (host) return check_status(h);
  return GAME_OK;
}

int game_set_state(game_t h, const float* pop, const double* fit, int64_t generation) {
  g_last_error.clear();
  if (!h || !pop) return fail(GAME_EINVAL, "NULL argument");
  if (generation < 0 || generation >= 0xFFFFFFFFll) return fail(GAME_EINVAL, "bad generation");
  int rc = copy_in(h, h->pop[h->cur], pop, (size_t)h->prm.P * h->Kg * sizeof(float));
  if (rc) return rc;
  if (fit) {
    rc = copy_in(h, h->fit, fit, (size_t)h->prm.P * sizeof(double));
    if (rc) return rc;
  } else {
    rc = eval_state(h);
    if (rc) return rc;
  }
  h->fit_valid = true;
  h->gen = generation;
  return check_status(h);
}

int game_eval_sse(game_t h, const float* pop, int32_t P, double* sse_out) {
  g_last_error.clear();
  if (!h || !sse_out) return fail(GAME_EINVAL, "NULL argument");
  if (!pop) P = h->prm.P;
  if (P < 1 || P > (1 << 24)) return fail(GAME_EINVAL, "P must be in 1..2^24");
  const bool dev_out = is_device_ptr(sse_out);
  if (pop && is_device_ptr(pop) != dev_out)
    return fail(GAME_EINVAL, "pop and sse_out must be in the same memory");
  const float* dpop = pop ? pop : h->pop[h->cur];
  int rc;
  if (pop && !dev_out) {
    rc = ensure_upload(h, P);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->upop, pop, (size_t)P * h->Kg * sizeof(float), cudaMemcpyHostToDevice,
                       h->st));
    dpop = h->upop;
  } else if (!dev_out) {
    rc = ensure_upload(h, P);
    if (rc) return rc;
  }
  double* dsse = dev_out ? sse_out : h->ufit;
  rc = eval_device(h, dpop, P, h->prm.precision, dsse, true);
  if (rc) return rc;
  if (!dev_out)
    CK(cudaMemcpyAsync(sse_out, dsse, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  return dev_out ? GAME_OK : check_status(h);
}

int game_breed(game_t h, uint64_t seed) {
  g_last_error.clear();
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  if (h->prm.surrogate)
    return fail(GAME_ESTATE, "surrogate handles breed inside game_generation only");
  if (!h->fit_valid) return fail(GAME_ESTATE, "the current population has no fitness");
  if (h->gen >= 0xFFFFFFFFll) return fail(GAME_ESTATE, "generation counter exhausted");
  cudaEvent_t t0 = stage_begin(h);
  CK(launch_generation(ga_dev(h), h->pop[h->cur], h->fit, seed, (uint32_t)h->gen, h->plan,
                       h->pop[h->cur ^ 1], h->st));
  stage_end(h, t0, kOperators);
  h->cur ^= 1;
  h->gen += 1;
  h->fit_valid = false;
  return GAME_OK;
}

int game_set_fitness(game_t h, const double* fit) {
  g_last_error.clear();
  if (!h || !fit) return fail(GAME_EINVAL, "NULL argument");
  int rc = copy_in(h, h->fit, fit, (size_t)h->prm.P * sizeof(double));
  if (rc) return rc;
  h->fit_valid = true;
  return is_device_ptr(fit) ? GAME_OK : check_status(h);
}

int game_set_timing(game_t h, int32_t enable) {
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  harvest_spans(h);
  for (int k = 0; k < 6; ++k) {
    h->tot_ms[k] = 0.0;
    h->count[k] = 0;
  }
  h->timing = enable != 0;
  return GAME_OK;
}

int game_get_timing(game_t h, game_timing* out) {
  if (!h || !out) return fail(GAME_EINVAL, "NULL argument");
  harvest_spans(h);
  out->fitness_ms = h->tot_ms[kFitness];
  out->pack_ms = h->tot_ms[kPack];
  out->reduce_ms = h->tot_ms[kReduce];
  out->operators_ms = h->tot_ms[kOperators];
  out->fitness_launches = h->count[kFitness];
  out->pack_launches = h->count[kPack];
  out->reduce_launches = h->count[kReduce];
  out->operators_launches = h->count[kOperators];
  out->rescore_ms = h->tot_ms[kRescore];
  out->rescore_launches = h->count[kRescore];
  out->surrogate_ms = h->tot_ms[kSurrogate];
  out->surrogate_launches = h->count[kSurrogate];
  return GAME_OK;
}

// ---- fitness surrogate ----

namespace {
// Device copies of caller arrays for the surrogate calls (n rows).
int surrogate_inputs(game_ctx* h, const float* pop, const double* fit, int n) {
  if (n > h->sur_cap) {
    dev_free(h->uX);
    dev_free(h->ufitd);
    dev_free(h->upred);
    h->uX = nullptr;
    h->ufitd = nullptr;
    h->upred = nullptr;
    h->sur_cap = 0;
    if (dev_alloc(&h->uX, (size_t)n * h->Kg) != cudaSuccess ||
        dev_alloc(&h->ufitd, (size_t)n) != cudaSuccess ||
        dev_alloc(&h->upred, (size_t)n) != cudaSuccess) {
      cudaGetLastError();
      return fail(GAME_ENOMEM, "surrogate inputs");
    }
    h->sur_cap = n;
  }
  CK(cudaMemcpyAsync(h->uX, pop, (size_t)n * h->Kg * sizeof(float), cudaMemcpyDefault, h->st));
  if (fit) CK(cudaMemcpyAsync(h->ufitd, fit, (size_t)n * sizeof(double), cudaMemcpyDefault, h->st));
  return ensure_surrogate(h, n);
}
}  // namespace

int game_surrogate_predict(game_t h, const float* pop, int32_t n, float* pred_out) {
  g_last_error.clear();
  if (!h || !pop || !pred_out || n < 1) return fail(GAME_EINVAL, "bad argument");
  int rc = surrogate_inputs(h, pop, nullptr, n);
  if (rc) return rc;
  CK(surrogate_forward(h->sd, h->uX, n, h->upred, h->st));
  CK(cudaMemcpyAsync(pred_out, h->upred, (size_t)n * sizeof(float), cudaMemcpyDefault, h->st));
  return check_status(h);
}

int game_surrogate_grad(game_t h, const float* pop, const double* fit, int32_t n,
                        float* grad_out, float* loss_out) {
  g_last_error.clear();
  if (!h || !pop || !fit || !grad_out || n < 1) return fail(GAME_EINVAL, "bad argument");
  int rc = surrogate_inputs(h, pop, fit, n);
  if (rc) return rc;
  CK(surrogate_forward(h->sd, h->uX, n, h->sd.out, h->st));
  CK(surrogate_backward(h->sd, h->uX, h->ufitd, n, h->st));
  CK(cudaMemcpyAsync(grad_out, h->sd.g, surrogate_param_count(h->Kg) * sizeof(float),
                     cudaMemcpyDefault, h->st));
  if (loss_out) CK(cudaMemcpyAsync(loss_out, h->sd.loss, sizeof(float), cudaMemcpyDefault, h->st));
  return check_status(h);
}

int game_surrogate_train(game_t h, const float* pop, const double* fit, int32_t n) {
  g_last_error.clear();
  if (!h || !pop || !fit || n < 1) return fail(GAME_EINVAL, "bad argument");
  int rc = surrogate_inputs(h, pop, fit, n);
  if (rc) return rc;
  rc = surrogate_step(h, h->uX, h->ufitd, n);
  if (rc) return rc;
  return check_status(h);
}

int game_surrogate_params(game_t h, float* w_out, int64_t* count) {
  g_last_error.clear();
  if (!h || !count) return fail(GAME_EINVAL, "bad argument");
  *count = surrogate_param_count(h->Kg);
  if (!w_out) return GAME_OK;
  int rc = ensure_surrogate(h, 1);
  if (rc) return rc;
  CK(cudaMemcpyAsync(w_out, h->sd.w, *count * sizeof(float), cudaMemcpyDefault, h->st));
  return check_status(h);
}

int game_surrogate_set_params(game_t h, const float* w) {
  g_last_error.clear();
  if (!h || !w) return fail(GAME_EINVAL, "bad argument");
  int rc = ensure_surrogate(h, 1);
  if (rc) return rc;
  const int64_t n = surrogate_param_count(h->Kg);
  CK(cudaMemcpyAsync(h->sd.w, w, n * sizeof(float), cudaMemcpyDefault, h->st));
  CK(cudaMemsetAsync(h->sd.m, 0, n * sizeof(float), h->st));
  CK(cudaMemsetAsync(h->sd.v, 0, n * sizeof(float), h->st));
  h->sd.step = 0;
  return check_status(h);
}

int game_surrogate_last(game_t h, float* pred_out, int32_t* keep_out, int32_t* n_out,
                        int32_t* trusted_out, float* r_out) {
  g_last_error.clear();
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  if (n_out) *n_out = h->last_n;
  if (h->last_n == 0) return GAME_OK;
  if (trusted_out)
    CK(cudaMemcpyAsync(trusted_out, h->trust + 1, sizeof(int32_t), cudaMemcpyDefault, h->st));
  if (r_out) CK(cudaMemcpyAsync(r_out, h->trust_r, sizeof(float), cudaMemcpyDefault, h->st));
  if (pred_out)
    CK(cudaMemcpyAsync(pred_out, h->pred, (size_t)h->last_n * sizeof(float), cudaMemcpyDefault,
                       h->st));
  if (keep_out)
    CK(cudaMemcpyAsync(keep_out, h->flag, (size_t)h->last_n * sizeof(int32_t), cudaMemcpyDefault,
                       h->st));
  return check_status(h);
}

int game_gram(game_t h, double* G_out, double* b_out, double* yy_out) {
  g_last_error.clear();
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  int rc = ensure_gram(h);
  if (rc) return rc;
  const int K = h->Kg;
  if (G_out) CK(cudaMemcpyAsync(G_out, h->G, (size_t)K * K * sizeof(double), cudaMemcpyDefault, h->st));
  if (b_out) CK(cudaMemcpyAsync(b_out, h->gb, (size_t)K * sizeof(double), cudaMemcpyDefault, h->st));
  if (yy_out) CK(cudaMemcpyAsync(yy_out, h->gyy, sizeof(double), cudaMemcpyDefault, h->st));
  return check_status(h);
}

namespace {

// Device copy of a host or device array for the duration of one call.
struct DevCopy {
  void* p = nullptr;
  bool owned = false;
  ~DevCopy() {
    if (owned) cudaFree(p);
  }
};

int dev_view(game_ctx* h, const void* src, size_t bytes, DevCopy* out) {
  if (!src || bytes == 0) return GAME_OK;
  if (is_device_ptr(src)) {
    out->p = const_cast<void*>(src);
    return GAME_OK;
  }
  if (cudaMalloc(&out->p, bytes) != cudaSuccess) {
    cudaGetLastError();
    out->p = nullptr;
    return fail(GAME_ENOMEM, "device copy of a caller array");
  }
  out->owned = true;
  CK(cudaMemcpyAsync(out->p, src, bytes, cudaMemcpyHostToDevice, h->st));
  return GAME_OK;
}

// Shared argument handling of game_predict / game_classify: the chromosome
// and the patterns (the training set when X is NULL) on the device.
int predict_inputs(game_ctx* h, const float* chrom, const float* X, const float* y, int64_t M,
                   bool need_y, DevCopy* dchrom, DevCopy* dX, DevCopy* dy, bool* tiled) {
  if (!chrom) return fail(GAME_EINVAL, "chrom is NULL");
  if (M < 0) return fail(GAME_EINVAL, "M must be >= 0");
  if (!X) {
    if (need_y && y) return fail(GAME_EINVAL, "X and y must both be given or both be NULL");
    if (M != h->s.M) return fail(GAME_EINVAL, "M must equal the training set's M when X is NULL");
    *tiled = true;
  } else {
    if (need_y && !y) return fail(GAME_EINVAL, "y is NULL");
    *tiled = false;
  }
  int rc = dev_view(h, chrom, (size_t)h->Kg * sizeof(float), dchrom);
  if (!rc && X) rc = dev_view(h, X, (size_t)M * h->s.N * sizeof(float), dX);
  if (!rc && X && need_y) rc = dev_view(h, y, (size_t)M * sizeof(float), dy);
  return rc;
}

}  // namespace

int game_predict(game_t h, const float* chrom, const float* X, int64_t M, double* out) {
  g_last_error.clear();
  if (!h || !out) return fail(GAME_EINVAL, "NULL argument");
  DevCopy dchrom, dX, dy, dout;
  bool tiled = false;
  int rc = predict_inputs(h, chrom, X, nullptr, M, false, &dchrom, &dX, &dy, &tiled);
  if (rc) return rc;
  if (M == 0) return GAME_OK;
  const bool dev_out = is_device_ptr(out);
  if (dev_out) {
    dout.p = out;
  } else if (cudaMalloc(&dout.p, (size_t)M * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    dout.p = nullptr;
    return fail(GAME_ENOMEM, "device outputs");
  } else {
    dout.owned = true;
  }
  const float* Xd = tiled ? h->Xt : static_cast<const float*>(dX.p);
  CK(launch_predict(h->s, h->prm.tied, h->Kg, Xd, tiled, M, static_cast<const float*>(dchrom.p),
                    nullptr, 0.0, static_cast<double*>(dout.p), nullptr, h->num_sms, h->st));
  if (dev_out && !dchrom.owned && !dX.owned) return GAME_OK;   // enqueued only
  if (!dev_out)
    CK(cudaMemcpyAsync(out, dout.p, (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));   // before the temporary copies are freed
  return check_status(h);
}

int game_classify(game_t h, const float* chrom, const float* X, const float* y, int64_t M,
                  double threshold, game_confusion* out) {
  g_last_error.clear();
  if (!h || !out) return fail(GAME_EINVAL, "NULL argument");
  if (threshold != threshold) return fail(GAME_EINVAL, "threshold is NaN");
  DevCopy dchrom, dX, dy, dcnt;
  bool tiled = false;
  int rc = predict_inputs(h, chrom, X, y, M, true, &dchrom, &dX, &dy, &tiled);
  if (rc) return rc;
  unsigned long long cnt[4] = {0, 0, 0, 0};
  if (M > 0) {
    if (cudaMalloc(&dcnt.p, 4 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      dcnt.p = nullptr;
      return fail(GAME_ENOMEM, "counters");
    }
    dcnt.owned = true;
    CK(cudaMemsetAsync(dcnt.p, 0, 4 * sizeof(unsigned long long), h->st));
    const float* Xd = tiled ? h->Xt : static_cast<const float*>(dX.p);
    const float* yd = tiled ? h->y : static_cast<const float*>(dy.p);
    CK(launch_predict(h->s, h->prm.tied, h->Kg, Xd, tiled, M,
                      static_cast<const float*>(dchrom.p), yd, threshold, nullptr,
                      static_cast<unsigned long long*>(dcnt.p), h->num_sms, h->st));
    CK(cudaMemcpyAsync(cnt, dcnt.p, sizeof(cnt), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    rc = check_status(h);
    if (rc) return rc;
  }
  out->tp = (int64_t)cnt[0];
  out->fp = (int64_t)cnt[1];
  out->tn = (int64_t)cnt[2];
  out->fn = (int64_t)cnt[3];
  const int64_t total = out->tp + out->fp + out->tn + out->fn;
  out->accuracy = total ? (double)(out->tp + out->tn) / (double)total : 0.0;
  out->completeness = out->tp + out->fn ? (double)out->tp / (double)(out->tp + out->fn) : 0.0;
  out->contamination = out->tp + out->fp ? (double)out->fp / (double)(out->tp + out->fp) : 0.0;
  return GAME_OK;
}

namespace {

// ---- checkpoint file ----
// Layout (host byte order): CkptHeader, pop [P][K] FP32, fit [P] FP64; with
// the surrogate, then w, m, v [n] FP32, trust [2] int32, trust_r FP32, the
// replay ring rX [2][P][K] FP32 and rfit [2][P] FP64.
constexpr char kCkptMagic[8] = {'G', 'A', 'M', 'E', 'C', 'K', 'P', '1'};

struct CkptHeader {
  char magic[8];
  int64_t M, generation, sur_step, sur_params;
  uint64_t seed;
  int32_t N, degree, basis, tied, K, P, surrogate, ring_n, ring_head, last_n;
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

// host staging of one device array, written to / read from the file
int dump(game_ctx* h, FILE* f, const void* dev, size_t bytes) {
  std::vector<char> buf(bytes);
  CK(cudaMemcpyAsync(buf.data(), dev, bytes, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (fwrite(buf.data(), 1, bytes, f) != bytes) return fail(GAME_EINVAL, "checkpoint write failed");
  return GAME_OK;
}

int undump(game_ctx* h, FILE* f, void* dev, size_t bytes) {
  std::vector<char> buf(bytes);
  if (fread(buf.data(), 1, bytes, f) != bytes) return fail(GAME_EINVAL, "checkpoint truncated");
  CK(cudaMemcpyAsync(dev, buf.data(), bytes, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return GAME_OK;
}

CkptHeader header_of(const game_ctx* h) {
  CkptHeader c;
  memset(&c, 0, sizeof(c));
  memcpy(c.magic, kCkptMagic, 8);
  c.M = h->s.M;
  c.generation = h->gen;
  c.seed = h->prm.seed;
  c.N = h->s.N;
  c.degree = h->s.d;
  c.basis = h->s.basis;
  c.tied = h->prm.tied;
  c.K = h->Kg;
  c.P = h->prm.P;
  c.surrogate = h->prm.surrogate;
  if (h->prm.surrogate) {
    c.sur_step = h->sd.step;
    c.sur_params = surrogate_param_count(h->Kg);
    c.ring_n = h->ring_n;
    c.ring_head = h->ring_head;
    c.last_n = h->last_n;
  }
  return c;
}

}  // namespace

int game_save(game_t h, const char* path) {
  g_last_error.clear();
  if (!h || !path) return fail(GAME_EINVAL, "NULL argument");
  if (!h->fit_valid) {
    int rc = eval_state(h);
    if (rc) return rc;
    h->fit_valid = true;
  }
  CK(cudaStreamSynchronize(h->st));
  int rc = check_status(h);
  if (rc) return rc;
  const std::string tmp = std::string(path) + ".tmp";
  File file;
  file.f = fopen(tmp.c_str(), "wb");
  if (!file.f) return fail(GAME_EINVAL, "cannot open the checkpoint file for writing");
  const CkptHeader c = header_of(h);
  const size_t P = (size_t)h->prm.P, K = (size_t)h->Kg;
  if (fwrite(&c, sizeof(c), 1, file.f) != 1) return fail(GAME_EINVAL, "checkpoint write failed");
  rc = dump(h, file.f, h->pop[h->cur], P * K * sizeof(float));
  if (!rc) rc = dump(h, file.f, h->fit, P * sizeof(double));
  if (!rc && h->prm.surrogate) {
    const size_t n = (size_t)c.sur_params * sizeof(float);
    rc = dump(h, file.f, h->sd.w, n);
    if (!rc) rc = dump(h, file.f, h->sd.m, n);
    if (!rc) rc = dump(h, file.f, h->sd.v, n);
    if (!rc) rc = dump(h, file.f, h->trust, 2 * sizeof(int));
    if (!rc) rc = dump(h, file.f, h->trust_r, sizeof(float));
    for (int i = 0; i < 2 && !rc; ++i) rc = dump(h, file.f, h->rX[i], P * K * sizeof(float));
    for (int i = 0; i < 2 && !rc; ++i) rc = dump(h, file.f, h->rfit[i], P * sizeof(double));
  }
  if (rc) return rc;
  if (fclose(file.f) != 0) {
    file.f = nullptr;
    return fail(GAME_EINVAL, "checkpoint write failed");
  }
  file.f = nullptr;
  if (rename(tmp.c_str(), path) != 0) return fail(GAME_EINVAL, "cannot move the checkpoint in place");
  return GAME_OK;
}

int game_load(game_t h, const char* path) {
  g_last_error.clear();
  if (!h || !path) return fail(GAME_EINVAL, "NULL argument");
  File file;
  file.f = fopen(path, "rb");
  if (!file.f) return fail(GAME_EINVAL, "cannot open the checkpoint file");
  CkptHeader c;
  if (fread(&c, sizeof(c), 1, file.f) != 1) return fail(GAME_EINVAL, "checkpoint truncated");
  const CkptHeader mine = header_of(h);
  if (memcmp(c.magic, kCkptMagic, 8) != 0) return fail(GAME_EINVAL, "not a GAME checkpoint");
  if (c.M != mine.M || c.N != mine.N || c.degree != mine.degree || c.basis != mine.basis ||
      c.tied != mine.tied || c.K != mine.K || c.P != mine.P || c.surrogate != mine.surrogate ||
      (c.surrogate && c.sur_params != mine.sur_params))
    return fail(GAME_EINVAL, "checkpoint of a different shape or settings");
  if (c.generation < 0 || c.generation >= 0xFFFFFFFFll ||
      (c.surrogate && (c.ring_n < 0 || c.ring_n > 2 || c.ring_head < 0 || c.ring_head > 1 ||
                       c.sur_step < 0 || c.last_n < 0)))
    return fail(GAME_EINVAL, "corrupt checkpoint header");
  const size_t P = (size_t)h->prm.P, K = (size_t)h->Kg;
  // the whole file is checked for its length before any state is replaced
  size_t want = sizeof(CkptHeader) + P * K * sizeof(float) + P * sizeof(double);
  if (c.surrogate)
    want += 3 * (size_t)c.sur_params * sizeof(float) + 2 * sizeof(int) + sizeof(float) +
            2 * P * K * sizeof(float) + 2 * P * sizeof(double);
  if (fseek(file.f, 0, SEEK_END) != 0 || ftell(file.f) != (long)want ||
      fseek(file.f, (long)sizeof(CkptHeader), SEEK_SET) != 0)
    return fail(GAME_EINVAL, "checkpoint of the wrong length");
  int rc = undump(h, file.f, h->pop[h->cur], P * K * sizeof(float));
  if (!rc) rc = undump(h, file.f, h->fit, P * sizeof(double));
  if (!rc && c.surrogate) {
    const size_t n = (size_t)c.sur_params * sizeof(float);
    rc = undump(h, file.f, h->sd.w, n);
    if (!rc) rc = undump(h, file.f, h->sd.m, n);
    if (!rc) rc = undump(h, file.f, h->sd.v, n);
    if (!rc) rc = undump(h, file.f, h->trust, 2 * sizeof(int));
    if (!rc) rc = undump(h, file.f, h->trust_r, sizeof(float));
    for (int i = 0; i < 2 && !rc; ++i) rc = undump(h, file.f, h->rX[i], P * K * sizeof(float));
    for (int i = 0; i < 2 && !rc; ++i) rc = undump(h, file.f, h->rfit[i], P * sizeof(double));
    if (!rc) {
      h->sd.step = c.sur_step;
      h->ring_n = c.ring_n;
      h->ring_head = c.ring_head;
      h->last_n = c.last_n;
    }
  }
  if (rc) {
    h->fit_valid = false;   // state partly replaced: re-evaluated before use
    return rc;
  }
  h->fit_valid = true;
  h->gen = c.generation;
  return GAME_OK;
}

int game_sync(game_t h) {
  if (!h) return fail(GAME_EINVAL, "NULL handle");
  return check_status(h);
}

int game_destroy(game_t h) {
  destroy_ctx(h);
  return GAME_OK;
}

}  // extern "C"
