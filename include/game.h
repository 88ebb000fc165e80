/*
 * game.h -- C ABI of libgame.so: GAME population fitness evaluation and
 * genetic operators on one NVIDIA GB300 (sm_103a).
 *
 * Method: Cavuoti, Garofalo, Brescia, Pescape, Longo, Ventre, "Genetic
 * Algorithm Modeling with GPU Parallel Computing Technology",
 * arXiv:1211.5481. Section numbers and equations below are that paper's.
 *
 * Notation: M patterns (the paper's NP), N features per pattern, d degree,
 * B = 1 (Chebyshev basis T_j) or 2 (trigonometric basis cos(jx), sin(jx),
 * the paper's "polytrigo", Eq. 6), K = B*N*d + 1 genes per chromosome,
 * P chromosomes. Chromosome p is a row pop[p][0..K-1] of FP32 genes:
 * gene 0 is the bias a_0 and gene 1 + i*B*d + b*d + (j-1) weights
 * phi_{b,j}(x_i) (b = 0: T_j or cos(j x); b = 1: sin(j x)).
 *
 * Fitness is the mean squared error of Eq. 3 over all M patterns
 * (Section 3; Section 5 sets MSE as the error function), lower is better.
 * Also offered (game_params.error): its square root (RMSE) and the mean
 * absolute difference (MAE), the other errors Section 3 names.
 *
 * Shared genes (game_params.tied = 1): Eq. 2 as printed indexes the genes by
 * basis group and degree only, common to every feature, so a chromosome has
 * K = B*d + 1 genes (Eq. 5): gene 0 is a_0 and gene 1 + b*d + (j-1) weights
 * sum_i phi_{b,j}(x_i). Every K below is then B*d + 1.
 *
 * Conventions for every call:
 *  - Returns GAME_OK (0) or a negative GAME_E* code; game_last_error()
 *    then describes the failure (thread-local string, valid until the
 *    calling thread's next call).
 *  - Pointers are "host or device": the library asks the CUDA driver which
 *    kind each pointer is. Device pointers must be on the handle's device.
 *  - All GPU work goes on the stream given to game_create. Calls with host
 *    output pointers synchronise that stream before returning; calls whose
 *    outputs are device pointers only enqueue work (use game_sync).
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Arrays are row-major and owned by the caller; the handle owns its own
 *    device copies.
 */
#ifndef GAME_H
#define GAME_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GAME_OK 0
#define GAME_EINVAL (-1)   /* bad argument, shape, value or non-finite data */
#define GAME_ENOMEM (-2)   /* host or device allocation failed */
#define GAME_ECUDA (-3)    /* CUDA runtime error (message has the details) */
#define GAME_ETIMEOUT (-4) /* a kernel's bounded wait ran out; results void */
#define GAME_ESTATE (-5)   /* call not valid in the handle's current state */

#define GAME_BASIS_CHEB 0
#define GAME_BASIS_TRIG 1

/* Error function of the fitness (game_params.error). */
#define GAME_ERR_MSE 0     /* (1/M) sum_m (y_m - Out(m))^2 (Eq. 3, averaged) */
#define GAME_ERR_RMSE 1    /* sqrt of the MSE */
#define GAME_ERR_MAE 2     /* (1/M) sum_m |y_m - Out(m)| */

/* Parent selection (game_params.selection; Section 5 names ranking and
 * roulette). Each parent takes its random words from one Philox4x32-10
 * call (counter: generation, pair, parent, purpose). */
#define GAME_SEL_TOURNAMENT 0 /* best of `tournament` uniform draws */
#define GAME_SEL_RANKING 1    /* linear ranking: the chromosome of rank r
                                 (0 = best by fitness, then lower index;
                                 NaN last) drawn with weight P - r;
                                 P <= 16384 */
#define GAME_SEL_ROULETTE 2   /* fitness-proportionate on 1 / (1 + fit):
                                 integer weight floor(2^32 RN(1/RN(1 + fit))),
                                 0 for NaN or infinite fit; uniform draws
                                 when every weight is 0 */

/* Arithmetic of the fitness contraction (the expansion-times-genes sum). In
 * every direct form the residuals of Eq. 3 are squared (absolute values for
 * the MAE) in FP32 and the sum over patterns ends in FP64. */
#define GAME_PREC_FP32 0   /* FP32 CUDA-core FFMA, FP32 accumulation */
#define GAME_PREC_BF16 1   /* tcgen05 BF16 x BF16 -> FP32 in tensor memory;
                              the expansion tile of all K - 1 columns stays
                              in shared memory, which limits K - 1 to 2560
                              at N <= 128 (GAME_EINVAL beyond) */
#define GAME_PREC_BF16X3 2 /* tcgen05 split products: genes and expansion split
                              into BF16 hi + lo, three MMAs (hi*hi + hi*lo +
                              lo*hi) into one FP32 accumulator; both split
                              operands must fit in shared memory, which limits
                              K - 1 to 1216 at N <= 64 (GAME_EINVAL beyond) */
#define GAME_PREC_FP8 3    /* tcgen05 FP8 E4M3 x E4M3 -> FP32: expansion column
                              k scaled by 448 / max_m |phi_k(x_m)| (taken once
                              from the training set), genes by the inverse
                              and a per-chromosome factor restored in the
                              epilogue; K - 1 up to 4096 at N <= 128 */
#define GAME_PREC_GRAM 4   /* Gram form of the MSE in FP64: with
                              phi~ = (1, phi_1, ..., phi_{K-1}),
                              fit = (y.y - 2 a.b + a^T G a) / M where
                              G = sum phi~ phi~^T and b = sum y phi~ are built
                              once per handle (FP64 expansion and sums); a
                              generation then costs P K^2 FP64 multiply-adds
                              instead of M P K; exact to FP64 rounding (no
                              re-scoring) */

typedef struct game_ctx* game_t;

/* GA and evaluation settings. Section 5 lists the paper's own settings:
 * crossover rate 0.9, mutation rate 0.2, 2 elites, MSE stop threshold
 * 0.001, roulette/ranking selection. The defaults here keep crossover 0.9
 * and 2 elites, use tournaments of 3, per-gene mutation rate 0.02 with
 * Gaussian steps of sd 0.1, and no stop threshold. */
typedef struct {
  int32_t P;            /* chromosomes; 0 = B*N + 1 (Eq. 4) */
  int32_t elitism;      /* E >= 0 best chromosomes copied unchanged */
  int32_t tournament;   /* candidates per tournament, 1..64 */
  int32_t precision;    /* GAME_PREC_* */
  int32_t immigrants;   /* fresh random chromosomes per generation (Section 4) */
  int32_t check_every;  /* generations between stop-rule checks in game_train */
  float pc;             /* crossover probability, [0, 1] */
  float pm;             /* per-gene mutation probability, [0, 1] */
  float sigma;          /* sd of the Gaussian mutation step, >= 0 */
  float reserved_f;
  double mse_threshold; /* game_train stops once best fitness < this; <= 0 off */
  uint64_t seed;        /* key of the counter-based generator (Philox4x32-10) */
  int32_t rescore_top;  /* 0..16: after every evaluation of the GA population
                           in a reduced-precision form (not GAME_PREC_FP32),
                           the rescore_top best chromosomes are re-scored as
                           game_rescore_top does, before the operators rank
                           them; 0 = off; the default 16 keeps the ten best
                           of the ranked vector those of FP64 */
  int32_t surrogate;    /* 1: screen oversampled offspring with the fitness
                           surrogate (game_surrogate_*), 0: off */
  int32_t oversample;   /* offspring per kept child when screening (>= 1,
                           oversample * (P - elitism) <= 16384) */
  int32_t selection;    /* GAME_SEL_* (default tournament) */
  int32_t tied;         /* 1: shared genes, K = B*d + 1 (Eq. 2 as printed,
                           Eq. 5); 0: one gene per feature, basis group and
                           degree, K = B*N*d + 1 (default) */
  int32_t error;        /* GAME_ERR_* (default MSE). GAME_ERR_MAE has no
                           Gram form: it needs a direct precision
                           (not GAME_PREC_GRAM) and rescore_top = 0 */
  int32_t surrogate_steps; /* with the surrogate: Adam steps per generation
                           on each of the last two generations' exact
                           (chromosome, fitness) pairs, 1..64 (default 8:
                           with fewer, the trust check below rarely passes
                           and the screening falls back to the unscreened
                           children) */
  int32_t reserved[1];  /* must be zero */
} game_params;

/* Fills *out with the defaults listed above (and rescore_top = 16,
 * oversample = 8, surrogate_steps = 8, tournament selection, per-feature
 * genes, MSE). */
int game_params_default(game_params* out);

/* Creates a handle for one training set and copies it to the device.
 *   X [M][N] FP32 features, y [M] FP32 targets (host or device memory).
 *   degree d >= 1; basis GAME_BASIS_CHEB or GAME_BASIS_TRIG.
 *   prm: settings (NULL = defaults); cuda_stream: a cudaStream_t, or NULL
 *   for the legacy default stream.
 * Validation (GAME_EINVAL): M < 1, N < 1, d < 1, unknown basis, NaN/Inf in
 * X or y, |x| > 1 with the Chebyshev basis, P < E + immigrants + 2,
 * tournament outside 1..64, rates outside [0, 1], sigma < 0, B*N*d + 1 >
 * 4097, an unknown selection / error function, ranking with P > 16384, the
 * MAE with the Gram form or re-scoring, surrogate settings out of range,
 * non-zero reserved fields.
 * The population is initialised with genes uniform in [-1, 1) (Section 3)
 * from prm->seed and evaluated, so the handle starts at generation 0 with
 * a valid fitness vector. Synchronous. */
int game_create(const float* X, const float* y, int64_t M, int32_t N,
                int32_t degree, int32_t basis, const game_params* prm,
                void* cuda_stream, game_t* out);

/* Shape queries. */
int game_get_shape(game_t h, int64_t* M, int32_t* N, int32_t* K, int32_t* P);

/* Fitness of a caller-supplied population (Eq. 2, Eq. 3; the handle's
 * error function):
 *   pop [P][K] FP32 genes, fit_out [P] FP64, both host or both device.
 * P >= 1 may differ from the handle's population size. Uses the handle's
 * precision. Does not touch the handle's GA state. */
int game_eval_fitness(game_t h, const float* pop, int32_t P, double* fit_out);

/* Like game_eval_fitness with the contraction arithmetic chosen per call
 * (GAME_PREC_*). */
int game_eval_fitness_prec(game_t h, const float* pop, int32_t P,
                           int32_t precision, double* fit_out);

/* The launch plan game_eval_fitness_prec would use for P chromosomes in the
 * given precision (host-side, nothing is launched), for tests and reports:
 *   info[0] kernel: GAME_KERNEL_FP32 (CUDA-core FFMA), GAME_KERNEL_TC (tcgen05
 *           on one SM per pattern tile), GAME_KERNEL_TC_PAIR (tcgen05 on SM
 *           pairs: 2-CTA clusters sharing each MMA, for the BF16 form where
 *           one SM would need a tile narrower than 256 patterns),
 *           GAME_KERNEL_GRAM (FP64 quadratic forms);
 *   info[1] patterns per tile; info[2] K-blocks of the contraction;
 *   info[3] gene stages; info[4] expansion K-block slots; info[5] 1 if the
 *   features are staged in shared memory (0: read from L2); info[6] CTAs;
 *   info[7] dynamic shared memory per CTA in bytes (tensor-core plans).
 * Fields that do not apply are 0. GAME_EINVAL for a contraction the
 * precision cannot take. */
#define GAME_KERNEL_FP32 1
#define GAME_KERNEL_TC 2
#define GAME_KERNEL_TC_PAIR 3
#define GAME_KERNEL_GRAM 4
int game_plan_info(game_t h, int32_t precision, int32_t P, int32_t* info);

/* Elite re-scoring. The n best chromosomes of fit (by fitness, then lower
 * index; NaN ranks last) are evaluated again in FP64 by the Gram form of the
 * MSE (see GAME_PREC_GRAM: exact to FP64 rounding; the handle builds its G
 * on first use), and their entries of fit are replaced. Its purpose is the
 * elitism decision of Section 3 (2 elites, Section 5) when fit came from a
 * reduced-precision contraction: the best candidates are then ranked by
 * accurate values.
 *   pop [P][K] FP32, fit [P] FP64 (in: any fitness vector of pop; out: the
 *   same with n entries replaced), both host or both device;
 *   1 <= n <= min(16, P); idx_out [n] (may be NULL; host or device) receives
 *   the candidates' indices, best first.
 * With GAME_ERR_RMSE the replaced entries are the square roots of the
 * Gram-form MSE; GAME_ERR_MAE handles refuse (GAME_EINVAL).
 * Entries other than the n candidates are not modified. Host arguments
 * synchronise; device arguments only enqueue. */
int game_rescore_top(game_t h, const float* pop, int32_t P, double* fit,
                     int32_t n, int32_t* idx_out);

/* One generation g -> g+1 of the GA state: elitism, parent selection,
 * one-point crossover, per-gene Gaussian mutation, clamping to [-1, 1]
 * (Section 3 names the operators; Section 5 the rates), then the fitness of
 * the new population. All random decisions come from Philox4x32-10 keyed
 * by `seed` with counters built from (g, slot, gene, purpose), so a run is
 * reproducible and resumable. Enqueues only. */
int game_generation(game_t h, uint64_t seed);

/* Runs up to `generations` generations with prm->seed, stopping early once
 * the best fitness drops below prm->mse_threshold (checked every
 * check_every generations; Section 4: training stops at the iteration limit
 * or the error threshold). *generations_run (may be NULL) receives the
 * count. Synchronous. */
int game_train(game_t h, int32_t generations, int32_t* generations_run);

/* Copies out the current population [P][K] FP32, its fitness [P] FP64 and
 * the generation counter; any output may be NULL. Host or device outputs
 * (pop_out and fit_out in the same kind of memory). */
int game_get_population(game_t h, float* pop_out, double* fit_out,
                        int64_t* generation);

/* Replaces the GA state: population [P][K] (the handle's P), its fitness
 * [P] (NULL = evaluate it now) and the generation counter. Together with
 * game_get_population this is checkpoint / resume. */
int game_set_state(game_t h, const float* pop, const double* fit,
                   int64_t generation);

/* ---- Pattern sharding ----
 * The fitness of Eq. 3 is a sum over patterns, so the training set can be
 * split into slices held by separate handles (on separate GPUs; the paper
 * names several GPUs as future work, Section 6): each slice gives the
 * unnormalised error sum of every chromosome, the sums of all slices added
 * in a fixed order and divided by the total M are the fitness, and every
 * handle then breeds the same next population from the same (seed,
 * generation) counters. These three calls are the per-slice steps. */

/* Error sums of a population over the handle's own patterns:
 *   sse_out[p] = sum_m (y_m - Out_p(m))^2 for GAME_ERR_MSE and GAME_ERR_RMSE
 *   handles, sum_m |y_m - Out_p(m)| for GAME_ERR_MAE; FP64, unnormalised.
 * Computed by the handle's precision, which must be a direct form (not
 * GAME_PREC_GRAM: GAME_EINVAL), without elite re-scoring.
 *   pop [P][K] FP32 genes, or NULL for the handle's current population (P is
 *   then ignored); pop and sse_out host or device (both the same kind when
 *   pop is given). Host outputs synchronise; device ones only enqueue. */
int game_eval_sse(game_t h, const float* pop, int32_t P, double* sse_out);

/* The operators of one generation alone (those of game_generation: elitism,
 * selection, crossover, mutation, clamping; generation g -> g + 1), without
 * evaluating the new population. Until game_set_fitness (or
 * game_set_state) gives it a fitness vector, game_breed returns
 * GAME_ESTATE, and game_generation / game_train evaluate it on the
 * handle's own patterns first. GAME_ESTATE also for surrogate handles.
 * Enqueues only. */
int game_breed(game_t h, uint64_t seed);

/* Sets the fitness vector of the current population: fit [P] FP64, host or
 * device (the handle's P). Host input synchronises. */
int game_set_fitness(game_t h, const double* fit);

/* Checkpoint file of the GA state: population, fitness and generation and,
 * with the surrogate, its parameters, Adam moments and step, the trust
 * check's verdict and the replay ring, so that game_load followed by the same calls
 * continues the run exactly. The file records M, N, degree, basis, tied, K,
 * P and the surrogate setting; game_load refuses (GAME_EINVAL) a file of a
 * different shape or a truncated or foreign one. The training set itself
 * is not stored: load into a handle created on the same data and settings.
 * game_save writes `path`.tmp and renames it to `path`. Synchronous. */
int game_save(game_t h, const char* path);
int game_load(game_t h, const char* path);

/* Per-stage device timing (CUDA events recorded on the handle's stream
 * around each kernel launch of the stages below). */
typedef struct {
  double fitness_ms;        /* fused fitness contraction kernel */
  double pack_ms;           /* population -> contraction operand layout */
  double reduce_ms;         /* cross-tile FP64 error sum */
  double operators_ms;      /* selection / crossover / mutation kernels */
  int64_t fitness_launches;
  int64_t pack_launches;
  int64_t reduce_launches;
  int64_t operators_launches; /* calls; two kernels each (plan, breeding), one
                               fused kernel for populations of at most 1024
                               chromosomes and 65,536 genes, plus a selection
                               table kernel for ranking or roulette above that */
  double rescore_ms;        /* elite candidate selection and re-scoring */
  int64_t rescore_launches; /* calls; three kernels each (selection, quadratic
                               forms, final sums) */
  double surrogate_ms;      /* surrogate screening and training */
  int64_t surrogate_launches; /* generations screened */
} game_timing;

/* enable != 0 starts recording (and clears the totals); 0 stops. */
int game_set_timing(game_t h, int32_t enable);
/* Synchronises the stream and returns the totals since the last enable. */
int game_get_timing(game_t h, game_timing* out);

/* Fitness of a population without any device allocation, for callers that
 * cannot call cudaMalloc: plug-ins inside a host application that owns the
 * device-memory budget and hands out only what it pre-allocated, and
 * runtimes that forbid allocation after start-up (an allocation can fail,
 * and cudaMalloc / cudaFree may synchronise the device, stalling every other
 * stream). The paper has no counterpart of this call. It returns the same
 * FP32 MSE that game_eval_fitness computes with GAME_PREC_FP32 (FP32
 * CUDA-core contraction, FP64 cross-tile sum), without a handle.
 *   X [M][N] FP32 row-major, y [M] FP32, pop [P][K] FP32 (K = B*N*d + 1),
 *   fit_out [P] FP64: all device (or managed) memory of the current device,
 *   owned by the caller. Inputs are used as given (no NaN / domain checks).
 *   cuda_stream: a cudaStream_t or NULL. Only enqueues work.
 * The only intermediate buffer is a fixed 4 MiB array of FP64 partial sums
 * that the library holds on every GPU that loads it, until the process
 * exits. P above 524288 (the array's capacity in chromosome rows) is
 * rejected with GAME_EINVAL before any launch. The first call on a device
 * looks up that array's address and caches it (make it before any stream
 * capture); after cudaDeviceReset of that device the cached address is
 * stale, so no call may follow a reset in the same process. All calls share
 * the array: calls that overlap on the GPU race on it, so the caller must
 * serialise them. Errors: GAME_EINVAL (arguments, host pointers, memory of
 * another device), GAME_ECUDA; the reason is in game_last_error(). */
int game_eval_fitness_static(const float* X, const float* y, int64_t M,
                             int32_t N, int32_t degree, int32_t basis,
                             const float* pop, int32_t P, double* fit_out,
                             void* cuda_stream);

/* ---- Fitness surrogate ----
 * Not in the paper: a small MLP (genes -> 256 -> 256 -> 1, GELU, BF16
 * operands with FP32 accumulation in the two hidden layers, FP32 master
 * weights, Adam lr 1e-3) that predicts log(MSE) of a chromosome. With
 * prm->surrogate, every generation breeds oversample * (P - E) children with
 * the operators of game_generation (tournaments from the current
 * population), keeps the P - E children with the lowest predicted fitness
 * (ties by slot) in slot order after the E elites, evaluates that population
 * exactly (the handle's precision and re-scoring), and then trains the
 * surrogate with surrogate_steps rounds of one Adam step on each of the last
 * two generations' exact (chromosome, fitness) pairs. The exact fitness also
 * checks the surrogate
 * (game_surrogate_last): while its predictions do not correlate with the
 * exact fitness of the children they kept, screening keeps the children an
 * unscreened generation would have. The surrogate of a fresh handle is initialised
 * from prm->seed and trained with 20 steps on generation 0.
 * Parameter vector (FP32): W1 [256][K], b1 [256], W2 [256][256], b2 [256],
 * w3 [256], b3 [1]. Arrays may be host or device memory. */
/* Predictions for n chromosomes pop [n][K] into pred_out [n] (FP32, on the
 * standardised log-fitness scale of the training batches). */
int game_surrogate_predict(game_t h, const float* pop, int32_t n, float* pred_out);
/* Gradient of the training loss mean((out - t)^2), t the log-fitness
 * standardised over the batch (mean 0, sd 1), over the pairs
 * (pop [n][K], fit [n]) at the current parameters, into grad_out [count];
 * loss_out (may be NULL) receives the loss. Parameters are not changed. */
int game_surrogate_grad(game_t h, const float* pop, const double* fit, int32_t n,
                        float* grad_out, float* loss_out);
/* One Adam step on the pairs (pop [n][K], fit [n]). */
int game_surrogate_train(game_t h, const float* pop, const double* fit, int32_t n);
/* The parameter count (count may not be NULL) and, if w_out is not NULL, the
 * FP32 parameters. */
int game_surrogate_params(game_t h, float* w_out, int64_t* count);
/* Replaces the parameters (w [count]) and resets the Adam state. */
int game_surrogate_set_params(game_t h, const float* w);
/* The last screening: *n_out children (slot E + i), their predictions
 * pred_out [n], kept flags keep_out [n], whether the screening trusted the
 * surrogate (*trusted_out; if not it kept the first P - E children, those of
 * the unscreened generation), and the trust check's correlation *r_out measured on
 * the children it kept (any output may be NULL; pass NULL arrays first to
 * learn n). The trust check: the next screening trusts the surrogate iff the
 * Pearson correlation of the kept children's predictions with their exact
 * log-fitness exceeds 0.25; a fresh handle starts untrusted. */
int game_surrogate_last(game_t h, float* pred_out, int32_t* keep_out, int32_t* n_out,
                        int32_t* trusted_out, float* r_out);

/* ---- Batched runs ----
 * Many independent GA runs, each the method above on its own training set,
 * degree, basis, population size and seed, advanced together: one launch
 * per stage for all runs (operators, operand pack, fused fitness, FP64
 * reduce), the stages of a generation replayed from a CUDA graph. The
 * contraction is BF16 on the tensor cores (GAME_PREC_BF16), the GA state
 * FP32. Run r with seed s follows the operators of a single handle keyed by
 * s given the same fitness values. */
typedef struct game_batch* game_batch_t;

typedef struct {
  const float* X;   /* [M][N] FP32 features (host or device; copied) */
  const float* y;   /* [M] FP32 targets */
  int64_t M;
  int32_t N, degree, basis;
  int32_t P;        /* chromosomes, elitism + immigrants + 2 .. 2^20 */
  uint64_t seed;    /* the run's Philox key */
} game_run_desc;

/* Creates a batch of R runs. prm gives the GA settings shared by all runs
 * (elitism, tournament, pc, pm, sigma, immigrants; its P, precision, seed,
 * rescore_top and stop threshold are ignored). tiles: the pattern-tile width
 * of each run's fitness items (32, 64, 128 or 256; NULL = choose): with
 * autotune != 0, starting from the widest width that fits every run, each
 * group of runs with the same K-block count class, widest width and
 * chromosome-tile count is tried at its other widths while the whole
 * fitness launch is timed, and
 * a width kept when that launch gets at least 0.5% faster; with autotune ==
 * 0 the widest that fits. Fitness values depend on the tile width in their
 * last bits (FP32 sums inside a tile): pass the widths game_batch_get_tiles
 * returns to reproduce a run exactly. Validation as game_create per run
 * (GAME_EINVAL naming the run), plus K - 1 <= 2048 and N <= 256; batched
 * runs use tournament selection, per-feature genes and the MSE. The initial
 * populations are generated and evaluated. Synchronous. */
int game_batch_create(const game_run_desc* runs, int32_t R, const game_params* prm,
                      const int32_t* tiles, int32_t autotune, void* cuda_stream,
                      game_batch_t* out);
/* One generation of every run (one graph launch). Enqueues only. */
int game_batch_generation(game_batch_t b);
/* Population [P_r][K_r], fitness [P_r] and generation of run r (host or
 * device outputs; any may be NULL). Synchronises. */
int game_batch_get_run(game_batch_t b, int32_t r, float* pop_out, double* fit_out,
                       int64_t* generation);
/* The tile width of every run, tiles_out[R]. */
int game_batch_get_tiles(game_batch_t b, int32_t* tiles_out);
/* Mean device time of the batched fitness launch over reps launches on the
 * current populations (CUDA events on the batch's stream). Synchronises. */
int game_batch_fitness_ms(game_batch_t b, int32_t reps, double* ms_out);
/* Waits for the batch's stream and reports a kernel timeout, if any. */
int game_batch_sync(game_batch_t b);
/* Releases the batch (NULL is accepted). */
int game_batch_destroy(game_batch_t b);

/* The Gram form's G [K][K], b [K] and y.y (FP64; built on first use; any
 * output may be NULL; host or device). For a shared-gene handle the
 * expansion is psi_{b,j}(x) = sum_i phi_{b,j}(x_i) (K = B*d + 1).
 * Synchronises. */
int game_gram(game_t h, double* G_out, double* b_out, double* yy_out);

/* Outputs Out(m) of one chromosome (Eq. 2) on a set of patterns, computed
 * in FP64 on the GPU (FP64 expansion, FP64 sum in gene order):
 *   chrom [K] FP32 genes in the handle's layout (host or device);
 *   X [M][N] FP32 features, row-major, host or device, with N the handle's;
 *   NULL = the handle's training set (M must then equal its M);
 *   out [M] FP64, host or device.
 * M = 0 is allowed (nothing to do). The Chebyshev polynomials are evaluated
 * by their recurrence at any x (the [-1, 1] check applies to the training
 * set only). Host outputs synchronise; a device out only enqueues. */
int game_predict(game_t h, const float* chrom, const float* X, int64_t M,
                 double* out);

/* Binary classification by one chromosome. Section 5 reports accuracy,
 * completeness and contamination without defining them; here a pattern is
 * a positive when its target y_m > threshold and is predicted positive when
 * Out(m) > threshold (Out in FP64 as game_predict), and
 *   accuracy = (tp + tn) / M, completeness = tp / (tp + fn),
 *   contamination = fp / (tp + fp)   (0 when a denominator is 0). */
typedef struct {
  int64_t tp, fp, tn, fn;
  double accuracy, completeness, contamination;
} game_confusion;

/* X [M][N], y [M] FP32 (host or device; both NULL = the training set, M
 * then equal to its M); chrom [K] as game_predict; *out on the host.
 * Synchronous. */
int game_classify(game_t h, const float* chrom, const float* X, const float* y,
                  int64_t M, double threshold, game_confusion* out);

/* Waits for the handle's stream and reports a kernel timeout, if any. */
int game_sync(game_t h);

/* Test hooks: process-wide switches that make the library's failure paths
 * reachable without any fault on the GPU (the paper has no counterpart).
 *   GAME_HOOK_FAIL_ALLOC, value k >= 1: the k-th device allocation made by
 *     the library from now on fails as if the device were out of memory
 *     (the call then returns GAME_ENOMEM after releasing what it holds);
 *     0 switches the hook off.
 *   GAME_HOOK_STALL_NS, value t in 1..10^9: the next launch of the
 *     tensor-core fitness kernel makes its MMA issuer wait up to t ns on a
 *     barrier phase that nothing completes; the wait runs out, and the kernel
 *     abandons the launch the way every expired wait does (raises the
 *     handle's status word, drains its own copies and MMAs, frees its tensor
 *     memory, returns), so the call reports GAME_ETIMEOUT and the handle
 *     stays usable; 0 cancels a pending stall.
 *   GAME_HOOK_SMEM_SLACK, value s in 1..1024: the tensor-core launch plans
 *     keep s bytes for aligning the kernel's dynamic shared memory instead
 *     of the padding that game_create's probe found (1024 gives the plans of
 *     a device whose shared memory needs the full alignment: the large
 *     classification plan then reads its targets from global memory instead
 *     of staging them); 0 returns to the probed padding. A slack below the
 *     real padding makes the kernel end before touching shared memory and
 *     the call report GAME_ECUDA.
 * Returns GAME_EINVAL for an unknown hook or a value out of range. */
#define GAME_HOOK_FAIL_ALLOC 1
#define GAME_HOOK_STALL_NS 2
#define GAME_HOOK_SMEM_SLACK 3
int game_test_hook(int32_t hook, int64_t value);

/* Releases the handle and all its device memory (NULL is accepted). */
int game_destroy(game_t h);

/* Description of the calling thread's last failure ("" if none). */
const char* game_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
