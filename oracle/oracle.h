/*
 * oracle.h -- FP64 CPU oracle for GAME (Cavuoti et al., arXiv:1211.5481).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline, reference and accuracy legs load this library. It shares no code, header,
 * table or constant with the CUDA path, and neither side includes the other.
 *
 * Notation (paper, Section 3):
 *   M  patterns (the paper's NP), N features, d polynomial degree,
 *   B  basis multiplicity (1 = Chebyshev, 2 = trigonometric "polytrigo"),
 *   K  genes per chromosome = B*N*d + 1 (one gene per feature, basis group
 *      and degree, plus one bias gene a_0), P chromosomes, E elites.
 *   Gene k = 1 + i*B*d + b*d + (j-1) weights phi_{b,j}(x_i),
 *   phi_{0,j} = T_j (Chebyshev) or cos(j x) (trigonometric),
 *   phi_{1,j} = sin(j x) (trigonometric only).
 *
 * All arrays are row-major and owned by the caller. Functions return 0 on
 * success and a negative value on invalid arguments.
 */
#ifndef GAME_ORACLE_H
#define GAME_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_CHEB = 0, ORACLE_TRIG = 1 };
enum { ORACLE_ERR_MSE = 0, ORACLE_ERR_RMSE = 1, ORACLE_ERR_MAE = 2 };
enum { ORACLE_SEL_TOURNAMENT = 0, ORACLE_SEL_RANKING = 1, ORACLE_SEL_ROULETTE = 2 };

/* Section 3, Eq. 4: population size B*N + 1. */
int64_t oracle_num_chromosomes(int32_t N, int32_t basis);
/* Section 3, Eq. 5: genes of the paper's shared-gene chromosome, B*d + 1. */
int64_t oracle_num_genes_tied(int32_t d, int32_t basis);
/* Per-feature genes: B*N*d + 1. */
int64_t oracle_num_genes(int32_t N, int32_t d, int32_t basis);

/* Section 3, Eq. 1 and Eq. 6: the B*d basis values of one feature value x. */
int oracle_basis(int32_t basis, int32_t d, double x, double* out);

/* Section 3, Eq. 2: Out(pat) for one pattern x[N] and one chromosome a[K]. */
double oracle_output(const double* a, const double* x, int32_t N, int32_t d,
                     int32_t basis);

/* Section 3, Eq. 3 and the MSE that follows it (Section 5 fixes MSE):
 * fit[p] = (1/M) sum_m (y_m - Out_p(x_m))^2, direct triple loop, OpenMP over p.
 * X[M][N], y[M], pop[P][K] (K = B*N*d + 1). */
int oracle_fitness(const double* X, const double* y, int64_t M, int32_t N,
                   int32_t d, int32_t basis, const double* pop, int32_t P,
                   double* fit);

/* Same, with the error function selectable: ORACLE_ERR_MSE (Eq. 3 averaged),
 * ORACLE_ERR_RMSE (its square root) or ORACLE_ERR_MAE (mean absolute
 * difference, the "absolute difference" error of Section 3). */
int oracle_fitness_err(const double* X, const double* y, int64_t M, int32_t N,
                       int32_t d, int32_t basis, const double* pop, int32_t P,
                       int32_t err_kind, double* fit);

/* Paper-literal shared-gene form (Eq. 2 with a_j common to all features,
 * Eq. 5 chromosome length): pop[P][B*d + 1]. */
int oracle_fitness_tied(const double* X, const double* y, int64_t M, int32_t N,
                        int32_t d, int32_t basis, const double* pop, int32_t P,
                        double* fit);

/* Outputs of one chromosome a[K] (Eq. 2) on M patterns X[M][N]: out[M]. */
int oracle_predict(const double* X, int64_t M, int32_t N, int32_t d, int32_t basis,
                   const double* a, double* out);

/* Binary classification counts of one chromosome (Section 5 reports
 * accuracy, completeness and contamination without defining them): a
 * pattern is a positive when y_m > threshold and is predicted positive when
 * Out(m) > threshold. counts[4] = {TP, FP, TN, FN}. */
int oracle_classify(const double* X, const double* y, int64_t M, int32_t N,
                    int32_t d, int32_t basis, const double* a, double threshold,
                    int64_t* counts);

/* Gram form of the MSE: with phi~(x) = (1, phi_1(x), ..., phi_{K-1}(x)),
 * G = sum_m phi~ phi~^T [K][K], b = sum_m y_m phi~ [K], yy = sum_m y_m^2,
 * SSE_p = yy - 2 a_p^T b + a_p^T G a_p. */
int oracle_gram(const double* X, const double* y, int64_t M, int32_t N,
                int32_t d, int32_t basis, double* G, double* b, double* yy);
int oracle_fitness_gram(const double* G, const double* b, double yy, int64_t M,
                        int32_t K, const double* pop, int32_t P, double* fit);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = bijection of the
 * 128-bit counter ctr under the 64-bit key (key[0] low word). */
void oracle_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4],
                          uint32_t out[4]);

/* GA operator parameters. thr_pc = floor(pc * 2^24), thr_pm = floor(pm * 2^24).
 * selection (Section 5 names roulette and ranking selection):
 *  ORACLE_SEL_TOURNAMENT: the best of `tournament` uniform draws;
 *  ORACLE_SEL_RANKING: linear ranking, rank r (0 = best by (fitness, index))
 *    drawn with weight P - r (needs P <= 65535);
 *  ORACLE_SEL_ROULETTE: fitness-proportionate on the maximised transform
 *    1 / (1 + fit), as the integer weight floor(2^32 RN(1 / RN(1 + fit)))
 *    (0 for a NaN, negative or infinite fit; uniform draws when every
 *    weight is 0). */
typedef struct {
  int32_t elitism;     /* E */
  int32_t tournament;  /* candidates per tournament */
  uint32_t thr_pc;
  uint32_t thr_pm;
  float sigma;         /* Gaussian mutation step */
  int32_t immigrants;  /* fresh random chromosomes per generation */
  int32_t selection;   /* ORACLE_SEL_* */
} oracle_ga_params;

/* Gene initialisation, uniform in [-1, 1) (Section 3: genes generated at
 * random, normalised between -1 and +1). pop[P][K]. */
int oracle_init_population(uint64_t seed, int32_t P, int32_t K, float* pop);

/* One generation g -> g+1 (elitism, selection, one-point crossover,
 * Gaussian mutation, clamp to [-1, 1]). pop[P][K], fit[P],
 * next[P][K]; next must not alias pop. */
int oracle_generation(const float* pop, const double* fit, int32_t P,
                      int32_t K, const oracle_ga_params* prm, uint64_t seed,
                      uint32_t g, float* next);

/* The n best chromosomes by (fitness, index), NaN ranking as +infinity:
 * idx[0..n-1], best first (the ranking elitism uses, Section 3). */
int oracle_select_best(const double* fit, int32_t P, int32_t n, int32_t* idx);

/* Elite re-scoring: fit_out = fit_in with the entries of the n best (by
 * oracle_select_best on fit_in) replaced by their FP64 fitness (the direct
 * form of oracle_fitness). idx[n] receives the candidates, best first.
 * pop[P][K] FP32 genes. */
int oracle_rescore(const double* X, const double* y, int64_t M, int32_t N,
                   int32_t d, int32_t basis, const float* pop, int32_t P,
                   const double* fit_in, int32_t n, double* fit_out,
                   int32_t* idx);

/* The operators of oracle_generation with n_out output slots instead of P
 * (oversampled offspring): slots 0..E-1 the elites, E..n_out-1 children of
 * parents selected from the P current chromosomes, the last I slots
 * immigrants; next[n_out][K]. n_out = P is oracle_generation. */
int oracle_offspring(const float* pop, const double* fit, int32_t P, int32_t K,
                     const oracle_ga_params* prm, uint64_t seed, uint32_t g,
                     int32_t n_out, float* next);

/* Whole GA run: init, then G times (fitness, generation), with the fitness
 * computed by the direct form (use_gram = 0) or the Gram form (1).
 * best[G+1] receives the best fitness after init and after each generation.
 * On return pop[P][K] and fit[P] hold generation G. */
int oracle_train(const double* X, const double* y, int64_t M, int32_t N,
                 int32_t d, int32_t basis, int32_t P,
                 const oracle_ga_params* prm, uint64_t seed, int32_t G,
                 int32_t use_gram, float* pop, double* fit, double* best);

/* The same run on shared-gene chromosomes (Eq. 5, K = B*d + 1), the
 * fitness by the direct form of oracle_fitness_tied. pop[P][B*d + 1]. */
int oracle_train_tied(const double* X, const double* y, int64_t M, int32_t N,
                      int32_t d, int32_t basis, int32_t P,
                      const oracle_ga_params* prm, uint64_t seed, int32_t G,
                      float* pop, double* fit, double* best);

/* Threads the OpenMP loops may use (0 = runtime default); returns the count
 * in effect. */
int oracle_set_threads(int32_t n);

#ifdef __cplusplus
}
#endif
#endif
