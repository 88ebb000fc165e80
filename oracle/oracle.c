/*
 * oracle.c -- FP64 CPU oracle for GAME population fitness evaluation and the
 * GA operators (Cavuoti et al., "Genetic Algorithm Modeling with GPU Parallel
 * Computing Technology", arXiv:1211.5481).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline, reference and accuracy legs load this library;
 * the CUDA path never does.
 * It is written to be read against the paper, not to be fast: every
 * function is the plain definition, with no blocking, fusion or reordering.
 *
 * Floating point: fitness is FP64 throughout. The GA state (genes) is FP32,
 * so the operators compute gene updates in FP32 with one rounding per
 * operation; build with -ffp-contract=off so that no FMA is formed.
 *
 * Readings of the paper used here (the paper is ambiguous or silent):
 *  - Eq. 1 writes powers g^j(f); Eq. 6 and the serial listing of Section 4
 *    use cos(j x), sin(j x). g^j is read as the j-th basis function; the
 *    Chebyshev basis T_j is the second family offered.
 *  - Eq. 2 indexes genes by degree only (shared by all features). The
 *    per-feature reading, one gene per (feature, basis group, degree), is the
 *    main form; the shared-gene form is oracle_fitness_tied, and replicating
 *    its genes over features gives the same fitness.
 *  - One bias gene a_0 (Eq. 2), so K = B*N*d + 1.
 *  - Fitness is the MSE (Section 3 after Eq. 3; Section 5), minimised; ties
 *    are broken by the lower index and a NaN fitness ranks as +infinity.
 *  - The operators are named (Section 3: crossover, mutation, elitism;
 *    Section 5: rates, 2 elites, ranking and roulette selection) but not
 *    defined. The definitions below (tournament, linear-ranking and
 *    roulette selection, one-point crossover, per-gene Gaussian mutation
 *    with an Irwin-Hall normal, clamp to [-1, 1], counter-based Philox
 *    draws) are this project's. Roulette turns on 1 / (1 + fit), a
 *    positive transform that is larger for a better (smaller) MSE.
 *  - Section 4 replaces older individuals by fresh random chromosomes each
 *    generation, without a count: `immigrants` slots at the end of the
 *    population are refilled (0 by default).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Counter tags: the fourth counter word separates the uses of one draw. */
enum {
  TAG_INIT = 1,
  TAG_TOUR = 2,
  TAG_XO = 3,
  TAG_MUT = 4,
  TAG_G0 = 5,
  TAG_G1 = 6,
  TAG_G2 = 7,
  TAG_IMM = 8
};

static int basis_mult(int32_t basis) { return basis == ORACLE_TRIG ? 2 : 1; }

static int valid_basis(int32_t basis) {
  return basis == ORACLE_CHEB || basis == ORACLE_TRIG;
}

int64_t oracle_num_chromosomes(int32_t N, int32_t basis) {
  if (N < 1 || !valid_basis(basis)) return -1;
  return (int64_t)basis_mult(basis) * N + 1;
}

int64_t oracle_num_genes_tied(int32_t d, int32_t basis) {
  if (d < 1 || !valid_basis(basis)) return -1;
  return (int64_t)basis_mult(basis) * d + 1;
}

int64_t oracle_num_genes(int32_t N, int32_t d, int32_t basis) {
  if (N < 1 || d < 1 || !valid_basis(basis)) return -1;
  return (int64_t)basis_mult(basis) * N * d + 1;
}

/* Chebyshev polynomial of the first kind by its three-term recurrence:
 * T_0 = 1, T_1 = x, T_{j+1} = 2 x T_j - T_{j-1}. */
static double cheb_T(int j, double x) {
  if (j == 0) return 1.0;
  double tm1 = 1.0, t = x;
  for (int n = 1; n < j; ++n) {
    double tp1 = 2.0 * x * t - tm1;
    tm1 = t;
    t = tp1;
  }
  return t;
}

/* phi_{b,j}(x): Chebyshev T_j, or cos(j x) / sin(j x) (Eq. 6). */
static double phi(int32_t basis, int b, int j, double x) {
  if (basis == ORACLE_CHEB) return cheb_T(j, x);
  return b == 0 ? cos((double)j * x) : sin((double)j * x);
}

int oracle_basis(int32_t basis, int32_t d, double x, double* out) {
  if (d < 1 || !valid_basis(basis) || !out) return -1;
  const int B = basis_mult(basis);
  for (int b = 0; b < B; ++b)
    for (int j = 1; j <= d; ++j) out[b * d + (j - 1)] = phi(basis, b, j, x);
  return 0;
}

/* Eq. 2: a_0 + sum_i sum_b sum_j a_{1 + i*B*d + b*d + j-1} phi_{b,j}(x_i). */
double oracle_output(const double* a, const double* x, int32_t N, int32_t d,
                     int32_t basis) {
  const int B = basis_mult(basis);
  double out = a[0];
  for (int i = 0; i < N; ++i)
    for (int b = 0; b < B; ++b)
      for (int j = 1; j <= d; ++j)
        out += a[1 + (int64_t)i * B * d + b * d + (j - 1)] *
               phi(basis, b, j, x[i]);
  return out;
}

int oracle_fitness_err(const double* X, const double* y, int64_t M, int32_t N,
                       int32_t d, int32_t basis, const double* pop, int32_t P,
                       int32_t err_kind, double* fit) {
  if (M < 1 || N < 1 || d < 1 || P < 0 || !valid_basis(basis)) return -1;
  if (err_kind < ORACLE_ERR_MSE || err_kind > ORACLE_ERR_MAE) return -1;
  const int64_t K = oracle_num_genes(N, d, basis);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t p = 0; p < P; ++p) {
    const double* a = pop + (int64_t)p * K;
    double acc = 0.0;
    for (int64_t m = 0; m < M; ++m) {
      /* Eq. 3: E_k = (t_k - Out(pat_k))^2 */
      double r = y[m] - oracle_output(a, X + m * N, N, d, basis);
      acc += (err_kind == ORACLE_ERR_MAE) ? fabs(r) : r * r;
    }
    double mean = acc / (double)M;
    fit[p] = (err_kind == ORACLE_ERR_RMSE) ? sqrt(mean) : mean;
  }
  return 0;
}

int oracle_predict(const double* X, int64_t M, int32_t N, int32_t d, int32_t basis,
                   const double* a, double* out) {
  if (M < 0 || N < 1 || d < 1 || !valid_basis(basis) || !a || !out) return -1;
  for (int64_t m = 0; m < M; ++m) out[m] = oracle_output(a, X + m * N, N, d, basis);
  return 0;
}

int oracle_classify(const double* X, const double* y, int64_t M, int32_t N,
                    int32_t d, int32_t basis, const double* a, double threshold,
                    int64_t* counts) {
  if (M < 0 || N < 1 || d < 1 || !valid_basis(basis) || !a || !counts) return -1;
  counts[0] = counts[1] = counts[2] = counts[3] = 0;
  for (int64_t m = 0; m < M; ++m) {
    const int actual = y[m] > threshold;
    const int predicted = oracle_output(a, X + m * N, N, d, basis) > threshold;
    if (predicted && actual) counts[0] += 1;        /* true positive */
    else if (predicted) counts[1] += 1;             /* false positive */
    else if (!actual) counts[2] += 1;               /* true negative */
    else counts[3] += 1;                            /* false negative */
  }
  return 0;
}

int oracle_fitness(const double* X, const double* y, int64_t M, int32_t N,
                   int32_t d, int32_t basis, const double* pop, int32_t P,
                   double* fit) {
  return oracle_fitness_err(X, y, M, N, d, basis, pop, P, ORACLE_ERR_MSE, fit);
}

int oracle_fitness_tied(const double* X, const double* y, int64_t M, int32_t N,
                        int32_t d, int32_t basis, const double* pop, int32_t P,
                        double* fit) {
  if (M < 1 || N < 1 || d < 1 || P < 0 || !valid_basis(basis)) return -1;
  const int B = basis_mult(basis);
  const int64_t K = (int64_t)B * d + 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t p = 0; p < P; ++p) {
    const double* a = pop + (int64_t)p * K;
    double sse = 0.0;
    for (int64_t m = 0; m < M; ++m) {
      /* Eq. 2 as printed: one a_0, genes a_j (and b_j) shared by features. */
      double out = a[0];
      for (int i = 0; i < N; ++i)
        for (int b = 0; b < B; ++b)
          for (int j = 1; j <= d; ++j)
            out += a[1 + b * d + (j - 1)] * phi(basis, b, j, X[m * N + i]);
      double r = y[m] - out;
      sse += r * r;
    }
    fit[p] = sse / (double)M;
  }
  return 0;
}

int oracle_gram(const double* X, const double* y, int64_t M, int32_t N,
                int32_t d, int32_t basis, double* G, double* b, double* yy) {
  if (M < 1 || N < 1 || d < 1 || !valid_basis(basis)) return -1;
  const int B = basis_mult(basis);
  const int64_t K = oracle_num_genes(N, d, basis);
  const int64_t CH = 512; /* patterns per block of the design matrix */
  double* Phi = (double*)malloc(sizeof(double) * CH * K);
  if (!Phi) return -2;
  memset(G, 0, sizeof(double) * K * K);
  memset(b, 0, sizeof(double) * K);
  double s = 0.0;
  for (int64_t m0 = 0; m0 < M; m0 += CH) {
    const int64_t mc = (M - m0 < CH) ? (M - m0) : CH;
    for (int64_t r = 0; r < mc; ++r) {
      const double* x = X + (m0 + r) * N;
      double* row = Phi + r * K;
      row[0] = 1.0;
      for (int i = 0; i < N; ++i)
        for (int bb = 0; bb < B; ++bb)
          for (int j = 1; j <= d; ++j)
            row[1 + (int64_t)i * B * d + bb * d + (j - 1)] =
                phi(basis, bb, j, x[i]);
    }
    /* G += Phi^T Phi, b += Phi^T y, rows of G split over threads. */
#pragma omp parallel for schedule(static)
    for (int64_t k1 = 0; k1 < K; ++k1) {
      for (int64_t r = 0; r < mc; ++r) {
        const double v = Phi[r * K + k1];
        for (int64_t k2 = 0; k2 < K; ++k2) G[k1 * K + k2] += v * Phi[r * K + k2];
        b[k1] += v * y[m0 + r];
      }
    }
    for (int64_t r = 0; r < mc; ++r) s += y[m0 + r] * y[m0 + r];
  }
  *yy = s;
  free(Phi);
  return 0;
}

int oracle_fitness_gram(const double* G, const double* b, double yy, int64_t M,
                        int32_t K, const double* pop, int32_t P, double* fit) {
  if (M < 1 || K < 1 || P < 0) return -1;
#pragma omp parallel for schedule(static)
  for (int32_t p = 0; p < P; ++p) {
    const double* a = pop + (int64_t)p * K;
    double aGa = 0.0, ab = 0.0;
    for (int32_t k1 = 0; k1 < K; ++k1) {
      double row = 0.0;
      for (int32_t k2 = 0; k2 < K; ++k2) row += G[(int64_t)k1 * K + k2] * a[k2];
      aGa += a[k1] * row;
      ab += a[k1] * b[k1];
    }
    fit[p] = (yy - 2.0 * ab + aGa) / (double)M;
  }
  return 0;
}

/* Philox4x32-10: ten rounds of two 32x32->64 multiplies (multipliers
 * 0xD2511F53, 0xCD9E8D57) with the key bumped by the Weyl constants
 * 0x9E3779B9, 0xBB67AE85 after each round. */
void oracle_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4],
                          uint32_t out[4]) {
  uint32_t k0 = key[0], k1 = key[1];
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int round = 0; round < 10; ++round) {
    const uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    const uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    const uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)prod1;
    const uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)prod0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                 uint32_t c3, uint32_t w[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {c0, c1, c2, c3};
  oracle_philox4x32_10(key, ctr, w);
}

/* Uniform gene in [-1, 1): a signed 24-bit integer times 2^-23 (exact). */
static float uniform_gene(uint32_t w) {
  return (float)((int32_t)(w >> 8) - 8388608) * (1.0f / 8388608.0f);
}

int oracle_init_population(uint64_t seed, int32_t P, int32_t K, float* pop) {
  if (P < 0 || K < 1 || !pop) return -1;
  for (int32_t p = 0; p < P; ++p)
    for (int32_t k = 0; k < K; ++k) {
      uint32_t w[4];
      draw(seed, 0u, (uint32_t)p, (uint32_t)k, TAG_INIT, w);
      pop[(int64_t)p * K + k] = uniform_gene(w[0]);
    }
  return 0;
}

/* Ranking key: lower fitness is better, NaN counts as +infinity, equal
 * fitness goes to the lower index. Returns nonzero if (fa, a) beats (fb, b). */
static int better(double fa, int32_t a, double fb, int32_t b) {
  if (isnan(fa)) fa = INFINITY;
  if (isnan(fb)) fb = INFINITY;
  if (fa < fb) return 1;
  if (fa > fb) return 0;
  return a < b;
}

/* Standard normal from the Irwin-Hall sum of twelve 24-bit uniforms:
 * z = (sum_i u_i - 6 * 2^24) * 2^-24, the sum exact in 64-bit integers and
 * converted to FP32 with round-to-nearest-even. */
static float irwin_hall_12(uint64_t seed, uint32_t g, uint32_t s, uint32_t k) {
  int64_t sum = 0;
  const uint32_t tags[3] = {TAG_G0, TAG_G1, TAG_G2};
  for (int t = 0; t < 3; ++t) {
    uint32_t w[4];
    draw(seed, g, s, k, tags[t], w);
    for (int i = 0; i < 4; ++i) sum += (int64_t)(w[i] >> 8);
  }
  const float centred = (float)(sum - (int64_t)6 * 16777216);
  return centred * (1.0f / 16777216.0f);
}

/* Roulette weight of a fitness value (lower fitness is better, so the wheel
 * turns on the maximised transform 1 / (1 + fit)): the integer
 * floor(2^32 * (1 / (1 + fit))) with FP64 rounding of the sum and the
 * quotient; 0 for a NaN, negative or infinite fitness. */
static uint64_t roulette_weight(double f) {
  if (!(f >= 0.0) || isinf(f)) return 0;
  const double w = 1.0 / (1.0 + f);
  return (uint64_t)(w * 4294967296.0);
}

/* Selection tables over the P current chromosomes: for ranking, order[r] =
 * the chromosome of rank r (0 = best); for roulette, the weights and their
 * total. */
typedef struct {
  int32_t* order;
  uint64_t* weight;
  uint64_t total;
} selection_tables;

/* Parent r (0 or 1) of pair q. Every mode takes its random words from
 * Philox(seed; g, q, r, TOUR | call << 8). */
static int32_t select_parent(const double* fit, int32_t P, const oracle_ga_params* prm,
                             const selection_tables* tab, uint64_t seed, uint32_t g,
                             uint32_t q, uint32_t r) {
  uint32_t w[4];
  if (prm->selection == ORACLE_SEL_RANKING) {
    /* u uniform on [0, W), W = P (P + 1) / 2; rank k covers the u with
     * sum_{j<k} (P - j) <= u < sum_{j<=k} (P - j). */
    draw(seed, g, q, r, TAG_TOUR, w);
    const uint64_t u = ((uint64_t)w[0] * tab->total) >> 32;
    uint64_t cum = 0;
    for (int32_t k = 0; k < P; ++k) {
      cum += (uint64_t)(P - k);
      if (u < cum) return tab->order[k];
    }
    return tab->order[P - 1];
  }
  if (prm->selection == ORACLE_SEL_ROULETTE) {
    /* u uniform on [0, W) from 64 random bits, W = sum of the weights;
     * chromosome p covers [sum_{j<p} w_j, sum_{j<=p} w_j). */
    draw(seed, g, q, r, TAG_TOUR, w);
    if (tab->total == 0) return (int32_t)(((uint64_t)w[0] * (uint64_t)P) >> 32);
    const uint64_t bits = ((uint64_t)w[0] << 32) | w[1];
    const uint64_t u = (uint64_t)(((unsigned __int128)bits * tab->total) >> 64);
    uint64_t cum = 0;
    for (int32_t p = 0; p < P; ++p) {
      cum += tab->weight[p];
      if (u < cum) return p;
    }
    return P - 1;
  }
  /* tournament: the best of T uniform candidates */
  int32_t win = -1;
  for (int32_t s = 0; s < prm->tournament; ++s) {
    if (s % 4 == 0) draw(seed, g, q, r, TAG_TOUR | ((uint32_t)(s / 4) << 8), w);
    const int32_t c = (int32_t)(((uint64_t)w[s % 4] * (uint64_t)P) >> 32);
    if (win < 0 || better(fit[c], c, fit[win], win)) win = c;
  }
  return win;
}

int oracle_generation(const float* pop, const double* fit, int32_t P,
                      int32_t K, const oracle_ga_params* prm, uint64_t seed,
                      uint32_t g, float* next) {
  return oracle_offspring(pop, fit, P, K, prm, seed, g, P, next);
}

int oracle_offspring(const float* pop, const double* fit, int32_t P, int32_t K,
                     const oracle_ga_params* prm, uint64_t seed, uint32_t g,
                     int32_t n_out, float* next) {
  if (!pop || !fit || !next || !prm || K < 1) return -1;
  const int32_t E = prm->elitism, T = prm->tournament, I = prm->immigrants;
  if (E < 0 || T < 1 || I < 0 || P < E + I + 2 || n_out < E + I + 2) return -1;
  if (prm->selection < ORACLE_SEL_TOURNAMENT || prm->selection > ORACLE_SEL_ROULETTE) return -1;
  if (prm->selection == ORACLE_SEL_RANKING && P > 65535) return -1;

  /* 0. Selection tables (ranking: the order by (fitness, index), each
   * chromosome's rank counted as the number that beat it; roulette: the
   * weights). */
  selection_tables tab = {NULL, NULL, 0};
  if (prm->selection == ORACLE_SEL_RANKING) {
    tab.order = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
    if (!tab.order) return -2;
    for (int32_t p = 0; p < P; ++p) {
      int32_t rank = 0;
      for (int32_t q = 0; q < P; ++q) rank += better(fit[q], q, fit[p], p);
      tab.order[rank] = p;
    }
    tab.total = (uint64_t)P * (uint64_t)(P + 1) / 2;
  } else if (prm->selection == ORACLE_SEL_ROULETTE) {
    tab.weight = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)P);
    if (!tab.weight) return -2;
    for (int32_t p = 0; p < P; ++p) {
      tab.weight[p] = roulette_weight(fit[p]);
      tab.total += tab.weight[p];
    }
  }

  /* 1. Elitism: the E best by (fitness, index) are copied unchanged. */
  int32_t* chosen = (int32_t*)calloc((size_t)P, sizeof(int32_t));
  if (!chosen) {
    free(tab.order);
    free(tab.weight);
    return -2;
  }
  for (int32_t e = 0; e < E; ++e) {
    int32_t best = -1;
    for (int32_t p = 0; p < P; ++p)
      if (!chosen[p] && (best < 0 || better(fit[p], p, fit[best], best)))
        best = p;
    chosen[best] = 1;
    memcpy(next + (int64_t)e * K, pop + (int64_t)best * K, sizeof(float) * K);
  }
  free(chosen);

  /* 2.-3. Pairs of parents selected from the P current chromosomes,
   * one-point crossover, children in slots E.. n_out-1. */
  const int32_t npairs = (n_out - E + 1) / 2;
  for (int32_t q = 0; q < npairs; ++q) {
    int32_t parent[2];
    for (int r = 0; r < 2; ++r)
      parent[r] = select_parent(fit, P, prm, &tab, seed, g, (uint32_t)q, (uint32_t)r);
    uint32_t w[4];
    draw(seed, g, (uint32_t)q, 0u, TAG_XO, w);
    int32_t cut = K; /* no crossover: children are copies of the parents */
    if ((w[0] >> 8) < prm->thr_pc)
      cut = 1 + (int32_t)(((uint64_t)w[1] * (uint64_t)(K - 1)) >> 32);
    const float* p0 = pop + (int64_t)parent[0] * K;
    const float* p1 = pop + (int64_t)parent[1] * K;
    for (int c = 0; c < 2; ++c) {
      const int32_t slot = E + 2 * q + c;
      if (slot >= n_out) continue;
      const float* head = c == 0 ? p0 : p1;
      const float* tail = c == 0 ? p1 : p0;
      float* child = next + (int64_t)slot * K;
      for (int32_t k = 0; k < K; ++k) child[k] = k < cut ? head[k] : tail[k];
    }
  }

  /* 4. Per-gene Gaussian mutation of every non-elite slot, then clamp. */
  for (int32_t s = E; s < n_out; ++s)
    for (int32_t k = 0; k < K; ++k) {
      uint32_t w[4];
      draw(seed, g, (uint32_t)s, (uint32_t)k, TAG_MUT, w);
      if ((w[0] >> 8) >= prm->thr_pm) continue;
      const float z = irwin_hall_12(seed, g, (uint32_t)s, (uint32_t)k);
      const float step = prm->sigma * z;
      float v = next[(int64_t)s * K + k] + step;
      if (v < -1.0f) v = -1.0f;
      if (v > 1.0f) v = 1.0f;
      next[(int64_t)s * K + k] = v;
    }

  /* 5. Immigrants: the last I slots are replaced by fresh random genes. */
  for (int32_t s = n_out - I; s < n_out; ++s)
    for (int32_t k = 0; k < K; ++k) {
      uint32_t w[4];
      draw(seed, g, (uint32_t)s, (uint32_t)k, TAG_IMM, w);
      next[(int64_t)s * K + k] = uniform_gene(w[0]);
    }
  free(tab.order);
  free(tab.weight);
  return 0;
}

int oracle_select_best(const double* fit, int32_t P, int32_t n, int32_t* idx) {
  if (!fit || !idx || P < 1 || n < 0 || n > P) return -1;
  unsigned char* taken = (unsigned char*)calloc((size_t)P, 1);
  if (!taken) return -2;
  for (int32_t r = 0; r < n; ++r) {
    int32_t best = -1;
    for (int32_t p = 0; p < P; ++p)
      if (!taken[p] && (best < 0 || better(fit[p], p, fit[best], best))) best = p;
    taken[best] = 1;
    idx[r] = best;
  }
  free(taken);
  return 0;
}

int oracle_rescore(const double* X, const double* y, int64_t M, int32_t N,
                   int32_t d, int32_t basis, const float* pop, int32_t P,
                   const double* fit_in, int32_t n, double* fit_out,
                   int32_t* idx) {
  const int64_t K = oracle_num_genes(N, d, basis);
  if (K < 1 || !pop || !fit_in || !fit_out || !idx) return -1;
  int rc = oracle_select_best(fit_in, P, n, idx);
  if (rc) return rc;
  memcpy(fit_out, fit_in, sizeof(double) * P);
  double* a = (double*)malloc(sizeof(double) * K);
  if (!a) return -2;
  for (int32_t r = 0; r < n && !rc; ++r) {
    for (int64_t k = 0; k < K; ++k) a[k] = (double)pop[(int64_t)idx[r] * K + k];
    rc = oracle_fitness(X, y, M, N, d, basis, a, 1, &fit_out[idx[r]]);
  }
  free(a);
  return rc;
}

/* The GA run behind oracle_train (tied = 0) and oracle_train_tied (1). */
static int train_run(const double* X, const double* y, int64_t M, int32_t N,
                     int32_t d, int32_t basis, int32_t P,
                     const oracle_ga_params* prm, uint64_t seed, int32_t G,
                     int32_t use_gram, int32_t tied, float* pop, double* fit,
                     double* best) {
  const int64_t K = tied ? oracle_num_genes_tied(d, basis) : oracle_num_genes(N, d, basis);
  if (K < 1 || M < 1 || G < 0 || !prm || P < prm->elitism + prm->immigrants + 2 ||
      (tied && use_gram))
    return -1;
  double* Gm = NULL;
  double* bv = NULL;
  double yy = 0.0;
  double* popd = (double*)malloc(sizeof(double) * P * K);
  float* next = (float*)malloc(sizeof(float) * P * K);
  int rc = (popd && next) ? 0 : -2;
  if (!rc && use_gram) {
    Gm = (double*)malloc(sizeof(double) * K * K);
    bv = (double*)malloc(sizeof(double) * K);
    rc = (Gm && bv) ? oracle_gram(X, y, M, N, d, basis, Gm, bv, &yy) : -2;
  }
  if (!rc) rc = oracle_init_population(seed, P, (int32_t)K, pop);
  for (int32_t g = 0; !rc && g <= G; ++g) {
    if (g > 0) {
      rc = oracle_generation(pop, fit, P, (int32_t)K, prm, seed,
                             (uint32_t)(g - 1), next);
      memcpy(pop, next, sizeof(float) * P * K);
    }
    for (int64_t i = 0; i < P * K; ++i) popd[i] = (double)pop[i];
    if (!rc)
      rc = use_gram ? oracle_fitness_gram(Gm, bv, yy, M, (int32_t)K, popd, P, fit)
           : tied   ? oracle_fitness_tied(X, y, M, N, d, basis, popd, P, fit)
                    : oracle_fitness(X, y, M, N, d, basis, popd, P, fit);
    double bf = INFINITY;
    for (int32_t p = 0; p < P; ++p)
      if (fit[p] < bf) bf = fit[p];
    if (best) best[g] = bf;
  }
  free(popd);
  free(next);
  free(Gm);
  free(bv);
  return rc;
}

int oracle_train(const double* X, const double* y, int64_t M, int32_t N,
                 int32_t d, int32_t basis, int32_t P,
                 const oracle_ga_params* prm, uint64_t seed, int32_t G,
                 int32_t use_gram, float* pop, double* fit, double* best) {
  return train_run(X, y, M, N, d, basis, P, prm, seed, G, use_gram, 0, pop, fit, best);
}

int oracle_train_tied(const double* X, const double* y, int64_t M, int32_t N,
                      int32_t d, int32_t basis, int32_t P,
                      const oracle_ga_params* prm, uint64_t seed, int32_t G,
                      float* pop, double* fit, double* best) {
  return train_run(X, y, M, N, d, basis, P, prm, seed, G, 0, 1, pop, fit, best);
}

int oracle_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
