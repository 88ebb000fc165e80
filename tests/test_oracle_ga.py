"""Pins of the oracle's GA operators by invariants the definitions fix:
constant population size, verbatim elites, crossover that only exchanges
genes inside a parent pair, genes kept in [-1, 1], elitist best fitness that
never worsens, exact resume, and the rates of the random decisions."""
import numpy as np
import pytest

from paper_1211_5481_gb300 import datagen as dg

CHEB = 0


def _fit_key(f):
    return np.where(np.isnan(f), np.inf, f)


def _elites(fit, E):
    order = np.lexsort((np.arange(fit.size), _fit_key(fit)))
    return order[:E]


def test_init_population_range_and_uniformity(orc):
    pop = orc.init_population(42, 256, 33)
    assert pop.dtype == np.float32 and pop.shape == (256, 33)
    assert pop.min() >= -1.0 and pop.max() < 1.0
    # U[-1,1): mean 0, variance 1/3
    assert abs(pop.mean()) < 0.01 and abs(pop.var() - 1 / 3) < 0.01
    # genes are multiples of 2^-23
    assert np.all(pop * 2.0**23 == np.round(pop * 2.0**23))
    # different seeds give different populations, same seed the same one
    assert not np.array_equal(pop, orc.init_population(43, 256, 33))
    assert np.array_equal(pop, orc.init_population(42, 256, 33))


@pytest.mark.parametrize("P,E", [(64, 2), (65, 2), (10, 0), (9, 3)])
def test_generation_invariants(orc, P, E):
    K = 17
    rng = np.random.default_rng(P + E)
    pop = orc.init_population(7, P, K)
    fit = rng.uniform(0, 1, P)
    fit[3] = fit[5]  # a tie, broken by the lower index
    prm = orc.ga_params(elitism=E, pm=0.0)   # no mutation: pure crossover
    nxt = orc.generation(pop, fit, 77, 3, prm)
    assert nxt.shape == pop.shape
    # elites verbatim, in rank order
    for e, src in enumerate(_elites(fit, E)):
        np.testing.assert_array_equal(nxt[e], pop[src])
    # every child gene comes from a population member at the same locus, and
    # each pair's two children hold, per locus, the genes of two parents
    for s in range(E, P):
        for k in range(K):
            assert nxt[s, k] in pop[:, k]
    for q in range((P - E) // 2):
        a, b = nxt[E + 2 * q], nxt[E + 2 * q + 1]
        # find the parents: members whose genes match at locus 0 and K-1
        pa = [p for p in range(P) if pop[p, 0] == a[0]]
        pb = [p for p in range(P) if pop[p, 0] == b[0]]
        ok = False
        for i in pa:
            for j in pb:
                if all(sorted((a[k], b[k])) == sorted((pop[i, k], pop[j, k]))
                       for k in range(K)):
                    ok = True
        assert ok, f"pair {q} is not a crossover of two members"
    assert np.all(np.abs(nxt) <= 1.0)


def _tagged_population(P, K):
    """Member p holds gene (p*K + k) * 2^-20 at locus k, so the source member
    and locus of any copied gene can be read back exactly."""
    assert P * K < 2**20
    return ((np.arange(P)[:, None] * K + np.arange(K)[None, :]) * 2.0**-20).astype(np.float32)


def _source(pop_tagged, v, K):
    idx = np.round(np.asarray(v, dtype=np.float64) * 2.0**20).astype(np.int64)
    return idx // K, idx % K


def test_crossover_is_one_point(orc):
    """Each child is a head of one parent joined to the tail of the other at a
    single cut in [1, K-1] (or an unchanged copy); genes keep their locus."""
    P, K = 40, 25
    pop = _tagged_population(P, K)
    fit = np.linspace(1, 2, P)
    nxt = orc.generation(pop, fit, 5, 0, orc.ga_params(elitism=2, pm=0.0))
    for s in range(2, P):
        member, locus = _source(pop, nxt[s], K)
        np.testing.assert_array_equal(locus, np.arange(K))
        assert np.count_nonzero(np.diff(member)) <= 1
    for q in range((P - 2) // 2):
        ma, _ = _source(pop, nxt[2 + 2 * q], K)
        mb, _ = _source(pop, nxt[3 + 2 * q], K)
        # the two children hold complementary parents at every locus
        for k in range(K):
            assert sorted((ma[k], mb[k])) == sorted((ma[0], mb[0]))
        cut_a = np.nonzero(np.diff(ma))[0]
        cut_b = np.nonzero(np.diff(mb))[0]
        np.testing.assert_array_equal(cut_a, cut_b)


def test_rates(orc):
    """Crossover happens for ~pc of the pairs, mutation for ~pm of the
    genes, and the Irwin-Hall steps have mean 0 and sd sigma."""
    P, K = 402, 65
    pop = _tagged_population(P, K)
    fit = np.arange(P, dtype=np.float64)
    pc = 0.6
    crossed = pairs = same = 0
    for g in range(10):
        nxt = orc.generation(pop, fit, 11, g, orc.ga_params(elitism=2, pc=pc, pm=0.0))
        for q in range((P - 2) // 2):
            ma, _ = _source(pop, nxt[2 + 2 * q], K)
            mb, _ = _source(pop, nxt[3 + 2 * q], K)
            same += ma[0] == mb[0]
            crossed += ma[0] != ma[-1]
            pairs += 1
    # a crossed pair of identical parents looks uncrossed; count those out
    assert abs(crossed / (pairs - same) - pc) < 0.04
    pm, sigma = 0.05, 0.01
    zero = np.zeros((P, K), dtype=np.float32)   # children = sigma * z exactly
    steps = []
    for g in range(4):
        nxt = orc.generation(zero, fit, 13, g, orc.ga_params(elitism=2, pc=0.9, pm=pm,
                                                            sigma=sigma))
        assert np.all(nxt[:2] == 0)
        steps.append(nxt[2:].reshape(-1))
    steps = np.concatenate(steps).astype(np.float64)
    mutated = steps[steps != 0]
    assert abs(mutated.size / steps.size - pm) < 0.004
    assert abs(mutated.mean()) < 0.05 * sigma
    assert abs(mutated.std() / sigma - 1) < 0.05
    # Irwin-Hall-12 is bounded by 6 sd
    assert np.abs(mutated).max() <= 6 * sigma * (1 + 1e-6)


def test_tournament_prefers_fitter(orc):
    """With tournaments of 3 the chance of selecting the best-ranked member
    is 1 - (1 - 1/P)^3 per draw; the top decile dominates the parents."""
    P, K = 200, 9
    pop = np.zeros((P, K), dtype=np.float32)
    pop[:, 0] = np.arange(P) / 256.0       # identifies the member
    fit = np.arange(P, dtype=np.float64)   # member p has rank p
    prm = orc.ga_params(elitism=0, pc=0.0, pm=0.0)
    ranks = []
    for g in range(20):
        nxt = orc.generation(pop, fit, 21, g, prm)
        ranks.extend((nxt[:, 0] * 256).round().astype(int).tolist())
    ranks = np.array(ranks)
    # P(rank < P/10) for the min of 3 uniform draws = 1 - 0.9^3 = 0.271
    assert abs(np.mean(ranks < P // 10) - 0.271) < 0.03
    # the worst member can only win when drawn three times
    assert np.mean(ranks == P - 1) < 0.001


@pytest.mark.parametrize("T", [1, 2, 3])
def test_tournament_win_probability_closed_form(orc, T):
    """Tournaments draw T candidates uniformly with replacement and keep the
    best, so the member of rank r (0 = best) wins with probability
    ((P - r)^T - (P - r - 1)^T) / P^T; with T = 1 the draw is uniform, and
    even the worst member wins when every candidate is it."""
    P = 6
    fit = np.array([0.4, 0.1, 0.9, 0.3, 0.6, 0.2])   # ranks 3 0 5 2 4 1
    rank = np.argsort(np.argsort(fit))
    counts = _parent_counts(orc, fit, orc.SEL_TOURNAMENT, 60000, tournament=T)
    prob = ((P - rank) ** T - (P - rank - 1.0) ** T) / float(P) ** T
    assert _within_binomial(counts, prob)
    assert counts[np.argmax(rank)] > 0


def test_nan_fitness_never_elite(orc):
    P, K = 12, 5
    pop = orc.init_population(1, P, K)
    fit = np.linspace(0.1, 1.0, P)
    fit[0] = np.nan
    nxt = orc.generation(pop, fit, 2, 0, orc.ga_params(elitism=2))
    np.testing.assert_array_equal(nxt[0], pop[1])
    np.testing.assert_array_equal(nxt[1], pop[2])


def test_immigrants_fill_last_slots(orc):
    P, K, I = 20, 7, 3
    pop = orc.init_population(1, P, K)
    fit = np.linspace(0.1, 1.0, P)
    nxt = orc.generation(pop, fit, 4, 2, orc.ga_params(elitism=2, immigrants=I))
    fresh = nxt[P - I:]
    assert np.all(fresh >= -1) and np.all(fresh < 1)
    assert np.all(fresh * 2.0**23 == np.round(fresh * 2.0**23))
    assert not np.any([np.any(np.all(pop == r, axis=1)) for r in fresh])


def test_generation_rejects_bad_params(orc):
    pop = orc.init_population(1, 4, 5)
    with pytest.raises(ValueError):
        orc.generation(pop, np.zeros(4), 1, 0, orc.ga_params(elitism=3))
    with pytest.raises(ValueError):
        orc.generation(pop, np.zeros(4), 1, 0, orc.ga_params(tournament=0))


def test_train_elitist_best_never_worsens(orc):
    pr = dg.regression(21, 400, 4, 3, 0.05, degree=3)
    _, fit, best = orc.train(pr.X, pr.y, 3, CHEB, 24, 30, seed=5)
    assert np.all(np.diff(best) <= 0.0)
    assert best[-1] < best[0]
    assert best[-1] == fit.min()


def test_train_resume_is_exact(orc):
    """Counter-based draws depend only on (seed, g, slot, gene): running
    G1 generations, then continuing from that state, equals one run of
    G1 + G2 generations."""
    pr = dg.regression(22, 300, 3, 2, 0.05, degree=2)
    prm = orc.ga_params()
    pop_full, fit_full, _ = orc.train(pr.X, pr.y, 2, CHEB, 16, 12, seed=8, prm=prm)
    pop, fit, _ = orc.train(pr.X, pr.y, 2, CHEB, 16, 5, seed=8, prm=prm)
    for g in range(5, 12):
        pop = orc.generation(pop, fit, 8, g, prm)
        fit = orc.fitness(pr.X, pr.y, pop, 2, CHEB)
    np.testing.assert_array_equal(pop, pop_full)
    np.testing.assert_array_equal(fit, fit_full)


def test_train_gram_matches_direct(orc):
    pr = dg.regression(23, 300, 3, 2, 0.05, degree=2)
    pd_, fd, bd = orc.train(pr.X, pr.y, 2, CHEB, 16, 6, seed=9)
    pg, fg, bg = orc.train(pr.X, pr.y, 2, CHEB, 16, 6, seed=9, use_gram=True)
    np.testing.assert_allclose(bg, bd, rtol=1e-9)


def test_cut_points_uniform(orc):
    """The cut is uniform over [1, K-1]: with K = 5 each head length 1..4
    occurs for about a quarter of the crossed pairs."""
    P, K = 402, 5
    pop = _tagged_population(P, K)
    fit = np.arange(P, dtype=np.float64)
    heads = []
    for g in range(6):
        nxt = orc.generation(pop, fit, 17, g, orc.ga_params(elitism=2, pc=1.0, pm=0.0))
        for q in range((P - 2) // 2):
            ma, _ = _source(pop, nxt[2 + 2 * q], K)
            mb, _ = _source(pop, nxt[3 + 2 * q], K)
            if ma[0] == mb[0]:
                continue   # identical parents: the cut is invisible
            heads.append(int(np.count_nonzero(ma == ma[0])))
    counts = np.bincount(heads, minlength=K + 1)
    assert counts[0] == 0 and counts[K] == 0
    frac = counts[1:K] / len(heads)
    assert np.all(np.abs(frac - 0.25) < 0.04)


def test_mutation_clamps_both_ends(orc):
    """Genes at the bounds pushed by large steps stay in [-1, 1] and land
    exactly on the bound when the step overshoots."""
    P, K = 64, 33
    pop = np.ones((P, K), dtype=np.float32)
    pop[P // 2:] = -1.0
    fit = np.arange(P, dtype=np.float64)
    nxt = orc.generation(pop, fit, 3, 0, orc.ga_params(elitism=2, pc=0.0, pm=1.0, sigma=0.5))
    assert nxt.min() >= -1.0 and nxt.max() <= 1.0
    child = nxt[2:]
    # half the steps overshoot: many genes sit exactly on a bound, the rest
    # moved inwards
    assert np.count_nonzero(np.abs(child) == 1.0) > 0.3 * child.size
    assert np.count_nonzero(np.abs(child) < 1.0) > 0.3 * child.size


def _parent_counts(orc, fit, selection, n_out, seeds=(5,), g=0, tournament=3):
    """Selection frequencies: with no crossover, mutation, elites or
    immigrants each child slot is a copy of one selected parent, identified
    by gene 0."""
    P = fit.size
    pop = np.zeros((P, 3), dtype=np.float32)
    pop[:, 0] = np.arange(P) / 2.0**20
    prm = orc.ga_params(elitism=0, pc=0.0, pm=0.0, selection=selection, tournament=tournament)
    counts = np.zeros(P)
    for seed in seeds:
        nxt = orc.offspring(pop, fit, seed, g, n_out, prm)
        counts += np.bincount((nxt[:, 0] * 2.0**20).round().astype(int), minlength=P)
    return counts


def _within_binomial(counts, prob, z=5.0):
    n = counts.sum()
    sd = np.sqrt(n * prob * (1 - prob))
    return np.all(np.abs(counts - n * prob) <= z * sd + 1e-9)


def test_ranking_selection_is_linear_in_rank(orc):
    """Linear ranking: the member of rank r (0 = best) is drawn with
    probability (P - r) / (P (P + 1) / 2), whatever the fitness values."""
    P = 7
    fit = np.array([0.3, 5.0, 0.1, 2.0, 0.2, 9.0, 1.0])   # ranks 2 5 0 4 1 6 3
    rank = np.argsort(np.argsort(fit))
    counts = _parent_counts(orc, fit, orc.SEL_RANKING, 60000)
    prob = (P - rank) / (P * (P + 1) / 2)
    assert _within_binomial(counts, prob)
    # only the ranks matter: a monotone transform of fit draws the same parents
    np.testing.assert_array_equal(counts, _parent_counts(orc, np.exp(fit), orc.SEL_RANKING, 60000))


def test_ranking_ties_and_nan(orc):
    """Equal fitness ranks by index; NaN ranks last (weight 1)."""
    fit = np.array([1.0, 1.0, 1.0, np.nan])
    counts = _parent_counts(orc, fit, orc.SEL_RANKING, 40000)
    assert _within_binomial(counts, np.array([4, 3, 2, 1]) / 10.0)


def test_roulette_selection_is_proportional(orc):
    """Roulette on 1 / (1 + fit): probability proportional to it; NaN and
    infinite fitness are never drawn."""
    fit = np.array([0.0, 1.0, 3.0, 9.0, np.nan, np.inf, 0.5])
    w = np.where(np.isfinite(fit), 1.0 / (1.0 + np.nan_to_num(fit, nan=0.0)), 0.0)
    counts = _parent_counts(orc, fit, orc.SEL_ROULETTE, 60000)
    assert counts[4] == 0 and counts[5] == 0
    assert _within_binomial(counts, w / w.sum())


def test_roulette_all_zero_weights_is_uniform(orc):
    fit = np.full(5, np.nan)
    counts = _parent_counts(orc, fit, orc.SEL_ROULETTE, 50000)
    assert _within_binomial(counts, np.full(5, 0.2))


def test_roulette_exact_integer_weights(orc):
    """The weights are the integers floor(2^32 / (1 + fit)): fit = 2^32 - 1
    has weight exactly 1 and fit = 2^32 weight 0, so with weights (1, 0, 1, 1)
    u is uniform on {0, 1, 2} and member p covers [sum_{j<p} w_j,
    sum_{j<=p} w_j): members 0, 2, 3 each a third, member 1 never."""
    fit = np.array([2.0**32 - 1, 2.0**32, 2.0**32 - 1, 2.0**32 - 1])
    counts = _parent_counts(orc, fit, orc.SEL_ROULETTE, 30000)
    assert counts[1] == 0
    assert _within_binomial(counts, np.array([1, 0, 1, 1]) / 3.0)


def test_roulette_large_fitness_spread(orc):
    """A fitness of 1e12 has the integer weight floor(2^32 / (1 + 1e12)) = 0,
    so it is never drawn next to fit = 0 (weight 2^32)."""
    fit = np.array([1e12, 0.0])
    counts = _parent_counts(orc, fit, orc.SEL_ROULETTE, 2000)
    assert counts[0] == 0 and counts[1] == 2000


@pytest.mark.parametrize("selection", [1, 2])
def test_selection_modes_keep_invariants(orc, selection):
    """Elites verbatim, population size, genes in range, under every mode."""
    P, K, E = 33, 11, 2
    rng = np.random.default_rng(selection)
    pop = orc.init_population(3, P, K)
    fit = rng.uniform(0, 1, P)
    prm = orc.ga_params(elitism=E, selection=selection)
    nxt = orc.generation(pop, fit, 9, 1, prm)
    assert nxt.shape == pop.shape and np.all(np.abs(nxt) <= 1)
    for e, src in enumerate(_elites(fit, E)):
        np.testing.assert_array_equal(nxt[e], pop[src])


def test_selection_rejects_bad_mode(orc):
    pop = orc.init_population(1, 4, 5)
    with pytest.raises(ValueError):
        orc.generation(pop, np.zeros(4), 1, 0, orc.ga_params(elitism=0, selection=3))


def test_train_tied_with_one_feature_is_the_per_feature_run(orc):
    """With N = 1 the shared-gene chromosome is the per-feature one: both
    runs are identical, bit for bit."""
    pr = dg.regression(4, 300, 1, 3, 0.05, degree=4)
    prm = orc.ga_params(selection=orc.SEL_RANKING)
    a = orc.train(pr.X, pr.y, 4, CHEB, 20, 15, 7, prm)
    b = orc.train_tied(pr.X, pr.y, 4, CHEB, 20, 15, 7, prm)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_train_tied_elitist_and_shared_genes(orc):
    pr = dg.regression(6, 500, 5, 2, 0.05, degree=3, basis=1)
    pop, fit, best = orc.train_tied(pr.X, pr.y, 3, 1, 11, 30, 2,
                                    orc.ga_params(selection=orc.SEL_ROULETTE))
    assert pop.shape == (11, 7)
    assert np.all(np.diff(best) <= 0)
    np.testing.assert_allclose(fit, orc.fitness_tied(pr.X, pr.y, pop, 3, 1), rtol=1e-14)


def test_params_struct_layout_matches_the_c_header(orc, tmp_path):
    """The ctypes mirror of oracle_ga_params has the C compiler's size and
    field offsets, so the oracle reads the rates and counts it is given."""
    import ctypes
    import os
    import subprocess
    inc = os.path.dirname(orc.__file__)
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "oracle.h"', 'int main(void) {',
             '  printf("size %zu\\n", sizeof(oracle_ga_params));']
    for name, _ in orc.GAParams._fields_:
        lines.append(f'  printf("{name} %zu\\n", offsetof(oracle_ga_params, {name}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(orc.GAParams)
    for name, _ in orc.GAParams._fields_:
        assert int(got[name]) == getattr(orc.GAParams, name).offset, name
