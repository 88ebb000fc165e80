"""Pins of the oracle's elite re-scoring: the candidate ranking against
numpy's lexicographic sort (fitness, then index; NaN last), and the
re-scored values against an independent numpy design-matrix MSE."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, design_matrix
from paper_1211_5481_gb300 import datagen as dg


def lexsort_best(fit, n):
    key = np.where(np.isnan(fit), np.inf, fit)
    return np.lexsort((np.arange(fit.shape[0]), key))[:n]


@pytest.mark.parametrize("P,n,seed", [(1, 1, 0), (7, 7, 1), (64, 8, 2), (1024, 16, 3),
                                      (300, 5, 4), (33, 1, 5)])
def test_select_best_is_lexicographic(orc, P, n, seed):
    rng = np.random.default_rng(seed)
    fit = rng.choice([0.5, 1.0, 2.0, 3.0], P) if seed % 2 else rng.uniform(0, 1, P)
    fit = fit.astype(np.float64)
    fit[rng.integers(0, P, max(1, P // 10))] = np.nan
    got = orc.select_best(fit, n)
    np.testing.assert_array_equal(got, lexsort_best(fit, n))


def test_select_best_all_nan_and_ties(orc):
    fit = np.full(10, np.nan)
    np.testing.assert_array_equal(orc.select_best(fit, 10), np.arange(10))
    fit = np.array([2.0, 1.0, 1.0, np.inf, 1.0, np.nan])
    np.testing.assert_array_equal(orc.select_best(fit, 6), [1, 2, 4, 0, 3, 5])


@pytest.mark.parametrize("basis", [CHEB, TRIG])
def test_rescore_replaces_only_candidates(orc, basis):
    pr = dg.regression(9, 400, 5, 3, 0.05, degree=4, basis=basis)
    P, n = 40, 6
    pop = dg.random_population(11, P, pr.K)
    rng = np.random.default_rng(1)
    fit_in = rng.uniform(0.0, 1.0, P)       # any vector: the ranking uses it as given
    fit_in[3] = np.nan
    out, idx = orc.rescore(pr.X, pr.y, pop, 4, basis, fit_in, n)
    np.testing.assert_array_equal(idx, lexsort_best(fit_in, n))
    others = np.setdiff1d(np.arange(P), idx)
    np.testing.assert_array_equal(out[others], fit_in[others])
    Phi = design_matrix(pr.X, 4, basis)
    r = pr.y.astype(np.float64)[:, None] - Phi @ pop[idx].astype(np.float64).T
    np.testing.assert_allclose(out[idx], (r * r).mean(axis=0), rtol=1e-12, atol=0)


def test_rescore_of_exact_values_is_identity(orc):
    pr = dg.regression(2, 300, 4, 3, 0.05, degree=3)
    pop = dg.random_population(5, 20, pr.K)
    exact = orc.fitness(pr.X, pr.y, pop, 3, CHEB)
    out, _ = orc.rescore(pr.X, pr.y, pop, 3, CHEB, exact, 8)
    np.testing.assert_array_equal(out, exact)
