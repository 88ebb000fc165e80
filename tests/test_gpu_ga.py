"""The GPU operators are bit-exact against the oracle's: initial population,
and one generation (elitism, tournament, crossover, mutation, clamp,
immigrants) given the same population, fitness vector, seed and generation;
along a real training trajectory; and across checkpoint / resume."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, fp32_tol
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def problem_with_K(N, d, basis=CHEB, M=300, seed=1):
    return dg.regression(seed, M, N, min(d, 3), 0.05, degree=d, basis=basis)


@pytest.mark.parametrize("P,N,d,seed", [(64, 8, 4, 1), (33, 3, 2, 99), (1024, 32, 8, 2),
                                        (5, 1, 1, 2**40 + 7)])
def test_init_population_bit_exact(orc, P, N, d, seed):
    pr = problem_with_K(N, d)
    with game.Game(pr.X, pr.y, d, CHEB, P=P, seed=seed) as g:
        pop, fit, gen = g.population()
    assert gen == 0
    np.testing.assert_array_equal(bits(pop), bits(orc.init_population(seed, P, pr.K)))


OPS = [
    # P, N, d, E, T, I, pc, pm, sigma
    (64, 8, 4, 2, 3, 0, 0.9, 0.02, 0.1),
    (65, 8, 4, 2, 3, 0, 0.9, 0.02, 0.1),     # odd number of children
    (1024, 32, 8, 2, 3, 0, 0.9, 0.02, 0.1),
    (50, 3, 3, 0, 1, 0, 1.0, 0.5, 0.7),      # no elites, random selection, heavy clamping
    (40, 2, 5, 5, 7, 3, 0.5, 0.2, 0.3),      # tournament over two Philox calls, immigrants
    (9, 1, 1, 3, 64, 0, 0.9, 1.0, 2.0),      # K = 2, every gene mutated
    (2048, 48, 6, 2, 3, 0, 0.9, 0.02, 0.1),
]


@pytest.mark.parametrize("P,N,d,E,T,I,pc,pm,sigma", OPS)
def test_generation_bit_exact(orc, P, N, d, E, T, I, pc, pm, sigma):
    pr = problem_with_K(N, d)
    K = pr.K
    rng = np.random.default_rng(P * 7 + K)
    pop = dg.random_population(P + K, P, K)
    fit = rng.uniform(0.0, 2.0, P)
    fit[rng.integers(0, P, 3)] = fit[0]            # ties
    fit[rng.integers(0, P, 2)] = np.nan            # NaN ranks last
    prm = orc.ga_params(elitism=E, tournament=T, pc=pc, pm=pm, sigma=sigma, immigrants=I)
    for g_index, seed in [(0, 11), (7, 2**33 + 5), (123456, 3)]:
        with game.Game(pr.X, pr.y, d, CHEB, P=P, elitism=E, tournament=T, immigrants=I,
                       pc=pc, pm=pm, sigma=sigma) as g:
            g.set_state(pop, fit, g_index)
            g.generation(seed)
            nxt, _, gen = g.population()
        assert gen == g_index + 1
        ref = orc.generation(pop, fit, seed, g_index, prm)
        np.testing.assert_array_equal(bits(nxt), bits(ref))


@pytest.mark.parametrize("prec", [game.GAME_PREC_FP32, game.GAME_PREC_BF16])
def test_training_trajectory(orc, prec):
    """Each generation of a GPU run equals the oracle's operators applied to
    the GPU's own population and fitness; the fitness tracks the oracle's;
    the elitist best never worsens."""
    pr = dg.small_regression()
    seed = 17
    prm = orc.ga_params()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=seed, precision=prec) as g:
        pop, fit, gen = g.population()
        best = [fit.min()]
        for step in range(25):
            g.generation(seed)
            nxt, nfit, ngen = g.population()
            assert ngen == gen + 1
            np.testing.assert_array_equal(bits(nxt), bits(orc.generation(pop, fit, seed, gen,
                                                                         prm)))
            if prec == game.GAME_PREC_FP32 and step % 6 == 0:
                ref = orc.fitness(pr.X, pr.y, nxt, pr.degree, CHEB)
                assert np.all(np.abs(nfit - ref) <= fp32_tol(ref, pr.y))
            pop, fit, gen = nxt, nfit, ngen
            best.append(fit.min())
    assert np.all(np.diff(best) <= 0.0)
    assert best[-1] < best[0]


def test_train_and_resume():
    pr = dg.small_regression()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=5) as g:
        assert g.train(15) == 15
        pop_a, fit_a, gen_a = g.population()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=5) as g:
        g.train(6)
        ck = g.population()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=5) as g:
        g.set_state(ck[0], ck[1], ck[2])
        g.train(9)
        pop_b, fit_b, gen_b = g.population()
    assert gen_a == gen_b == 15
    np.testing.assert_array_equal(bits(pop_a), bits(pop_b))
    np.testing.assert_array_equal(fit_a, fit_b)


def test_train_stop_threshold():
    pr = dg.small_regression()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=5, mse_threshold=1e9,
                   check_every=1) as g:
        assert g.train(10) == 0      # already below the threshold
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=5, mse_threshold=1e-12) as g:
        assert g.train(4) == 4
