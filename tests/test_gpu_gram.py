"""The Gram form of the MSE on the GPU (FP64) against the oracle: G, b and
y.y against the oracle's Gram routine (itself pinned against the direct
form), and the fitness against the oracle's direct triple loop within the
FP64 rounding bound of the quadratic form."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, U64, quad_bound
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GRAM = game.GAME_PREC_GRAM

CASES = [
    (2000, 8, 4, CHEB, 64),
    (777, 3, 7, TRIG, 130),
    (1, 4, 2, CHEB, 5),
    (5000, 16, 10, TRIG, 257),
    (70001, 6, 5, CHEB, 33),    # several chunks of patterns? (one; rows split 8 ways)
    (3001, 48, 6, CHEB, 300),
]


@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
def test_gram_matches_oracle(orc, case):
    M, N, d, basis, P = case
    pr = dg.regression(M + 7, M, N, min(d, 4), 0.05, degree=d, basis=basis)
    pop = dg.random_population(P + 2, P, pr.K)
    Go, bo, yyo, _ = orc.gram(pr.X, pr.y, d, basis)
    with game.Game(pr.X, pr.y, d, basis, P=max(P, 4), precision=GRAM) as g:
        G, b, yy = g.gram()
        fit = g.eval_fitness(pop)
    # the two accumulations differ only in summation order and last-ulp
    # basis values: relative to the absolute sums (<= M for |phi| <= 1)
    scale = max(M, 1)
    assert np.max(np.abs(G - Go)) <= 64 * scale * U64 * 4
    assert np.max(np.abs(b - bo)) <= 64 * scale * U64 * (1 + np.max(np.abs(pr.y)))
    assert abs(yy - yyo) <= 64 * scale * U64 * np.max(pr.y.astype(np.float64) ** 2)
    np.testing.assert_array_equal(G, G.T)
    ref = orc.fitness(pr.X, pr.y, pop, d, basis)
    bound = quad_bound(Go, bo, yyo, pop, M) + np.abs(ref) * 1e-12
    assert np.all(np.abs(fit - ref) <= bound), np.max(np.abs(fit - ref) / bound)


def test_gram_ga_trajectory(orc):
    """Operators bit-exact given the device's Gram fitness; the fitness of
    the evolved population against the direct oracle."""
    pr = dg.small_regression()
    prm = orc.ga_params()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=12, precision=GRAM) as g:
        pop, fit, gen = g.population()
        for _ in range(10):
            g.generation(12)
            nxt, nfit, ngen = g.population()
            np.testing.assert_array_equal(nxt.view(np.uint32),
                                          orc.generation(pop, fit, 12, gen, prm).view(np.uint32))
            pop, fit, gen = nxt, nfit, ngen
    ref = orc.fitness(pr.X, pr.y, pop, pr.degree, CHEB)
    np.testing.assert_allclose(fit, ref, rtol=1e-9)


def test_gram_deterministic():
    pr = dg.regression(5, 3000, 12, 4, 0.05, degree=5)
    pop = dg.random_population(4, 200, pr.K)
    outs = []
    for _ in range(2):
        with game.Game(pr.X, pr.y, 5, CHEB, P=200, precision=GRAM) as g:
            outs.append((g.gram()[0], g.eval_fitness(pop)))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
