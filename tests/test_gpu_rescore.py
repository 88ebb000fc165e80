"""Elite re-scoring on the GPU against the oracle: the candidates are the
oracle's ranking of the same input vector (exact), the re-scored values are
within the FP64 rounding bound of the Gram form (the quadratic form's
roundings, tests/helpers.quad_bound, plus 1e-12 relative for the
expansion's last FP64 bits) of the FP64 oracle fitness -- an FP32 slip
anywhere in the re-score fails it -- and every other entry is unchanged;
and the GA state of a BF16 handle carries the re-scored values."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, quad_bound
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BF16 = game.GAME_PREC_BF16


def rescore_tol(orc, X, y, pop, d, basis, ref):
    """FP64 rounding bound of the Gram-form re-score of pop's rows."""
    G, b, yy, _ = orc.gram(X, y, d, basis)
    return quad_bound(G, b, yy, pop, X.shape[0]) + 1e-12 * np.abs(ref)


CASES = [
    # M, N, d, basis, P, n
    (2000, 8, 4, CHEB, 64, 8),
    (777, 3, 7, TRIG, 130, 16),     # two candidate groups, ragged M
    (1, 4, 2, CHEB, 5, 5),          # one pattern, n = P
    (5000, 16, 10, TRIG, 257, 9),   # second group with one candidate
    (513, 64, 10, TRIG, 33, 3),     # K' = 1280
    (70001, 32, 8, CHEB, 1024, 8),  # several pattern slices per CTA
]


@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
def test_rescore_matches_oracle(orc, case):
    M, N, d, basis, P, n = case
    pr = dg.regression(M + 3, M, N, min(d, 4), 0.05, degree=d, basis=basis)
    pop = dg.random_population(P + 1, P, pr.K)
    with game.Game(pr.X, pr.y, d, basis, P=max(P, 4), precision=BF16) as g:
        fbf = g.eval_fitness(pop)
        got, idx = g.rescore_top(pop, fbf, n)
    want_idx = orc.select_best(fbf, n)
    np.testing.assert_array_equal(idx, want_idx)
    others = np.setdiff1d(np.arange(P), idx)
    np.testing.assert_array_equal(got[others], fbf[others])
    ref = orc.fitness(pr.X, pr.y, pop[idx], d, basis)
    err = np.abs(got[idx] - ref)
    tol = rescore_tol(orc, pr.X, pr.y, pop[idx], d, basis, ref)
    assert np.all(err <= tol), (err / tol).max()


def test_rescore_ranking_with_ties_and_nan(orc):
    pr = dg.regression(4, 1000, 6, 3, 0.05, degree=3)
    P = 300
    pop = dg.random_population(8, P, pr.K)
    rng = np.random.default_rng(3)
    fit = rng.choice([0.25, 0.5, 1.0], P).astype(np.float64)
    fit[rng.integers(0, P, 20)] = np.nan
    with game.Game(pr.X, pr.y, 3, CHEB, P=8) as g:
        got, idx = g.rescore_top(pop, fit, 16)
    np.testing.assert_array_equal(idx, orc.select_best(fit, 16))
    ref = orc.fitness(pr.X, pr.y, pop[idx], 3, CHEB)
    assert np.all(np.abs(got[idx] - ref) <= rescore_tol(orc, pr.X, pr.y, pop[idx], 3, CHEB, ref))


def test_rescore_device_and_host_agree():
    pr = dg.small_regression()
    pop = dg.random_population(2, 64, pr.K)
    dev = torch.device("cuda:0")
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, precision=BF16) as g:
        fit = g.eval_fitness(pop)
        h_fit, h_idx = g.rescore_top(pop, fit, 8)
        d_fit, d_idx = g.rescore_top(torch.from_numpy(pop).to(dev),
                                     torch.from_numpy(fit).to(dev), 8)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(h_fit, d_fit.cpu().numpy())
    np.testing.assert_array_equal(h_idx, d_idx.cpu().numpy())


def test_rescore_rejects_bad_counts():
    pr = dg.small_regression()
    pop = dg.random_population(2, 10, pr.K)
    fit = np.zeros(10)
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=10) as g:
        for n in (0, 11, 17):
            with pytest.raises(game.GameError) as ei:
                g.rescore_top(pop, fit, n)
            assert ei.value.code == game.GAME_EINVAL
    with pytest.raises(game.GameError):
        game.Game(pr.X, pr.y, pr.degree, CHEB, P=10, rescore_top=17)


@pytest.mark.parametrize("top", [8, 0])
def test_ga_state_carries_rescored_values(orc, top):
    """A BF16 handle's fitness vector: its `top` best entries by the BF16
    contraction hold FP64-accurate values, the rest the BF16 values."""
    pr = dg.small_regression()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=3, precision=BF16,
                   rescore_top=top) as g:
        for _ in range(3):
            g.generation(3)
        pop, fit, _ = g.population()
        fbf = g.eval_fitness(pop)
    if top == 0:
        np.testing.assert_array_equal(fit, fbf)
        return
    idx = orc.select_best(fbf, top)
    others = np.setdiff1d(np.arange(64), idx)
    np.testing.assert_array_equal(fit[others], fbf[others])
    ref = orc.fitness(pr.X, pr.y, pop[idx], pr.degree, CHEB)
    assert np.all(np.abs(fit[idx] - ref) <= rescore_tol(orc, pr.X, pr.y, pop[idx], pr.degree,
                                                        CHEB, ref))


def test_full_size_rescore(orc):
    """The large classification workload (M = 10^6, N = 32, degree 8,
    P = 1024): the 8 re-scored candidates against the oracle."""
    pr = dg.large_classification()
    P = 1024
    pop = orc.init_population(2, P, pr.K)
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    with game.Game(Xd, yd, pr.degree, CHEB, P=P, precision=BF16) as g:
        fbf = g.eval_fitness(pop)
        got, idx = g.rescore_top(pop, fbf, 8)
    np.testing.assert_array_equal(idx, orc.select_best(fbf, 8))
    ref = orc.fitness(pr.X, pr.y, pop[idx], pr.degree, CHEB)
    assert np.all(np.abs(got[idx] - ref) <= rescore_tol(orc, pr.X, pr.y, pop[idx], pr.degree,
                                                        CHEB, ref))
