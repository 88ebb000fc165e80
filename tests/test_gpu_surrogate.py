"""The fitness surrogate and the screened generation against the oracle:
initial weights bit-exact, predictions within the rounding bound, gradients
and Adam steps close to the FP64 oracle, and a screened generation
bit-exact given the device's predictions (offspring, selection, assembly)."""
import numpy as np
import pytest

from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game
from oracle import surrogate as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BF16 = game.GAME_PREC_BF16


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


@pytest.fixture(scope="module")
def prob():
    return dg.small_regression()


def test_initial_weights_bit_exact(orc, prob):
    with game.Game(prob.X, prob.y, prob.degree, 0, P=64, seed=21) as g:
        w = g.surrogate_params()
    np.testing.assert_array_equal(bits(w), bits(sg.init_params(21, prob.K)))


@pytest.mark.parametrize("n", [1, 64, 1000])
def test_predictions_within_bound(orc, prob, n):
    rng = np.random.default_rng(n)
    with game.Game(prob.X, prob.y, prob.degree, 0, P=64, seed=5) as g:
        w = sg.init_params(5, prob.K)
        w = (w * 3 + rng.normal(0, 0.02, w.shape)).astype(np.float32)   # non-trivial biases too
        g.surrogate_set_params(w)
        pop = dg.random_population(n, n, prob.K)
        got = g.surrogate_predict(pop)
    ref, _ = sg.forward(w, pop, prob.K)
    bound = sg.forward_bound(w, pop, prob.K)
    assert np.all(np.abs(got - ref) <= bound + 1e-6 * np.abs(ref)), \
        np.max(np.abs(got - ref) / (bound + 1e-30))


def test_gradient_and_adam_step(orc, prob):
    rng = np.random.default_rng(1)
    pop = dg.random_population(9, 256, prob.K)
    fit = np.exp(rng.normal(0, 1, 256))
    with game.Game(prob.X, prob.y, prob.degree, 0, P=64, seed=3) as g:
        w0 = g.surrogate_params()
        gd, loss = g.surrogate_grad(pop, fit)
        g.surrogate_set_params(w0)
        g.surrogate_train(pop, fit)
        w1 = g.surrogate_params()
    lref, gref = sg.loss_and_grad(w0, pop, fit, prob.K)
    assert abs(loss - lref) <= 1e-4 * lref
    assert np.linalg.norm(gd - gref) <= 1e-3 * np.linalg.norm(gref)
    wref, _, _ = sg.adam(w0, gref, np.zeros_like(gref), np.zeros_like(gref), 1)
    big = np.abs(gref) > 1e-5
    # at t = 1 the step is lr g / (|g| + eps): close for every non-tiny gradient
    assert np.max(np.abs(w1[big] - wref[big])) <= 1e-2 * sg.LR + 1e-6
    assert np.max(np.abs(w1 - wref)) <= 2 * sg.LR + 1e-6


@pytest.mark.parametrize("P,E,S,seed", [(64, 2, 8, 4), (40, 3, 5, 2**35 + 1)])
def test_screened_generation_bit_exact(orc, prob, P, E, S, seed):
    """Offspring, screening and assembly bit-exact given the device's
    predictions; the trust check's correlation against the oracle's, and its
    verdict used by the next screening; the first screening (untrusted)
    equals the unscreened generation."""
    prm = orc.ga_params(elitism=E)
    with game.Game(prob.X, prob.y, prob.degree, 0, P=P, seed=seed, precision=BF16,
                   elitism=E, surrogate=1, oversample=S) as g:
        verdict = 0   # a fresh handle starts untrusted
        for step in range(6):
            pop, fit, gen = g.population()
            w = g.surrogate_params()
            g.generation(seed)
            nxt, nfit, ngen = g.population()
            pred, keep, trusted, r = g.surrogate_last()
            n = S * (P - E)
            assert ngen == gen + 1 and pred.shape == (n,)
            assert trusted == verdict
            off = orc.offspring(pop, fit, seed, gen, E + n, prm)
            # the device's predictions of the children, against the oracle's forward
            ref, _ = sg.forward(w, off[E:], prob.K)
            assert np.all(np.abs(pred - ref) <= sg.forward_bound(w, off[E:], prob.K)
                          + 1e-6 * np.abs(ref))
            # selection and assembly, exact given the device's predictions
            np.testing.assert_array_equal(keep, sg.select_keep(pred, P - E, trusted))
            np.testing.assert_array_equal(bits(nxt), bits(sg.screen(off, keep, E)))
            if step == 0:   # untrusted: the unscreened generation exactly
                np.testing.assert_array_equal(bits(nxt),
                                              bits(orc.generation(pop, fit, seed, gen, prm)))
            r_ref, verdict = sg.trust_check(pred, keep, nfit[E:])
            assert abs(r - r_ref) <= 1e-5
            verdict = int(verdict)


def test_screened_run_elitist(prob):
    """Elitism with exact fitness under screening: the best never worsens and
    improves over the run."""
    with game.Game(prob.X, prob.y, prob.degree, 0, P=64, seed=8, precision=BF16,
                   surrogate=1, oversample=8) as g:
        best = [g.population()[1].min()]
        for _ in range(30):
            g.generation(8)
            best.append(g.population()[1].min())
    assert np.all(np.diff(best) <= 1e-12 * np.abs(np.array(best[:-1])))
    assert best[-1] < best[0]


def test_surrogate_learns_fitness_ranking(prob):
    """Trained on 4096 random chromosomes with their exact fitness (200 Adam
    steps on batches of 1024), the surrogate ranks 1024 held-out chromosomes
    close to their exact ranking."""
    K = prob.K
    train = dg.random_population(31, 4096, K)
    test = dg.random_population(32, 1024, K)
    with game.Game(prob.X, prob.y, prob.degree, 0, P=64, seed=9) as g:
        ftrain = g.eval_fitness(train)
        ftest = g.eval_fitness(test)
        for step in range(200):
            i = (step % 4) * 1024
            g.surrogate_train(train[i:i + 1024], ftrain[i:i + 1024])
        pred = g.surrogate_predict(test)
    ranks = lambda a: np.argsort(np.argsort(a))
    rho = np.corrcoef(ranks(pred), ranks(ftest))[0, 1]
    assert rho > 0.8, rho
