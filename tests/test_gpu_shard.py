"""The per-slice steps of pattern sharding through the CUDA library, on one
GPU: two handles hold the two halves of a training set and play the two
ranks of paper_1211_5481_gb300/shard.py (their exchange is the in-process
sum of their error sums in rank order). Checked against the FP64 oracle:
each slice's error sums (game_eval_sse, FP32 and BF16 forms), the summed
fitness against the whole set's, and the populations both handles breed
(game_breed) from that fitness -- bit-identical to each other and to the
oracle's operators."""
import numpy as np
import pytest

from emulation import model
from helpers import CHEB, TRIG, fp32_tol
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game, shard

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
FP32, BF16 = game.GAME_PREC_FP32, game.GAME_PREC_BF16


@pytest.mark.parametrize("prec", [FP32, BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("basis", [CHEB, TRIG], ids=["cheb", "trig"])
def test_two_slices_follow_the_oracle(orc, prec, basis):
    pr = dg.regression(13, 6001, 6, 3, 0.05, degree=4, basis=basis)
    P, seed = 96, 17
    prm = orc.ga_params()
    sl = [shard.shard_bounds(pr.M, 2, r) for r in range(2)]
    hs = [game.Game(pr.X[b:e], pr.y[b:e], 4, basis, P=P, seed=seed, precision=prec,
                    rescore_top=0) for b, e in sl]
    whole = game.Game(pr.X, pr.y, 4, basis, P=P, seed=seed, precision=prec, rescore_top=0)
    try:
        pop, _, gen = hs[0].population()
        for g in range(4):
            sums = [h.eval_sse() for h in hs]
            # each slice's sums against the oracle's (FP32) or the form's model (BF16)
            for (b, e), s in zip(sl, sums):
                if prec == FP32:
                    ref = orc.fitness(pr.X[b:e], pr.y[b:e], pop, 4, basis)
                    tol = fp32_tol(ref, pr.y[b:e])
                else:
                    ref, tol = model("bf16", pr.X[b:e], pr.y[b:e], pop, 4, basis)
                assert np.all(np.abs(s / (e - b) - ref) <= tol)
            fit = (sums[0] + sums[1]) / pr.M
            if prec == FP32:
                exact = orc.fitness(pr.X, pr.y, pop, 4, basis)
                assert np.all(np.abs(fit - exact) <= fp32_tol(exact, pr.y))
            np.testing.assert_allclose(fit, whole.eval_fitness(pop), rtol=2e-5)
            for h in hs:
                h.set_fitness(fit)
                h.breed(seed)
            nxt = [h.population() for h in hs]
            np.testing.assert_array_equal(nxt[0][0].view(np.uint32), nxt[1][0].view(np.uint32))
            want = orc.generation(pop, fit, seed, gen, prm)
            np.testing.assert_array_equal(nxt[0][0].view(np.uint32), want.view(np.uint32))
            pop, gen = nxt[0][0], nxt[0][2]
            assert gen == g + 1
    finally:
        for h in hs + [whole]:
            h.close()


def test_device_sums_equal_host_sums():
    pr = dg.regression(3, 5000, 4, 3, 0.05, degree=5)
    with game.Game(pr.X, pr.y, 5, CHEB, P=64, precision=BF16, rescore_top=0) as g:
        pop = dg.random_population(1, 200, pr.K)
        host = g.eval_sse(pop)
        dev = g.eval_sse(torch.from_numpy(pop).cuda(),
                         out=torch.empty(200, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host, dev.cpu().numpy())
        cur = g.eval_sse()
        np.testing.assert_allclose(cur / pr.M, g.population()[1], rtol=1e-12)


def test_sharding_steps_refuse_what_they_cannot_do():
    pr = dg.small_regression()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=16, precision=game.GAME_PREC_GRAM) as g:
        with pytest.raises(game.GameError) as ei:
            g.eval_sse()
        assert ei.value.code == game.GAME_EINVAL
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=16) as g:
        g.breed(1)
        with pytest.raises(game.GameError) as ei:
            g.breed(1)                       # the bred population has no fitness yet
        assert ei.value.code == game.GAME_ESTATE
        g.set_fitness(np.ones(16))
        g.breed(1)
        with pytest.raises(ValueError):
            g.set_fitness(np.ones(15))
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=16, precision=BF16, surrogate=1,
                   oversample=2) as g:
        with pytest.raises(game.GameError) as ei:
            g.breed(1)
        assert ei.value.code == game.GAME_ESTATE
