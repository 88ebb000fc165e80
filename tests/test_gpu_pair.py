"""The paired-SM BF16 kernel (csrc/fitness_tc2.cu: 2-CTA clusters sharing
each tcgen05 MMA) on the shapes where the launch plan takes it -- the one-SM
kernel would need a tile narrower than 256 patterns -- against the CPU model
of the BF16 form (tests/emulation.py) for the three error functions of
Section 3, with staged and L2-read features, one and two chromosome pairs,
padded chromosome rows and ragged pattern tails; and the plan's choice
itself."""
import numpy as np
import pytest

from emulation import model
from helpers import CHEB, TRIG, bf16_bound
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BF16 = game.GAME_PREC_BF16
ERR = {"mse": game.GAME_ERR_MSE, "rmse": game.GAME_ERR_RMSE, "mae": game.GAME_ERR_MAE}

# (M, N, d, basis, P)
PAIR_CASES = [
    (3001, 48, 6, CHEB, 300),    # staged features (degree 6), two pairs, padded rows
    (2999, 48, 8, CHEB, 129),    # K' = 384, features read from L2, one pair, ragged tail
    (1537, 20, 7, TRIG, 257),    # trigonometric, K' = 280, two pairs (one nearly empty)
]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    game.load()
    return torch.device("cuda:0")


def test_plan_takes_pairs_only_where_one_sm_narrows(dev):
    for M, N, d, basis, P in PAIR_CASES:
        pr = dg.regression(M, M, N, 3, 0.05, degree=d, basis=basis)
        with game.Game(pr.X, pr.y, d, basis, P=P, precision=BF16) as g:
            pl = g.plan()
            assert pl["kernel"] == "fitness_tc2_kernel" and pl["tile"] == 256, pl
            assert g.plan(P=128)["kernel"] == "fitness_tc_kernel"      # one chromosome tile
            assert g.plan(game.GAME_PREC_FP8)["kernel"] == "fitness_tc_kernel"
    pr = dg.regression(1, 6000, 32, 3, 0.05, degree=8)
    with game.Game(pr.X, pr.y, 8, CHEB, P=1024, precision=BF16) as g:
        pl = g.plan()
        assert pl["kernel"] == "fitness_tc_kernel" and pl["tile"] == 256 and pl["staged"] == 0


@pytest.mark.parametrize("case", PAIR_CASES, ids=[str(c) for c in PAIR_CASES])
@pytest.mark.parametrize("error", ["mse", "rmse", "mae"])
def test_pair_kernel_matches_the_bf16_model(dev, case, error):
    M, N, d, basis, P = case
    pr = dg.regression(M + P, M, N, min(d, 4), 0.05, degree=d, basis=basis)
    pop = dg.random_population(P + 3, P, pr.K)
    want, tol = model("bf16", pr.X, pr.y, pop, d, basis, error=error)
    with game.Game(pr.X, pr.y, d, basis, P=P, precision=BF16, error=ERR[error],
                   rescore_top=0) as g:
        assert g.plan()["kernel"] == "fitness_tc2_kernel"
        got = g.eval_fitness(pop)
    err = np.abs(got - want)
    assert np.all(err <= tol), (error, err.max(), (err / tol).max())


def test_pair_kernel_against_the_oracle_and_a_generation(orc, dev):
    """The oracle's fitness within the BF16 worst-case bound, and one
    generation's operators bit-exact given the device's fitness."""
    M, N, d, basis, P = PAIR_CASES[0]
    pr = dg.regression(7, M, N, 4, 0.05, degree=d, basis=basis)
    pop = dg.random_population(9, P, pr.K)
    ref = orc.fitness(pr.X, pr.y, pop, d, basis)
    with game.Game(pr.X, pr.y, d, basis, P=P, seed=3, precision=BF16) as g:
        got = g.eval_fitness(pop)
        assert np.all(np.abs(got - ref) <= bf16_bound(ref, pr.X, pop, d, basis))
        p0, f0, g0 = g.population()
        g.generation(3)
        p1, _, g1 = g.population()
    want = orc.generation(p0, f0, 3, g0, orc.ga_params())
    assert g1 == g0 + 1
    np.testing.assert_array_equal(p1.view(np.uint32), want.view(np.uint32))
