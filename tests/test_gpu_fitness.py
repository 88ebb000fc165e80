"""Parity of the CUDA fitness kernels with the FP64 oracle, through the C ABI.

FP32 form (CUDA-core FFMA): |f - f_oracle| <= 1e-5 |f_oracle| + 1e-7 mean(y^2).
BF16 form (tcgen05): within the worst-case rounding bound of a BF16 x BF16 ->
FP32 contraction (helpers.bf16_bound), and its relative error is reported.
"""
import numpy as np
import pytest

from helpers import CHEB, TRIG, bf16_bound, bf16x3_bound, fp32_tol, fp8_bound
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32, BF16 = game.GAME_PREC_FP32, game.GAME_PREC_BF16
BF16X3, FP8 = game.GAME_PREC_BF16X3, game.GAME_PREC_FP8
BOUNDS = {BF16: bf16_bound, BF16X3: bf16x3_bound, FP8: fp8_bound}

# (M, N, d, basis, P): tile multiples, ragged tails, K not a multiple of 16,
# P below / above / not a multiple of 128, tiny and long contractions
CASES = [
    (2000, 8, 4, CHEB, 64),      # the small regression workload's shape
    (1003, 5, 3, CHEB, 70),      # K' = 15
    (777, 3, 7, TRIG, 130),      # trigonometric, P just above one tile
    (300, 1, 1, CHEB, 3),        # K = 2
    (1, 4, 2, CHEB, 5),          # a single pattern
    (5000, 16, 10, TRIG, 257),   # K' = 320, 6 K-blocks
    (4099, 40, 8, CHEB, 1),      # a single chromosome, K' = 320
    (513, 64, 10, TRIG, 33),     # K' = 1280, the longest batched contraction
    (6000, 32, 8, CHEB, 256),    # the large classification shape, reduced M
    (3001, 48, 6, CHEB, 300),    # the surrogate workload's shape: 192-pattern tiles
    # Chebyshev runs of 8 degrees (BF16: features from L2, spare expansion slots)
    (1000, 5, 8, CHEB, 100),     # one K-block, zero chunks after K' = 40
    (2999, 9, 8, CHEB, 130),     # K' = 72: the last MMA reads a zero chunk
    (1500, 3, 16, CHEB, 64),     # degree 16: chunks starting at degree 9
    (3000, 48, 8, CHEB, 200),    # K' = 384: 128-pattern tiles, ten slots
    # the narrowest tiles of every form, each at its longest contraction
    (1500, 128, 20, CHEB, 40),   # K' = 2560: BF16 at its limit, 32-pattern tiles
    (1300, 66, 10, TRIG, 70),    # K' = 1320: BF16 32-pattern tiles, trigonometric
    (1203, 64, 19, CHEB, 130),   # K' = 1216: bf16x3 at its limit, 32-pattern tiles
    (1100, 128, 32, CHEB, 40),   # K' = 4096: FP8 at its limit, 32-pattern tiles
    (2500, 50, 10, CHEB, 200),   # K' = 500: FP8 128-pattern tiles
]

# longest contraction K' each tensor-core form accepts at N <= 128 (the
# expansion tile of all K' columns stays in shared memory)
KP_LIMIT = {BF16: 2560, BF16X3: 1216, FP8: 4096, FP32: 4096}


def make_problem(M, N, d, basis, seed):
    pr = dg.regression(seed, M, N, min(d, 4), 0.05, degree=d, basis=basis)
    return pr


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    game.load()
    return torch.device("cuda:0")


@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
@pytest.mark.parametrize("prec", [FP32, BF16, BF16X3, FP8], ids=["fp32", "bf16", "bf16x3", "fp8"])
def test_fitness_matches_oracle(orc, dev, case, prec):
    M, N, d, basis, P = case
    pr = make_problem(M, N, d, basis, seed=M + N + d)
    pop = dg.random_population(7 + P, P, pr.K)
    ref = orc.fitness(pr.X, pr.y, pop, d, basis)
    if pr.K - 1 > KP_LIMIT[prec]:
        # the expansion tile no longer fits in shared memory: rejected
        with pytest.raises(game.GameError) as ei:
            game.Game(pr.X, pr.y, d, basis, P=max(P, 4), precision=prec)
        assert ei.value.code == game.GAME_EINVAL
        return
    with game.Game(pr.X, pr.y, d, basis, P=max(P, 4), precision=prec) as g:
        got = g.eval_fitness(pop)
    if prec == FP32:
        tol = fp32_tol(ref, pr.y)
    else:
        tol = BOUNDS[prec](ref, pr.X, pop, d, basis)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (f"max err {err.max():.3e}, worst ratio "
                                f"{(err / tol).max():.3f}, rel {np.max(err / np.abs(ref)):.3e}")


@pytest.mark.parametrize("prec", [FP32, BF16, BF16X3, FP8], ids=["fp32", "bf16", "bf16x3", "fp8"])
def test_trigonometric_wide_domain(orc, dev, prec):
    """Eq. 6 puts no limit on x: features spread over [-8, 8] exercise the
    argument reduction of sincosf and the recurrences far from [-1, 1]."""
    pr = dg.regression(41, 3000, 6, 3, 0.05, degree=5, basis=TRIG)
    X = (pr.X * np.float32(8.0)).astype(np.float32)
    assert np.abs(X).max() > 7.5
    P = 100
    pop = dg.random_population(43, P, pr.K)
    ref = orc.fitness(X, pr.y, pop, 5, TRIG)
    with game.Game(X, pr.y, 5, TRIG, P=P, precision=prec) as g:
        got = g.eval_fitness(pop)
    tol = fp32_tol(ref, pr.y) if prec == FP32 else BOUNDS[prec](ref, X, pop, 5, TRIG)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (f"max err {err.max():.3e}, worst ratio {(err / tol).max():.3f}")


def test_device_and_host_pointers_agree(dev):
    pr = dg.small_regression()
    pop = dg.random_population(3, 64, pr.K)
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    with game.Game(Xd, yd, pr.degree, CHEB, P=64) as g:
        host = g.eval_fitness(pop)
        dfit = g.eval_fitness(torch.from_numpy(pop).to(dev))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host, dfit.cpu().numpy())


def test_converged_population(orc, dev):
    """Near the generating coefficients the MSE is ~ noise^2 = 0.0025 and
    the residual sum cancels most: the FP32 bound still holds."""
    pr = dg.small_regression()
    rng = np.random.default_rng(5)
    pop = (pr.coef[None, :] + rng.normal(0, 0.01, (64, pr.K))).astype(np.float32)
    pop[0] = pr.coef
    ref = orc.fitness(pr.X, pr.y, pop, pr.degree, CHEB)
    assert ref.min() < 0.003
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64) as g:
        got = g.eval_fitness(pop)
        got_bf = g.eval_fitness(pop, precision=BF16)
    assert np.all(np.abs(got - ref) <= fp32_tol(ref, pr.y))
    assert np.all(np.abs(got_bf - ref) <= bf16_bound(ref, pr.X, pop, pr.degree, CHEB))


def test_deterministic(dev):
    pr = dg.regression(5, 3000, 12, 4, 0.05, degree=5)
    pop = dg.random_population(4, 200, pr.K)
    for prec in (FP32, BF16, BF16X3, FP8):
        with game.Game(pr.X, pr.y, 5, CHEB, P=200, precision=prec) as g:
            a = g.eval_fitness(pop)
            b = g.eval_fitness(pop)
        np.testing.assert_array_equal(a, b)


def test_full_size_sampled(orc, dev):
    """The large classification workload at full size (M = 10^6, N = 32,
    degree 8, P = 1024) in the benchmark's launch configuration; a sample of
    chromosomes is re-computed by the oracle one by one."""
    pr = dg.large_classification()
    P = 1024
    pop = orc.init_population(2, P, pr.K)
    sample = np.array([0, 1, 127, 128, 511, 640, 1000, 1023])
    ref = orc.fitness(pr.X, pr.y, pop[sample], pr.degree, CHEB)
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    with game.Game(Xd, yd, pr.degree, CHEB, P=P) as g:
        f32 = g.eval_fitness(pop)
        fbf = g.eval_fitness(pop, precision=BF16)
        fx3 = g.eval_fitness(pop, precision=BF16X3)
        ff8 = g.eval_fitness(pop, precision=FP8)
    assert np.all(np.abs(f32[sample] - ref) <= fp32_tol(ref, pr.y))
    # the bounds use every 50th pattern for their means of S: allow 10% for that
    for got, bound in ((fbf, bf16_bound), (fx3, bf16x3_bound), (ff8, fp8_bound)):
        b = bound(ref, pr.X[::50], pop[sample], pr.degree, CHEB)
        assert np.all(np.abs(got[sample] - ref) <= 1.1 * b)
    # all chromosomes: the two GPU forms agree within the BF16 bound scale
    rel = np.abs(fbf - f32) / f32
    assert np.median(rel) < 1e-2


def test_create_rejects_bad_data(dev):
    pr = dg.regression(3, 500, 4, 3, 0.0, degree=3)
    X = pr.X.copy()
    X[7, 2] = np.nan
    with pytest.raises(game.GameError) as ei:
        game.Game(X, pr.y, 3, CHEB, P=10)
    assert ei.value.code == game.GAME_EINVAL
    X = pr.X.copy()
    X[3, 1] = 1.5
    with pytest.raises(game.GameError) as ei:
        game.Game(X, pr.y, 3, CHEB, P=10)
    assert ei.value.code == game.GAME_EINVAL
    with game.Game(X, pr.y, 3, TRIG, P=10) as g:   # any x is in the trigonometric domain
        assert g.K == 2 * 4 * 3 + 1
    y = pr.y.copy()
    y[0] = np.inf
    with pytest.raises(game.GameError):
        game.Game(pr.X, y, 3, CHEB, P=10)


def test_staged_targets_bit_identical(dev):
    """With features read from L2 (BF16, degree 8, 256-pattern tiles) the plan
    stages each tile's targets in shared memory when the probe found the
    dynamic shared memory aligned, and reads them from global memory when the
    plan must keep the full 1 KB alignment slack (forced here with the test
    hook). Only where the same FP32 targets are read from differs, so the
    fitness is identical bit for bit; the plan's shared memory shows that
    both paths ran."""
    pr = dg.regression(77, 6000, 32, 4, 0.05, degree=8, basis=CHEB)
    pop = dg.random_population(5, 256, pr.K)
    with game.Game(pr.X, pr.y, 8, CHEB, P=256, precision=game.GAME_PREC_BF16) as g:
        plan_probe = g.plan()
        f_probe = g.eval_fitness(pop)
        game.game_test_hook(game.GAME_HOOK_SMEM_SLACK, 1024)
        try:
            plan_slack = g.plan()
            f_slack = g.eval_fitness(pop)
        finally:
            game.game_test_hook(game.GAME_HOOK_SMEM_SLACK, 0)
        assert g.plan() == plan_probe
    assert plan_probe["kernel"] == plan_slack["kernel"] == "fitness_tc_kernel"
    assert plan_probe["tile"] == plan_slack["tile"] == 256 and plan_probe["staged"] == 0
    # 2 KB of staged targets against 1 KB of slack: the probed plan is 1 KB
    # larger when the probe found the base aligned (else the plans agree)
    assert plan_probe["smem"] - plan_slack["smem"] in (0, 1024)
    np.testing.assert_array_equal(f_probe, f_slack)
