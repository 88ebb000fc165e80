"""The paper-literal options on the GPU against the oracle, through the C ABI:
ranking and roulette selection (Section 5) bit-exact; shared genes (Eq. 2 as
printed, Eq. 5: K = B*d + 1) in the FP32, BF16 and Gram forms; the RMSE and
MAE error functions (Section 3)."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, U_FP32, abs_weighted_sum, bf16_bound, fp32_tol
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32, BF16, GRAM = game.GAME_PREC_FP32, game.GAME_PREC_BF16, game.GAME_PREC_GRAM
RANKING, ROULETTE = game.GAME_SEL_RANKING, game.GAME_SEL_ROULETTE
RMSE, MAE = game.GAME_ERR_RMSE, game.GAME_ERR_MAE
U64 = 2.0 ** -53


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def problem(M, N, d, basis=CHEB, seed=1):
    return dg.regression(seed, M, N, min(d, 3), 0.05, degree=d, basis=basis)


# ---------------------------------------------------------------- selection

SEL_CASES = [
    # P, N, d, E, I, selection
    (64, 8, 4, 2, 0, RANKING),
    (65, 8, 4, 2, 0, ROULETTE),
    (1024, 32, 8, 2, 0, RANKING),
    (1024, 32, 8, 2, 0, ROULETTE),
    (333, 3, 3, 0, 3, RANKING),      # no elites, immigrants, P not a power of two
    (333, 3, 3, 0, 3, ROULETTE),
    (16384, 2, 2, 2, 0, RANKING),    # the largest ranking population (sort of 2^14 keys)
    (20000, 2, 2, 2, 0, ROULETTE),   # many weights per scanning thread
]


@pytest.mark.parametrize("P,N,d,E,I,sel", SEL_CASES, ids=[str(c) for c in SEL_CASES])
def test_selection_bit_exact(orc, P, N, d, E, I, sel):
    pr = problem(300, N, d)
    K = pr.K
    rng = np.random.default_rng(P * 3 + sel)
    pop = dg.random_population(P + K, P, K)
    fit = rng.uniform(0.0, 2.0, P)
    fit[rng.integers(0, P, 3)] = fit[0]     # ties
    fit[rng.integers(0, P, 2)] = np.nan     # weight 0 / ranked last
    fit[rng.integers(0, P, 1)] = np.inf
    fit[rng.integers(0, P, 1)] = 1e-17      # 1 + f rounds to 1
    fit[rng.integers(0, P, 1)] = 0.0
    prm = orc.ga_params(elitism=E, immigrants=I, selection=sel)
    for g_index, seed in [(0, 11), (99, 2**35 + 1)]:
        with game.Game(pr.X, pr.y, d, CHEB, P=P, elitism=E, immigrants=I, selection=sel) as g:
            g.set_state(pop, fit, g_index)
            g.generation(seed)
            nxt, _, gen = g.population()
        assert gen == g_index + 1
        ref = orc.generation(pop, fit, seed, g_index, prm)
        np.testing.assert_array_equal(bits(nxt), bits(ref))


def test_roulette_all_weights_zero(orc):
    pr = problem(200, 4, 3)
    P = 50
    pop = dg.random_population(5, P, pr.K)
    fit = np.full(P, np.nan)
    prm = orc.ga_params(elitism=0, selection=ROULETTE)
    with game.Game(pr.X, pr.y, 3, CHEB, P=P, elitism=0, selection=ROULETTE) as g:
        g.set_state(pop, fit, 4)
        g.generation(8)
        nxt, _, _ = g.population()
    np.testing.assert_array_equal(bits(nxt), bits(orc.generation(pop, fit, 8, 4, prm)))


@pytest.mark.parametrize("sel", [RANKING, ROULETTE])
def test_selection_training_trajectory(orc, sel):
    """Every generation of a run equals the oracle's operators applied to the
    GPU's own population and fitness; the elitist best never worsens."""
    pr = dg.small_regression()
    prm = orc.ga_params(selection=sel)
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=5, selection=sel) as g:
        pop, fit, gen = g.population()
        best = [fit.min()]
        for _ in range(15):
            g.generation(5)
            nxt, nfit, ngen = g.population()
            np.testing.assert_array_equal(bits(nxt), bits(orc.generation(pop, fit, 5, gen, prm)))
            best.append(nfit.min())
            pop, fit, gen = nxt, nfit, ngen
    assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))


# ------------------------------------------------------------- shared genes

TIED_CASES = [
    (2000, 8, 4, CHEB, 64),
    (777, 3, 7, TRIG, 130),
    (300, 1, 1, CHEB, 3),
    (5000, 16, 10, TRIG, 257),
    (3001, 48, 6, CHEB, 300),
]


def replicate(tied, N, B, d):
    """The per-feature chromosome with every feature's genes equal to the
    shared ones (gene 1 + i*B*d + c takes shared gene 1 + c)."""
    tied = np.asarray(tied, dtype=np.float32)
    full = np.zeros((tied.shape[0], B * N * d + 1), dtype=np.float32)
    full[:, 0] = tied[:, 0]
    for i in range(N):
        full[:, 1 + i * B * d:1 + (i + 1) * B * d] = tied[:, 1:]
    return full


def fold(G, b, N, B, d):
    """Gram matrix of the shared genes from the per-feature one: R^T G R and
    R^T b, R the replication map."""
    K = B * N * d + 1
    R = np.zeros((K, B * d + 1))
    R[0, 0] = 1.0
    for i in range(N):
        for c in range(B * d):
            R[1 + i * B * d + c, 1 + c] = 1.0
    return R.T @ G @ R, R.T @ b


def quad_bound(G, b, yy, pop, M):
    A = np.abs(np.asarray(pop, dtype=np.float64))
    K = A.shape[1]
    mag = yy + 2 * A @ np.abs(b) + np.einsum("pk,kl,pl->p", A, np.abs(G), A)
    return 4 * (K + 8) * U64 * mag / M + 1e-300


@pytest.mark.parametrize("case", TIED_CASES, ids=[str(c) for c in TIED_CASES])
@pytest.mark.parametrize("prec", [FP32, BF16, GRAM], ids=["fp32", "bf16", "gram"])
def test_tied_fitness(orc, case, prec):
    M, N, d, basis, P = case
    B = 2 if basis == TRIG else 1
    pr = problem(M, N, d, basis, seed=M + d)
    Kt = B * d + 1
    pop = dg.random_population(P + 1, P, Kt) / np.float32(N)   # outputs of order 1
    ref = orc.fitness_tied(pr.X, pr.y, pop, d, basis)
    with game.Game(pr.X, pr.y, d, basis, P=max(P, 4), tied=1, precision=prec) as g:
        assert g.K == Kt
        got = g.eval_fitness(pop)
        if prec == GRAM:
            G, b, yy = g.gram()
    full = replicate(pop, N, B, d)
    np.testing.assert_allclose(orc.fitness(pr.X, pr.y, full, d, basis), ref, rtol=1e-12)
    if prec == FP32:
        tol = fp32_tol(ref, pr.y)
    elif prec == BF16:
        tol = bf16_bound(ref, pr.X, full, d, basis)
    else:
        Go, bo, yyo, _ = orc.gram(pr.X, pr.y, d, basis)
        Gt, bt = fold(Go, bo, N, B, d)
        # the psi expansion: G of the sums over features
        scale = max(M, 1) * N * N
        assert np.max(np.abs(G - Gt)) <= 64 * scale * U64 * 4
        assert np.max(np.abs(b - bt)) <= 64 * scale * U64 * (1 + np.max(np.abs(pr.y)))
        np.testing.assert_array_equal(G, G.T)
        tol = quad_bound(Gt, bt, yyo, pop, M) + 1e-12 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (err.max(), (err / tol).max())


@pytest.mark.parametrize("prec", [FP32, GRAM])
def test_tied_generation_and_trajectory(orc, prec):
    """Operators on the B*d + 1 shared genes are bit-exact; the fitness of
    the evolved population tracks the oracle's shared-gene fitness."""
    pr = dg.small_regression()
    d = pr.degree
    prm = orc.ga_params()
    with game.Game(pr.X, pr.y, d, CHEB, P=64, seed=3, tied=1, precision=prec) as g:
        pop, fit, gen = g.population()
        assert pop.shape == (64, d + 1)
        np.testing.assert_array_equal(bits(pop), bits(orc.init_population(3, 64, d + 1)))
        best = [fit.min()]
        for _ in range(12):
            g.generation(3)
            nxt, nfit, ngen = g.population()
            np.testing.assert_array_equal(bits(nxt), bits(orc.generation(pop, fit, 3, gen, prm)))
            best.append(nfit.min())
            pop, fit, gen = nxt, nfit, ngen
    ref = orc.fitness_tied(pr.X, pr.y, pop, d, CHEB)
    if prec == FP32:
        assert np.all(np.abs(fit - ref) <= fp32_tol(ref, pr.y))
    else:
        np.testing.assert_allclose(fit, ref, rtol=1e-9)
    assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))


def test_tied_rescore_uses_shared_gram(orc):
    """BF16 fitness with elite re-scoring: the re-scored entries are the
    shared-gene Gram form's FP64 values."""
    pr = problem(4000, 12, 5, seed=9)
    P, Kt = 200, 6
    pop = dg.random_population(2, P, Kt) / np.float32(12)
    ref = orc.fitness_tied(pr.X, pr.y, pop, 5, CHEB)
    with game.Game(pr.X, pr.y, 5, CHEB, P=P, tied=1, precision=BF16) as g:
        fit = g.eval_fitness(pop)
        fit2, idx = g.rescore_top(pop, fit, 8)
    np.testing.assert_allclose(fit2[idx], ref[idx], rtol=1e-9)
    others = np.setdiff1d(np.arange(P), idx)
    np.testing.assert_array_equal(fit2[others], fit[others])


# ---------------------------------------------------------- error functions

ERR_CASES = [
    (2000, 8, 4, CHEB, 64),
    (777, 3, 7, TRIG, 130),
    (3001, 48, 6, CHEB, 300),
    (6000, 32, 8, CHEB, 256),
]


@pytest.mark.parametrize("case", ERR_CASES, ids=[str(c) for c in ERR_CASES])
@pytest.mark.parametrize("prec", [FP32, BF16, GRAM], ids=["fp32", "bf16", "gram"])
@pytest.mark.parametrize("err", [RMSE, MAE], ids=["rmse", "mae"])
def test_error_functions(orc, case, prec, err):
    M, N, d, basis, P = case
    pr = problem(M, N, d, basis, seed=N + d)
    pop = dg.random_population(P + 5, P, pr.K)
    kw = dict(P=max(P, 4), precision=prec, error=err, rescore_top=0 if err == MAE else 8)
    if prec == GRAM and err == MAE:
        with pytest.raises(game.GameError) as ei:
            game.Game(pr.X, pr.y, d, basis, **kw)
        assert ei.value.code == game.GAME_EINVAL
        return
    ref = orc.fitness(pr.X, pr.y, pop, d, basis, err=orc.ERR_RMSE if err == RMSE else orc.ERR_MAE)
    with game.Game(pr.X, pr.y, d, basis, **kw) as g:
        got = g.eval_fitness(pop)
    mse = orc.fitness(pr.X, pr.y, pop, d, basis)
    if prec == FP32:
        tol = 1e-5 * np.abs(ref) + 1e-7 * np.sqrt(np.mean(pr.y.astype(np.float64) ** 2))
    elif prec == BF16 and err == RMSE:
        # |sqrt(a) - sqrt(b)| <= |a - b| / sqrt(b)
        tol = bf16_bound(mse, pr.X, pop, d, basis) / np.sqrt(mse)
    elif prec == BF16:
        # |mean|r'| - mean|r|| <= mean|dOut| <= e mean(S), plus the FP32 tile sums
        K = pr.K
        e = 2 * 2.0 ** -8 + 2.0 ** -16 + K * U_FP32
        _, s1 = abs_weighted_sum(pr.X, pop, d, basis, with_mean=True)
        tol = e * s1 + 300 * U_FP32 * ref
    else:
        Go, bo, yyo, _ = orc.gram(pr.X, pr.y, d, basis)
        tol = (quad_bound(Go, bo, yyo, pop, M) + 1e-12 * mse) / np.sqrt(mse)
    e_abs = np.abs(got - ref)
    assert np.all(e_abs <= tol), (e_abs.max(), (e_abs / tol).max())


def test_rmse_rescore_and_training(orc):
    """RMSE handles re-score with the square root of the Gram MSE, and a GA
    run on the RMSE selects exactly as on the MSE (a monotone transform)."""
    pr = dg.small_regression()
    pop = dg.random_population(6, 64, pr.K)
    ref = orc.fitness(pr.X, pr.y, pop, pr.degree, CHEB, err=orc.ERR_RMSE)
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, precision=BF16, error=RMSE) as g:
        fit, idx = g.rescore_top(pop, g.eval_fitness(pop), 8)
    np.testing.assert_allclose(fit[idx], ref[idx], rtol=1e-9)
    runs = []
    for err in (game.GAME_ERR_MSE, RMSE):
        with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=4, precision=GRAM, error=err) as g:
            g.train(10)
            runs.append(g.population())
    np.testing.assert_array_equal(bits(runs[0][0]), bits(runs[1][0]))
    np.testing.assert_allclose(np.sqrt(np.maximum(runs[0][1], 0)), runs[1][1], rtol=1e-12)


def test_mae_refuses_rescore(orc):
    pr = dg.small_regression()
    pop = dg.random_population(6, 64, pr.K)
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, precision=BF16, error=MAE,
                   rescore_top=0) as g:
        fit = g.eval_fitness(pop)
        with pytest.raises(game.GameError) as ei:
            g.rescore_top(pop, fit, 4)
        assert ei.value.code == game.GAME_EINVAL
        with pytest.raises(game.GameError):
            g.eval_fitness(pop, precision=GRAM)


def test_tied_mae_roulette_together(orc):
    """Shared genes, the MAE and roulette selection in one handle: fitness
    against the oracle (the replicated chromosome's MAE) and one generation
    bit-exact against the oracle's operators on the shared genes."""
    pr = problem(3000, 12, 5, seed=2)
    P, Kt = 100, 6
    prm = orc.ga_params(selection=orc.SEL_ROULETTE)
    with game.Game(pr.X, pr.y, 5, CHEB, P=P, seed=6, tied=1, error=MAE, rescore_top=0,
                   selection=ROULETTE) as g:
        pop, fit, gen = g.population()
        ref = orc.fitness(pr.X, pr.y, replicate(pop, 12, 1, 5), 5, CHEB, err=orc.ERR_MAE)
        assert pop.shape == (P, Kt)
        assert np.all(np.abs(fit - ref) <= 1e-5 * np.abs(ref) + 1e-7)
        g.generation(6)
        nxt, _, _ = g.population()
    np.testing.assert_array_equal(bits(nxt), bits(orc.generation(pop, fit, 6, gen, prm)))


def test_tied_surrogate_run_is_elitist():
    """Shared genes with the surrogate screening (K = B d + 1 inputs to the
    MLP): the run proceeds and the elitist best never worsens."""
    pr = problem(4000, 10, 6, seed=3)
    with game.Game(pr.X, pr.y, 6, CHEB, P=64, seed=2, tied=1, precision=BF16, surrogate=1,
                   oversample=4) as g:
        assert g.K == 7
        best = [g.population()[1].min()]
        for _ in range(8):
            g.generation(2)
            best.append(g.population()[1].min())
        pred, keep, trusted, r = g.surrogate_last()
    assert pred.shape == (4 * 62,) and keep.sum() == 62
    assert all(b1 <= b0 * (1 + 1e-12) for b0, b1 in zip(best, best[1:]))
