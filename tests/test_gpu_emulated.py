"""Element-by-element parity of the reduced-precision tensor-core forms with
a CPU model of their own arithmetic (tests/emulation.py): operands rounded
to BF16, split into BF16 hi + lo, or scaled and quantised to E4M3 exactly as
the kernels round them, products and sums exact. The kernel may differ from
the model only by the FP32 accumulation order of its K' products, the
epilogue's FP32 residual and sums, and operands whose rounding is ambiguous
(trigonometric expansion values within a few FP32 ulps of a rounding
boundary); `emulation.tolerance` bounds exactly those, so a kernel error
far below the forms' own rounding error (a dropped product, a wrong scale,
a misplaced column) fails here even where the worst-case bounds against
the FP64 oracle in test_gpu_fitness.py would let it pass.

The cases reach every pattern-tile width each form can select (256, 192,
128, 64 and 32 for BF16; 256, 128, 64 and 32 for bf16x3 and FP8) and a
trigonometric set with features over [-8, 8]."""
import numpy as np
import pytest

from emulation import model
from helpers import CHEB, TRIG
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PREC = {"bf16": game.GAME_PREC_BF16, "bf16x3": game.GAME_PREC_BF16X3,
        "fp8": game.GAME_PREC_FP8}
KP_LIMIT = {"bf16": 2560, "bf16x3": 1216, "fp8": 4096}

# (M, N, d, basis, P, x scale)
CASES = [
    (2000, 8, 4, CHEB, 64, 1),       # 256-pattern tiles, one K-block
    (777, 3, 7, TRIG, 130, 1),       # trigonometric, ragged M, two chromosome tiles
    (6000, 32, 8, CHEB, 256, 1),     # the classification shape (features from L2 in BF16)
    (3001, 48, 6, CHEB, 300, 1),     # BF16 192-pattern tiles
    (3000, 48, 8, CHEB, 200, 1),     # K' = 384: BF16 128-pattern tiles
    (2500, 50, 10, CHEB, 200, 1),    # K' = 500: FP8 128, BF16 128
    (513, 64, 10, TRIG, 33, 1),      # K' = 1280: BF16 64, FP8 64
    (1300, 66, 10, TRIG, 70, 1),     # K' = 1320: BF16 32
    (1203, 64, 19, CHEB, 130, 1),    # K' = 1216: bf16x3 32 at its limit
    (1500, 128, 20, CHEB, 40, 1),    # K' = 2560: BF16 32 at its limit, FP8 32
    (1100, 128, 32, CHEB, 40, 1),    # K' = 4096: FP8 32 at its limit
    (3000, 6, 5, TRIG, 100, 8),      # features over [-8, 8]
    (1003, 5, 3, CHEB, 70, 1),       # K' = 15: a partial first MMA group
    (2999, 9, 8, CHEB, 130, 1),      # degree 8 from L2 in BF16: zero chunks past feature 9
]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    game.load()
    return torch.device("cuda:0")


@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
@pytest.mark.parametrize("form", ["bf16", "bf16x3", "fp8"])
def test_form_matches_its_cpu_model(dev, case, form):
    M, N, d, basis, P, xs = case
    pr = dg.regression(M + N + d, M, N, min(d, 4), 0.05, degree=d, basis=basis)
    X = (pr.X * np.float32(xs)).astype(np.float32)
    if pr.K - 1 > KP_LIMIT[form]:
        pytest.skip("contraction longer than the form accepts (refusal: test_gpu_fitness)")
    pop = dg.random_population(11 + P, P, pr.K)
    want, tol = model(form, X, pr.y, pop, d, basis)
    with game.Game(X, pr.y, d, basis, P=max(P, 4), precision=PREC[form]) as g:
        got = g.eval_fitness(pop)
    err = np.abs(got - want)
    assert np.all(err <= tol), (f"{form}: max err {err.max():.3e}, worst ratio "
                                f"{(err / tol).max():.3f}, rel {np.max(err / want):.3e}")


@pytest.mark.parametrize("form", ["bf16", "fp8"])
def test_converged_population_matches_model(dev, form):
    """Near the generating chromosome the fitness is about the noise (0.0025)
    and the residuals cancel most: the model still holds the kernel."""
    pr = dg.small_regression()
    rng = np.random.default_rng(5)
    pop = (pr.coef[None, :] + rng.normal(0, 0.01, (64, pr.K))).astype(np.float32)
    pop[0] = pr.coef
    want, tol = model(form, pr.X, pr.y, pop, pr.degree, CHEB)
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, precision=PREC[form]) as g:
        got = g.eval_fitness(pop)
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)
