"""Pins of the CPU model of the reduced-precision forms (tests/emulation.py)
against what fixes it independently: its BF16 and E4M3 roundings against
torch's own casts (round to nearest even, E4M3's subnormals), its FP32
expansion against the FP64 Chebyshev / trigonometric values within FP32
rounding, its width `delta` against the observed FP32 error, and the model
fitness against the FP64 oracle within the worst-case bounds of each form
(tests/helpers.py). With exact operands (values that BF16 and E4M3 hold
exactly) every form's model equals the oracle to FP64 rounding."""
import numpy as np
import pytest

from emulation import bf16, e4m3, expansion_fp32, model
from helpers import CHEB, TRIG, bf16_bound, bf16x3_bound, design_matrix, fp8_bound
from paper_1211_5481_gb300 import datagen as dg

torch = pytest.importorskip("torch")


def test_roundings_match_torch_casts():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 50, 50000), rng.uniform(-0.05, 0.05, 50000),
                        rng.uniform(-2.0 ** -8, 2.0 ** -8, 20000)]).astype(np.float32)
    x8 = x[np.abs(x) < 440]
    t8 = torch.from_numpy(x8).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(e4m3(x8), t8)
    np.testing.assert_array_equal(e4m3(np.array([500.0, -1e6], dtype=np.float32)), [448, -448])
    tb = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(bf16(x), tb)


@pytest.mark.parametrize("basis,d,scale", [(CHEB, 8, 1), (CHEB, 32, 1), (TRIG, 10, 1),
                                           (TRIG, 10, 8)])
def test_fp32_expansion_within_its_delta_of_fp64(basis, d, scale):
    rng = np.random.default_rng(d + scale)
    X = (rng.uniform(-1, 1, (3000, 4)) * scale).astype(np.float32)
    phi, delta = expansion_fp32(X, d, basis)
    exact = design_matrix(X, d, basis)[:, 1:]
    err = np.abs(phi - exact)
    # FP32 recurrence error of this kind stays within the stated width of
    # the kernel's deviation from the model (both are FP32 recurrences)
    assert np.all(err <= delta + 2.0 ** -20 * d * d)
    assert np.max(err) > 0          # a genuinely FP32 computation


@pytest.mark.parametrize("form,bound", [("bf16", bf16_bound), ("bf16x3", bf16x3_bound),
                                        ("fp8", fp8_bound)])
@pytest.mark.parametrize("case", [(1500, 8, 4, CHEB), (800, 3, 7, TRIG), (1200, 32, 8, CHEB)])
def test_model_within_the_worst_case_bound_of_the_oracle(orc, form, bound, case):
    M, N, d, basis = case
    pr = dg.regression(M + d, M, N, min(d, 3), 0.05, degree=d, basis=basis)
    pop = dg.random_population(3, 24, pr.K)
    ref = orc.fitness(pr.X, pr.y, pop, d, basis)
    fit, tol = model(form, pr.X, pr.y, pop, d, basis)
    assert np.all(np.abs(fit - ref) <= bound(ref, pr.X, pop, d, basis))
    # the model's own tolerance is far tighter than the worst case where the
    # operand rounding, not the FP32 summation, dominates the error
    if form != "bf16x3":
        assert np.median(tol) < 0.1 * np.median(bound(ref, pr.X, pop, d, basis))


def test_exact_operands_reproduce_the_oracle(orc):
    """Features 0 and +-1/2 (exact Chebyshev values in every format) and
    genes that are short binary fractions: the BF16 and split operands are
    exact, so those models are the oracle's fitness up to FP64 rounding (FP8
    rescales each chromosome's genes, which no choice keeps exact)."""
    rng = np.random.default_rng(2)
    M, N, d = 600, 3, 4
    X = rng.choice([-0.5, 0.0, 0.5], (M, N)).astype(np.float32)
    y = rng.choice([-1.0, 0.5, 2.0], M).astype(np.float32)
    K = N * d + 1
    pop = (rng.integers(-8, 9, (16, K)) / 16.0).astype(np.float32)
    pop[:, 1:] *= 2.0 ** -(np.arange(K - 1) % 3)
    ref = orc.fitness(X, y, pop, d, CHEB)
    for form in ("bf16", "bf16x3"):
        fit, _ = model(form, X, y, pop, d, CHEB)
        np.testing.assert_allclose(fit, ref, rtol=1e-12, err_msg=form)
