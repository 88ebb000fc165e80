"""Pins of the oracle's basis, output and fitness against facts that do not
come from the oracle itself: closed forms, numpy's independent Chebyshev
routines, brute force on tiny inputs, algebraic identities and the paper's
worked example (Section 3, Eq. 1-7)."""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from paper_1211_5481_gb300 import datagen as dg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CHEB, TRIG = 0, 1


def test_chebyshev_closed_form(orc):
    """T_k(cos t) = cos(k t): pins the three-term recurrence (a wrong
    coefficient or seed value breaks it at k >= 2)."""
    for t in np.linspace(0.0, math.pi, 37):
        vals = orc.basis_values(CHEB, 10, math.cos(t))
        for k in range(1, 11):
            assert abs(vals[k - 1] - math.cos(k * t)) < 1e-12


def test_trig_basis_against_libm(orc):
    """Eq. 6: the trigonometric group is cos(j x) for j=1..d, then sin(j x)."""
    for x in np.linspace(-3.0, 3.0, 25):
        vals = orc.basis_values(TRIG, 5, x)
        for j in range(1, 6):
            assert vals[j - 1] == pytest.approx(math.cos(j * x), abs=1e-15)
            assert vals[5 + j - 1] == pytest.approx(math.sin(j * x), abs=1e-15)


def test_degree_one_is_linear_model(orc):
    """Chebyshev degree 1: T_1(x) = x, so Out = a_0 + sum_i a_i x_i."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        N = int(rng.integers(1, 9))
        a = rng.uniform(-1, 1, N + 1)
        x = rng.uniform(-1, 1, N)
        assert orc.output(a, x, 1, CHEB) == pytest.approx(a[0] + a[1:] @ x, abs=1e-14)


def design_matrix_numpy(X, d, basis):
    """Design matrix built from numpy's chebvander / np.cos / np.sin in the
    gene order 1 + i*B*d + b*d + j-1 (bias column first)."""
    X = np.asarray(X, dtype=np.float64)
    cols = [np.ones(X.shape[0])]
    for i in range(X.shape[1]):
        if basis == CHEB:
            V = npcheb.chebvander(X[:, i], d)[:, 1:]
            cols.extend(V.T)
        else:
            for j in range(1, d + 1):
                cols.append(np.cos(j * X[:, i]))
            for j in range(1, d + 1):
                cols.append(np.sin(j * X[:, i]))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("basis", [CHEB, TRIG])
@pytest.mark.parametrize("N,d", [(1, 1), (3, 2), (5, 4), (2, 7)])
def test_brute_force_tiny(orc, basis, N, d):
    """Brute force on M <= 8: numpy design matrix, matrix-vector product and
    mean of squared residuals, compared with the oracle's direct loop."""
    rng = np.random.default_rng(N * 10 + d + basis)
    M = int(rng.integers(1, 9))
    X = rng.uniform(-1, 1, (M, N))
    y = rng.uniform(-2, 2, M)
    K = orc.num_genes(N, d, basis)
    pop = rng.uniform(-1, 1, (4, K))
    Phi = design_matrix_numpy(X, d, basis)
    assert Phi.shape[1] == K
    ref = ((y[None, :] - pop @ Phi.T) ** 2).mean(axis=1)
    got = orc.fitness(X, y, pop, d, basis)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_fitness_zero_for_generating_chromosome(orc):
    """A noiseless target built (by numpy's chebval) from a chromosome's own
    genes gives fitness 0 up to FP64 rounding; a sign error, a dropped term
    or a shifted gene index leaves a large residual."""
    pr = dg.regression(11, 300, 6, 4, 0.0, degree=4)
    y64 = pr.extra["target_fp64"]
    fit = orc.fitness(pr.X, y64, pr.coef[None, :], 4, CHEB)
    assert fit[0] <= 1e-28
    # one perturbed gene moves it well away from zero
    c2 = pr.coef.copy()
    c2[7] += 0.25
    assert orc.fitness(pr.X, y64, c2[None, :], 4, CHEB)[0] > 1e-3


def test_fitness_zero_higher_degree_basis(orc):
    """A degree-3 target lies in the span of a degree-5 chromosome: its genes
    at j <= 3 are the coefficients and those at j = 4, 5 are zero."""
    D, d, N = 3, 5, 4
    pr = dg.regression(12, 200, N, D, 0.0, degree=d)
    a = np.zeros(N * d + 1)
    a[0] = pr.coef[0]
    for i in range(N):
        a[1 + i * d: 1 + i * d + D] = pr.coef[1 + i * D: 1 + (i + 1) * D]
    assert orc.fitness(pr.X, pr.extra["target_fp64"], a, d, CHEB)[0] <= 1e-28


@pytest.mark.parametrize("basis", [CHEB, TRIG])
def test_gram_equals_direct(orc, basis):
    """SSE = |y|^2 - 2 a^T Phi^T y + a^T Phi^T Phi a (exact algebra)."""
    pr = dg.regression(13, 1500, 5, 3, 0.05, degree=3, basis=basis)
    pop = dg.random_population(5, 16, pr.K)
    direct = orc.fitness(pr.X, pr.y, pop, 3, basis)
    gram = orc.fitness_gram(orc.gram(pr.X, pr.y, 3, basis), pop)
    np.testing.assert_allclose(gram, direct, rtol=1e-10)


@pytest.mark.parametrize("basis", [CHEB, TRIG])
def test_tied_equals_replicated(orc, basis):
    """Eq. 2 as printed shares a_j over the features; the per-feature form
    with those genes replicated over features gives the same fitness."""
    pr = dg.regression(14, 400, 7, 3, 0.05, degree=3, basis=basis)
    d, N, B = 3, 7, (2 if basis == TRIG else 1)
    tied = dg.random_population(6, 5, B * d + 1)
    full = np.zeros((5, B * N * d + 1), dtype=np.float32)
    full[:, 0] = tied[:, 0]
    for i in range(N):
        full[:, 1 + i * B * d: 1 + (i + 1) * B * d] = tied[:, 1:]
    np.testing.assert_allclose(orc.fitness_tied(pr.X, pr.y, tied, d, basis),
                               orc.fitness(pr.X, pr.y, full, d, basis), rtol=1e-12)


def test_worked_example_counts(orc):
    """Section 3: 11 features, trigonometric degree 3 -> Eq. 4 gives 23
    chromosomes and Eq. 5 gives 7 genes [a0, a1..a3, b1..b3]."""
    with open(os.path.join(GOLDEN, "worked_example.json")) as f:
        ex = json.load(f)
    assert orc.num_chromosomes(ex["features"], TRIG) == ex["chromosomes"]
    assert orc.num_genes_tied(ex["degree"], TRIG) == ex["genes"]
    # the tied chromosome's gene order: cosine block, then sine block
    x = 0.37
    vals = orc.basis_values(TRIG, ex["degree"], x)
    names = ex["gene_order"][1:]
    for name, v in zip(names, vals):
        j = int(name[1])
        ref = math.cos(j * x) if name[0] == "a" else math.sin(j * x)
        assert v == pytest.approx(ref, abs=1e-15)


def test_fitness_is_quadratic_in_genes(orc):
    """MSE is a quadratic form in the genes: the second difference along a
    gene direction e is 2 |Phi e|^2 / M whatever the base point."""
    pr = dg.regression(15, 500, 3, 2, 0.05, degree=2)
    Phi = design_matrix_numpy(pr.X, 2, CHEB)
    rng = np.random.default_rng(3)
    a = rng.uniform(-1, 1, pr.K)
    e = np.zeros(pr.K)
    e[4] = 1.0
    h = 0.5
    f = orc.fitness(pr.X, pr.y, np.stack([a - h * e, a, a + h * e]), 2, CHEB)
    second = (f[0] - 2 * f[1] + f[2]) / h ** 2
    assert second == pytest.approx(2 * np.sum(Phi[:, 4] ** 2) / pr.M, rel=1e-9)


def test_error_kinds(orc):
    """RMSE is the root of the MSE; the mean absolute error never exceeds it."""
    pr = dg.regression(16, 300, 4, 3, 0.1, degree=3)
    pop = dg.random_population(8, 6, pr.K)
    mse = orc.fitness(pr.X, pr.y, pop, 3, CHEB, err=orc.ERR_MSE)
    rmse = orc.fitness(pr.X, pr.y, pop, 3, CHEB, err=orc.ERR_RMSE)
    mae = orc.fitness(pr.X, pr.y, pop, 3, CHEB, err=orc.ERR_MAE)
    np.testing.assert_allclose(rmse, np.sqrt(mse), rtol=1e-14)
    assert np.all(mae <= rmse * (1 + 1e-12))
    Phi = design_matrix_numpy(pr.X, 3, CHEB)
    np.testing.assert_allclose(mae, np.abs(pr.y[None, :] - pop.astype(np.float64) @ Phi.T)
                               .mean(axis=1), rtol=1e-12)


def test_invalid_arguments(orc):
    with pytest.raises(ValueError):
        orc.basis_values(5, 3, 0.1)
    assert orc.num_genes(0, 3, CHEB) == -1


def test_predict_matches_numpy_design_matrix(orc):
    for basis, d in [(CHEB, 5), (TRIG, 3)]:
        pr = dg.regression(21 + basis, 400, 5, 3, 0.1, degree=d, basis=basis)
        a = dg.random_population(4, 1, pr.K)[0]
        out = orc.predict(pr.X, a, d, basis)
        ref = design_matrix_numpy(pr.X, d, basis) @ a.astype(np.float64)
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_classify_hand_example(orc):
    """Degree 1, one feature, a = (0, 1): Out = x. Positives by target:
    patterns 0, 1; predicted positive: patterns 1, 2."""
    X = np.array([[-0.5], [0.2], [0.7], [-0.1]])
    y = np.array([1.0, 1.0, -1.0, -1.0])
    counts = orc.classify(X, y, np.array([0.0, 1.0]), 1, CHEB, 0.0)
    assert counts == (1, 1, 1, 1)
    assert orc.classification_metrics(counts) == (0.5, 0.5, 0.5)
    # a threshold beyond every target and output: all negatives / all positives
    assert orc.classify(X, y, np.array([0.0, 1.0]), 1, CHEB, 10.0) == (0, 0, 4, 0)
    assert orc.classify(X, y, np.array([0.0, 1.0]), 1, CHEB, -10.0) == (4, 0, 0, 0)
    # Out = 0.3 - x: predicted positive for x < 0.3 (patterns 0, 1, 3)
    assert orc.classify(X, y, np.array([0.3, -1.0]), 1, CHEB, 0.0) == (2, 1, 1, 0)


def test_classify_values_at_the_threshold_are_negative(orc):
    """Both comparisons are strict: a target or an output equal to the
    threshold counts as negative. Out = 0.25 + x is exactly 0.25 at x = 0."""
    X = np.array([[-0.5], [0.0], [0.0], [0.5]])
    y = np.array([0.25, 0.25, 1.0, 1.0])
    # pattern 0: y = t, Out < t (TN); 1: y = t, Out = t (TN);
    # 2: y > t, Out = t (FN); 3: y > t, Out > t (TP)
    assert orc.classify(X, y, np.array([0.25, 1.0]), 1, CHEB, 0.25) == (1, 0, 2, 1)


def test_classify_counts_brute_force(orc):
    pr = dg.regression(5, 700, 4, 3, 0.2, degree=3)
    a = dg.random_population(9, 1, pr.K, scale=0.3)[0]
    out = design_matrix_numpy(pr.X, 3, CHEB) @ a.astype(np.float64)
    thr = float(np.median(pr.y))
    assert np.min(np.abs(out - thr)) > 1e-9      # no decision at the rounding level
    act, pred = pr.y > thr, out > thr
    ref = (int(np.sum(pred & act)), int(np.sum(pred & ~act)), int(np.sum(~pred & ~act)),
           int(np.sum(~pred & act)))
    assert orc.classify(pr.X, pr.y, a, 3, CHEB, thr) == ref


def test_generating_chromosome_misclassifies_only_flipped_labels(orc):
    """The large classification set labels sign(target) with 5% flips: its
    generating chromosome predicts every unflipped label."""
    pr = dg.large_classification(M=5000)
    t = design_matrix_numpy(pr.X, 8, CHEB) @ pr.coef.astype(np.float64)
    flipped = int(np.sum(np.where(t >= 0, 1.0, -1.0) != pr.y))
    tp, fp, tn, fn = orc.classify(pr.X, pr.y, pr.coef, 8, CHEB, 0.0)
    assert tp + fp + tn + fn == 5000
    assert fp + fn == flipped and 150 < flipped < 350
