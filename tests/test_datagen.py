"""The synthetic input recipes (the stand-ins for the paper's data set) hold
the properties they are documented with: shapes, ranges, noise level, label
flips, feature correlation, the batched workload's parameter ranges, and
seeded determinism. None of this touches GAME's arithmetic."""
import numpy as np
import pytest

from paper_1211_5481_gb300 import datagen as dg


def test_small_regression_recipe():
    pr = dg.small_regression()
    assert pr.X.shape == (2000, 8) and pr.X.dtype == np.float32 and pr.y.dtype == np.float32
    assert (pr.degree, pr.basis, pr.P, pr.K) == (4, dg.CHEB, 64, 33)
    assert pr.X.min() >= -1.0 and pr.X.max() <= 1.0
    # noise = y - noiseless target: sd 0.05 within sampling error (2000 draws)
    t = dg.additive_chebyshev_target(pr.X, pr.coef, 4)
    r = pr.extra["target_fp64"] - t
    assert abs(r.std() - 0.05) < 0.005 and abs(r.mean()) < 0.005


def test_large_classification_recipe():
    M = 40000
    pr = dg.large_classification(M=M)
    assert pr.X.shape == (M, 32) and (pr.degree, pr.P, pr.K) == (8, 1024, 257)
    # min-max scaled per column: every column reaches both ends exactly
    np.testing.assert_array_equal(pr.X.min(axis=0), -1.0)
    np.testing.assert_array_equal(pr.X.max(axis=0), 1.0)
    assert set(np.unique(pr.y)) == {-1.0, 1.0}
    t = dg.additive_chebyshev_target(pr.X, pr.coef, 8)
    flipped = np.mean(np.where(t >= 0, 1.0, -1.0) != pr.y)
    assert abs(flipped - 0.05) < 5 * np.sqrt(0.05 * 0.95 / M)
    # the affine scaling keeps the correlation of x = L z: corr of S = W W^T / N + 0.1 I
    rng = dg._rng(2, dg._TAG_MIX)
    W = rng.standard_normal((32, 32))
    S = W @ W.T / 32 + 0.1 * np.eye(32)
    d = np.sqrt(np.diag(S))
    want = S / np.outer(d, d)
    got = np.corrcoef(pr.X.astype(np.float64), rowvar=False)
    assert np.max(np.abs(got - want)) < 0.03


def test_small_classification_has_the_paper_shape():
    pr = dg.small_classification()
    assert pr.X.shape == (2100, 9) and pr.basis == dg.TRIG
    assert pr.P == 2 * 9 + 1          # Eq. 4: B N + 1
    assert set(np.unique(pr.y)) == {-1.0, 1.0}


def test_surrogate_regression_recipe_small_sample():
    pr = dg.surrogate_regression(M=5000)
    assert pr.X.shape == (5000, 48) and (pr.degree, pr.P, pr.K) == (6, 2048, 289)


def test_batched_runs_ranges():
    runs = dg.batched_runs(R=256)
    M = np.array([r.M for r in runs])
    N = np.array([r.N for r in runs])
    d = np.array([r.degree for r in runs])
    P = np.array([r.P for r in runs])
    B = np.array([2 if r.basis == dg.TRIG else 1 for r in runs])
    assert len(runs) == 256
    assert M.min() >= 1000 and M.max() <= 200_000
    assert N.min() >= 4 and N.max() <= 64 and d.min() >= 2 and d.max() <= 10
    assert P.min() >= 32 and P.max() <= 512
    assert 0 < np.sum(B == 2) < 256
    K = np.array([r.K for r in runs])
    np.testing.assert_array_equal(K, B * N * d + 1)
    assert K.min() >= 9 and K.max() <= 2 * 64 * 10 + 1
    # log-uniform M: the median sits near the geometric mean of the range
    assert abs(np.log(np.median(M)) - np.log(np.sqrt(1000 * 200_000))) < 0.5


@pytest.mark.parametrize("make", [dg.small_regression, lambda: dg.large_classification(M=3000),
                                  dg.small_classification])
def test_seeded_and_deterministic(make):
    a, b = make(), make()
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.y, b.y)


def test_streams_differ_by_seed_and_purpose():
    a = dg.regression(1, 500, 4, 2, 0.1)
    b = dg.regression(2, 500, 4, 2, 0.1)
    assert not np.array_equal(a.X, b.X)
    # features and coefficients of one seed come from different streams
    assert not np.allclose(a.X.ravel()[:a.coef.size], a.coef)
