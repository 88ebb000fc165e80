"""Outputs (Eq. 2, FP64 on the GPU) and binary classification counts of one
chromosome against the oracle, through the C ABI: on the training set and
on caller data, per-feature and shared genes, both bases."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, design_matrix
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
U64 = 2.0 ** -53


def out_tol(X, a, d, basis):
    """FP64 rounding of the sum and the recurrences: a few K u64 of the
    absolute terms."""
    Phi = np.abs(design_matrix(X, d, basis))
    K = Phi.shape[1]
    return 8 * (K + d * d) * U64 * (Phi @ np.abs(np.asarray(a, dtype=np.float64))) + 1e-300


@pytest.mark.parametrize("M,N,d,basis", [(3001, 8, 4, CHEB), (777, 3, 7, TRIG), (1, 2, 2, CHEB),
                                         (5000, 32, 8, CHEB)])
def test_predict_training_set_and_caller_data(orc, M, N, d, basis):
    pr = dg.regression(M + N, M, N, min(d, 3), 0.05, degree=d, basis=basis)
    a = dg.random_population(3, 1, pr.K)[0]
    ref = orc.predict(pr.X, a, d, basis)
    tol = out_tol(pr.X, a, d, basis)
    other = dg.regression(M + 1, 257, N, 2, 0.0, degree=d, basis=basis).X
    ref_o = orc.predict(other, a, d, basis)
    with game.Game(pr.X, pr.y, d, basis, P=8) as g:
        got = g.predict(a)
        got_o = g.predict(a, other)
        got_dev = g.predict(torch.from_numpy(a).cuda(), torch.from_numpy(other).cuda())
        torch.cuda.synchronize()
        assert g.predict(a, other[:0]).shape == (0,)
    assert np.all(np.abs(got - ref) <= tol)
    assert np.all(np.abs(got_o - ref_o) <= out_tol(other, a, d, basis))
    np.testing.assert_array_equal(got_dev.cpu().numpy(), got_o)


def test_predict_shared_genes(orc):
    pr = dg.regression(3, 2000, 6, 3, 0.05, degree=5, basis=TRIG)
    tied = dg.random_population(4, 1, 11)[0]
    full = np.concatenate([tied[:1]] + [tied[1:]] * 6)
    ref = orc.predict(pr.X, full, 5, TRIG)
    with game.Game(pr.X, pr.y, 5, TRIG, P=8, tied=1) as g:
        got = g.predict(tied)
    assert np.all(np.abs(got - ref) <= out_tol(pr.X, full, 5, TRIG))


def _assert_same_counts(res, ref):
    assert (res["tp"], res["fp"], res["tn"], res["fn"]) == ref
    acc, comp, cont = (ref[0] + ref[2]) / sum(ref), ref[0] / (ref[0] + ref[3]), \
        ref[1] / (ref[0] + ref[1])
    assert res["accuracy"] == pytest.approx(acc, rel=1e-15)
    assert res["completeness"] == pytest.approx(comp, rel=1e-15)
    assert res["contamination"] == pytest.approx(cont, rel=1e-15)


def test_classify_large_classification_generating_chromosome(orc):
    """The classification workload's generating chromosome: exactly the
    flipped labels are misclassified; counts equal the oracle's."""
    pr = dg.large_classification(M=60000)
    out = orc.predict(pr.X, pr.coef, 8, CHEB)
    assert np.min(np.abs(out)) > 1e-9   # no decision at the rounding level
    ref = orc.classify(pr.X, pr.y, pr.coef, 8, CHEB, 0.0)
    with game.Game(pr.X, pr.y, 8, CHEB, P=8) as g:
        res = g.classify(pr.coef)
        res_ext = g.classify(pr.coef, pr.X[:1000], pr.y[:1000])
    _assert_same_counts(res, ref)
    assert res["fp"] + res["fn"] == int(np.sum(np.where(out >= 0, 1.0, -1.0) != pr.y))
    _assert_same_counts(res_ext, orc.classify(pr.X[:1000], pr.y[:1000], pr.coef, 8, CHEB, 0.0))


def test_classify_threshold_and_edge_cases(orc):
    pr = dg.regression(8, 4000, 5, 3, 0.3, degree=3)
    a = dg.random_population(10, 1, pr.K, scale=0.4)[0]
    thr = float(np.median(pr.y))
    out = orc.predict(pr.X, a, 3, CHEB)
    assert np.min(np.abs(out - thr)) > 1e-9
    with game.Game(pr.X, pr.y, 3, CHEB, P=8) as g:
        _assert_same_counts(g.classify(a, threshold=thr), orc.classify(pr.X, pr.y, a, 3, CHEB, thr))
        empty = g.classify(a, pr.X[:0], pr.y[:0])
        assert (empty["tp"], empty["fp"], empty["tn"], empty["fn"]) == (0, 0, 0, 0)
        assert empty["accuracy"] == 0.0
        big = g.classify(a, threshold=1e300)
        assert (big["tp"], big["fp"], big["fn"]) == (0, 0, 0) and big["tn"] == pr.M
        with pytest.raises(game.GameError):
            g.classify(a, threshold=float("nan"))
        with pytest.raises(game.GameError):   # the training set has M patterns
            game._check(game.load().game_predict(g.h, game._ptr(a), None, pr.M - 1,
                                                 game._ptr(np.zeros(pr.M))))
