"""Checkpoint files (game_save / game_load) through the C ABI: a run resumed
from a file continues exactly, bit for bit, with and without the surrogate;
files of another shape, truncated or foreign files are refused."""
import os

import numpy as np
import pytest

from helpers import CHEB, TRIG
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


@pytest.mark.parametrize("kw", [
    dict(precision=game.GAME_PREC_BF16),
    dict(precision=game.GAME_PREC_GRAM, tied=1, selection=game.GAME_SEL_ROULETTE),
    dict(precision=game.GAME_PREC_FP32, selection=game.GAME_SEL_RANKING, immigrants=2),
], ids=["bf16", "tied-gram-roulette", "fp32-ranking"])
def test_resume_from_file_is_exact(tmp_path, kw):
    pr = dg.small_regression()
    path = str(tmp_path / "run.ckpt")
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=21, **kw) as g:
        g.train(5)
        g.save(path)
        g.train(7)
        ref = g.population()
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64, seed=21, **kw) as g:
        g.load(path)
        assert g.population()[2] == 5
        g.train(7)
        got = g.population()
    assert got[2] == ref[2] == 12
    np.testing.assert_array_equal(bits(got[0]), bits(ref[0]))
    np.testing.assert_array_equal(bits(got[1]), bits(ref[1]))
    assert not os.path.exists(path + ".tmp")


def test_resume_with_surrogate_is_exact(tmp_path):
    """The surrogate's weights, Adam state, verdict and replay ring travel
    with the file: the screened run continues exactly."""
    pr = dg.regression(3, 3000, 12, 4, 0.05, degree=4)
    path = str(tmp_path / "sur.ckpt")
    kw = dict(P=128, seed=5, precision=game.GAME_PREC_BF16, surrogate=1, oversample=4)
    with game.Game(pr.X, pr.y, 4, CHEB, **kw) as g:
        g.train(4)
        g.save(path)
        g.train(4)
        ref = g.population()
        ref_w = g.surrogate_params()
    with game.Game(pr.X, pr.y, 4, CHEB, **kw) as g:
        g.train(2)   # a different surrogate state, replaced by the file's
        g.load(path)
        g.train(4)
        got = g.population()
        got_w = g.surrogate_params()
    np.testing.assert_array_equal(bits(got[0]), bits(ref[0]))
    np.testing.assert_array_equal(bits(got[1]), bits(ref[1]))
    np.testing.assert_array_equal(bits(got_w), bits(ref_w))


def test_load_refuses_other_shapes_and_bad_files(tmp_path):
    pr = dg.small_regression()
    path = str(tmp_path / "a.ckpt")
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64) as g:
        g.save(path)
        before = g.population()
    cases = [dict(P=65), dict(P=64, tied=1), dict(P=64, surrogate=1, oversample=2)]
    for kw in cases:
        with game.Game(pr.X, pr.y, pr.degree, CHEB, **kw) as g:
            with pytest.raises(game.GameError) as ei:
                g.load(path)
            assert ei.value.code == game.GAME_EINVAL
    with game.Game(pr.X, pr.y, pr.degree, TRIG, P=64) as g:   # other basis
        with pytest.raises(game.GameError):
            g.load(path)
    data = open(path, "rb").read()
    short = str(tmp_path / "short.ckpt")
    open(short, "wb").write(data[:len(data) // 2])
    foreign = str(tmp_path / "foreign.ckpt")
    open(foreign, "wb").write(b"x" * len(data))
    with game.Game(pr.X, pr.y, pr.degree, CHEB, P=64) as g:
        for bad in (short, foreign, str(tmp_path / "missing.ckpt")):
            with pytest.raises(game.GameError) as ei:
                g.load(bad)
            assert ei.value.code == game.GAME_EINVAL
        g.load(path)   # a good file still loads after the refusals
        got = g.population()
    np.testing.assert_array_equal(bits(got[0]), bits(before[0]))
