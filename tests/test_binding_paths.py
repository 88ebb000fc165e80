"""Every method of the Python binding's Game and Batch wrappers runs its
argument handling (conversions, type checks, output allocation, result
unpacking) against a stand-in for the library that accepts every call, with
numpy arrays and with torch tensors. No device is involved: this covers the
binding's own Python, which the GPU tests otherwise reach only on a GPU."""
import ctypes

import numpy as np
import pytest

from paper_1211_5481_gb300 import game

torch = pytest.importorskip("torch")


class _StandIn:
    """Returns GAME_OK for every entry point; fills the few outputs the
    binding reads back."""

    def __init__(self, real):
        self.real = real

    def __getattr__(self, name):
        if name == "game_params_default":
            return self.real.game_params_default
        if name == "game_last_error":
            return lambda: b"stand-in"
        if name == "game_get_shape":
            def shape(h, M, N, K, P):
                M._obj.value, N._obj.value, K._obj.value, P._obj.value = 100, 3, 13, 8
                return 0
            return shape
        if name == "game_surrogate_last":
            def last(h, pred, keep, n, tr, r):
                n._obj.value = 0
                return 0
            return last
        if name == "game_surrogate_params":
            def params(h, w, n):
                n._obj.value = 5
                return 0
            return params
        if name == "game_train":
            def train(h, g, run):
                run._obj.value = g
                return 0
            return train
        return lambda *a: 0


@pytest.fixture
def stand_in(monkeypatch):
    monkeypatch.setattr(game, "_lib", _StandIn(game.load()))


def test_game_methods_with_numpy(stand_in, tmp_path):
    X = np.zeros((100, 3))           # float64: converted by the wrapper
    y = np.zeros(100)
    pop = np.zeros((8, 13), dtype=np.float32)
    with game.Game(X, y, 2, game.GAME_BASIS_TRIG, P=8, seed=1) as g:
        assert (g.M, g.N, g.K, g.P) == (100, 3, 13, 8)
        assert g.eval_fitness(pop).dtype == np.float64
        assert g.eval_fitness(pop.astype(np.float64), precision=game.GAME_PREC_BF16).shape == (8,)
        fit, idx = g.rescore_top(pop, np.zeros(8), 4)
        assert fit.dtype == np.float64 and idx.dtype == np.int32 and idx.shape == (4,)
        assert g.predict(pop[0]).shape == (100,) and g.predict(pop[0], X[:10]).shape == (10,)
        assert set(g.classify(pop[0])) == {"tp", "fp", "tn", "fn", "accuracy", "completeness",
                                           "contamination"}
        g.classify(pop[0], X[:10], y[:10], threshold=0.5)
        g.set_state(pop.astype(np.float64), np.zeros(8, dtype=np.float32), 3)
        g.generation(5)
        assert g.train(7) == 7
        p, f, gen = g.population()
        assert p.shape == (8, 13) and f.shape == (8,)
        assert g.surrogate_last()[0].shape == (0,) and g.surrogate_params().shape == (5,)
        g.surrogate_predict(pop)
        g.surrogate_train(pop, np.ones(8))
        g.surrogate_grad(pop, np.ones(8))
        g.surrogate_set_params(np.zeros(5))
        g.save(str(tmp_path / "c.ckpt"))
        g.load(str(tmp_path / "c.ckpt"))
        g.set_timing(True)
        assert "fitness_ms" in g.timing()
        g.sync()
        assert g.eval_sse().shape == (8,) and g.eval_sse(pop).dtype == np.float64
        g.breed(3)
        g.set_fitness(np.zeros(8, dtype=np.float32))
        with pytest.raises(ValueError):
            g.set_fitness(np.zeros(7))
        with pytest.raises(TypeError):
            g.eval_sse(pop, out=np.zeros(8, dtype=np.float32))


def test_game_methods_with_tensors(stand_in):
    X = torch.zeros((100, 3), dtype=torch.float32)
    y = torch.zeros(100, dtype=torch.float32)
    pop = torch.zeros((8, 13), dtype=torch.float32)
    with game.Game(X, y, 2, game.GAME_BASIS_TRIG, P=8) as g:
        assert g.eval_fitness(pop).dtype == torch.float64
        fit, idx = g.rescore_top(pop, torch.zeros(8, dtype=torch.float64), 4)
        assert idx.dtype == torch.int32
        assert g.predict(pop[0], X).dtype == torch.float64
        with pytest.raises(TypeError):
            g.eval_fitness(pop.double())
        with pytest.raises(TypeError):
            g.predict(pop[0], X.half())
    with pytest.raises(TypeError):
        game.Game(X.double(), y, 2, game.GAME_BASIS_TRIG)


def test_batch_methods(stand_in):
    X = np.zeros((100, 3), dtype=np.float32)
    y = np.zeros(100, dtype=np.float32)
    with game.Batch([(X, y, 2, 0, 8, 1), (X, y, 3, 1, 16, 2)], tiles=[64, 128]) as b:
        b.generation()
        pop, fit, gen = b.run(1)
        assert pop.shape == (16, 2 * 3 * 3 + 1)
        assert b.tiles().shape == (2,)
        b.fitness_ms()
        b.sync()


class _OnDevice:
    """A CPU tensor that reports itself as a CUDA tensor: the allocation-free
    wrapper checks device residence, contiguity and shapes before it takes
    raw pointers, and the stand-in library never dereferences them."""

    def __init__(self, t):
        self.t = t
        self.dtype, self.shape, self.is_cuda = t.dtype, t.shape, True

    def dim(self):
        return self.t.dim()

    def numel(self):
        return self.t.numel()

    def is_contiguous(self):
        return self.t.is_contiguous()

    def data_ptr(self):
        return self.t.data_ptr()


def test_static_wrapper_checks_shapes(stand_in):
    f32, f64 = torch.float32, torch.float64
    M, N, d = 50, 3, 2
    K = 2 * N * d + 1          # trigonometric basis
    X, y = torch.zeros((M, N), dtype=f32), torch.zeros(M, dtype=f32)
    pop, fit = torch.zeros((6, K), dtype=f32), torch.zeros(6, dtype=f64)
    dv = _OnDevice
    trig = game.GAME_BASIS_TRIG
    out = game.game_eval_fitness_static(dv(X), dv(y), d, trig, dv(pop), dv(fit))
    assert out.t is fit
    with pytest.raises(TypeError):          # host tensors
        game.game_eval_fitness_static(X, dv(y), d, trig, dv(pop), dv(fit))
    with pytest.raises(TypeError):          # element type
        game.game_eval_fitness_static(dv(X), dv(y), d, trig, dv(pop.double()), dv(fit))
    with pytest.raises(ValueError):         # K of the Chebyshev basis, not the trigonometric one
        game.game_eval_fitness_static(dv(X), dv(y), d, game.GAME_BASIS_CHEB, dv(pop), dv(fit))
    with pytest.raises(ValueError):         # y shorter than X
        game.game_eval_fitness_static(dv(X), dv(y[:-1]), d, trig, dv(pop), dv(fit))
    with pytest.raises(ValueError):         # fit_out shorter than P
        game.game_eval_fitness_static(dv(X), dv(y), d, trig, dv(pop), dv(fit[:5]))
    with pytest.raises(ValueError):         # a transposed (strided) view
        game.game_eval_fitness_static(dv(X.t()), dv(y), d, trig, dv(pop), dv(fit))
