"""Thin ctypes binding of libgame.so (include/game.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
library. Arrays may be numpy arrays (host memory) or torch CUDA tensors
(device memory); torch supplies device memory and the stream. If the
library has not been built the import of the functions fails loudly: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GAME_OK = 0
GAME_EINVAL = -1
GAME_ENOMEM = -2
GAME_ECUDA = -3
GAME_ETIMEOUT = -4
GAME_ESTATE = -5

GAME_BASIS_CHEB = 0
GAME_BASIS_TRIG = 1
GAME_PREC_FP32 = 0
GAME_PREC_BF16 = 1
GAME_PREC_BF16X3 = 2
GAME_PREC_FP8 = 3
GAME_PREC_GRAM = 4
GAME_ERR_MSE = 0
GAME_ERR_RMSE = 1
GAME_ERR_MAE = 2
GAME_SEL_TOURNAMENT = 0
GAME_SEL_RANKING = 1
GAME_SEL_ROULETTE = 2
GAME_HOOK_FAIL_ALLOC = 1
GAME_HOOK_STALL_NS = 2
GAME_HOOK_SMEM_SLACK = 3
GAME_KERNEL_FP32 = 1
GAME_KERNEL_TC = 2
GAME_KERNEL_TC_PAIR = 3
GAME_KERNEL_GRAM = 4

_ERR_NAMES = {GAME_EINVAL: "GAME_EINVAL", GAME_ENOMEM: "GAME_ENOMEM", GAME_ECUDA: "GAME_ECUDA",
              GAME_ETIMEOUT: "GAME_ETIMEOUT", GAME_ESTATE: "GAME_ESTATE"}

# every symbol include/game.h declares
EXPORTED = ("game_params_default", "game_create", "game_get_shape", "game_eval_fitness",
            "game_eval_fitness_prec", "game_generation", "game_train", "game_get_population",
            "game_set_state", "game_set_timing", "game_get_timing", "game_sync",
            "game_destroy", "game_last_error", "game_eval_fitness_static", "game_rescore_top",
            "game_batch_create", "game_batch_generation", "game_batch_get_run",
            "game_batch_get_tiles", "game_batch_fitness_ms", "game_batch_sync",
            "game_batch_destroy", "game_surrogate_predict", "game_surrogate_grad",
            "game_surrogate_train", "game_surrogate_params", "game_surrogate_set_params",
            "game_surrogate_last", "game_gram", "game_predict", "game_classify",
            "game_save", "game_load", "game_test_hook", "game_eval_sse", "game_breed",
            "game_set_fitness", "game_plan_info")


class GameError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class game_params(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_int32),
        ("elitism", ctypes.c_int32),
        ("tournament", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("immigrants", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("pc", ctypes.c_float),
        ("pm", ctypes.c_float),
        ("sigma", ctypes.c_float),
        ("reserved_f", ctypes.c_float),
        ("mse_threshold", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("rescore_top", ctypes.c_int32),
        ("surrogate", ctypes.c_int32),
        ("oversample", ctypes.c_int32),
        ("selection", ctypes.c_int32),
        ("tied", ctypes.c_int32),
        ("error", ctypes.c_int32),
        ("surrogate_steps", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class game_timing(ctypes.Structure):
    _fields_ = [
        ("fitness_ms", ctypes.c_double),
        ("pack_ms", ctypes.c_double),
        ("reduce_ms", ctypes.c_double),
        ("operators_ms", ctypes.c_double),
        ("fitness_launches", ctypes.c_int64),
        ("pack_launches", ctypes.c_int64),
        ("reduce_launches", ctypes.c_int64),
        ("operators_launches", ctypes.c_int64),
        ("rescore_ms", ctypes.c_double),
        ("rescore_launches", ctypes.c_int64),
        ("surrogate_ms", ctypes.c_double),
        ("surrogate_launches", ctypes.c_int64),
    ]


class game_confusion(ctypes.Structure):
    _fields_ = [
        ("tp", ctypes.c_int64),
        ("fp", ctypes.c_int64),
        ("tn", ctypes.c_int64),
        ("fn", ctypes.c_int64),
        ("accuracy", ctypes.c_double),
        ("completeness", ctypes.c_double),
        ("contamination", ctypes.c_double),
    ]


class game_run_desc(ctypes.Structure):
    _fields_ = [
        ("X", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("M", ctypes.c_int64),
        ("N", ctypes.c_int32),
        ("degree", ctypes.c_int32),
        ("basis", ctypes.c_int32),
        ("P", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgame.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libgame.so not built at {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    vp, i32, i64, u64, dp = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_void_p)
    sig = {
        "game_params_default": [ctypes.POINTER(game_params)],
        "game_create": [vp, vp, i64, i32, i32, i32, ctypes.POINTER(game_params), vp,
                        ctypes.POINTER(vp)],
        "game_get_shape": [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                           ctypes.POINTER(i32)],
        "game_eval_fitness": [vp, vp, i32, dp],
        "game_eval_fitness_prec": [vp, vp, i32, i32, dp],
        "game_generation": [vp, u64],
        "game_train": [vp, i32, ctypes.POINTER(i32)],
        "game_get_population": [vp, vp, dp, ctypes.POINTER(i64)],
        "game_set_state": [vp, vp, dp, i64],
        "game_set_timing": [vp, i32],
        "game_get_timing": [vp, ctypes.POINTER(game_timing)],
        "game_sync": [vp],
        "game_destroy": [vp],
        "game_eval_fitness_static": [vp, vp, i64, i32, i32, i32, vp, i32, dp, vp],
        "game_rescore_top": [vp, vp, i32, dp, i32, vp],
        "game_batch_create": [ctypes.POINTER(game_run_desc), i32, ctypes.POINTER(game_params),
                              vp, i32, vp, ctypes.POINTER(vp)],
        "game_batch_generation": [vp],
        "game_batch_get_run": [vp, i32, vp, dp, ctypes.POINTER(i64)],
        "game_batch_get_tiles": [vp, vp],
        "game_batch_fitness_ms": [vp, i32, ctypes.POINTER(ctypes.c_double)],
        "game_batch_sync": [vp],
        "game_batch_destroy": [vp],
        "game_surrogate_predict": [vp, vp, i32, vp],
        "game_surrogate_grad": [vp, vp, dp, i32, vp, vp],
        "game_surrogate_train": [vp, vp, dp, i32],
        "game_surrogate_params": [vp, vp, ctypes.POINTER(i64)],
        "game_surrogate_set_params": [vp, vp],
        "game_surrogate_last": [vp, vp, vp, ctypes.POINTER(i32), vp, vp],
        "game_gram": [vp, vp, vp, vp],
        "game_predict": [vp, vp, vp, i64, dp],
        "game_save": [vp, ctypes.c_char_p],
        "game_load": [vp, ctypes.c_char_p],
        "game_test_hook": [i32, i64],
        "game_eval_sse": [vp, vp, i32, dp],
        "game_breed": [vp, u64],
        "game_set_fitness": [vp, dp],
        "game_plan_info": [vp, i32, i32, vp],
        "game_classify": [vp, vp, vp, vp, i64, ctypes.c_double, ctypes.POINTER(game_confusion)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.game_last_error.argtypes = []
    lib.game_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc: int):
    if rc != GAME_OK:
        raise GameError(rc, load().game_last_error().decode())


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr()


def _need(a, dtype: str, name: str):
    """a (numpy array, torch tensor or None) unchanged if it holds `dtype`
    ("float32", "float64", "int32"); TypeError otherwise. The library sees
    raw pointers, so a wrong element type would be misread (or read past the
    end of the buffer)."""
    if a is None:
        return a
    got = str(a.dtype).replace("torch.", "")
    if got != dtype:
        raise TypeError(f"{name} must be {dtype}, got {got}")
    return a


def _f32(a):
    """A contiguous float32 copy or view of a numpy array; tensors must
    already be float32."""
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    return _need(a, "float32", "tensor")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def game_params_default() -> game_params:
    p = game_params()
    _check(load().game_params_default(ctypes.byref(p)))
    return p


def game_create(X, y, degree: int, basis: int, prm: game_params | None = None, stream=None):
    """X [M][N] float32, y [M] float32 (numpy or CUDA tensors)."""
    M, N = X.shape
    _need(X, "float32", "X")
    _need(y, "float32", "y")
    h = ctypes.c_void_p()
    _check(load().game_create(_ptr(X), _ptr(y), M, N, degree, basis,
                              ctypes.byref(prm) if prm is not None else None,
                              _stream_ptr(stream), ctypes.byref(h)))
    return h


def game_get_shape(h):
    M, N, K, P = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().game_get_shape(h, ctypes.byref(M), ctypes.byref(N), ctypes.byref(K),
                                 ctypes.byref(P)))
    return M.value, N.value, K.value, P.value


def game_eval_fitness(h, pop, fit_out, precision: int | None = None):
    """pop [P][K] float32, fit_out [P] float64; both numpy or both CUDA tensors."""
    P = pop.shape[0]
    _need(pop, "float32", "pop")
    _need(fit_out, "float64", "fit_out")
    if precision is None:
        _check(load().game_eval_fitness(h, _ptr(pop), P, _ptr(fit_out)))
    else:
        _check(load().game_eval_fitness_prec(h, _ptr(pop), P, precision, _ptr(fit_out)))
    return fit_out


def game_rescore_top(h, pop, fit, n: int, idx_out=None):
    """pop [P][K] float32, fit [P] float64 (updated in place), idx_out [n] int32;
    numpy arrays or CUDA tensors (pop and fit in the same memory)."""
    _need(pop, "float32", "pop")
    _need(fit, "float64", "fit")
    _need(idx_out, "int32", "idx_out")
    _check(load().game_rescore_top(h, _ptr(pop), pop.shape[0], _ptr(fit), n, _ptr(idx_out)))
    return fit


def game_generation(h, seed: int):
    _check(load().game_generation(h, seed))


def game_train(h, generations: int) -> int:
    run = ctypes.c_int32()
    _check(load().game_train(h, generations, ctypes.byref(run)))
    return run.value


def game_get_population(h, pop_out=None, fit_out=None) -> int:
    g = ctypes.c_int64()
    _check(load().game_get_population(h, _ptr(pop_out), _ptr(fit_out), ctypes.byref(g)))
    return g.value


def game_set_state(h, pop, fit=None, generation: int = 0):
    _need(pop, "float32", "pop")
    _need(fit, "float64", "fit")
    _check(load().game_set_state(h, _ptr(pop), _ptr(fit), generation))


def game_set_timing(h, enable: bool):
    _check(load().game_set_timing(h, int(bool(enable))))


def game_get_timing(h) -> dict:
    t = game_timing()
    _check(load().game_get_timing(h, ctypes.byref(t)))
    return {name: getattr(t, name) for name, _ in game_timing._fields_}


def game_eval_fitness_static(X, y, degree: int, basis: int, pop, fit_out, stream=None):
    """Allocation-free FP32 fitness. X [M][N], y [M], pop [P][K] float32 and
    fit_out [>= P] float64, all contiguous CUDA tensors (the library reads
    them through raw pointers, so every shape is checked here first)."""
    for a, dt, name in ((X, "float32", "X"), (y, "float32", "y"), (pop, "float32", "pop"),
                        (fit_out, "float64", "fit_out")):
        _need(a, dt, name)
        if not getattr(a, "is_cuda", False):
            raise TypeError(f"{name} must be a CUDA tensor")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if X.dim() != 2 or pop.dim() != 2:
        raise ValueError("X and pop must be 2-D")
    M, N = X.shape
    B = 2 if basis == GAME_BASIS_TRIG else 1
    K = B * N * degree + 1
    P = pop.shape[0]
    if y.numel() != M:
        raise ValueError(f"y has {y.numel()} elements, X has {M} rows")
    if pop.shape[1] != K:
        raise ValueError(f"pop has {pop.shape[1]} genes per chromosome, B*N*d + 1 = {K}")
    if fit_out.numel() < P:
        raise ValueError(f"fit_out holds {fit_out.numel()} values, P = {P}")
    _check(load().game_eval_fitness_static(_ptr(X), _ptr(y), M, N, degree, basis, _ptr(pop),
                                           P, _ptr(fit_out), _stream_ptr(stream)))
    return fit_out


def game_sync(h):
    _check(load().game_sync(h))


def game_test_hook(hook: int, value: int):
    """Arms a test hook (GAME_HOOK_FAIL_ALLOC: the value-th device
    allocation from now fails; GAME_HOOK_STALL_NS: the next tensor-core
    fitness launch runs into an expired wait after value ns;
    GAME_HOOK_SMEM_SLACK: tensor-core plans keep value bytes of alignment
    slack; 0 = off)."""
    _check(load().game_test_hook(hook, value))


def game_destroy(h):
    if h:
        _check(load().game_destroy(h))


def _params(params) -> game_params:
    """The defaults with the named fields replaced; an unknown name raises
    (ctypes would otherwise accept it as a plain attribute and ignore it)."""
    prm = game_params_default()
    names = {name for name, _ in game_params._fields_}
    for k, v in params.items():
        if k not in names:
            raise TypeError(f"unknown game_params field {k!r}")
        setattr(prm, k, v)
    return prm


class Game:
    """Owning wrapper of a handle with numpy convenience accessors."""

    def __init__(self, X, y, degree, basis=GAME_BASIS_CHEB, stream=None, **params):
        self.h = None
        prm = _params(params)
        X, y = _f32(X), _f32(y)
        self._keep = (X, y)
        self.h = game_create(X, y, degree, basis, prm, stream)
        self.M, self.N, self.K, self.P = game_get_shape(self.h)
        self.precision = prm.precision

    def eval_fitness(self, pop, precision=None):
        if isinstance(pop, np.ndarray):
            pop = np.ascontiguousarray(pop, dtype=np.float32)
            fit = np.zeros(pop.shape[0], dtype=np.float64)
        else:
            import torch
            fit = torch.empty(pop.shape[0], dtype=torch.float64, device=pop.device)
        return game_eval_fitness(self.h, pop, fit, precision)

    def rescore_top(self, pop, fit, n):
        """Returns (fit with the n best re-scored, their indices best first)."""
        if isinstance(pop, np.ndarray):
            pop = np.ascontiguousarray(pop, dtype=np.float32)
            fit = np.array(fit, dtype=np.float64)
            idx = np.zeros(n, dtype=np.int32)
        else:
            import torch
            fit = fit.clone()
            idx = torch.empty(n, dtype=torch.int32, device=pop.device)
        game_rescore_top(self.h, pop, fit, n, idx)
        return fit, idx

    def generation(self, seed):
        game_generation(self.h, seed)

    def gram(self):
        """(G [K][K], b [K], y.y) of the Gram form, FP64."""
        G = np.zeros((self.K, self.K), dtype=np.float64)
        b = np.zeros(self.K, dtype=np.float64)
        yy = np.zeros(1, dtype=np.float64)
        _check(load().game_gram(self.h, _ptr(G), _ptr(b), _ptr(yy)))
        return G, b, float(yy[0])

    def predict(self, chrom, X=None):
        """Outputs Out(m) (Eq. 2, FP64) of one chromosome on X [M][N] (numpy
        or CUDA tensor; None = the training set)."""
        chrom = _f32(chrom)
        M = self.M if X is None else X.shape[0]
        if X is not None:
            X = _f32(X)
        if X is None or isinstance(X, np.ndarray):
            out = np.zeros(M, dtype=np.float64)
        else:
            import torch
            out = torch.empty(M, dtype=torch.float64, device=X.device)
        _check(load().game_predict(self.h, _ptr(chrom), _ptr(X), M, _ptr(out)))
        return out

    def classify(self, chrom, X=None, y=None, threshold=0.0):
        """game_confusion of one chromosome on (X, y) (None = the training
        set) as a dict."""
        chrom = _f32(chrom)
        M = self.M if X is None else X.shape[0]
        if X is not None:
            X, y = _f32(X), _f32(y)
        c = game_confusion()
        _check(load().game_classify(self.h, _ptr(chrom), _ptr(X), _ptr(y), M, float(threshold),
                                    ctypes.byref(c)))
        return {name: getattr(c, name) for name, _ in game_confusion._fields_}

    # ---- fitness surrogate (numpy in / out) ----
    def surrogate_predict(self, pop):
        pop = np.ascontiguousarray(pop, dtype=np.float32)
        out = np.zeros(pop.shape[0], dtype=np.float32)
        _check(load().game_surrogate_predict(self.h, _ptr(pop), pop.shape[0], _ptr(out)))
        return out

    def surrogate_grad(self, pop, fit):
        pop = np.ascontiguousarray(pop, dtype=np.float32)
        fit = np.ascontiguousarray(fit, dtype=np.float64)
        n = ctypes.c_int64()
        _check(load().game_surrogate_params(self.h, None, ctypes.byref(n)))
        g = np.zeros(n.value, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(load().game_surrogate_grad(self.h, _ptr(pop), _ptr(fit), pop.shape[0], _ptr(g),
                                          _ptr(loss)))
        return g, float(loss[0])

    def surrogate_train(self, pop, fit):
        pop = np.ascontiguousarray(pop, dtype=np.float32)
        fit = np.ascontiguousarray(fit, dtype=np.float64)
        _check(load().game_surrogate_train(self.h, _ptr(pop), _ptr(fit), pop.shape[0]))

    def surrogate_params(self):
        n = ctypes.c_int64()
        _check(load().game_surrogate_params(self.h, None, ctypes.byref(n)))
        w = np.zeros(n.value, dtype=np.float32)
        _check(load().game_surrogate_params(self.h, _ptr(w), ctypes.byref(n)))
        return w

    def surrogate_set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().game_surrogate_set_params(self.h, _ptr(w)))

    def surrogate_last(self):
        """(predictions, kept flags, trusted flag used, trust check's correlation)"""
        n = ctypes.c_int32()
        _check(load().game_surrogate_last(self.h, None, None, ctypes.byref(n), None, None))
        pred = np.zeros(n.value, dtype=np.float32)
        keep = np.zeros(n.value, dtype=np.int32)
        tr = np.zeros(1, dtype=np.int32)
        r = np.zeros(1, dtype=np.float32)
        if n.value:
            _check(load().game_surrogate_last(self.h, _ptr(pred), _ptr(keep), ctypes.byref(n),
                                              _ptr(tr), _ptr(r)))
        return pred, keep, int(tr[0]), float(r[0])

    def train(self, generations):
        return game_train(self.h, generations)

    # ---- pattern sharding: per-slice steps ----
    def eval_sse(self, pop=None, out=None):
        """Unnormalised error sums over this handle's patterns (FP64 [P]) of
        pop (None = the current population). out: a float64 numpy array or
        CUDA tensor to fill (default: a new numpy array)."""
        P = self.P if pop is None else pop.shape[0]
        if pop is not None and isinstance(pop, np.ndarray):
            pop = np.ascontiguousarray(pop, dtype=np.float32)
        _need(pop, "float32", "pop")
        if out is None:
            out = np.zeros(P, dtype=np.float64)
        _need(out, "float64", "out")
        if out.shape[0] < P:
            raise ValueError("out holds fewer than P values")
        _check(load().game_eval_sse(self.h, _ptr(pop), P, _ptr(out)))
        return out

    def plan(self, precision=None, P=None):
        """The launch plan of an evaluation (game_plan_info) as a dict."""
        info = np.zeros(8, dtype=np.int32)
        prec = self.precision if precision is None else precision
        _check(load().game_plan_info(self.h, prec, self.P if P is None else P, _ptr(info)))
        names = {GAME_KERNEL_FP32: "fitness_fp32_kernel", GAME_KERNEL_TC: "fitness_tc_kernel",
                 GAME_KERNEL_TC_PAIR: "fitness_tc2_kernel", GAME_KERNEL_GRAM: "quad_kernel"}
        keys = ("kernel", "tile", "kblocks", "stages", "slots", "staged", "ctas", "smem")
        d = dict(zip(keys, (int(v) for v in info)))
        d["kernel"] = names[d["kernel"]]
        return d

    def breed(self, seed):
        """The operators of one generation, without evaluating the result."""
        _check(load().game_breed(self.h, seed))

    def set_fitness(self, fit):
        """Fitness [P] FP64 of the current population (numpy or CUDA tensor)."""
        if isinstance(fit, np.ndarray):
            fit = np.ascontiguousarray(fit, dtype=np.float64)
        _need(fit, "float64", "fit")
        if fit.shape[0] != self.P:
            raise ValueError(f"fit has {fit.shape[0]} values, P = {self.P}")
        _check(load().game_set_fitness(self.h, _ptr(fit)))

    def population(self):
        pop = np.zeros((self.P, self.K), dtype=np.float32)
        fit = np.zeros(self.P, dtype=np.float64)
        g = game_get_population(self.h, pop, fit)
        return pop, fit, g

    def save(self, path):
        _check(load().game_save(self.h, os.fsencode(path)))

    def load(self, path):
        _check(load().game_load(self.h, os.fsencode(path)))

    def set_state(self, pop, fit=None, generation=0):
        pop = np.ascontiguousarray(pop, dtype=np.float32) if isinstance(pop, np.ndarray) else pop
        if fit is not None and isinstance(fit, np.ndarray):
            fit = np.ascontiguousarray(fit, dtype=np.float64)
        game_set_state(self.h, pop, fit, generation)

    def sync(self):
        game_sync(self.h)

    def set_timing(self, enable=True):
        game_set_timing(self.h, enable)

    def timing(self):
        return game_get_timing(self.h)

    def close(self):
        if self.h:
            game_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Owning wrapper of a batch of independent runs (game_batch_*).

    runs: sequence of (X, y, degree, basis, P, seed) with X [M][N] float32 and
    y [M] float32 numpy arrays or CUDA tensors."""

    def __init__(self, runs, tiles=None, autotune=True, stream=None, **params):
        self.h = None
        prm = _params(params)
        descs = (game_run_desc * len(runs))()
        self._keep = []
        self.shapes = []
        for r, (X, y, degree, basis, P, seed) in enumerate(runs):
            X, y = _f32(X), _f32(y)
            self._keep.append((X, y))
            M, N = X.shape
            descs[r] = game_run_desc(_ptr(X), _ptr(y), M, N, degree, basis, P, seed)
            B = 2 if basis == GAME_BASIS_TRIG else 1
            self.shapes.append((M, N, B * N * degree + 1, P))
        t = None
        if tiles is not None:
            t = np.ascontiguousarray(tiles, dtype=np.int32)
            self._keep.append(t)
        h = ctypes.c_void_p()
        _check(load().game_batch_create(descs, len(runs), ctypes.byref(prm),
                                        _ptr(t) if t is not None else None, int(bool(autotune)),
                                        _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.R = len(runs)

    def generation(self):
        _check(load().game_batch_generation(self.h))

    def run(self, r):
        M, N, K, P = self.shapes[r]
        pop = np.zeros((P, K), dtype=np.float32)
        fit = np.zeros(P, dtype=np.float64)
        g = ctypes.c_int64()
        _check(load().game_batch_get_run(self.h, r, _ptr(pop), _ptr(fit), ctypes.byref(g)))
        return pop, fit, g.value

    def tiles(self):
        t = np.zeros(self.R, dtype=np.int32)
        _check(load().game_batch_get_tiles(self.h, _ptr(t)))
        return t

    def fitness_ms(self, reps=10):
        ms = ctypes.c_double()
        _check(load().game_batch_fitness_ms(self.h, reps, ctypes.byref(ms)))
        return ms.value

    def sync(self):
        _check(load().game_batch_sync(self.h))

    def close(self):
        if self.h:
            _check(load().game_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
