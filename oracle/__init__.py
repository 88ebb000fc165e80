"""FP64 CPU oracle for GAME fitness evaluation and GA operators.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline, reference and accuracy legs of ``bench.py`` import this
package. It shares no code with the CUDA path (``paper_1211_5481_gb300``)
and neither imports the other.

``GAME_ORACLE_SOURCE`` and ``GAME_ORACLE_SURROGATE_SOURCE`` (tests only)
name another copy of ``oracle.c`` or ``surrogate.py`` to load instead: the
planted-mistake tests run the pins against copies with one mistake each.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over
chromosomes); this module only compiles it and marshals numpy arrays.
Citations are to Cavuoti et al., arXiv:1211.5481 (Section 3, Eq. 1-6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.environ.get("GAME_ORACLE_SOURCE") or os.path.join(_HERE, "oracle.c")
_LIB = (os.path.join(_HERE, "liboracle.so") if _SRC == os.path.join(_HERE, "oracle.c")
        else os.path.splitext(_SRC)[0] + ".so")
_lock = threading.Lock()
_lib = None

CHEB, TRIG = 0, 1
ERR_MSE, ERR_RMSE, ERR_MAE = 0, 1, 2
SEL_TOURNAMENT, SEL_RANKING, SEL_ROULETTE = 0, 1, 2


class GAParams(ctypes.Structure):
    _fields_ = [
        ("elitism", ctypes.c_int32),
        ("tournament", ctypes.c_int32),
        ("thr_pc", ctypes.c_uint32),
        ("thr_pm", ctypes.c_uint32),
        ("sigma", ctypes.c_float),
        ("immigrants", ctypes.c_int32),
        ("selection", ctypes.c_int32),
    ]


def ga_params(elitism=2, tournament=3, pc=0.9, pm=0.02, sigma=0.1, immigrants=0,
              selection=SEL_TOURNAMENT):
    """Operator parameters; the rates become 24-bit integer thresholds
    floor(rate * 2^24), computed once in FP64."""
    return GAParams(elitism, tournament, int(np.floor(pc * 2.0**24)),
                    int(np.floor(pm * 2.0**24)), float(np.float32(sigma)), immigrants,
                    selection)


def compile_source(src: str, lib: str) -> str:
    """gcc, -O2, OpenMP, no FP contraction so that FP32 gene updates round
    once per operation; ``oracle.h`` is taken from this directory."""
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-I", _HERE, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source unless it is up to date."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        return compile_source(_SRC, _LIB)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d, i32, i64, u32, u64 = (ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_uint32, ctypes.c_uint64)
        vp = ctypes.c_void_p
        lib.oracle_num_chromosomes.restype = i64
        lib.oracle_num_chromosomes.argtypes = [i32, i32]
        lib.oracle_num_genes_tied.restype = i64
        lib.oracle_num_genes_tied.argtypes = [i32, i32]
        lib.oracle_num_genes.restype = i64
        lib.oracle_num_genes.argtypes = [i32, i32, i32]
        lib.oracle_basis.argtypes = [i32, i32, d, vp]
        lib.oracle_output.restype = d
        lib.oracle_output.argtypes = [vp, vp, i32, i32, i32]
        lib.oracle_fitness.argtypes = [vp, vp, i64, i32, i32, i32, vp, i32, vp]
        lib.oracle_fitness_err.argtypes = [vp, vp, i64, i32, i32, i32, vp, i32, i32, vp]
        lib.oracle_fitness_tied.argtypes = [vp, vp, i64, i32, i32, i32, vp, i32, vp]
        lib.oracle_gram.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, vp]
        lib.oracle_predict.argtypes = [vp, i64, i32, i32, i32, vp, vp]
        lib.oracle_train_tied.argtypes = [vp, vp, i64, i32, i32, i32, i32, vp, u64, i32, vp, vp,
                                          vp]
        lib.oracle_classify.argtypes = [vp, vp, i64, i32, i32, i32, vp, d, vp]
        lib.oracle_fitness_gram.argtypes = [vp, vp, d, i64, i32, vp, i32, vp]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        lib.oracle_init_population.argtypes = [u64, i32, i32, vp]
        lib.oracle_generation.argtypes = [vp, vp, i32, i32, ctypes.POINTER(GAParams),
                                          u64, u32, vp]
        lib.oracle_train.argtypes = [vp, vp, i64, i32, i32, i32, i32,
                                     ctypes.POINTER(GAParams), u64, i32, i32, vp, vp, vp]
        lib.oracle_select_best.argtypes = [vp, i32, i32, vp]
        lib.oracle_offspring.argtypes = [vp, vp, i32, i32, ctypes.POINTER(GAParams), u64, u32,
                                         i32, vp]
        lib.oracle_rescore.argtypes = [vp, vp, i64, i32, i32, i32, vp, i32, vp, i32, vp, vp]
        lib.oracle_set_threads.argtypes = [i32]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what}: oracle returned {rc}")


def set_threads(n: int = 0) -> int:
    return _load().oracle_set_threads(n)


def num_genes(N, d, basis):
    return int(_load().oracle_num_genes(N, d, basis))


def num_genes_tied(d, basis):
    return int(_load().oracle_num_genes_tied(d, basis))


def num_chromosomes(N, basis):
    return int(_load().oracle_num_chromosomes(N, basis))


def basis_values(basis, d, x):
    """Eq. 1 / Eq. 6: the B*d basis values of the scalar x."""
    B = 2 if basis == TRIG else 1
    out = np.zeros(B * d, dtype=np.float64)
    _check(_load().oracle_basis(basis, d, float(x), _ptr(out)), "basis")
    return out


def output(a, x, d, basis):
    """Eq. 2 for one chromosome a[K] and one pattern x[N]."""
    a, x = _f64(a), _f64(x)
    return float(_load().oracle_output(_ptr(a), _ptr(x), x.shape[0], d, basis))


def fitness(X, y, pop, d, basis, err=ERR_MSE):
    """Eq. 3 averaged over the M patterns (MSE), one value per chromosome."""
    X, y, pop = _f64(X), _f64(y), _f64(np.atleast_2d(pop))
    M, N = X.shape
    P = pop.shape[0]
    assert pop.shape[1] == num_genes(N, d, basis), "chromosome length"
    fit = np.zeros(P, dtype=np.float64)
    _check(_load().oracle_fitness_err(_ptr(X), _ptr(y), M, N, d, basis, _ptr(pop), P,
                                      err, _ptr(fit)), "fitness")
    return fit


def fitness_tied(X, y, pop, d, basis):
    X, y, pop = _f64(X), _f64(y), _f64(np.atleast_2d(pop))
    M, N = X.shape
    fit = np.zeros(pop.shape[0], dtype=np.float64)
    assert pop.shape[1] == num_genes_tied(d, basis)
    _check(_load().oracle_fitness_tied(_ptr(X), _ptr(y), M, N, d, basis, _ptr(pop),
                                       pop.shape[0], _ptr(fit)), "fitness_tied")
    return fit


def predict(X, a, d, basis):
    """Outputs Out(m) of one chromosome a[K] (Eq. 2) on the patterns X."""
    X, a = _f64(X), _f64(np.ravel(a))
    M, N = X.shape
    assert a.shape[0] == num_genes(N, d, basis), "chromosome length"
    out = np.zeros(M, dtype=np.float64)
    _check(_load().oracle_predict(_ptr(X), M, N, d, basis, _ptr(a), _ptr(out)), "predict")
    return out


def classify(X, y, a, d, basis, threshold=0.0):
    """(TP, FP, TN, FN): positive when y > threshold, predicted positive
    when Out > threshold."""
    X, y, a = _f64(X), _f64(y), _f64(np.ravel(a))
    M, N = X.shape
    assert a.shape[0] == num_genes(N, d, basis), "chromosome length"
    counts = np.zeros(4, dtype=np.int64)
    _check(_load().oracle_classify(_ptr(X), _ptr(y), M, N, d, basis, _ptr(a), float(threshold),
                                   _ptr(counts)), "classify")
    return tuple(int(c) for c in counts)


def classification_metrics(counts):
    """accuracy = (TP + TN) / M, completeness = TP / (TP + FN),
    contamination = FP / (TP + FP) (0 for an empty denominator)."""
    tp, fp, tn, fn = counts
    M = tp + fp + tn + fn
    return ((tp + tn) / M if M else 0.0, tp / (tp + fn) if tp + fn else 0.0,
            fp / (tp + fp) if tp + fp else 0.0)


def gram(X, y, d, basis):
    X, y = _f64(X), _f64(y)
    M, N = X.shape
    K = num_genes(N, d, basis)
    G = np.zeros((K, K), dtype=np.float64)
    b = np.zeros(K, dtype=np.float64)
    yy = np.zeros(1, dtype=np.float64)
    _check(_load().oracle_gram(_ptr(X), _ptr(y), M, N, d, basis, _ptr(G), _ptr(b),
                               _ptr(yy)), "gram")
    return G, b, float(yy[0]), M


def fitness_gram(gram_state, pop):
    G, b, yy, M = gram_state
    pop = _f64(np.atleast_2d(pop))
    fit = np.zeros(pop.shape[0], dtype=np.float64)
    _check(_load().oracle_fitness_gram(_ptr(G), _ptr(b), yy, M, G.shape[0], _ptr(pop),
                                       pop.shape[0], _ptr(fit)), "fitness_gram")
    return fit


def philox4x32_10(key, ctr):
    """Philox4x32-10 of counters ctr[n][4] under the 64-bit key."""
    ctr = np.ascontiguousarray(np.atleast_2d(ctr), dtype=np.uint32)
    k = np.array([key & 0xFFFFFFFF, (key >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    out = np.zeros_like(ctr)
    lib = _load()
    for n in range(ctr.shape[0]):
        lib.oracle_philox4x32_10(_ptr(k), _ptr(ctr[n]), _ptr(out[n]))
    return out


def init_population(seed, P, K):
    pop = np.zeros((P, K), dtype=np.float32)
    _check(_load().oracle_init_population(seed, P, K, _ptr(pop)), "init_population")
    return pop


def generation(pop, fit, seed, g, prm=None):
    prm = prm or ga_params()
    pop = np.ascontiguousarray(pop, dtype=np.float32)
    fit = _f64(fit)
    P, K = pop.shape
    nxt = np.zeros_like(pop)
    _check(_load().oracle_generation(_ptr(pop), _ptr(fit), P, K, ctypes.byref(prm),
                                     seed, g, _ptr(nxt)), "generation")
    return nxt


def select_best(fit, n):
    """Indices of the n best by (fitness, index), NaN last, best first."""
    fit = _f64(fit)
    idx = np.zeros(n, dtype=np.int32)
    _check(_load().oracle_select_best(_ptr(fit), fit.shape[0], n, _ptr(idx)), "select_best")
    return idx


def rescore(X, y, pop, d, basis, fit, n):
    """fit with its n best entries replaced by their FP64 fitness; returns
    (new fit, candidate indices best first)."""
    X, y, fit = _f64(X), _f64(y), _f64(fit)
    pop = np.ascontiguousarray(pop, dtype=np.float32)
    M, N = X.shape
    P = pop.shape[0]
    out = np.zeros(P, dtype=np.float64)
    idx = np.zeros(n, dtype=np.int32)
    _check(_load().oracle_rescore(_ptr(X), _ptr(y), M, N, d, basis, _ptr(pop), P, _ptr(fit),
                                  n, _ptr(out), _ptr(idx)), "rescore")
    return out, idx


def offspring(pop, fit, seed, g, n_out, prm=None):
    """The generation's operators with n_out output slots (oversampling)."""
    prm = prm or ga_params()
    pop = np.ascontiguousarray(pop, dtype=np.float32)
    fit = _f64(fit)
    P, K = pop.shape
    nxt = np.zeros((n_out, K), dtype=np.float32)
    _check(_load().oracle_offspring(_ptr(pop), _ptr(fit), P, K, ctypes.byref(prm), seed, g,
                                    n_out, _ptr(nxt)), "offspring")
    return nxt


def train(X, y, d, basis, P, G, seed, prm=None, use_gram=False):
    """Whole GA run; returns (pop[P][K] float32, fit[P], best[G+1])."""
    prm = prm or ga_params()
    X, y = _f64(X), _f64(y)
    M, N = X.shape
    K = num_genes(N, d, basis)
    pop = np.zeros((P, K), dtype=np.float32)
    fit = np.zeros(P, dtype=np.float64)
    best = np.zeros(G + 1, dtype=np.float64)
    _check(_load().oracle_train(_ptr(X), _ptr(y), M, N, d, basis, P, ctypes.byref(prm),
                                seed, G, int(use_gram), _ptr(pop), _ptr(fit),
                                _ptr(best)), "train")
    return pop, fit, best


def train_tied(X, y, d, basis, P, G, seed, prm=None):
    """Whole GA run on shared-gene chromosomes (K = B*d + 1)."""
    prm = prm or ga_params()
    X, y = _f64(X), _f64(y)
    M, N = X.shape
    K = num_genes_tied(d, basis)
    pop = np.zeros((P, K), dtype=np.float32)
    fit = np.zeros(P, dtype=np.float64)
    best = np.zeros(G + 1, dtype=np.float64)
    _check(_load().oracle_train_tied(_ptr(X), _ptr(y), M, N, d, basis, P, ctypes.byref(prm),
                                     seed, G, _ptr(pop), _ptr(fit), _ptr(best)), "train_tied")
    return pop, fit, best


def _load_surrogate_copy(path):
    """Tests only: load another copy of surrogate.py as oracle.surrogate."""
    import importlib.util
    import sys
    spec = importlib.util.spec_from_file_location(__name__ + ".surrogate", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    globals()["surrogate"] = mod


if os.environ.get("GAME_ORACLE_SURROGATE_SOURCE"):
    _load_surrogate_copy(os.environ["GAME_ORACLE_SURROGATE_SOURCE"])
