"""Seeded synthetic inputs for GAME workloads.

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests. It holds none of GAME's arithmetic: it draws features and
target coefficients from numpy's Philox-based generator and evaluates the
target polynomials with numpy's own Chebyshev routine
(``numpy.polynomial.chebyshev.chebval``), never with code from either side.

Workloads (the paper's data set, 2100 Globular-Cluster candidates of the
NGC1399 field with 7-11 features, Section 5, is not available; these
synthetic sets stand in for it at its shape and beyond):

* ``small_regression``: M=2000 patterns, N=8 features iid U[-1,1], target an
  additive degree-4 Chebyshev polynomial of the features with U[-1,1]
  coefficients plus N(0, 0.05^2) noise; fitted with Chebyshev degree 4
  (K = 33), P = 64.
* ``large_classification``: M=1,000,000, N=32 correlated Gaussian features
  (x = L z with L = chol(W W^T / N + 0.1 I), W ~ N(0,1)^{NxN}) min-max scaled
  per column to [-1, 1]; target sign(t) of an additive degree-8 Chebyshev
  polynomial t with 5% of the labels flipped (sign(0) = +1); Chebyshev
  degree 8 (K = 257), P = 1024.
* ``batched_runs``: 256 independent problems, M log-uniform in [1e3, 2e5],
  N uniform in {4..64}, basis Chebyshev or trigonometric, degree uniform in
  {2..10}, P log-uniform in [32, 512], regression targets as in the small
  workload.
* ``surrogate_regression``: M=4,000,000, N=48 iid U[-1,1], additive degree-6
  Chebyshev target + N(0, 0.05^2) noise; degree 6 (K = 289), P = 2048.
* ``small_classification``: the shape of the paper's own experiment
  (Section 5: 2100 patterns, 11 columns of which two are the class, so 9
  input features): M=2100, N=9 iid U[-1,1], labels +-1 = sign(t) of an
  additive degree-3 Chebyshev polynomial with 5% flipped; fitted with the
  trigonometric basis and shared genes (Eq. 5), P = B N + 1 = 19 (Eq. 4).

The additive target t = c_0 + sum_i sum_{j=1..D} c_{ij} T_j(x_i) lies in the
span of a Chebyshev chromosome of degree >= D, so with zero noise the
chromosome holding c (in gene order 1 + i*d + j-1) has fitness exactly 0 up
to rounding.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial import chebyshev as npcheb

CHEB, TRIG = 0, 1

# data-stream tags, so that features, coefficients and noise of one seed
# never share a stream
_TAG_X, _TAG_COEF, _TAG_NOISE, _TAG_FLIP, _TAG_MIX, _TAG_RUNS = range(1, 7)


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, tag]))


@dataclass
class Problem:
    """One data set plus the GA settings it is fitted with."""
    name: str
    X: np.ndarray          # [M][N] float32, row-major
    y: np.ndarray          # [M] float32
    degree: int
    basis: int
    P: int
    generations: int
    coef: np.ndarray | None = None   # generating chromosome (float32, K genes)
    extra: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.X.shape[0])

    @property
    def N(self) -> int:
        return int(self.X.shape[1])

    @property
    def K(self) -> int:
        return (2 if self.basis == TRIG else 1) * self.N * self.degree + 1


def additive_chebyshev_target(X: np.ndarray, coef: np.ndarray, D: int) -> np.ndarray:
    """t_m = c_0 + sum_i sum_{j=1..D} c[1 + i*D + j-1] T_j(x_mi), evaluated in
    FP64 by numpy's Chebyshev series routine."""
    X = np.asarray(X, dtype=np.float64)
    c = np.asarray(coef, dtype=np.float64)
    t = np.full(X.shape[0], c[0], dtype=np.float64)
    for i in range(X.shape[1]):
        series = np.concatenate([[0.0], c[1 + i * D: 1 + (i + 1) * D]])
        t += npcheb.chebval(X[:, i], series)
    return t


def regression(seed: int, M: int, N: int, D: int, noise: float, *, degree: int | None = None,
               basis: int = CHEB, P: int = 64, generations: int = 100,
               name: str = "regression") -> Problem:
    """U[-1,1] features, additive degree-D Chebyshev target, Gaussian noise."""
    X = _rng(seed, _TAG_X).uniform(-1.0, 1.0, size=(M, N)).astype(np.float32)
    coef = _rng(seed, _TAG_COEF).uniform(-1.0, 1.0, size=N * D + 1).astype(np.float32)
    t = additive_chebyshev_target(X, coef, D)
    if noise > 0:
        t = t + _rng(seed, _TAG_NOISE).normal(0.0, noise, size=M)
    return Problem(name, X, t.astype(np.float32), degree or D, basis, P, generations,
                   coef=coef, extra={"target_degree": D, "noise": noise,
                                     "target_fp64": t})


def small_regression(seed: int = 1) -> Problem:
    return regression(seed, 2000, 8, 4, 0.05, degree=4, P=64, generations=100,
                      name="M2000_N8_cheb4_P64")


def correlated_features(seed: int, M: int, N: int) -> np.ndarray:
    rng = _rng(seed, _TAG_MIX)
    W = rng.standard_normal((N, N))
    S = W @ W.T / N + 0.1 * np.eye(N)
    L = np.linalg.cholesky(S)
    Z = _rng(seed, _TAG_X).standard_normal((M, N))
    Xr = Z @ L.T
    lo, hi = Xr.min(axis=0), Xr.max(axis=0)
    X = 2.0 * (Xr - lo) / (hi - lo) - 1.0
    return np.clip(X.astype(np.float32), -1.0, 1.0)


def large_classification(seed: int = 2, M: int = 1_000_000) -> Problem:
    N, D = 32, 8
    X = correlated_features(seed, M, N)
    coef = _rng(seed, _TAG_COEF).uniform(-1.0, 1.0, size=N * D + 1).astype(np.float32)
    t = additive_chebyshev_target(X, coef, D)
    lab = np.where(t >= 0.0, 1.0, -1.0)
    flip = _rng(seed, _TAG_FLIP).random(M) < 0.05
    lab[flip] = -lab[flip]
    return Problem(f"M{M}_N32_cheb8_P1024_cls", X, lab.astype(np.float32), 8, CHEB,
                   1024, 200, coef=coef, extra={"flip_rate": 0.05})


def small_classification(seed: int = 5, M: int = 2100, N: int = 9) -> Problem:
    X = _rng(seed, _TAG_X).uniform(-1.0, 1.0, size=(M, N)).astype(np.float32)
    coef = _rng(seed, _TAG_COEF).uniform(-1.0, 1.0, size=N * 3 + 1).astype(np.float32)
    t = additive_chebyshev_target(X, coef, 3)
    lab = np.where(t >= 0.0, 1.0, -1.0)
    flip = _rng(seed, _TAG_FLIP).random(M) < 0.05
    lab[flip] = -lab[flip]
    return Problem(f"M{M}_N{N}_gc_shape_cls", X, lab.astype(np.float32), 8, TRIG, 2 * N + 1,
                   40000, coef=None, extra={"flip_rate": 0.05, "target_degree": 3})


def surrogate_regression(seed: int = 4, M: int = 4_000_000) -> Problem:
    return regression(seed, M, 48, 6, 0.05, degree=6, P=2048, generations=300,
                      name=f"M{M}_N48_cheb6_P2048")


def batched_runs(seed: int = 3, R: int = 256, m_range=(1_000, 200_000),
                 n_range=(4, 64), d_range=(2, 10), p_range=(32, 512)) -> list[Problem]:
    """R independent problems of uneven shape (log-uniform M and P)."""
    rng = _rng(seed, _TAG_RUNS)
    runs = []
    for r in range(R):
        M = int(round(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1])))))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        basis = int(rng.integers(0, 2))
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        P = int(round(np.exp(rng.uniform(np.log(p_range[0]), np.log(p_range[1])))))
        pr = regression(seed * 100_003 + r + 1, M, N, 4, 0.05, degree=d, basis=basis,
                        P=P, generations=100, name=f"run{r}")
        runs.append(pr)
    return runs


def random_population(seed: int, P: int, K: int, scale: float = 1.0) -> np.ndarray:
    """Test populations: genes U[-scale, scale] as float32."""
    return _rng(seed, 99).uniform(-scale, scale, size=(P, K)).astype(np.float32)
