"""Test-side helpers: an independent numpy design matrix (numpy's chebvander
and np.cos/np.sin, gene order 1 + i*B*d + b*d + j-1) and the tolerances of
the parity tests."""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

CHEB, TRIG = 0, 1
U_BF16 = 2.0 ** -8   # unit roundoff of bfloat16 (8 significant bits)
U_FP32 = 2.0 ** -24


def design_matrix(X, d, basis, dtype=np.float64):
    X = np.asarray(X, dtype=np.float64)
    cols = [np.ones(X.shape[0])]
    for i in range(X.shape[1]):
        if basis == CHEB:
            cols.extend(npcheb.chebvander(X[:, i], d)[:, 1:].T)
        else:
            cols.extend(np.cos(j * X[:, i]) for j in range(1, d + 1))
            cols.extend(np.sin(j * X[:, i]) for j in range(1, d + 1))
    return np.stack(cols, axis=1).astype(dtype)


def fp32_tol(f_oracle, y):
    """|f - f_oracle| <= 1e-5 |f_oracle| + 1e-7 mean(y^2): relative error of
    the FP32 form, with an absolute floor for fitness near zero."""
    y = np.asarray(y, dtype=np.float64)
    return 1e-5 * np.abs(f_oracle) + 1e-7 * np.mean(y * y)


def abs_weighted_sum(X, pop, d, basis, chunk=65536):
    """S[p][m] = sum_k |a_pk phi_k(x_m)| without the bias, returned as the
    per-chromosome mean of S^2 (for the BF16 bound)."""
    pop = np.abs(np.asarray(pop, dtype=np.float64))[:, 1:]
    acc = np.zeros(pop.shape[0])
    M = X.shape[0]
    for m0 in range(0, M, chunk):
        Phi = np.abs(design_matrix(X[m0:m0 + chunk], d, basis)[:, 1:])
        S = Phi @ pop.T
        acc += (S * S).sum(axis=0)
    return acc / M


def bf16_bound(f_oracle, X, pop, d, basis):
    """Worst-case fitness error of a BF16 x BF16 -> FP32 contraction: each
    product a_k phi_k carries a relative error <= 2u + u^2 (both operands
    rounded, u = 2^-8), plus FP32 accumulation (K u_32 of the same sum), so
    |dOut_m| <= e S_m with e = 2u + u^2 + K u_32, and
    |df| <= 2 sqrt(f) sqrt(mean dOut^2) + mean dOut^2."""
    K = np.asarray(pop).shape[1]
    e = 2 * U_BF16 + U_BF16 ** 2 + K * U_FP32
    ms = abs_weighted_sum(X, pop, d, basis) * e * e
    return 2 * np.sqrt(np.asarray(f_oracle)) * np.sqrt(ms) + ms
