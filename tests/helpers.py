"""Test-side helpers: an independent numpy design matrix (numpy's chebvander
and np.cos/np.sin, gene order 1 + i*B*d + b*d + j-1) and the tolerances of
the parity tests."""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

CHEB, TRIG = 0, 1
U_BF16 = 2.0 ** -8   # unit roundoff of bfloat16 (8 significant bits)
U_FP32 = 2.0 ** -24
U_E4M3 = 2.0 ** -4   # unit roundoff of FP8 E4M3 (4 significant bits)
U64 = 2.0 ** -53


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


def abs_weighted_sum(X, pop, d, basis, chunk=65536, with_mean=False):
    """S[p][m] = sum_k |a_pk phi_k(x_m)| without the bias, returned as the
    per-chromosome mean of S^2 (and of S)."""
    pop = np.abs(np.asarray(pop, dtype=np.float64))[:, 1:]
    acc = np.zeros(pop.shape[0])
    acc1 = np.zeros(pop.shape[0])
    M = X.shape[0]
    for m0 in range(0, M, chunk):
        Phi = np.abs(design_matrix(X[m0:m0 + chunk], d, basis)[:, 1:])
        S = Phi @ pop.T
        acc += (S * S).sum(axis=0)
        acc1 += S.sum(axis=0)
    return (acc / M, acc1 / M) if with_mean else acc / M


def out_error_bound(f_oracle, X, pop, d, basis, e, c=0.0):
    """Fitness error when every output carries |dOut_m| <= e S_m + c:
    |df| <= 2 sqrt(f) sqrt(mean dOut^2) + mean dOut^2, with
    mean dOut^2 <= e^2 mean(S^2) + 2 e c mean(S) + c^2."""
    s2, s1 = abs_weighted_sum(X, pop, d, basis, with_mean=True)
    ms = e * e * s2 + 2 * e * c * s1 + c * c
    return 2 * np.sqrt(np.asarray(f_oracle)) * np.sqrt(ms) + ms


def bf16x3_bound(f_oracle, X, pop, d, basis):
    """Split products: x = hi + lo + r with hi = bf16(x), lo = bf16(x - hi),
    |lo| <= u|x|, |r| <= u^2 |x|; the three products hi*hi + hi*lo + lo*hi
    miss lo*lo and the r terms, |a phi - computed| <= 3 u^2 |a phi| (+ u^3
    terms, covered by the factor 4), plus FP32 accumulation K u_32."""
    K = np.asarray(pop).shape[1]
    e = 4 * U_BF16 ** 2 + K * U_FP32
    return out_error_bound(f_oracle, X, pop, d, basis, e)


def fp8_bound(f_oracle, X, pop, d, basis):
    """FP8 E4M3 operands after scaling into [-448, 448]: relative rounding
    2u + u^2 per product (u = 2^-4) in the normal range; below E4M3's
    smallest normal (2^-6) the absolute error is at most 2^-10 in scaled
    units, i.e. <= 2^-10 * 448 * u_p per product term in output units, with
    u_p <= max|a| max|phi| / 448^2 (the per-chromosome gene scale), summed
    over K terms; plus FP32 accumulation."""
    pop = np.asarray(pop, dtype=np.float64)
    K = pop.shape[1]
    e = 2 * U_E4M3 + U_E4M3 ** 2 + K * U_FP32
    up = np.abs(pop[:, 1:]).max(axis=1) / 448.0 ** 2
    c = K * 2 * 2.0 ** -10 * 448 * up
    return out_error_bound(f_oracle, X, pop, d, basis, e, c)


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


def quad_bound(G, b, yy, pop, M):
    """|fit - fit_exact| <= c u (y.y + 2 |a|.|b| + |a|^T |G| |a|) / M with
    c = 4 (K + 8): each of the three sums carries at most K + 8 roundings
    of its own magnitude in FP64, plus the rounding of G and b themselves
    (their accumulation over the patterns, bounded the same way relative to
    the absolute sums, which |G| and |b| dominate)."""
    A = np.abs(np.asarray(pop, dtype=np.float64))
    K = A.shape[1]
    mag = yy + 2 * A @ np.abs(b) + np.einsum("pk,kl,pl->p", A, np.abs(G), A)
    return 4 * (K + 8) * U64 * mag / M + 1e-300
