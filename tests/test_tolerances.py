"""The parity tolerances of the reduced-precision forms (tests/helpers.py)
are sound bounds of the arithmetic they describe: an emulation of each form
(operands rounded to BF16, split into BF16 hi + lo, or quantised to FP8
E4M3 with the column and chromosome scales; products summed in FP32, the
residual squared in FP32 and the sum over patterns in FP64) never leaves
its bound around the FP64 oracle. The bounds are worst-case (every
rounding error aligned, over the K products of an output and over the M
patterns of a fitness), so they sit 300 to 6000 times above the errors the
emulation shows; the test also holds them under 10^4 times, so that a
change making them vacuous fails here."""
import numpy as np
import pytest

from emulation import bf16, e4m3
from helpers import CHEB, TRIG, bf16_bound, bf16x3_bound, design_matrix, fp8_bound
from paper_1211_5481_gb300 import datagen as dg


def fitness_from_products(y, a0, D):
    """Residual and square in FP32, sum over patterns in FP64, as the
    epilogue and the reduce do."""
    r = (y.astype(np.float32)[:, None] - a0.astype(np.float32)[None, :]) - D.astype(np.float32)
    return np.mean((r * r).astype(np.float64), axis=0)


def emulate(form, X, y, pop, d, basis):
    Phi = design_matrix(X, d, basis)[:, 1:].astype(np.float32)
    A = pop[:, 1:].astype(np.float32)
    if form == "bf16":
        D = bf16(Phi) @ bf16(A).T
    elif form == "bf16x3":
        ph, ah = bf16(Phi), bf16(A)
        pl, al = bf16(Phi - ph), bf16(A - ah)
        D = ph @ ah.T + ph @ al.T + pl @ ah.T
    else:
        s = np.abs(Phi).max(axis=0).astype(np.float64) / 448.0
        s[s == 0] = 1.0
        As = A.astype(np.float64) * s
        u = np.abs(As).max(axis=1) / 448.0
        u[u == 0] = 1.0
        D = (e4m3(Phi / s) @ e4m3(As / u[:, None]).T) * u[None, :].astype(np.float32)
    return fitness_from_products(y, pop[:, 0], D)


CASES = [(1500, 8, 4, CHEB, 0.05), (800, 3, 7, TRIG, 0.05), (2000, 32, 8, CHEB, 0.05),
         (1200, 16, 3, TRIG, 0.0)]
BOUNDS = {"bf16": bf16_bound, "bf16x3": bf16x3_bound, "fp8": fp8_bound}


@pytest.mark.parametrize("form", ["bf16", "bf16x3", "fp8"])
@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
def test_emulated_form_stays_within_its_bound(orc, form, case):
    M, N, d, basis, noise = case
    pr = dg.regression(M + d, M, N, min(d, 3), noise, degree=d, basis=basis)
    pops = [dg.random_population(3, 24, pr.K)]
    if basis == CHEB:
        # near the generating chromosome: small fitness, where cancellation is worst
        near = np.zeros((8, pr.K), dtype=np.float32)
        c = np.zeros(pr.K)
        c[0] = pr.coef[0]
        for i in range(N):
            D = min(d, 3)
            c[1 + i * d: 1 + i * d + D] = pr.coef[1 + i * D: 1 + (i + 1) * D]
        near[:] = c + dg.random_population(5, 8, pr.K, scale=1e-3)
        pops.append(near)
    for pop in pops:
        ref = orc.fitness(pr.X, pr.y, pop, d, basis)
        got = emulate(form, pr.X, pr.y, pop, d, basis)
        bound = BOUNDS[form](ref, pr.X, pop, d, basis)
        err = np.abs(got - ref)
        assert np.all(err <= bound), (form, float(np.max(err / bound)))
        assert np.max(bound) < 1e4 * max(np.max(err), 1e-300) or np.max(err) == 0
