"""CPU model of the reduced-precision fitness forms, for element-by-element
parity of the tensor-core kernels.

Each form rounds its operands in a fixed way before the contraction: the
expansion values phi (FP32 recurrences, Section 3 Eq. 1 / Eq. 6) and the
genes are rounded to BF16, split into BF16 hi + lo, or scaled and quantised
to FP8 E4M3. This module applies the same roundings on the CPU and then
forms every output exactly (FP64 sums of the rounded operands' products,
which are exact), so that what is left between it and a kernel is

  * the FP32 accumulation of the K' products in tensor memory (any order),
  * the FP32 residual, square and per-tile sum of the epilogue, and
  * operand values whose rounding is ambiguous: the kernel's FP32 expansion
    values are reproduced bit for bit for the Chebyshev basis (the same
    fused multiply-add recurrence), but only to within a few FP32 ulps for
    the trigonometric basis (sincosf is not correctly rounded); where such
    a value lies that close to a BF16 or E4M3 rounding boundary, either
    neighbour is accepted.

`tolerance` turns these three into a per-chromosome bound on the fitness
difference. The FP64 oracle stays the reference of what the method computes;
this model states what each reduced-precision form computes.
"""
import numpy as np

from helpers import CHEB

U32 = 2.0 ** -24


# ---- rounding of FP32 values ----

def bf16(x):
    """Round FP32 values to BF16 (round to nearest, ties to even)."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def bf16_gap(x):
    """Spacing of BF16 values at |x| (8 significant bits)."""
    a = np.maximum(np.abs(np.asarray(x, dtype=np.float64)), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def e4m3(x):
    """Round to the nearest E4M3 value (3 fraction bits, subnormal quantum
    2^-9), ties to even, saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.maximum(np.floor(np.log2(np.maximum(a, 2.0 ** -9))), -6)
    q = 2.0 ** (e - 3)
    return (np.sign(x) * np.minimum(np.round(a / q) * q, 448.0)).astype(np.float32)


def e4m3_gap(x):
    """Spacing of E4M3 values at |x| (normal range from 2^-6, quantum 2^-9
    below)."""
    a = np.abs(np.asarray(x, dtype=np.float64))
    e = np.maximum(np.floor(np.log2(np.maximum(a, 2.0 ** -9))), -6)
    return 2.0 ** (e - 3)


def ambiguous(v, w, rnd):
    """True where the interval [v - w, v + w] rounds (by `rnd`) to more than
    one value, i.e. holds a rounding boundary."""
    v = np.asarray(v, dtype=np.float64)
    lo = rnd((v - w).astype(np.float32)).astype(np.float64)
    hi = rnd((v + w).astype(np.float32)).astype(np.float64)
    mid = rnd(v.astype(np.float32)).astype(np.float64)
    return (lo != mid) | (hi != mid)


# ---- the kernels' FP32 expansion ----

def _fma32(a, b, c):
    """fmaf(a, b, c) for FP32 arrays: the product of two FP32 values is exact
    in FP64 and the sum rounds there before the final rounding to FP32 (a
    double rounding that differs from one rounding only when the FP64 value
    sits on an FP32 midpoint, which the ambiguity width covers)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def expansion_fp32(X, d, basis):
    """phi [M][K'] as the kernels compute it in FP32, and a bound delta
    [M][K'] on |kernel value - this value|.

    Chebyshev: T_0 = 1, T_1 = x, T_{j+1} = fma(2x, T_j, -T_{j-1}) in FP32,
    reproduced exactly (delta: two FP32 ulps for the double rounding above).
    Trigonometric: cos(jx), sin(jx) by f_{j+1} = fma(2c, f_j, -f_{j-1}) from
    c = cos x, s = sin x rounded to FP32. The kernels' sincosf is within 2.5
    FP32 ulps of those; a perturbation of the start values and the two
    sides' different roundings (each at most 3.5 * 2^-23 per step) grow
    through the recurrence by at most the Chebyshev U polynomials (|U_j| <=
    j + 1), so delta_j = ((j + 1)(j + 2) * 2 + (j + 1)) * 2^-23."""
    X = np.asarray(X, dtype=np.float32)
    M, N = X.shape
    cols, dels = [], []
    for i in range(N):
        x = X[:, i]
        if basis == CHEB:
            x2 = (x + x).astype(np.float32)
            tm, t = np.ones(M, dtype=np.float32), x.copy()
            for j in range(1, d + 1):
                cols.append(t)
                dels.append(2.0 * U32 * 2 * np.maximum(np.abs(t.astype(np.float64)), 2.0 ** -100))
                tm, t = t, _fma32(x2, t, -tm)
        else:
            xd = x.astype(np.float64)
            c1 = np.cos(xd).astype(np.float32)
            s1 = np.sin(xd).astype(np.float32)
            c2 = (c1 + c1).astype(np.float32)
            for f_m, f in ((np.ones(M, dtype=np.float32), c1), (np.zeros(M, dtype=np.float32), s1)):
                for j in range(1, d + 1):
                    cols.append(f)
                    dels.append(np.full(M, ((j + 1) * (j + 2) * 2 + (j + 1)) * 2.0 ** -23))
                    f_m, f = f, _fma32(c2, f, -f_m)
    return np.stack(cols, axis=1), np.stack(dels, axis=1)


# ---- the three forms ----

def _gene_rows(pop):
    pop = np.asarray(pop, dtype=np.float32)
    return pop[:, 0], pop[:, 1:]


def bf16_operands(X, pop, d, basis):
    """Rounded operands of the BF16 form and the per-output allowance for
    ambiguous roundings: returns (a0, A~ [P][K'], Phi~ [M][K'],
    amb [M][K'] = BF16 spacing where phi's rounding is ambiguous, else 0)."""
    phi, delta = expansion_fp32(X, d, basis)
    a0, A = _gene_rows(pop)
    amb = np.where(ambiguous(phi, delta, bf16), bf16_gap(phi), 0.0)
    return a0, bf16(A).astype(np.float64), bf16(phi).astype(np.float64), amb


def model(form, X, y, pop, d, basis, error="mse"):
    """Fitness of every chromosome under the form's operand roundings, with
    exact products and sums, and the per-chromosome tolerance of a kernel
    around it (see `tolerance`). error: "mse", "rmse" or "mae" (mean
    absolute residual). Returns (fit [P], tol [P])."""
    y = np.asarray(y, dtype=np.float32)
    a0, A = _gene_rows(pop)
    phi, delta = expansion_fp32(X, d, basis)
    Kp = phi.shape[1]
    if form == "bf16":
        Ar, Pr = bf16(A).astype(np.float64), bf16(phi).astype(np.float64)
        D = Pr @ Ar.T
        S = np.abs(Pr) @ np.abs(Ar).T
        amb = np.where(ambiguous(phi, delta, bf16), bf16_gap(phi), 0.0)
        dD = 2 * Kp * U32 * S + amb @ np.abs(Ar).T
        u = np.ones(len(a0))
    elif form == "bf16x3":
        ah = bf16(A)
        al = bf16((A - ah).astype(np.float32))
        ph = bf16(phi)
        pl = bf16((phi - ph).astype(np.float32))
        ah, al, ph, pl = (v.astype(np.float64) for v in (ah, al, ph, pl))
        D = ph @ ah.T + ph @ al.T + pl @ ah.T
        S = np.abs(ph) @ np.abs(ah).T + np.abs(ph) @ np.abs(al).T + np.abs(pl) @ np.abs(ah).T
        # the kernel's phi differs by at most delta; where hi's rounding is
        # ambiguous, hi + lo still equals phi up to lo's rounding (lo's
        # spacing, at most 2^-8 of hi's); where lo's is, by lo's spacing
        lo_v = (phi - bf16(phi)).astype(np.float32)
        amb = delta + np.where(ambiguous(phi, delta, bf16), bf16_gap(phi) * 2.0 ** -7, 0.0) \
            + np.where(ambiguous(lo_v, delta, bf16), bf16_gap(lo_v), 0.0)
        dD = 3 * 2 * Kp * U32 * S + amb @ (np.abs(ah) + np.abs(al)).T
        u = np.ones(len(a0))
    elif form == "fp8":
        # column scales from the FP32 expansion's column maxima (computed
        # over the same values), gene scales per chromosome
        mx = np.abs(phi).max(axis=0).astype(np.float32)
        colscale = (mx.astype(np.float64) / 448.0).astype(np.float32)
        with np.errstate(divide="ignore"):
            colinv = np.where(mx > 0, (448.0 / mx.astype(np.float64)), 0.0).astype(np.float32)
        gs = (A.astype(np.float64) * colscale.astype(np.float64)).astype(np.float32)
        mg = np.abs(gs).max(axis=1).astype(np.float64)
        u = np.where(mg > 0, (mg / 448.0).astype(np.float32), 1.0).astype(np.float32)
        g = (gs.astype(np.float64) / u.astype(np.float64)[:, None]).astype(np.float32)
        ps = (phi.astype(np.float64) * colinv.astype(np.float64)).astype(np.float32)
        A8, P8 = e4m3(g).astype(np.float64), e4m3(ps).astype(np.float64)
        D = P8 @ A8.T
        S = np.abs(P8) @ np.abs(A8).T
        # the trigonometric expansion's column maxima, and with them every
        # scale, are known to within delta / max (relative): widen the
        # scaled values' intervals by that, and the genes' likewise
        rho = np.where(mx > 0, delta.max(axis=0) / np.maximum(mx.astype(np.float64), 1e-30), 0.0)
        rho = rho if basis != CHEB else np.zeros_like(rho)
        w_phi = delta * colinv.astype(np.float64) + np.abs(ps) * (2 * rho + 2 * U32)
        amb_phi = np.where(ambiguous(ps, w_phi, e4m3), e4m3_gap(ps), 0.0)
        rg = 4 * rho.max() + 4 * U32 if basis != CHEB else 2 * U32
        w_g = np.abs(g.astype(np.float64)) * rg
        amb_g = np.where(ambiguous(g, w_g, e4m3), e4m3_gap(g), 0.0)
        dD = 2 * Kp * U32 * S + amb_phi @ np.abs(A8).T + np.abs(P8) @ amb_g.T + \
            (4 * rho.max() if basis != CHEB else 0.0) * S
        u = u.astype(np.float64)
    else:
        raise ValueError(form)
    ya = (y[:, None].astype(np.float32) - a0[None, :].astype(np.float32)).astype(np.float32)
    r = ya.astype(np.float64) - u[None, :] * D
    dOut = u[None, :] * dD
    if error == "mae":
        # |mean |r'| - mean |r|| <= mean |dOut|, plus the epilogue's FP32 sums
        fit = np.mean(np.abs(r), axis=0)
        yv = np.asarray(y, dtype=np.float64)
        return fit, np.mean(dOut, axis=0) + 1e-5 * fit + 1e-7 * np.sqrt(np.mean(yv * yv))
    fit = np.mean(r * r, axis=0)
    tol = tolerance(fit, dOut, y)
    if error == "rmse":
        # |sqrt(a) - sqrt(b)| <= |a - b| / sqrt(b)
        return np.sqrt(fit), tol / np.sqrt(fit)
    return fit, tol


def tolerance(fit, dOut, y):
    """Bound on |kernel fitness - model fitness| when every output Out_pm
    differs by at most dOut[m][p]: |df| <= 2 sqrt(f) sqrt(mean dOut^2) +
    mean dOut^2, plus the epilogue's FP32 residual, square and per-tile sums
    (at most 1e-5 of the fitness, as for the FP32 form) and the FP32 form's
    floor 1e-7 mean(y^2)."""
    ms = np.mean(dOut * dOut, axis=0)
    y = np.asarray(y, dtype=np.float64)
    return 2 * np.sqrt(fit) * np.sqrt(ms) + ms + 1e-5 * fit + 1e-7 * np.mean(y * y)
