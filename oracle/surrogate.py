"""FP64 oracle of the fitness surrogate: a K -> H -> H -> 1 MLP with GELU (tanh
form), trained by Adam on (chromosome, log fitness) pairs, and the screening
of oversampled offspring by its predictions.

TEST INFRASTRUCTURE (see the package docstring): plain numpy, no code shared
with the CUDA path. The surrogate is not part of the paper; it serves the
paper's GA (Section 3) by deciding which offspring get the exact fitness of
Eq. 3.

Definitions (the same as the CUDA path, written from them):
  * parameters, FP32, in this order: W1 [H][K], b1 [H], W2 [H][H], b2 [H],
    w3 [H], b3 [1];
  * initial weights: u * a with u = (r >> 8) 2^-23 - 1, r the first word of
    Philox4x32-10 under the seed with counter (layer, index, 0, 9), a =
    1 / sqrt(fan_in) in FP32; biases 0;
  * forward, with BF16 rounding (round to nearest even) of the inputs, of W1,
    W2 and of the first hidden activations:
      Z1 = bf(x) bf(W1)^T + b1, H1 = bf(g(Z1)), Z2 = H1 bf(W2)^T + b2,
      H2 = g(Z2), out = H2 . w3 + b3,
    g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
  * target: l = log(max(fit, 1e-30)) standardised over the batch,
    t = (l - mean l) / sd l (sd 0 counts as 1);
  * loss = mean over the batch of (out - t)^2; gradients pass the rounding
    points unchanged;
  * Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
  * screening: of n children keep the n_keep with the smallest prediction,
    ties by slot, predictions ordered as IEEE-754 total order (NaN last) --
    or, when the surrogate is not trusted, the first n_keep children; the
    next population is the elites followed by the kept children in slot order;
  * trust check: the Pearson correlation r of the kept children's predictions with
    their exact log-fitness; the next screening trusts the surrogate iff
    r > 0.25.
"""
from __future__ import annotations

import numpy as np

from . import philox4x32_10

H_DEFAULT = 256
TAG_SURROGATE = 9
GELU_C = np.sqrt(2.0 / np.pi)
GELU_A = 0.044715
LR, B1, B2, EPS = 1e-3, 0.9, 0.999, 1e-8


def param_count(K, H=H_DEFAULT):
    return H * K + H + H * H + H + H + 1


def unpack(w, K, H=H_DEFAULT):
    w = np.asarray(w)
    o = 0
    out = {}
    for name, shape in (("W1", (H, K)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("w3", (H,)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.ravel(p[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def init_params(seed, K, H=H_DEFAULT):
    """The initial FP32 parameters (bit-exact with the CUDA path)."""
    def layer(idx_layer, n, fan_in):
        ctr = np.zeros((n, 4), dtype=np.uint32)
        ctr[:, 0] = idx_layer
        ctr[:, 1] = np.arange(n, dtype=np.uint32)
        ctr[:, 3] = TAG_SURROGATE
        r = philox4x32_10(seed, ctr)[:, 0]
        u = (r >> 8).astype(np.float32) * np.float32(1.0 / 8388608.0) - np.float32(1.0)
        a = np.float32(1.0) / np.sqrt(np.float32(fan_in))
        return (u * a).astype(np.float32)
    p = {"W1": layer(1, H * K, K).reshape(H, K), "b1": np.zeros(H, np.float32),
         "W2": layer(2, H * H, H).reshape(H, H), "b2": np.zeros(H, np.float32),
         "w3": layer(3, H, H), "b3": np.zeros(1, np.float32)}
    return pack(p).astype(np.float32)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def _round(x, on):
    return bf16(x) if on else np.asarray(x, dtype=np.float64)


def forward(w, X, K, H=H_DEFAULT, rounding=True):
    p = {k: v.astype(np.float64) for k, v in unpack(w, K, H).items()}
    Xb = _round(X, rounding)
    W1b, W2b = _round(p["W1"], rounding), _round(p["W2"], rounding)
    Z1 = Xb @ W1b.T + p["b1"]
    H1 = _round(gelu(Z1), rounding)
    Z2 = H1 @ W2b.T + p["b2"]
    H2 = gelu(Z2)
    out = H2 @ p["w3"] + p["b3"][0]
    return out, {"Xb": Xb, "W1b": W1b, "W2b": W2b, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "p": p}


def targets(fit):
    l = np.log(np.maximum(np.asarray(fit, dtype=np.float64), 1e-30))
    mu = l.mean()
    sd = np.sqrt(np.mean((l - mu) ** 2))
    return (l - mu) / (sd if sd > 0 else 1.0)


def loss_and_grad(w, X, fit, K, H=H_DEFAULT, rounding=True):
    out, c = forward(w, X, K, H, rounding)
    B = out.shape[0]
    r = out - targets(fit)
    loss = np.mean(r * r)
    d_out = 2.0 * r / B
    g = {"w3": c["H2"].T @ d_out, "b3": np.array([d_out.sum()])}
    dZ2 = np.outer(d_out, c["p"]["w3"]) * gelu_grad(c["Z2"])
    g["W2"] = dZ2.T @ c["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ c["W2b"]) * gelu_grad(c["Z1"])
    g["W1"] = dZ1.T @ c["Xb"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, pack(g)


def adam(w, g, m, v, t):
    """One Adam step (t = step number after this step, from 1)."""
    w, g, m, v = (np.asarray(a, dtype=np.float64) for a in (w, g, m, v))
    m = B1 * m + (1 - B1) * g
    v = B2 * v + (1 - B2) * g * g
    mh = m / (1 - B1 ** t)
    vh = v / (1 - B2 ** t)
    return w - LR * mh / (np.sqrt(vh) + EPS), m, v


def forward_bound(w, X, K, H=H_DEFAULT):
    """Bound on |out_device - out_oracle| per row: the two sides round the
    same BF16 operands; they differ by FP32 accumulation (K u32 of the
    absolute sums per layer), FP32 GELU (a few ulp), and a possible one-ulp
    BF16 flip of H1 where the FP32 and FP64 values straddle a rounding
    boundary (u |H1|), propagated with |g'| <= 1.13."""
    u32, ub = 2.0 ** -24, 2.0 ** -8
    out, c = forward(w, X, K, H)
    A1 = np.abs(c["Xb"]) @ np.abs(c["W1b"]).T + np.abs(c["p"]["b1"])
    dZ1 = (K + 2) * u32 * A1
    dH1 = 1.13 * dZ1 + ub * np.abs(c["H1"]) + 8 * u32 * (np.abs(c["H1"]) + 1e-30)
    A2 = np.abs(c["H1"]) @ np.abs(c["W2b"]).T + np.abs(c["p"]["b2"])
    dZ2 = dH1 @ np.abs(c["W2b"]).T + (H + 2) * u32 * A2
    dH2 = 1.13 * dZ2 + 8 * u32 * np.abs(c["H2"])
    A3 = np.abs(c["H2"]) @ np.abs(c["p"]["w3"]) + abs(c["p"]["b3"][0])
    return dH2 @ np.abs(c["p"]["w3"]) + (H + 2) * u32 * A3


def total_order_key(pred):
    """IEEE-754 total order of FP32 values as unsigned keys (NaN as +inf)."""
    p = np.asarray(pred, dtype=np.float32).copy()
    p[np.isnan(p)] = np.inf
    u = p.view(np.uint32).astype(np.uint64)
    neg = (u & 0x80000000) != 0
    return np.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000)


def select_keep(pred, n_keep, trusted=True):
    """Flags of the n_keep children with the smallest predictions (ties by
    slot); the first n_keep children when the surrogate is not trusted."""
    if not trusted:
        keep = np.zeros(len(pred), dtype=np.int32)
        keep[:n_keep] = 1
        return keep
    key = total_order_key(pred)
    order = np.lexsort((np.arange(key.shape[0]), key))
    keep = np.zeros(key.shape[0], dtype=np.int32)
    keep[order[:n_keep]] = 1
    return keep


def screen(offspring, keep, E):
    """Elites (rows 0..E-1) then the kept children (rows E + i) in slot order."""
    off = np.asarray(offspring)
    kept = off[E:][np.asarray(keep).astype(bool)]
    return np.concatenate([off[:E], kept], axis=0)


def trust_check(pred, keep, fit_kept):
    """(r, trusted): Pearson correlation of the kept children's predictions
    with their exact log-fitness (fit_kept in slot order), and r > 0.25."""
    x = np.asarray(pred, dtype=np.float64)[np.asarray(keep).astype(bool)]
    y = np.log(np.maximum(np.asarray(fit_kept, dtype=np.float64), 1e-30))
    if x.shape[0] < 2 or x.std() == 0 or y.std() == 0:
        return 0.0, False
    r = float(np.corrcoef(x, y)[0, 1])
    return r, r > 0.25
