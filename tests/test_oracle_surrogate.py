"""Pins of the surrogate oracle: gradients against central finite
differences, GELU against its derivative and the erf form, Adam's first step
against its closed form, the initial weights' range, and the screening
selection against brute-force sorting."""
import math

import numpy as np
import pytest

from oracle import surrogate as sg


def test_gelu_derivative_and_erf_form():
    z = np.linspace(-6, 6, 1001)
    h = 1e-6
    num = (sg.gelu(z + h) - sg.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(sg.gelu_grad(z), num, rtol=1e-6, atol=1e-8)
    erf_form = np.array([0.5 * t * (1 + math.erf(t / math.sqrt(2))) for t in z])
    assert np.max(np.abs(sg.gelu(z) - erf_form)) < 1e-3   # the tanh form's known accuracy


@pytest.mark.parametrize("K,H,B", [(3, 4, 5), (7, 6, 9)])
def test_gradient_matches_finite_differences(orc, K, H, B):
    rng = np.random.default_rng(K * 10 + H)
    w = rng.normal(0, 0.5, sg.param_count(K, H))
    X = rng.uniform(-1, 1, (B, K))
    fit = np.exp(rng.normal(0, 1, B))
    loss, g = sg.loss_and_grad(w, X, fit, K, H, rounding=False)
    num = np.zeros_like(w)
    h = 1e-6
    for i in range(w.shape[0]):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        num[i] = (sg.loss_and_grad(wp, X, fit, K, H, False)[0]
                  - sg.loss_and_grad(wm, X, fit, K, H, False)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_adam_first_step_closed_form():
    g = np.array([1.0, -2.0, 1e-3, -5.0])
    w0 = np.zeros(4)
    w1, m, v = sg.adam(w0, g, np.zeros(4), np.zeros(4), 1)
    # t = 1: m_hat = g, v_hat = g^2, so the step is lr g / (|g| + eps)
    np.testing.assert_allclose(w1, -sg.LR * g / (np.abs(g) + sg.EPS), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_init_range_and_determinism(orc):
    K = 33
    w = sg.init_params(7, K)
    p = sg.unpack(w, K)
    a1, a2 = 1 / np.sqrt(np.float32(K)), 1 / np.sqrt(np.float32(256))
    assert w.dtype == np.float32 and w.shape[0] == sg.param_count(K)
    assert np.all(np.abs(p["W1"]) <= a1) and np.all(np.abs(p["W2"]) <= a2)
    assert np.all(p["b1"] == 0) and np.all(p["b2"] == 0) and p["b3"][0] == 0
    assert abs(p["W1"].mean()) < 0.02 * a1 and abs(p["W2"].std() - a2 / np.sqrt(3)) < 0.01 * a2
    np.testing.assert_array_equal(w, sg.init_params(7, K))
    assert not np.array_equal(w, sg.init_params(8, K))


def test_select_keep_brute_force():
    rng = np.random.default_rng(3)
    pred = rng.choice([0.5, -1.0, 2.0, 0.0], 40).astype(np.float32)
    pred[[3, 17]] = np.nan
    pred[5] = -0.0
    for n_keep in (1, 7, 20, 40):
        keep = sg.select_keep(pred, n_keep)
        key = [(math.inf if math.isnan(p) else float(p), math.copysign(1, p) > 0, i)
               for i, p in enumerate(pred)]
        want = sorted(range(40), key=lambda i: key[i])[:n_keep]
        assert set(np.nonzero(keep)[0]) == set(want)


def test_screen_keeps_slot_order():
    off = np.arange(12, dtype=np.float32).reshape(6, 2)
    keep = np.array([0, 1, 0, 1], dtype=np.int32)
    nxt = sg.screen(off, keep, 2)
    np.testing.assert_array_equal(nxt, off[[0, 1, 3, 5]])


def test_standardised_targets_and_trust_check():
    fit = np.array([1.0, np.e, np.e ** 2, np.e ** 3])
    t = sg.targets(fit)
    np.testing.assert_allclose(t, (np.arange(4) - 1.5) / np.sqrt(1.25), rtol=1e-12)
    np.testing.assert_allclose(sg.targets(np.full(5, 3.0)), 0.0)   # sd 0 counts as 1
    pred = np.array([0.1, 5.0, 0.2, 0.3], dtype=np.float32)
    keep = np.array([1, 0, 1, 1])
    r, ok = sg.trust_check(pred, keep, np.exp([1.0, 2.0, 3.0]))
    assert abs(r - 1.0) < 1e-12 and ok
    r, ok = sg.trust_check(pred, keep, np.exp([3.0, 2.0, 1.0]))
    assert abs(r + 1.0) < 1e-12 and not ok
    np.testing.assert_array_equal(sg.select_keep(pred, 2, trusted=False), [1, 1, 0, 0])


def test_trust_threshold_on_hand_computed_correlations():
    """Pearson r by hand: predictions 1..6 against log-fitness
    (1, 2, 2, 1, 1, 2) give sum dx dy = 0.5, sum dx^2 = 17.5, sum dy^2 = 1.5,
    r = 0.5 / sqrt(26.25) = 0.0976: positive but below 0.25, untrusted.
    Predictions 1..4 against (1, 1, 3, 1) give r = 1 / sqrt(15) = 0.258,
    just above 0.25: trusted."""
    r, ok = sg.trust_check(np.arange(1.0, 7.0), np.ones(6), np.exp([1.0, 2, 2, 1, 1, 2]))
    assert r == pytest.approx(0.5 / math.sqrt(26.25), rel=1e-12) and not ok
    r, ok = sg.trust_check(np.arange(1.0, 5.0), np.ones(4), np.exp([1.0, 1, 3, 1]))
    assert r == pytest.approx(1 / math.sqrt(15), rel=1e-12) and ok


def test_bf16_rounding_matches_torch():
    """BF16 rounding (nearest, ties to even) equals torch's float32 ->
    bfloat16 conversion on random bit patterns, 5000 of them exact ties."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2**32, size=100000, dtype=np.uint64).astype(np.uint32)
    bits[:5000] = (bits[:5000] & 0xFFFF0000) | 0x8000
    v = bits.view(np.float32)
    v = v[np.isfinite(v)]
    ref = torch.from_numpy(v.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(sg.bf16(v), ref)


def test_forward_rounds_at_each_stated_point():
    """A hand-built K = 1, H = 2 network whose input, W1 and W2 lie just off
    BF16 values (1 + 2^-10, 0.75 + 2^-12, 1 + 2^-10 round to 1, 0.75, 1):
    Z1 = 0.75, H1 = bf16(g(0.75)), Z2 = H1, out = g(bf16(g(0.75))), with the
    rounding taken from torch. Dropping any rounding point changes out."""
    torch = pytest.importorskip("torch")
    K, H = 1, 2
    p = {"W1": np.array([[0.75 + 2**-12], [0.0]]), "b1": np.zeros(2),
         "W2": np.array([[1 + 2**-10, 0.0], [0.0, 1.0]]), "b2": np.zeros(2),
         "w3": np.array([1.0, 0.0]), "b3": np.zeros(1)}
    w = sg.pack(p).astype(np.float32)
    out, _ = sg.forward(w, np.array([[1 + 2**-10]]), K, H)
    h1 = float(torch.tensor(sg.gelu(0.75), dtype=torch.float32).to(torch.bfloat16))
    assert out[0] == pytest.approx(sg.gelu(h1), rel=1e-12)
    assert abs(h1 - sg.gelu(0.75)) > 1e-3          # the rounding matters here
    raw, _ = sg.forward(w, np.array([[1 + 2**-10]]), K, H, rounding=False)
    assert abs(raw[0] - out[0]) > 1e-4