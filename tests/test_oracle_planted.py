"""Planted mistakes: each case rewrites one passage of a scratch copy of
oracle/oracle.c (or of the surrogate oracle, oracle/surrogate.py) into a
plausible slip (a dropped term, a wrong sign, index
or bound, a swapped word), builds the copy, and runs the oracle's pins
against it in a child process. Every slip must make at least one pin fail:
a pin set that lets one through does not pin the oracle. Each rewritten
passage must occur exactly once in the oracle, so that an edit of the oracle
that moves it shows up here rather than silently testing nothing.

Every rewrite keeps all memory accesses inside the caller's arrays, so a
mutant fails by its values, not by a crash (a crash would not count)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
SRC_SURROGATE = os.path.join(ROOT, "oracle", "surrogate.py")
PINS = ["tests/test_oracle_fitness.py", "tests/test_oracle_rescore.py",
        "tests/test_oracle_ga.py", "tests/test_oracle_philox.py"]
PINS_SURROGATE = ["tests/test_oracle_surrogate.py"]

# (name, passage of oracle.c, its replacement)
MISTAKES = [
    # basis (Eq. 1, Eq. 6)
    ("chebyshev-recurrence-sign",
     "double tp1 = 2.0 * x * t - tm1;", "double tp1 = 2.0 * x * t + tm1;"),
    ("cos-sin-swapped",
     "return b == 0 ? cos((double)j * x) : sin((double)j * x);",
     "return b == 0 ? sin((double)j * x) : cos((double)j * x);"),
    # output (Eq. 2) and the gene index
    ("bias-gene-dropped",
     "  double out = a[0];\n  for", "  double out = 0.0;\n  for"),
    ("gene-index-interleaved",
     "out += a[1 + (int64_t)i * B * d + b * d + (j - 1)] *",
     "out += a[1 + (int64_t)i * B * d + (j - 1) * B + b] *"),
    ("gene-index-feature-stride",
     "out += a[1 + (int64_t)i * B * d + b * d + (j - 1)] *",
     "out += a[1 + (int64_t)i * d + b * d + (j - 1)] *"),
    ("gene-index-degree-reversed",
     "out += a[1 + (int64_t)i * B * d + b * d + (j - 1)] *",
     "out += a[1 + (int64_t)i * B * d + b * d + (d - j)] *"),
    # error (Eq. 3) and its variants
    ("mse-over-m-minus-one",
     "double mean = acc / (double)M;", "double mean = acc / (double)(M > 1 ? M - 1 : 1);"),
    ("residual-sign-inside-mae",
     "? fabs(r) : r * r;", "? r : r * r;"),
    ("rmse-without-root",
     "fit[p] = (err_kind == ORACLE_ERR_RMSE) ? sqrt(mean) : mean;", "fit[p] = mean;"),
    # shared genes (Eq. 5)
    ("shared-genes-groups-merged",
     "out += a[1 + b * d + (j - 1)] * phi(", "out += a[1 + (j - 1)] * phi("),
    # Gram form
    ("gram-cross-term-halved",
     "fit[p] = (yy - 2.0 * ab + aGa) / (double)M;", "fit[p] = (yy - ab + aGa) / (double)M;"),
    ("gram-b-wrong-pattern",
     "b[k1] += v * y[m0 + r];", "b[k1] += v * y[m0];"),
    ("gram-diagonal-only-bias",
     "      row[0] = 1.0;\n", "      row[0] = 0.0;\n"),
    # Philox4x32-10
    ("philox-output-words-swapped",
     "  out[0] = c0;\n  out[1] = c1;", "  out[0] = c1;\n  out[1] = c0;"),
    ("philox-second-weyl-constant",
     "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    ("philox-nine-rounds",
     "for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 9; ++round)"),
    # initial genes
    ("uniform-gene-one-sided",
     "return (float)((int32_t)(w >> 8) - 8388608) * (1.0f / 8388608.0f);",
     "return (float)((int32_t)(w >> 9) - 8388608) * (1.0f / 8388608.0f);"),
    # ranking key: ties and NaN
    ("ties-to-higher-index", "  return a < b;\n}", "  return a > b;\n}"),
    ("nan-ranked-first",
     "if (isnan(fa)) fa = INFINITY;\n  if (isnan(fb)) fb = INFINITY;",
     "if (isnan(fa)) fa = -INFINITY;\n  if (isnan(fb)) fb = -INFINITY;"),
    # selection
    ("tournament-never-draws-last",
     "const int32_t c = (int32_t)(((uint64_t)w[s % 4] * (uint64_t)P) >> 32);",
     "const int32_t c = (int32_t)(((uint64_t)w[s % 4] * (uint64_t)(P - 1)) >> 32);"),
    ("tournament-worst-wins",
     "if (win < 0 || better(fit[c], c, fit[win], win)) win = c;",
     "if (win < 0 || better(fit[win], win, fit[c], c)) win = c;"),
    ("ranking-weights-reversed",
     "cum += (uint64_t)(P - k);", "cum += (uint64_t)(k + 1);"),
    ("ranking-order-by-worse",
     "for (int32_t q = 0; q < P; ++q) rank += better(fit[q], q, fit[p], p);",
     "for (int32_t q = 0; q < P; ++q) rank += better(fit[p], p, fit[q], q);"),
    ("roulette-on-f-over-one-plus-f",
     "const double w = 1.0 / (1.0 + f);", "const double w = f / (1.0 + f);"),
    ("roulette-nan-weighted",
     "if (!(f >= 0.0) || isinf(f)) return 0;",
     "if (isnan(f)) return (uint64_t)1 << 31;\n  if (f < 0.0 || isinf(f)) return 0;"),
    ("roulette-cover-inclusive",
     "      cum += tab->weight[p];\n      if (u < cum) return p;",
     "      cum += tab->weight[p];\n      if (u <= cum) return p;"),
    # elitism
    ("elites-in-reverse-order",
     "memcpy(next + (int64_t)e * K, pop + (int64_t)best * K, sizeof(float) * K);",
     "memcpy(next + (int64_t)(E - 1 - e) * K, pop + (int64_t)best * K, sizeof(float) * K);"),
    # crossover
    ("crossover-cut-may-be-zero",
     "cut = 1 + (int32_t)(((uint64_t)w[1] * (uint64_t)(K - 1)) >> 32);",
     "cut = (int32_t)(((uint64_t)w[1] * (uint64_t)(K - 1)) >> 32);"),
    ("crossover-children-not-complementary",
     "const float* tail = c == 0 ? p1 : p0;", "const float* tail = p1;"),
    ("crossover-threshold-inverted",
     "if ((w[0] >> 8) < prm->thr_pc)", "if ((w[0] >> 8) >= prm->thr_pc)"),
    # mutation
    ("mutation-rate-doubled",
     "if ((w[0] >> 8) >= prm->thr_pm) continue;", "if ((w[0] >> 9) >= prm->thr_pm) continue;"),
    ("mutation-step-halved-uniforms",
     "sum += (int64_t)(w[i] >> 8);", "sum += (int64_t)(w[i] >> 9);"),
    ("mutation-step-unscaled",
     "const float step = prm->sigma * z;", "const float step = z;"),
    ("clamp-upper-dropped", "      if (v > 1.0f) v = 1.0f;\n", ""),
    ("clamp-lower-dropped", "      if (v < -1.0f) v = -1.0f;\n", ""),
    # immigrants (Section 4)
    ("immigrants-one-slot-early",
     "for (int32_t s = n_out - I; s < n_out; ++s)", "for (int32_t s = n_out - I - 1; s < n_out; ++s)"),
    # elite re-scoring
    ("rescore-writes-rank-slot",
     "&fit_out[idx[r]]);", "&fit_out[r]);"),
    # the GA run
    ("train-generation-counter-shifted",
     "(uint32_t)(g - 1), next);", "(uint32_t)g, next);"),
    ("train-best-is-slot-zero",
     "if (best) best[g] = bf;", "if (best) best[g] = fit[0];"),
    ("elites-all-the-same-best",
     "    chosen[best] = 1;\n", "    chosen[best] = 0;\n"),
    ("odd-child-slot-left-empty",
     "const int32_t npairs = (n_out - E + 1) / 2;", "const int32_t npairs = (n_out - E) / 2;"),
    ("select-best-repeats-the-best",
     "    taken[best] = 1;\n    idx[r] = best;", "    idx[r] = best;"),
    ("gram-squares-one-column",
     "G[k1 * K + k2] += v * Phi[r * K + k2];", "G[k1 * K + k2] += v * Phi[r * K + k1];"),
    ("gram-row-times-wrong-gene",
     "row += G[(int64_t)k1 * K + k2] * a[k2];", "row += G[(int64_t)k1 * K + k2] * a[k1];"),
    ("shared-genes-mean-over-features",
     "fit[p] = sse / (double)M;", "fit[p] = sse / (double)(M * N);"),
    # classification (Section 5 metrics)
    ("label-threshold-inclusive",
     "const int actual = y[m] > threshold;", "const int actual = y[m] >= threshold;"),
    ("prediction-threshold-inclusive",
     "N, d, basis) > threshold;", "N, d, basis) >= threshold;"),
    ("false-positive-counted-as-negative",
     "else if (predicted) counts[1] += 1;", "else if (predicted) counts[3] += 1;"),
]

# the same for the surrogate oracle (numpy)
SURROGATE_MISTAKES = [
    ("gelu-drops-input-factor",
     "return 0.5 * z * (1.0 + np.tanh(", "return 0.5 * (1.0 + np.tanh("),
    ("gelu-grad-cubic-term",
     "(1.0 + 3.0 * GELU_A * z * z)", "(1.0 + GELU_A * z * z)"),
    ("loss-grad-without-two",
     "d_out = 2.0 * r / B", "d_out = r / B"),
    ("w2-grad-from-wrong-activation",
     'g["W2"] = dZ2.T @ c["H1"]', 'g["W2"] = dZ2.T @ c["H2"]'),
    ("backprop-through-transposed-w2",
     'dZ1 = (dZ2 @ c["W2b"]) * gelu_grad', 'dZ1 = (dZ2 @ c["W2b"].T) * gelu_grad'),
    ("b1-grad-halved",
     'g["b1"] = dZ1.sum(axis=0)', 'g["b1"] = dZ1.sum(axis=0) * 0.5'),
    ("adam-without-bias-correction",
     "mh = m / (1 - B1 ** t)", "mh = m"),
    ("adam-without-root",
     "return w - LR * mh / (np.sqrt(vh) + EPS), m, v", "return w - LR * mh / (vh + EPS), m, v"),
    ("init-scale-over-fan-in",
     "a = np.float32(1.0) / np.sqrt(np.float32(fan_in))", "a = np.float32(1.0) / np.float32(fan_in)"),
    ("init-one-sided",
     "u = (r >> 8).astype(np.float32)", "u = (r >> 9).astype(np.float32)"),
    ("targets-not-centred",
     "return (l - mu) / (sd if sd > 0 else 1.0)", "return l / (sd if sd > 0 else 1.0)"),
    ("screen-keeps-largest",
     "keep[order[:n_keep]] = 1\n    return keep", "keep[order[-n_keep:]] = 1\n    return keep"),
    ("screen-ties-to-higher-slot",
     "order = np.lexsort((np.arange(key.shape[0]), key))",
     "order = np.lexsort((-np.arange(key.shape[0]), key))"),
    ("screen-nan-first",
     "p[np.isnan(p)] = np.inf", "p[np.isnan(p)] = -np.inf"),
    ("untrusted-keeps-last-children",
     "keep[:n_keep] = 1", "keep[-n_keep:] = 1"),
    ("bf16-ties-away-from-zero",
     "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = (u + 0x8000) & 0xFFFF0000"),
    ("forward-skips-h1-rounding",
     'H1 = _round(gelu(Z1), rounding)', 'H1 = gelu(Z1)'),
    ("forward-skips-w2-rounding",
     'W1b, W2b = _round(p["W1"], rounding), _round(p["W2"], rounding)',
     'W1b, W2b = _round(p["W1"], rounding), p["W2"]'),
    ("trust-threshold-zero",
     "return r, r > 0.25", "return r, r > 0.0"),
]


def _run_pins(name, old, new, tmp, surrogate=False):
    path = SRC_SURROGATE if surrogate else SRC
    src = open(path).read()
    assert src.count(old) == 1, f"{name}: the passage must occur once in {os.path.basename(path)}"
    mutant = os.path.join(tmp, name + (".py" if surrogate else ".c"))
    with open(mutant, "w") as f:
        f.write(src.replace(old, new))
    if surrogate:
        env = dict(os.environ, GAME_ORACLE_SURROGATE_SOURCE=mutant, OMP_NUM_THREADS="1")
        pins = PINS_SURROGATE
    else:
        sys.path.insert(0, ROOT)
        import oracle
        oracle.compile_source(mutant, os.path.splitext(mutant)[0] + ".so")
        env = dict(os.environ, GAME_ORACLE_SOURCE=mutant, OMP_NUM_THREADS="1")
        pins = PINS
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           "-m", "not gpu", *pins]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return res.returncode, res.stdout[-3000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("planted"))
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {m[0]: ex.submit(_run_pins, *m, tmp) for m in MISTAKES}
        futs.update({m[0]: ex.submit(_run_pins, *m, tmp, True) for m in SURROGATE_MISTAKES})
        return {k: f.result() for k, f in futs.items()}


def test_names_are_unique():
    names = [m[0] for m in MISTAKES + SURROGATE_MISTAKES]
    assert len(set(names)) == len(names)


@pytest.mark.parametrize("name", [m[0] for m in MISTAKES + SURROGATE_MISTAKES])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    # 1 = some test failed; a crash, an interrupt or a collection error is
    # not a pin catching the mistake
    assert rc == 1 and " failed" in out, f"{name} slipped through the pins:\n{out}"
