"""Batched runs: many independent problems advanced by one launch per stage
under a CUDA graph. Each run is checked against the oracle as if it were a
single problem: the initial population bit for bit, the fitness within the
BF16 bound, and every generation's operators bit for bit given the run's
own fitness vector."""
import numpy as np
import pytest

from helpers import CHEB, TRIG, bf16_bound
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


# (M, N, d, basis, P, seed): tile multiples, ragged tails, a single pattern,
# K' from 2 to 1280, P below / above / across chromosome tiles
RUNS = [
    (2000, 8, 4, CHEB, 64, 11),
    (777, 3, 7, TRIG, 130, 12),
    (1, 4, 2, CHEB, 5, 13),
    (5000, 16, 10, TRIG, 257, 2**40 + 1),
    (300, 1, 1, CHEB, 9, 15),
    (513, 64, 10, TRIG, 33, 16),
    (6000, 32, 8, CHEB, 256, 17),
]


def make_runs(spec=RUNS):
    probs = []
    for (M, N, d, basis, P, seed) in spec:
        pr = dg.regression(M + N, M, N, min(d, 4), 0.05, degree=d, basis=basis)
        probs.append((pr, P, seed))
    return probs


def as_args(probs):
    return [(pr.X, pr.y, pr.degree, pr.basis, P, seed) for pr, P, seed in probs]


@pytest.fixture(scope="module")
def probs():
    return make_runs()


@pytest.mark.parametrize("tiles", ["heuristic", "autotune", "narrow"])
def test_batch_matches_oracle(orc, probs, tiles):
    kw = {"autotune": tiles == "autotune"}
    if tiles == "narrow":
        kw["tiles"] = [32] * len(probs)
    prm = orc.ga_params()
    with game.Batch(as_args(probs), **kw) as b:
        t = b.tiles()
        assert set(t.tolist()) <= {32, 64, 128, 256}
        states = [b.run(r) for r in range(b.R)]
        for r, (pr, P, seed) in enumerate(probs):
            pop, fit, gen = states[r]
            assert gen == 0
            np.testing.assert_array_equal(bits(pop), bits(orc.init_population(seed, P, pr.K)))
            ref = orc.fitness(pr.X, pr.y, pop, pr.degree, pr.basis)
            assert np.all(np.abs(fit - ref) <= bf16_bound(ref, pr.X, pop, pr.degree, pr.basis))
        for step in range(3):
            b.generation()
            nxt = [b.run(r) for r in range(b.R)]
            for r, (pr, P, seed) in enumerate(probs):
                pop, fit, gen = states[r]
                npop, nfit, ngen = nxt[r]
                assert ngen == gen + 1
                want = orc.generation(pop, fit, seed, gen, prm)
                np.testing.assert_array_equal(bits(npop), bits(want))
                if step == 2:
                    ref = orc.fitness(pr.X, pr.y, npop, pr.degree, pr.basis)
                    assert np.all(np.abs(nfit - ref) <=
                                  bf16_bound(ref, pr.X, npop, pr.degree, pr.basis))
            states = nxt


def test_batch_reproducible_with_given_tiles(probs):
    with game.Batch(as_args(probs), autotune=True) as b:
        t = b.tiles()
        for _ in range(4):
            b.generation()
        a = [b.run(r) for r in range(b.R)]
    with game.Batch(as_args(probs), tiles=t) as b:
        for _ in range(4):
            b.generation()
        c = [b.run(r) for r in range(b.R)]
    for (p1, f1, g1), (p2, f2, g2) in zip(a, c):
        assert g1 == g2 == 4
        np.testing.assert_array_equal(bits(p1), bits(p2))
        np.testing.assert_array_equal(f1, f2)


def test_batch_device_inputs_and_stream(probs):
    dev = torch.device("cuda:0")
    s = torch.cuda.Stream()
    args = [(torch.from_numpy(pr.X).to(dev), torch.from_numpy(pr.y).to(dev), pr.degree,
             pr.basis, P, seed) for pr, P, seed in probs]
    with game.Batch(args, autotune=False, stream=s) as b1, \
            game.Batch(as_args(probs), autotune=False) as b2:
        for _ in range(2):
            b1.generation()
            b2.generation()
        for r in range(len(probs)):
            p1, f1, _ = b1.run(r)
            p2, f2, _ = b2.run(r)
            np.testing.assert_array_equal(bits(p1), bits(p2))
            np.testing.assert_array_equal(f1, f2)


def test_batch_rejects_bad_runs(probs):
    args = as_args(probs)
    with pytest.raises(game.GameError) as ei:
        game.Batch(args, tiles=[48] * len(args))
    assert ei.value.code == game.GAME_EINVAL
    bad = dg.regression(1, 100, 3, 2, 0.0, degree=2)
    X = bad.X.copy()
    X[5, 1] = np.nan
    with pytest.raises(game.GameError) as ei:
        game.Batch(args[:2] + [(X, bad.y, 2, CHEB, 16, 1)])
    assert ei.value.code == game.GAME_EINVAL and "run 2" in str(ei.value)
    with pytest.raises(game.GameError):   # K - 1 = 2 * 64 * 17 > 2048
        long = dg.regression(1, 100, 64, 2, 0.0, degree=17, basis=TRIG)
        game.Batch([(long.X, long.y, 17, TRIG, 16, 1)])


def test_batched_workload_sample(orc):
    """The batched workload's generator (256 runs of uneven M, N, degree,
    basis, P) at 1/50 of its pattern counts: sampled runs against the oracle
    after two generations."""
    runs = dg.batched_runs(R=256, m_range=(20, 4000))
    args = [(pr.X, pr.y, pr.degree, pr.basis, pr.P, 1000 + r) for r, pr in enumerate(runs)]
    prm = orc.ga_params()
    with game.Batch(args, autotune=True) as b:
        b.generation()
        before = {r: b.run(r) for r in (0, 7, 100, 255)}
        b.generation()
        for r, (pop, fit, gen) in before.items():
            pr = runs[r]
            npop, nfit, ngen = b.run(r)
            assert ngen == gen + 1
            np.testing.assert_array_equal(bits(npop),
                                          bits(orc.generation(pop, fit, 1000 + r, gen, prm)))
            ref = orc.fitness(pr.X, pr.y, npop, pr.degree, pr.basis)
            assert np.all(np.abs(nfit - ref) <= bf16_bound(ref, pr.X, npop, pr.degree, pr.basis))


# every degree the batched generator specialises (1..10) and two it does not
# (11, 12: the generic chunk generator), for both bases; feature counts chosen
# so that feature groups, 8-column chunks and 64-column K-blocks meet at
# different offsets; trigonometric features over [-3, 3]
DEGREE_RUNS = [(200 + 97 * d + 31 * b, [3, 7, 13, 5, 9, 11, 4, 6, 10, 12, 2, 8][d - 1] + b,
                d, basis, 20 + 13 * d, 100 + 16 * d + b)
               for b, basis in enumerate((CHEB, TRIG)) for d in range(1, 13)]


@pytest.mark.parametrize("tiles", [None, 32, 64, 128])
def test_batch_every_degree_matches_cpu_model(tiles):
    """Each run's fitness against the CPU model of the BF16 form (operands
    rounded as the kernel rounds them, exact products): only the FP32
    accumulation order and ambiguous roundings may differ. Tile widths of
    32, 64 and 128 patterns put 8, 4 and 2 expansion threads on each pattern
    row (each a contiguous range of whole features)."""
    from emulation import model
    args, probs = [], []
    for (M, N, d, basis, P, seed) in DEGREE_RUNS:
        pr = dg.regression(seed, M, N, min(d, 4), 0.05, degree=d, basis=basis)
        X = (pr.X * np.float32(3.0 if basis == TRIG else 1.0)).astype(np.float32)
        args.append((X, pr.y, d, basis, P, seed))
        probs.append((X, pr.y, d, basis))
    kw = {"autotune": False}
    if tiles is not None:
        kw["tiles"] = [tiles] * len(args)
    with game.Batch(args, **kw) as b:
        if tiles is not None:
            assert b.tiles().tolist() == [tiles] * len(args)
        for gen in range(2):
            if gen:
                b.generation()
            for r, (X, y, d, basis) in enumerate(probs):
                pop, fit, _ = b.run(r)
                want, tol = model("bf16", X, y, pop, d, basis)
                err = np.abs(fit - want)
                assert np.all(err <= tol), (r, DEGREE_RUNS[r], float((err / tol).max()))


# Runs whose contraction is longer than their tile's expansion slots hold:
# one chromosome tile at 256 patterns, K-blocks cycling through a ring of four
# slots (K' from 320 to 2048, templated and generic degrees, ragged tails);
# two chromosome tiles at 128 patterns, a ring of eight slots filled by two
# threads per row (beyond 16 K-blocks the second thread's range starts past
# the ring's first pass); three or four at 64 patterns, sixteen slots and four
# threads per row; next to runs that use one slot per K-block at 256, 128
# and 64 patterns, so that the kernel passes between ring and plain items
# and between widths.
RING_RUNS = [
    (1500, 40, 8, CHEB, 100, 301),     # K' = 320: 5 K-blocks
    (2100, 33, 10, TRIG, 128, 302),    # 660: 11
    (900, 70, 12, CHEB, 64, 303),      # 840: 14, generic generator
    (700, 90, 11, TRIG, 17, 304),      # 1980: 31, generic
    (600, 128, 16, CHEB, 50, 305),     # 2048: 32, generic
    (1201, 96, 3, TRIG, 96, 306),      # 576: 9
    (1200, 64, 4, CHEB, 120, 307),     # 256: 4 K-blocks, one slot each
    (1000, 20, 9, TRIG, 200, 308),     # 360, two chromosome tiles: 128 patterns
    (800, 60, 10, CHEB, 300, 309),     # 600, three tiles: 64 patterns
    (1100, 50, 7, TRIG, 256, 310),     # 700, two tiles: 11 K-blocks in 8 slots at 128
    (900, 64, 8, TRIG, 140, 311),      # 1024, two tiles: 16 K-blocks in 8 slots
    (700, 68, 8, TRIG, 150, 312),      # 1088, two tiles: 17 K-blocks in 8 slots
    (600, 128, 8, TRIG, 200, 313),     # 2048, two tiles: 32 K-blocks in 8 slots
    (500, 128, 6, TRIG, 300, 314),     # 1536, three tiles: 24 K-blocks in 16 slots at 64
    (400, 128, 8, TRIG, 450, 315),     # 2048, four tiles: 32 K-blocks in 16 slots
    (333, 250, 5, CHEB, 390, 316),     # 1250, four tiles: 20 K-blocks in 16 slots
    (1, 128, 8, TRIG, 5, 317),         # 2048, one pattern: a ragged ring tile
    (129, 100, 7, CHEB, 129, 318),     # 700, two tiles: 128 + 1 patterns, 129 chromosomes
]


def test_batch_ring_items_match_cpu_model():
    """Ring items against the CPU model of the BF16 form, element by element,
    over two generations."""
    from emulation import model
    args, probs = [], []
    for (M, N, d, basis, P, seed) in RING_RUNS:
        pr = dg.regression(seed, M, N, min(d, 4), 0.05, degree=d, basis=basis)
        X = (pr.X * np.float32(3.0 if basis == TRIG else 1.0)).astype(np.float32)
        args.append((X, pr.y, d, basis, P, seed))
        probs.append((X, pr.y, d, basis))
    with game.Batch(args, autotune=False) as b:
        assert b.tiles().tolist() == ([256] * 7 + [128, 64, 128, 128, 128, 128, 64, 64, 64]
                                      + [256, 128])
        for gen in range(2):
            if gen:
                b.generation()
            for r, (X, y, d, basis) in enumerate(probs):
                pop, fit, _ = b.run(r)
                want, tol = model("bf16", X, y, pop, d, basis)
                err = np.abs(fit - want)
                assert np.all(err <= tol), (r, RING_RUNS[r], float((err / tol).max()))
