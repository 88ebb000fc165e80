"""Pattern sharding of one GA run (paper_1211_5481_gb300/shard.py) on two
gloo ranks on the CPU: each rank holds half of the patterns; per generation
both breed from the same counters, exchange their slices' error sums and add
them in rank order. Checked: both ranks end with bit-identical populations
and fitness; that state equals a single process doing the same slice sums in
the same order (so nothing but the sums crosses ranks); the fitness is the
whole set's within FP64 rounding; and the populations are the oracle's
operators applied to that fitness, bit for bit.

The per-slice evaluator here is the FP64 oracle (a stand-in with the
per-slice steps of game.Game); the GPU test test_gpu_shard.py runs the same
steps through the CUDA library."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")
torch = pytest.importorskip("torch")

G = 6
SEED = 21


class OracleSlice:
    """The per-slice steps of game.Game (eval_sse, breed, set_fitness,
    population, P) on one slice of the patterns, by the FP64 oracle."""

    def __init__(self, orc, X, y, d, basis, P, seed, prm):
        self.orc, self.X, self.y, self.d, self.basis, self.prm = orc, X, y, d, basis, prm
        self.P = P
        self.pop = orc.init_population(seed, P, orc.num_genes(X.shape[1], d, basis))
        self.fit = None
        self.gen = 0

    def eval_sse(self, out=None):
        s = self.orc.fitness(self.X, self.y, self.pop, self.d, self.basis) * self.X.shape[0]
        if out is not None:
            out[:] = s
            return out
        return s

    def breed(self, seed):
        self.pop = self.orc.generation(self.pop, self.fit, seed, self.gen, self.prm)
        self.gen += 1

    def set_fitness(self, fit):
        self.fit = np.array(fit, dtype=np.float64)

    def population(self):
        return self.pop.copy(), self.fit.copy(), self.gen


def _problem():
    from paper_1211_5481_gb300 import datagen as dg
    return dg.regression(8, 3001, 5, 3, 0.05, degree=4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path[:0] = [ROOT, TESTS]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1211_5481_gb300 import shard
    from test_shard_ranks import OracleSlice, _problem
    pr = _problem()
    b, e = shard.shard_bounds(pr.M, world, rank)
    ev = OracleSlice(oracle, pr.X[b:e], pr.y[b:e], 4, 0, 40, SEED, oracle.ga_params())
    ga = shard.ShardedGA(pr.X[b:e], pr.y[b:e], 4, 0, pr.M, evaluator=ev)
    for _ in range(G):
        ga.generation(SEED)
    q.put((rank,) + ga.population())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_cover_the_patterns():
    from paper_1211_5481_gb300 import shard
    for M in (1, 7, 3001, 10 ** 6):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(M, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == M
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)


def test_two_gloo_ranks_hold_identical_state(orc):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, pop0, fit0, g0), (_, pop1, fit1, g1) = got
    assert g0 == g1 == G
    np.testing.assert_array_equal(pop0.view(np.uint32), pop1.view(np.uint32))
    np.testing.assert_array_equal(fit0.view(np.uint64), fit1.view(np.uint64))

    # the same slice sums in the same order on one process
    from paper_1211_5481_gb300 import shard
    pr = _problem()
    prm = orc.ga_params()
    sl = [shard.shard_bounds(pr.M, 2, r) for r in range(2)]
    K = orc.num_genes(pr.N, 4, 0)
    pop = orc.init_population(SEED, 40, K)

    def fitness(pop):
        s = [orc.fitness(pr.X[b:e], pr.y[b:e], pop, 4, 0) * (e - b) for b, e in sl]
        return (s[0] + s[1]) / pr.M

    fit = fitness(pop)
    for g in range(G):
        pop = orc.generation(pop, fit, SEED, g, prm)
        fit = fitness(pop)
    np.testing.assert_array_equal(pop0.view(np.uint32), pop.view(np.uint32))
    np.testing.assert_array_equal(fit0.view(np.uint64), fit.view(np.uint64))
    # the fitness is the whole set's, up to FP64 rounding of the slice sums
    np.testing.assert_allclose(fit0, orc.fitness(pr.X, pr.y, pop0, 4, 0), rtol=1e-12)
