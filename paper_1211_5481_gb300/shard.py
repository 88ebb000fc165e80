"""One GA run with its training set split over several ranks (one process
per GPU, torch.distributed).

The fitness of Eq. 3 is a sum over patterns, so a run shards over patterns
(the paper lists several GPUs as future work, Section 6): each rank holds a
contiguous slice of the patterns in its own handle, and per generation every
rank

  1. breeds the next population (game_breed) from the same fitness vector
     and the same Philox (seed, generation) counters, so every rank holds the
     bit-identical population without any population being sent;
  2. evaluates its slice's unnormalised error sums (game_eval_sse);
  3. exchanges those P values with every rank (all_gather: P doubles per
     rank and generation, NCCL between GPUs) and adds the slices in rank
     order, the same FP64 additions on every rank, so the totals are
     bit-identical across ranks;
  4. sets the fitness sum / M (its square root for the RMSE) on its handle
     (game_set_fitness).

The exchange is a plain all_gather of device (or, with gloo, host) tensors;
no device kernel waits on another rank. The handles must be created with the
same settings and seed, a direct precision form and no elite re-scoring (the
re-score's Gram form would need the G of all slices) or surrogate."""
from __future__ import annotations

from . import game


def shard_bounds(M: int, world: int, rank: int) -> tuple[int, int]:
    """[begin, end) of rank's contiguous slice of M patterns; slice sizes
    differ by at most one, earlier ranks take the larger ones."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    base, extra = divmod(M, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


class ShardedGA:
    """The GA state of one run whose patterns are split over the ranks of
    `group` (torch.distributed). X, y: this rank's slice; M_total: the
    patterns of all slices. evaluator: anything with the per-slice steps of
    game.Game (eval_sse, breed, set_fitness, population, P); default: a
    game.Game on this rank's slice, built from degree, basis and params."""

    def __init__(self, X, y, degree, basis, M_total, group=None, evaluator=None, stream=None,
                 **params):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.M_total = int(M_total)
        self.error = params.get("error", game.GAME_ERR_MSE)
        if evaluator is None:
            if params.get("precision", game.GAME_PREC_FP32) == game.GAME_PREC_GRAM:
                raise ValueError("sharded runs need a direct precision form")
            if params.get("surrogate", 0):
                raise ValueError("sharded runs have no surrogate screening")
            params = dict(params, rescore_top=0)
            evaluator = game.Game(X, y, degree, basis, stream=stream, **params)
        self.ev = evaluator
        self.P = evaluator.P
        on_gpu = self.world > 1 and dist.get_backend(group) == "nccl"
        self.device = torch.device("cuda", torch.cuda.current_device()) if on_gpu else None
        # the initial population is the same on every rank (same seed); its
        # fitness is that of all slices
        self._exchange_and_set()

    def _local_sums(self):
        torch = self.torch
        if self.device is not None:
            out = torch.empty(self.P, dtype=torch.float64, device=self.device)
            return self.ev.eval_sse(out=out)
        return torch.from_numpy(self.ev.eval_sse())

    def sum_over_ranks(self, local):
        """The slices' sums added in rank order (identical on every rank)."""
        if self.world == 1:
            return local.clone()
        parts = [self.torch.empty_like(local) for _ in range(self.world)]
        self.dist.all_gather(parts, local, group=self.group)
        total = parts[0].clone()
        for p in parts[1:]:
            total += p
        return total

    def fitness_from_sums(self, total):
        fit = total / float(self.M_total)
        return fit.sqrt() if self.error == game.GAME_ERR_RMSE else fit

    def _exchange_and_set(self):
        fit = self.fitness_from_sums(self.sum_over_ranks(self._local_sums()))
        self.ev.set_fitness(fit if self.device is not None else fit.numpy())
        return fit

    def generation(self, seed: int):
        """One generation of the whole run (every rank calls it)."""
        self.ev.breed(seed)
        return self._exchange_and_set()

    def population(self):
        """(population [P][K] FP32, fitness [P] FP64, generation) on the host."""
        return self.ev.population()

    def close(self):
        if hasattr(self.ev, "close"):
            self.ev.close()

