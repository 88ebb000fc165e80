"""Failure paths on the GPU, reached through the library's test hooks and
never through a fault:

  * an expired wait: the next tensor-core fitness launch waits on a barrier
    phase that nothing completes; its bounded wait runs out, the kernel
    abandons the launch (status word, drained copies and MMAs, tensor memory
    freed), the call returns GAME_ETIMEOUT, and the same handle then
    evaluates correctly -- which also shows that the abandoned launch freed
    its tensor memory, since the next launch allocates it again;
  * allocation failures: the k-th device allocation of a handle's or a
    batch's creation fails, for every k the creation makes; each attempt
    returns GAME_ENOMEM, releases what it had allocated (device memory does
    not shrink over the attempts), and a creation afterwards succeeds."""
import numpy as np
import pytest

from emulation import model
from helpers import CHEB
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def disarm():
    game.load()
    yield
    game.game_test_hook(game.GAME_HOOK_FAIL_ALLOC, 0)
    game.game_test_hook(game.GAME_HOOK_STALL_NS, 0)


# one-SM kernel: staged features (degree 4), features read from L2
# (Chebyshev degree 8), FP8 and the split form; paired-SM kernel: 48 features
# of degree 6 (the one-SM plan would narrow its tile)
@pytest.mark.parametrize("N,degree,form,kernel", [
    (8, 4, "bf16", "fitness_tc_kernel"), (8, 8, "bf16", "fitness_tc_kernel"),
    (8, 4, "fp8", "fitness_tc_kernel"), (8, 4, "bf16x3", "fitness_tc_kernel"),
    (48, 6, "bf16", "fitness_tc2_kernel")])
def test_expired_wait_reports_timeout_and_the_handle_recovers(N, degree, form, kernel):
    prec = {"bf16": game.GAME_PREC_BF16, "fp8": game.GAME_PREC_FP8,
            "bf16x3": game.GAME_PREC_BF16X3}[form]
    pr = dg.regression(17, 20000, N, 3, 0.05, degree=degree)
    pop = dg.random_population(5, 300, pr.K)
    want, tol = model(form, pr.X, pr.y, pop, degree, CHEB)
    with game.Game(pr.X, pr.y, degree, CHEB, P=64, precision=prec, rescore_top=0) as g:
        assert g.plan(P=300)["kernel"] == kernel
        game.game_test_hook(game.GAME_HOOK_STALL_NS, 20_000_000)    # 20 ms
        with pytest.raises(game.GameError) as ei:
            g.eval_fitness(pop)
        assert ei.value.code == game.GAME_ETIMEOUT
        g.sync()                                  # the status word was cleared
        got = g.eval_fitness(pop)
        assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)
        g.generation(3)
        g.sync()


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _attempts(create):
    """Arms the allocation hook at k = 1, 2, ... until a creation succeeds;
    returns the number of failed attempts."""
    for k in range(1, 200):
        game.game_test_hook(game.GAME_HOOK_FAIL_ALLOC, k)
        try:
            obj = create()
        except game.GameError as e:
            assert e.code == game.GAME_ENOMEM, (k, str(e))
            continue
        finally:
            game.game_test_hook(game.GAME_HOOK_FAIL_ALLOC, 0)
        obj.close()
        return k - 1
    raise AssertionError("creation kept failing")


def test_every_allocation_failure_of_a_handle_is_clean():
    # large enough that a leaked training-set copy (9.6 MB) would show
    pr = dg.regression(23, 300_000, 8, 3, 0.05, degree=4)
    Xd = torch.from_numpy(pr.X).cuda()
    yd = torch.from_numpy(pr.y).cuda()
    kinds = [dict(precision=game.GAME_PREC_BF16),
             dict(precision=game.GAME_PREC_FP8, selection=game.GAME_SEL_RANKING),
             dict(precision=game.GAME_PREC_BF16, surrogate=1, oversample=2,
                  selection=game.GAME_SEL_ROULETTE)]
    for kw in kinds:
        for X, y in ((pr.X, pr.y), (Xd, yd)):    # host inputs take staging copies
            _attempts(lambda: game.Game(X, y, 4, CHEB, P=128, **kw))   # warm: lazy set-up
            before = _free_bytes()
            n = _attempts(lambda: game.Game(X, y, 4, CHEB, P=128, **kw))
            assert n >= 8, n
            assert _free_bytes() >= before - (16 << 20)
    with game.Game(pr.X, pr.y, 4, CHEB, P=128, precision=game.GAME_PREC_BF16) as g:
        g.generation(1)
        g.sync()


def test_every_allocation_failure_of_a_batch_is_clean():
    runs = [dg.regression(31 + r, 40_000 + 777 * r, 5 + r, 3, 0.05, degree=3 + r)
            for r in range(3)]
    args = [(pr.X, pr.y, pr.degree, CHEB, 64 + 32 * r, 9 + r) for r, pr in enumerate(runs)]
    _attempts(lambda: game.Batch(args, autotune=False))
    before = _free_bytes()
    n = _attempts(lambda: game.Batch(args, autotune=False))
    assert n >= 10, n
    assert _free_bytes() >= before - (16 << 20)
    with game.Batch(args, autotune=False) as b:
        b.generation()
        b.sync()
