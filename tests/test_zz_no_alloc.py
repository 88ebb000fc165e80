"""game_eval_fitness_static: the fitness call for callers that cannot
allocate device memory -- plug-ins inside a host application that owns the
device-memory budget, and runtimes that forbid allocation after start-up
(cudaMalloc can fail and may synchronise the device). It keeps its only
scratch, the FP64 partial sums, in a fixed array inside the library, so two
calls in a row must each give what the ordinary handle-based FP32
evaluation (game_eval_fitness) gives on the same inputs, and both must match
the FP64 oracle within the FP32 tolerance, with nothing left over from the
previous call.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import CHEB, TRIG, fp32_tol
from paper_1211_5481_gb300 import datagen as dg
from paper_1211_5481_gb300 import game

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _static_call(lib, Xd, yd, d, basis, popd, fitd, stream):
    M, N = Xd.shape
    return lib.game_eval_fitness_static(Xd.data_ptr(), yd.data_ptr(), M, N, d, basis,
                                        popd.data_ptr(), popd.shape[0], fitd.data_ptr(),
                                        stream.cuda_stream)


@pytest.mark.parametrize("M,N,d,basis,P", [(5003, 6, 5, CHEB, 200), (2000, 3, 4, TRIG, 70)])
def test_static_matches_handle_path_two_calls(orc, M, N, d, basis, P):
    assert torch.cuda.is_available()
    lib = game.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    pr = dg.regression(M + d, M, N, min(d, 3), 0.05, degree=d, basis=basis)
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    pops = [dg.random_population(1 + s, P, pr.K) for s in range(2)]
    with game.Game(pr.X, pr.y, d, basis, P=max(P, 4), precision=game.GAME_PREC_FP32) as g:
        handle = [g.eval_fitness(p) for p in pops]
    oracle = [orc.fitness(pr.X, pr.y, p, d, basis) for p in pops]
    # two calls in a row on different populations through the C ABI
    for pop, ref, exact in zip(pops, handle, oracle):
        popd = torch.from_numpy(pop).to(dev)
        fitd = torch.full((P,), float("nan"), dtype=torch.float64, device=dev)
        rc = _static_call(lib, Xd, yd, d, basis, popd, fitd, stream)
        assert rc == game.GAME_OK, lib.game_last_error().decode()
        torch.cuda.synchronize()
        got = fitd.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= fp32_tol(ref, pr.y)), np.max(np.abs(got - ref) / ref)
        assert np.all(np.abs(got - exact) <= fp32_tol(exact, pr.y)), \
            np.max(np.abs(got - exact) / exact)


def test_static_rejects_oversized_and_host_inputs():
    lib = game.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    Xd = torch.zeros((10, 2), dtype=torch.float32, device=dev)
    yd = torch.zeros(10, dtype=torch.float32, device=dev)
    fitd = torch.zeros(4, dtype=torch.float64, device=dev)
    popd = torch.zeros((4, 2 * 3 + 1), dtype=torch.float32, device=dev)
    # P beyond the static scratch (checked before any launch)
    rc = lib.game_eval_fitness_static(Xd.data_ptr(), yd.data_ptr(), 10, 2, 3, CHEB,
                                      popd.data_ptr(), 524289, fitd.data_ptr(),
                                      stream.cuda_stream)
    assert rc == game.GAME_EINVAL
    assert b"static scratch" in lib.game_last_error()
    host = np.zeros((4, 7), dtype=np.float32)
    rc = lib.game_eval_fitness_static(Xd.data_ptr(), yd.data_ptr(), 10, 2, 3, CHEB,
                                      host.ctypes.data, 4, fitd.data_ptr(), stream.cuda_stream)
    assert rc == game.GAME_EINVAL
    rc = lib.game_eval_fitness_static(Xd.data_ptr(), yd.data_ptr(), 10, 2, 3, CHEB,
                                      popd.data_ptr(), 4, fitd.data_ptr(), stream.cuda_stream)
    assert rc == game.GAME_OK
    torch.cuda.synchronize()
