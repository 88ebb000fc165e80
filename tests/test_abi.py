"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/game.h declares; argument checks that precede any GPU work reject
bad shapes without a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1211_5481_gb300 import build as gbuild
from paper_1211_5481_gb300 import game

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "game.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(game_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    lib = gbuild.build()
    assert os.path.exists(lib)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (game_[a-z_0-9]+)$", out, flags=re.M))
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    missing = [s for s in decl if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert set(decl) == set(game.EXPORTED)


def test_build_targets_sm103a_only():
    assert gbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_side_argument_checks():
    lib = game.load()
    p = game.game_params_default()
    assert p.elitism == 2 and p.tournament == 3 and abs(p.pc - 0.9) < 1e-7
    h = ctypes.c_void_p()
    X = np.zeros((4, 2), dtype=np.float32)
    y = np.zeros(4, dtype=np.float32)
    for M, N, d, basis in [(0, 2, 3, 0), (4, 0, 3, 0), (4, 2, 0, 0), (4, 2, 3, 7)]:
        rc = lib.game_create(X.ctypes.data, y.ctypes.data, M, N, d, basis, None, None,
                             ctypes.byref(h))
        assert rc == game.GAME_EINVAL
        assert lib.game_last_error()
    # K above the supported maximum
    rc = lib.game_create(X.ctypes.data, y.ctypes.data, 4, 2049, 2, 0, None, None,
                         ctypes.byref(h))
    assert rc == game.GAME_EINVAL
    bad = game.game_params_default()
    bad.P = 3   # < elitism + 2
    rc = lib.game_create(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, ctypes.byref(bad), None,
                         ctypes.byref(h))
    assert rc == game.GAME_EINVAL
    bad = game.game_params_default()
    bad.tournament = 0
    rc = lib.game_create(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, ctypes.byref(bad), None,
                         ctypes.byref(h))
    assert rc == game.GAME_EINVAL
    assert p.selection == game.GAME_SEL_TOURNAMENT and p.tied == 0
    assert p.error == game.GAME_ERR_MSE and p.surrogate_steps == 8
    # selection, shared genes and error function settings
    for field, value, extra in [("selection", 3, {}), ("selection", -1, {}),
                                ("selection", game.GAME_SEL_RANKING, {"P": 16385}),
                                ("tied", 2, {}), ("error", 3, {}),
                                ("error", game.GAME_ERR_MAE, {}),   # rescore_top = 16
                                ("error", game.GAME_ERR_MAE,
                                 {"rescore_top": 0, "precision": game.GAME_PREC_GRAM}),
                                ("surrogate_steps", 65, {}),
                                ("surrogate_steps", 0, {"surrogate": 1})]:
        bad = game.game_params_default()
        setattr(bad, field, value)
        for k, v in extra.items():
            setattr(bad, k, v)
        rc = lib.game_create(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, ctypes.byref(bad), None,
                             ctypes.byref(h))
        assert rc == game.GAME_EINVAL, (field, value, extra)
    bad = game.game_params_default()
    bad.reserved[0] = 1
    rc = lib.game_create(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, ctypes.byref(bad), None,
                         ctypes.byref(h))
    assert rc == game.GAME_EINVAL
    assert lib.game_destroy(None) == game.GAME_OK


def test_batch_refuses_paper_mode_settings():
    """Batched runs take tournament selection, per-feature genes and the MSE
    only; the check precedes any device work."""
    lib = game.load()
    X = np.zeros((4, 2), dtype=np.float32)
    y = np.zeros(4, dtype=np.float32)
    runs = (game.game_run_desc * 1)()
    runs[0] = game.game_run_desc(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, 8, 1)
    b = ctypes.c_void_p()
    for field, value in [("selection", game.GAME_SEL_RANKING), ("tied", 1),
                         ("error", game.GAME_ERR_RMSE)]:
        prm = game.game_params_default()
        setattr(prm, field, value)
        rc = lib.game_batch_create(runs, 1, ctypes.byref(prm), None, 1, None, ctypes.byref(b))
        assert rc == game.GAME_EINVAL, field


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the CUDA library the binding raises instead of
    computing anything, and the oracle is not imported by the package."""
    import sys as _sys
    monkeypatch.setattr(game, "_lib", None)
    monkeypatch.setattr(gbuild, "LIB", str(tmp_path / "missing" / "libgame.so"))
    with pytest.raises(ImportError):
        game.load(build_if_missing=False)
    # the product package never loads the oracle
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([_sys.executable, "-c",
                          "import sys; import paper_1211_5481_gb300.game, paper_1211_5481_gb300.datagen; "
                          "print('oracle' in sys.modules)"],
                         cwd=root, capture_output=True, text=True, check=True).stdout.strip()
    assert out == "False"
    for f in (game.__file__, gbuild.__file__):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src


def test_unknown_parameter_names_are_refused():
    """A misspelt setting raises before any device work instead of being
    kept as a stray attribute and silently ignored."""
    X = np.zeros((4, 2), dtype=np.float32)
    y = np.zeros(4, dtype=np.float32)
    with pytest.raises(TypeError, match="selction"):
        game.Game(X, y, 3, selction=game.GAME_SEL_RANKING)
    with pytest.raises(TypeError, match="elitsm"):
        game.Batch([(X, y, 3, 0, 8, 1)], elitsm=2)
    assert game._params({"selection": game.GAME_SEL_RANKING}).selection == game.GAME_SEL_RANKING


def test_element_types_are_checked_before_the_call():
    """The library sees raw pointers: arrays of the wrong element type are
    refused in the binding (numpy inputs of Game are converted instead)."""
    torch = pytest.importorskip("torch")
    pop64 = np.zeros((4, 7))
    with pytest.raises(TypeError, match="pop must be float32"):
        game.game_eval_fitness(None, pop64, np.zeros(4))
    with pytest.raises(TypeError, match="fit_out must be float64"):
        game.game_eval_fitness(None, pop64.astype(np.float32), np.zeros(4, dtype=np.float32))
    with pytest.raises(TypeError, match="X must be float32"):
        game.game_create(torch.zeros((4, 2), dtype=torch.float16), torch.zeros(4), 3, 0)
    with pytest.raises(TypeError, match="idx_out must be int32"):
        game.game_rescore_top(None, pop64.astype(np.float32), np.zeros(4), 2,
                              np.zeros(2, dtype=np.int64))
    with pytest.raises(TypeError, match="must be float32"):
        game._f32(torch.zeros(3, dtype=torch.float64))
    assert game._f32(np.zeros(3)).dtype == np.float32


@pytest.mark.parametrize("field,value,extra", [
    ("elitism", -1, {}), ("elitism", 257, {}), ("tournament", 65, {}), ("immigrants", -1, {}),
    ("P", (1 << 24) + 1, {}), ("immigrants", 7, {"P": 10}),
    ("pc", 1.5, {}), ("pm", -0.1, {}), ("pc", float("nan"), {}),
    ("sigma", -1.0, {}), ("sigma", float("inf"), {}), ("precision", 9, {}),
    ("surrogate", 2, {}), ("oversample", 0, {"surrogate": 1}),
    ("oversample", 300, {"surrogate": 1, "P": 64}),
    ("rescore_top", 17, {}), ("rescore_top", -1, {}), ("check_every", -1, {}),
], ids=lambda v: str(v))
def test_every_settings_check_precedes_device_work(field, value, extra):
    """Each refusal of game_params happens on the host, before any device
    call, with GAME_EINVAL and a message."""
    lib = game.load()
    X = np.zeros((4, 2), dtype=np.float32)
    y = np.zeros(4, dtype=np.float32)
    bad = game.game_params_default()
    setattr(bad, field, value)
    for k, v in extra.items():
        setattr(bad, k, v)
    h = ctypes.c_void_p()
    rc = lib.game_create(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, ctypes.byref(bad), None,
                         ctypes.byref(h))
    assert rc == game.GAME_EINVAL
    assert lib.game_last_error()


@pytest.mark.parametrize("case", ["no runs", "too many runs", "bad elitism", "bad rate",
                                  "bad sigma", "null out"])
def test_batch_refusals_precede_device_work(case):
    lib = game.load()
    X = np.zeros((4, 2), dtype=np.float32)
    y = np.zeros(4, dtype=np.float32)
    R = {"no runs": 0, "too many runs": 65536}.get(case, 1)
    runs = (game.game_run_desc * max(R, 1))()
    for r in range(max(R, 1)):
        runs[r] = game.game_run_desc(X.ctypes.data, y.ctypes.data, 4, 2, 3, 0, 8, 1)
    prm = game.game_params_default()
    if case == "bad elitism":
        prm.elitism = 257
    elif case == "bad rate":
        prm.pc = 2.0
    elif case == "bad sigma":
        prm.sigma = float("nan")
    b = ctypes.c_void_p()
    out = None if case == "null out" else ctypes.byref(b)
    rc = lib.game_batch_create(runs, R, ctypes.byref(prm), None, 0, None, out)
    assert rc == game.GAME_EINVAL
    assert lib.game_last_error()


def test_every_entry_point_refuses_a_null_handle():
    """Called with a NULL handle (and NULL arrays), every entry point returns
    GAME_EINVAL with a message; destroying NULL is a no-op."""
    lib = game.load()
    skip = {"game_last_error", "game_params_default", "game_create", "game_batch_create",
            "game_eval_fitness_static", "game_test_hook"}
    for name in game.EXPORTED:
        if name in skip:
            continue
        fn = getattr(lib, name)
        args = [1 if t in (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64) else
                0.0 if t is ctypes.c_double else None for t in fn.argtypes]
        rc = fn(*args)
        if name in ("game_destroy", "game_batch_destroy"):
            assert rc == game.GAME_OK, name
        else:
            assert rc == game.GAME_EINVAL, name
            assert lib.game_last_error(), name


def test_test_hook_refusals():
    """The test hooks take no handle: unknown hooks and out-of-range values
    are refused; 0 disarms each (left disarmed for the rest of the run)."""
    lib = game.load()
    assert lib.game_test_hook(99, 1) == game.GAME_EINVAL
    assert lib.game_test_hook(game.GAME_HOOK_FAIL_ALLOC, -1) == game.GAME_EINVAL
    assert lib.game_test_hook(game.GAME_HOOK_STALL_NS, 2_000_000_000) == game.GAME_EINVAL
    assert lib.game_test_hook(game.GAME_HOOK_SMEM_SLACK, 1025) == game.GAME_EINVAL
    assert lib.game_last_error()
    assert lib.game_test_hook(game.GAME_HOOK_FAIL_ALLOC, 0) == game.GAME_OK
    assert lib.game_test_hook(game.GAME_HOOK_STALL_NS, 0) == game.GAME_OK
    assert lib.game_test_hook(game.GAME_HOOK_SMEM_SLACK, 0) == game.GAME_OK
