"""The boundary is plain C: include/game.h compiles as C99 and C++ with all
warnings as errors, a C program links against libgame.so and calls it, and
every struct the Python binding mirrors has the same size and field offsets
as the C compiler gives it (a mismatch would hand the library shifted
settings). No GPU is needed: only game_params_default runs."""
import ctypes
import os
import subprocess

import pytest

from paper_1211_5481_gb300 import build as gbuild
from paper_1211_5481_gb300 import game

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

STRUCTS = [("game_params", game.game_params), ("game_timing", game.game_timing),
           ("game_run_desc", game.game_run_desc), ("game_confusion", game.game_confusion)]


def _layout_program():
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "game.h"', 'int main(void) {']
    for cname, cls in STRUCTS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  game_params p;', '  if (game_params_default(&p) != GAME_OK) return 1;',
              '  printf("default P %d elitism %d tournament %d rescore_top %d oversample %d\\n",',
              '         p.P, p.elitism, p.tournament, p.rescore_top, p.oversample);',
              '  return 0;', '}']
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_cleanly(tmp_path, lang, std):
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "game.h"\nint main(void) { return 0; }\n')
    cc = "gcc" if lang == "c" else "g++"
    subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INC,
                    "-fsyntax-only", str(src)], check=True)


def test_c_caller_and_ctypes_layouts_agree(tmp_path):
    lib = gbuild.build()
    src = tmp_path / "layout.c"
    src.write_text(_layout_program())
    exe = tmp_path / "layout"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", INC, str(src), "-o", str(exe),
                    "-L", libdir, "-lgame", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.splitlines() if not line.startswith("default"))
    for cname, cls in STRUCTS:
        assert int(got[f"{cname} size"]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"
    p = game.game_params_default()
    want = (f"default P {p.P} elitism {p.elitism} tournament {p.tournament} "
            f"rescore_top {p.rescore_top} oversample {p.oversample}")
    assert want in out


def test_binding_constants_equal_the_header_defines():
    """Every GAME_* value the header defines has the same value in the
    binding, and the binding defines no GAME_* value the header lacks."""
    import re
    src = open(os.path.join(INC, "game.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"^#define (GAME_[A-Z0-9_]+) \(?(-?\d+)\)?", src, flags=re.M)}
    assert len(defs) >= 19
    for name, value in defs.items():
        assert getattr(game, name) == value, name
    mirrored = {n for n in dir(game) if re.fullmatch(r"GAME_[A-Z0-9_]+", n)
                and isinstance(getattr(game, n), int)}
    assert mirrored == set(defs)


def test_binding_signatures_have_the_header_arity():
    """Every entry point's ctypes argtypes has as many arguments as its
    declaration in the header."""
    import re
    src = open(os.path.join(INC, "game.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lib = game.load()
    decls = re.findall(r"\b(?:int|const char\*)\s+(game_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src)
    assert len(decls) == len(game.EXPORTED)
    for name, args in decls:
        args = args.strip()
        n = 0 if args in ("", "void") else args.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name


def test_binding_signatures_have_the_header_types():
    """Each argument's ctypes type has the width and kind of its C type:
    integers of the declared width, doubles, and pointers (handles, arrays,
    structs and strings) as pointer types."""
    import re
    src = open(os.path.join(INC, "game.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lib = game.load()
    scalar = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
              "double": ctypes.c_double, "float": ctypes.c_float}
    decls = re.findall(r"\b(?:int|const char\*)\s+(game_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src)
    checked = 0
    for name, args in decls:
        args = args.strip()
        if args in ("", "void"):
            continue
        for arg, ct in zip(args.split(","), getattr(lib, name).argtypes):
            words = arg.split()
            if "*" in arg or words[0] in ("game_t", "game_batch_t"):
                # pointers and handles: a pointer type, not an integer
                assert ctypes.sizeof(ct) == ctypes.sizeof(ctypes.c_void_p), (name, arg)
                assert ct not in scalar.values(), (name, arg)
            else:
                assert ct is scalar[words[-2]], (name, arg, ct)
            checked += 1
    assert checked > 60
