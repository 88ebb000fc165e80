"""The oracle's ctypes signatures match oracle.h: the same functions, each
argument of the declared width and kind (integers of the declared width,
doubles, pointers as pointer types), and the declared return width, so the
oracle receives the sizes and values the tests give it."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCALAR = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
          "uint32_t": ctypes.c_uint32, "double": ctypes.c_double, "float": ctypes.c_float}


def test_oracle_signatures_match_the_header(orc):
    src = open(os.path.join(ROOT, "oracle", "oracle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"^(int64_t|int|double|void)\s+(oracle_[a-z_0-9]+)\s*\(([^)]*)\)\s*;",
                       src, flags=re.M)
    lib = orc._load()
    assert len(decls) == 21
    for ret, name, args in decls:
        fn = getattr(lib, name)
        want_ret = {"int64_t": ctypes.c_int64, "double": ctypes.c_double, "void": None,
                    "int": ctypes.c_int}[ret]
        assert fn.restype is want_ret, name
        args = [a for a in " ".join(args.split()).split(",") if a.strip()]
        assert len(fn.argtypes) == len(args), name
        for arg, ct in zip(args, fn.argtypes):
            words = arg.split()
            if "*" in arg or "[" in arg:
                assert ctypes.sizeof(ct) == ctypes.sizeof(ctypes.c_void_p), (name, arg)
                assert ct not in SCALAR.values(), (name, arg)
            else:
                assert ct is SCALAR[words[-2]], (name, arg, ct)
