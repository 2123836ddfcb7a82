"""The oracle's ctypes declarations against the C definitions they call: every
exported oracle_* function of ising_oracle.c is declared in oracle.lib() with
the same parameter count, pointer-or-scalar kind and scalar width, and the
same return type.  A mismatch would silently truncate a seed or shift every
later argument."""
import ctypes
import os
import re

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCALAR = {"int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32, "int64_t": ctypes.c_int64,
          "uint64_t": ctypes.c_uint64, "int": ctypes.c_int, "double": ctypes.c_double}
RET = {"void": None, "int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
       "uint32_t": ctypes.c_uint32}


def _definitions():
    src = open(os.path.join(ROOT, "oracle", "ising_oracle.c")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for m in re.finditer(r"^(void|int|int32_t|int64_t|uint32_t)\s+(oracle_\w+)\(([^)]*)\)\s*\{", src, flags=re.M):
        yield m.group(1), m.group(2), [p.strip() for p in " ".join(m.group(3).split()).split(",")]


def test_oracle_ctypes_declarations_match_the_c_definitions():
    L = oracle.lib()
    names = []
    for ret, name, params in _definitions():
        names.append(name)
        fn = getattr(L, name)
        assert fn.restype is RET[ret], (name, fn.restype)
        assert len(fn.argtypes) == len(params), (name, params)
        for p, t in zip(params, fn.argtypes):
            pointer = "*" in p or "[" in p
            if pointer:
                assert t is ctypes.c_void_p or issubclass(t, ctypes._Pointer), (name, p, t)
            else:
                base = re.sub(r"\s*\b\w+$", "", p).replace("const ", "").strip()
                assert t is SCALAR[base], (name, p, t)
    assert {"oracle_anneal", "oracle_anneal_bits", "oracle_anneal_trace", "oracle_anneal_graph", "oracle_cut",
            "oracle_energy", "oracle_thresholds", "oracle_thresholds16", "oracle_draw",
            "oracle_philox4x32_10"} <= set(names)
