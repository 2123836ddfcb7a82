"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad instances before touching CUDA."""
import ctypes

import numpy as np
import pytest

import synth
from paper_2505_18508_gb300 import _abi
from paper_2505_18508_gb300 import build as lib_build


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return _abi.lib()


def test_every_declared_symbol_is_exported(L):
    names = _abi.declared_symbols()
    assert {"ising_create", "ising_destroy", "ising_anneal", "ising_anneal_batched", "ising_cut",
            "ising_strerror"} <= set(names)
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(_abi._SIGNATURES), "binding and header disagree"


def test_strerror_names_every_code(L):
    for code in range(0, -9, -1):
        msg = L.ising_strerror(code).decode()
        assert msg and msg != "unknown status code"
    assert L.ising_strerror(-99).decode() == "unknown status code"


def _create(L, inst, X=None, Y=None, n=None, h=None, J=None, col=None, row_ptr=None):
    X = inst["X"] if X is None else X
    Y = inst["Y"] if Y is None else Y
    n = inst["n"] if n is None else n
    rp = np.ascontiguousarray(inst["row_ptr"] if row_ptr is None else row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(inst["col"] if col is None else col, dtype=np.int32)
    JJ = np.ascontiguousarray(inst["J"] if J is None else J, dtype=np.int8)
    hp = None
    if h is not None:
        h = np.ascontiguousarray(h, dtype=np.int8)
        hp = h.ctypes.data_as(ctypes.c_void_p)
    out = ctypes.c_void_p()
    rc = L.ising_create(n, rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                        JJ.ctypes.data_as(ctypes.c_void_p), hp, X, Y, ctypes.byref(out))
    return rc, out


def test_create_rejects_bad_instances(L):
    inst = synth.torus_instance(6, 4, 1)
    # shape mismatch / tiny / odd
    assert _create(L, inst, n=23)[0] == _abi.ISING_ERR_ARG
    small = synth.torus_instance(2, 4, 1)
    assert _create(L, small)[0] == _abi.ISING_ERR_ARG
    odd = synth.torus_instance(5, 4, 1)
    assert _create(L, odd)[0] == _abi.ISING_ERR_ODD_DIM
    odd2 = synth.torus_instance(6, 5, 1)
    assert _create(L, odd2)[0] == _abi.ISING_ERR_ODD_DIM
    # weights must be +-1
    J = inst["J"].copy(); J[3] = 2
    assert _create(L, inst, J=J)[0] == _abi.ISING_ERR_ARG
    J = inst["J"].copy(); J[5] = 0
    assert _create(L, inst, J=J)[0] == _abi.ISING_ERR_ARG
    # asymmetric coupling
    J = inst["J"].copy(); J[0] = -J[0]
    assert _create(L, inst, J=J)[0] == _abi.ISING_ERR_NOT_TORUS
    # a wrong neighbour
    col = inst["col"].copy(); col[0] = (col[0] + 2) % inst["n"]
    assert _create(L, inst, col=col)[0] == _abi.ISING_ERR_NOT_TORUS
    # a row with 5 entries
    rp = inst["row_ptr"].copy(); rp[1] += 1
    assert _create(L, inst, row_ptr=rp)[0] == _abi.ISING_ERR_NOT_TORUS
    # non-zero h
    h = np.zeros(inst["n"], dtype=np.int8); h[7] = 1
    assert _create(L, inst, h=h)[0] == _abi.ISING_ERR_H_UNSUPPORTED
    # wrong shape given for a valid CSR (a 6x4 torus is not a 4x6 torus)
    assert _create(L, inst, X=4, Y=6)[0] == _abi.ISING_ERR_NOT_TORUS
    # NULL pointers
    out = ctypes.c_void_p()
    assert L.ising_create(24, None, None, None, None, 6, 4, ctypes.byref(out)) == _abi.ISING_ERR_ARG


def test_null_handles_are_rejected(L):
    assert L.ising_anneal(None, 1, None, 0, 0, 0, None, None, None, None) == _abi.ISING_ERR_ARG
    assert L.ising_cut(None, None, 0, None, None) == _abi.ISING_ERR_ARG
    assert L.ising_set_launch(None, 0, 0, 0) == _abi.ISING_ERR_ARG
    L.ising_destroy(None)


def test_valid_instance_without_gpu_reports_cuda_error(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    inst = synth.torus_instance(8, 6, 2)
    rc, _ = _create(L, inst)
    assert rc == _abi.ISING_ERR_CUDA


def test_synthetic_instances_are_tori():
    for X, Y in ((4, 4), (8, 6), (200, 100)):
        inst = synth.torus_instance(X, Y, 9)
        n = X * Y
        assert inst["row_ptr"][-1] == 4 * n
        assert set(np.unique(inst["J"])) <= {-1, 1}
        # symmetric
        rp, col, J = inst["row_ptr"], inst["col"], inst["J"]
        d = {}
        for i in range(n):
            for e in range(rp[i], rp[i + 1]):
                d[(i, int(col[e]))] = int(J[e])
        assert all(d[(j, i)] == v for (i, j), v in d.items())
    b = synth.linear_betas(0.1, 3.0, 10000)
    assert b[0] == 0.1 and abs(b[-1] - 3.0) < 1e-12 and b.shape == (10000,)
    assert synth.linear_betas(0.5, 3.0, 1).tolist() == [0.5]
    cfg = synth.batched_config()
    assert len(cfg) == 96 and {c["X"] for c in cfg} == {50, 100, 140, 200}
    assert min(c["trials"] for c in cfg) == 32 and max(c["trials"] for c in cfg) == 512
    assert min(c["sweeps"] for c in cfg) >= 2000 and max(c["sweeps"] for c in cfg) <= 20000


def test_every_status_returning_entry_point_documents_its_errors():
    """Each int-returning declaration of include/ising.h is preceded by a
    comment that states its error codes (a declaration directly after another
    shares that one's comment)."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ising.h")
    src = open(path).read()
    decls = list(re.finditer(r"\n(int|void|const char\*|size_t)\s+(ising_\w+)\(", src))
    missing, prev_end, prev_comment = [], 0, ""
    for m in decls:
        between = src[prev_end:m.start()]
        start = between.rfind("/*")
        comment = between[start:] if start >= 0 else prev_comment
        if m.group(1) == "int" and "rrors" not in comment:
            missing.append(m.group(2))
        prev_end, prev_comment = m.end(), comment
    assert len(decls) >= 40
    assert not missing, missing


def test_binding_signatures_match_the_header():
    """Every parameter of every declaration in include/ising.h has the width
    the ctypes table passes (pointers as pointers, int32_t as a 32-bit int,
    uint64_t as a 64-bit unsigned, size_t, float), and the return types agree."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ising.h")
    src = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    scalar = {"int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32, "int64_t": ctypes.c_int64,
              "uint64_t": ctypes.c_uint64, "size_t": ctypes.c_size_t, "float": ctypes.c_float, "int": ctypes.c_int,
              "double": ctypes.c_double}
    rets = {"int": ctypes.c_int, "void": None, "size_t": ctypes.c_size_t, "const char*": ctypes.c_char_p}
    seen = 0
    for m in re.finditer(r"\n(int|void|const char\*|size_t)\s+(ising_\w+)\(([^)]*)\);", src):
        ret, name, params = m.group(1), m.group(2), " ".join(m.group(3).split())
        want_ret, argtypes = _abi._SIGNATURES[name]
        assert want_ret is rets[ret], name
        params = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        assert len(params) == len(argtypes), (name, params)
        for p, t in zip(params, argtypes):
            ctype = re.sub(r"\s*\b\w+$", "", p) if not p.endswith("*") else p
            if "*" in ctype:
                ok = t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer)
                if t is ctypes.c_char_p:
                    ok = ok and "char" in ctype
                assert ok, (name, p, t)
            else:
                base = ctype.replace("const ", "").strip()
                assert t is scalar[base], (name, p, t)
        seen += 1
    assert seen == len(_abi._SIGNATURES)
