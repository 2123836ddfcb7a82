"""ctypes binding of include/ising.h: the same names, argument marshalling only.

Loading fails loudly when libising.so has not been built; there is no other
implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("ISING_LIBRARY") or os.path.join(HERE, "_build", "libising.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ising.h")

ISING_OK = 0
ISING_ERR_ARG = -1
ISING_ERR_NOT_TORUS = -2
ISING_ERR_ODD_DIM = -3
ISING_ERR_H_UNSUPPORTED = -4
ISING_ERR_OOM = -5
ISING_ERR_CUDA = -6
ISING_ERR_TIMEOUT = -7
ISING_ERR_UNSUPPORTED = -8

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i32p = ctypes.POINTER(ctypes.c_int32)

_SIGNATURES = {
    "ising_create": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.POINTER(_vp)]),
    "ising_destroy": (None, [_vp]),
    "ising_anneal": (ctypes.c_int, [_vp, _i32, _vp, _i32, _u64, _u32, _vp, _vp, _vp, _vp]),
    "ising_cut": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "ising_anneal_trace": (ctypes.c_int, [_vp, _i32, _vp, _i32, _u64, _u32, _vp, _vp, _vp, _i32, _vp, _vp, _vp,
                                          _vp]),
    "ising_anneal_noalloc": (ctypes.c_int, [_vp, _i32, _vp, _i32, _u64, _u32, _vp, _vp, _vp, _vp]),
    "ising_anneal_batched": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "ising_batch_create": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp,
                                          ctypes.POINTER(_vp)]),
    "ising_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "ising_batch_destroy": (None, [_vp]),
    "ising_set_launch": (ctypes.c_int, [_vp, _i32, _i32, _i32]),
    "ising_last_launch": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p, _i32p]),
    "ising_problem_info": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "ising_set_kernel": (ctypes.c_int, [_vp, _i32]),
    "ising_set_graph_threads_per_site": (ctypes.c_int, [_vp, _i32]),
    "ising_thresholds": (ctypes.c_int, [_vp, _i32, _i32, _vp]),
    "ising_flow_split": (ctypes.c_int, [_i32, _i32, _i32, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp]),
    "ising_batch_schedule": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp,
                                            _vp, _i32, _vp]),
    "ising_set_draw_bits": (ctypes.c_int, [_vp, _i32]),
    "ising_graph_create": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "ising_greedy_colouring": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp]),
    "ising_graph_info": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "ising_energy": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "ising_philox": (ctypes.c_int, [_vp, _u64, _i32, _vp, _vp]),
    "ising_spins_to_hex": (ctypes.c_int, [_vp, _i32, _vp, ctypes.c_int64]),
    "ising_hex_to_spins": (ctypes.c_int, [ctypes.c_char_p, _i32, _vp]),
    "ising_debug_fail_allocs": (ctypes.c_int, [_i32]),
    "ising_anneal_pt": (ctypes.c_int, [_vp, _i32, _vp, _i32, _i32, _i32, _u64, _vp, _vp, _vp, _vp]),
    "ising_last_kernel": (ctypes.c_int, [_vp, _i32p]),
    "ising_get_status": (ctypes.c_int, [_vp, _vp, _i32p]),
    "ising_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int64, _i32]),
    "ising_cnn_create": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "ising_cnn_destroy": (None, [_vp]),
    "ising_cnn_get_params": (ctypes.c_int, [_vp, _vp]),
    "ising_cnn_set_params": (ctypes.c_int, [_vp, _vp]),
    "ising_cnn_workspace_bytes": (ctypes.c_size_t, [_i32, _i32, _i32]),
    "ising_cnn_forward": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp, ctypes.c_size_t, _vp]),
    "ising_cnn_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "ising_cnn_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int64, _i32]),
    "ising_cnn_adam_step": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_float, _vp]),
    "ising_propose": (ctypes.c_int, [_vp, _vp, _i32, _vp, _i32, _vp, _vp]),
    "ising_flip_targets": (ctypes.c_int, [_vp, _vp, _i32, _i32, _vp, _vp]),
    "ising_propose_clusters": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _vp, _vp]),
    "ising_droplet_targets": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "ising_transcribe": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32, _i32, _vp, _vp]),
    "ising_learned_create": (ctypes.c_int, [_vp, _i32, _i32, _vp, _i32, _vp, _i32, _i32, _vp, _i32, _i32, _vp, _vp,
                                            _vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "ising_learned_launch": (ctypes.c_int, [_vp, _vp]),
    "ising_learned_destroy": (None, [_vp]),
    "ising_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


class IsingError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "unknown"
        try:
            msg = lib().ising_strerror(code).decode()
        except Exception:  # pragma: no cover
            pass
        super().__init__(f"{where} failed: {msg} (code {code})")


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != ISING_OK:
        raise IsingError(code, where)


def declared_symbols():
    """Names of the functions include/ising.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ising_[a-z_]+)\s*\(", text)))
