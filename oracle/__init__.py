"""CPU oracle for the toroidal Ising / Max-Cut annealer.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing on the product
path imports this package, and it imports nothing from the product package.

Two layers:

* ``ising_oracle.c`` (loaded through ctypes): Philox4x32-10, the per-sweep
  acceptance thresholds, the sequential Metropolis annealer on a CSR graph,
  Eq. 1 cut and Eq. 2 energy.
* plain numpy / Python below: Eq. 1 and Eq. 2 over an edge list, brute-force
  enumeration of tiny instances, the exact Boltzmann distribution, and the
  campaign statistics of Eq. 3-5.

Each function cites the passage of Zick 2025 ("Performance report of
heuristic algorithm that cracked the largest Gset Ising problems") or of
Salmon et al. 2011 (Philox) that it follows.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building on first use) the C oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_thresholds.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_thresholds.restype = ctypes.c_int
        L.oracle_cut.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_cut.restype = ctypes.c_int32
        L.oracle_energy.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_energy.restype = ctypes.c_int64
        L.oracle_anneal.argtypes = [
            ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,  # n, row_ptr, col, J
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,                      # X, t_begin, t_count
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,   # betas, S, seed, offset
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,   # init, spins, cuts, check
        ]
        L.oracle_anneal.restype = ctypes.c_int
        L.oracle_anneal_bits.argtypes = L.oracle_anneal.argtypes + [ctypes.c_int32]   # + draw_bits
        L.oracle_anneal_bits.restype = ctypes.c_int
        L.oracle_anneal_trace.argtypes = L.oracle_anneal_bits.argtypes + [
            ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]   # trace_every, trace, best, best spins
        L.oracle_anneal_trace.restype = ctypes.c_int
        L.oracle_greedy_colouring.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_greedy_colouring.restype = ctypes.c_int32
        L.oracle_energy_h.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 5
        L.oracle_energy_h.restype = ctypes.c_int64
        L.oracle_anneal_graph.argtypes = [
            ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,   # n, rp, col, J, h
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,                     # colour, ncol, t0, tc
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,                   # betas, S, seed, off
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]                   # init, spins, cuts, chk
        L.oracle_anneal_graph.restype = ctypes.c_int
        L.oracle_thresholds16.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_thresholds16.restype = ctypes.c_int
        L.oracle_draw.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32]
        L.oracle_draw.restype = ctypes.c_uint32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al. 2011) and the thresholds
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr = 4 uint32, key = 2 uint32 -> 4 uint32."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def thresholds(betas, draw_bits=32):
    """(T4, T8) uint32 arrays: T_d = min(floor(exp(-beta d) 2^B), 2^B - 1),
    B = draw_bits (32, or 16 for the 16-bit draw mode)."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    S = b.shape[0]
    T4 = np.zeros(S, dtype=np.uint32)
    T8 = np.zeros(S, dtype=np.uint32)
    fn = lib().oracle_thresholds16 if draw_bits == 16 else lib().oracle_thresholds
    rc = fn(_ptr(b), S, _ptr(T4), _ptr(T8))
    if rc != 0:
        raise ValueError("inverse temperatures must be positive")
    return T4, T8


def decision_draw(i, k, t, seed, draw_bits=32):
    """The uniform draw of trial t at site i in sweep k (32- or 16-bit mode)."""
    return int(lib().oracle_draw(int(i) & 0xFFFFFFFF, int(k) & 0xFFFFFFFF, int(t),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, int(draw_bits)))


# --------------------------------------------------------------------------
# The annealer (C) and Eq. 1 / Eq. 2 on the CSR (C)
# --------------------------------------------------------------------------
def anneal(inst, betas, seed, trials=None, t_begin=0, t_count=None, sweep_offset=0,
           init=None, check_fields=False, draw_bits=32):
    """Run the sequential Metropolis annealer on the CSR instance ``inst``.

    Trials t_begin .. t_begin+t_count-1 (global indices select the random
    stream).  draw_bits: 32 (the default stream) or 16 (the 16-bit draw
    mode).  Returns (spins int8 [t_count, n], cuts int32 [t_count]).
    """
    if t_count is None:
        t_count = trials if trials is not None else 0
    n = int(inst["n"])
    row_ptr = np.ascontiguousarray(inst["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(inst["col"], dtype=np.int32)
    J = np.ascontiguousarray(inst["J"], dtype=np.int8)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    spins = np.zeros((t_count, n), dtype=np.int8)
    cuts = np.zeros(t_count, dtype=np.int32)
    ini = None
    if init is not None:
        ini = np.ascontiguousarray(init, dtype=np.int8)
        assert ini.shape == (t_count, n)
    rc = lib().oracle_anneal_bits(n, _ptr(row_ptr), _ptr(col), _ptr(J), int(inst["X"]),
                                  int(t_begin), int(t_count), _ptr(b), int(b.shape[0]),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(sweep_offset) & 0xFFFFFFFF,
                                  _ptr(ini), _ptr(spins), _ptr(cuts), 1 if check_fields else 0,
                                  int(draw_bits))
    if rc == -3:
        raise AssertionError("incremental local fields diverged from recomputed fields")
    if rc != 0:
        raise ValueError(f"oracle_anneal failed with code {rc}")
    return spins, cuts


def anneal_trace(inst, betas, seed, trace_every, t_begin=0, t_count=0, sweep_offset=0, init=None,
                 draw_bits=32):
    """The annealer with read-out along the trajectory: after every sweep j
    (from 1) that is a multiple of trace_every, and after the last sweep, the
    Eq. 1 cut of every trial; the best of those cuts per trial and the first
    configuration reaching it.  Returns (spins, cuts, trace int32 [points,
    t_count], best int32 [t_count], best_spins int8 [t_count, n])."""
    n = int(inst["n"])
    b = np.ascontiguousarray(betas, dtype=np.float64)
    S = int(b.shape[0])
    points = (S + trace_every - 1) // trace_every
    spins = np.zeros((t_count, n), dtype=np.int8)
    cuts = np.zeros(t_count, dtype=np.int32)
    trace = np.zeros((points, t_count), dtype=np.int32)
    best = np.zeros(t_count, dtype=np.int32)
    best_spins = np.zeros((t_count, n), dtype=np.int8)
    ini = None if init is None else np.ascontiguousarray(init, dtype=np.int8)
    rc = lib().oracle_anneal_trace(n, _ptr(np.ascontiguousarray(inst["row_ptr"], dtype=np.int64)),
                                   _ptr(np.ascontiguousarray(inst["col"], dtype=np.int32)),
                                   _ptr(np.ascontiguousarray(inst["J"], dtype=np.int8)), int(inst["X"]),
                                   int(t_begin), int(t_count), _ptr(b), S, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                   int(sweep_offset) & 0xFFFFFFFF, _ptr(ini), _ptr(spins), _ptr(cuts), 0,
                                   int(draw_bits), int(trace_every), _ptr(trace), _ptr(best), _ptr(best_spins))
    if rc != 0:
        raise ValueError(f"oracle_anneal_trace failed with code {rc}")
    return spins, cuts, trace, best, best_spins


# --------------------------------------------------------------------------
# General sparse graphs (integer J, fields h): Eq. 2 in full
# --------------------------------------------------------------------------
def _graph_arrays(g):
    rp = np.ascontiguousarray(g["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(g["col"], dtype=np.int32)
    J = np.ascontiguousarray(g["J"], dtype=np.int8)
    h = None if g.get("h") is None else np.ascontiguousarray(g["h"], dtype=np.int8)
    return rp, col, J, h


def greedy_colouring(g):
    """First-fit colouring in index order: (colour int32 [n], number of colours)."""
    rp, col, _, _ = _graph_arrays(g)
    colour = np.zeros(int(g["n"]), dtype=np.int32)
    k = lib().oracle_greedy_colouring(int(g["n"]), _ptr(rp), _ptr(col), _ptr(colour))
    if k < 0:
        raise ValueError("colouring failed")
    return colour, int(k)


def energy_h(g, spins):
    """Eq. 2 with fields: H = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i."""
    rp, col, J, h = _graph_arrays(g)
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().oracle_energy_h(int(g["n"]), _ptr(rp), _ptr(col), _ptr(J), _ptr(h), _ptr(s)))


def anneal_graph(g, betas, seed, t_count, t_begin=0, sweep_offset=0, init=None, colour=None,
                 check_fields=False):
    """The Metropolis annealer on a general graph, colour classes in order
    (first-fit colouring unless given).  Returns (spins, cuts)."""
    rp, col, J, h = _graph_arrays(g)
    n = int(g["n"])
    if colour is None:
        colour, ncol = greedy_colouring(g)
    else:
        colour = np.ascontiguousarray(colour, dtype=np.int32)
        ncol = int(colour.max()) + 1 if n else 0
    b = np.ascontiguousarray(betas, dtype=np.float64)
    spins = np.zeros((t_count, n), dtype=np.int8)
    cuts = np.zeros(t_count, dtype=np.int32)
    ini = None if init is None else np.ascontiguousarray(init, dtype=np.int8)
    rc = lib().oracle_anneal_graph(n, _ptr(rp), _ptr(col), _ptr(J), _ptr(h), _ptr(colour), ncol,
                                   int(t_begin), int(t_count), _ptr(b), int(b.shape[0]),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, int(sweep_offset) & 0xFFFFFFFF,
                                   _ptr(ini), _ptr(spins), _ptr(cuts), 1 if check_fields else 0)
    if rc == -3:
        raise AssertionError("incremental local fields diverged from recomputed fields")
    if rc != 0:
        raise ValueError(f"oracle_anneal_graph failed with code {rc}")
    return spins, cuts


def cut_csr(inst, spins):
    """Eq. 1 evaluated on the CSR (C): cut of one configuration."""
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().oracle_cut(int(inst["n"]), _ptr(np.ascontiguousarray(inst["row_ptr"], dtype=np.int64)),
                                _ptr(np.ascontiguousarray(inst["col"], dtype=np.int32)),
                                _ptr(np.ascontiguousarray(inst["J"], dtype=np.int8)), _ptr(s)))


def energy_csr(inst, spins):
    """Eq. 2 (h = 0) evaluated on the CSR (C)."""
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().oracle_energy(int(inst["n"]), _ptr(np.ascontiguousarray(inst["row_ptr"], dtype=np.int64)),
                                   _ptr(np.ascontiguousarray(inst["col"], dtype=np.int32)),
                                   _ptr(np.ascontiguousarray(inst["J"], dtype=np.int8)), _ptr(s)))


# --------------------------------------------------------------------------
# numpy layer: edge lists, Eq. 1 / Eq. 2, brute force, Boltzmann
# --------------------------------------------------------------------------
def torus_edges(X, Y, w_right, w_down):
    """Edge list (i, j, w) of the torus: each site's right and down edge."""
    ii, jj, ww = [], [], []
    for y in range(Y):
        for x in range(X):
            i = y * X + x
            ii.append(i); jj.append(y * X + (x + 1) % X); ww.append(int(w_right[y, x]))
            ii.append(i); jj.append(((y + 1) % Y) * X + x); ww.append(int(w_down[y, x]))
    return np.array(ii), np.array(jj), np.array(ww, dtype=np.int64)


def cut_eq1(edges, x):
    """Eq. 1: 1/2 sum_{edges} w_ij (1 - x_i x_j), x in {-1,+1} (batched on x)."""
    i, j, w = edges
    x = np.asarray(x, dtype=np.int64)
    return (w * (1 - x[..., i] * x[..., j])).sum(axis=-1) // 2


def energy_eq2(edges, s):
    """Eq. 2 with J = -w, h = 0: H = -sum J_ij s_i s_j = sum w_ij s_i s_j."""
    i, j, w = edges
    s = np.asarray(s, dtype=np.int64)
    J = -w
    return -(J * s[..., i] * s[..., j]).sum(axis=-1)


def all_states(n):
    """All 2^n configurations as int8 [2^n, n] in {-1,+1} (n <= 20)."""
    assert n <= 20
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8)


def brute_force(edges, n):
    """Exhaustive search: (min energy, max cut, energies of all states)."""
    S = all_states(n)
    E = energy_eq2(edges, S)
    C = cut_eq1(edges, S)
    return int(E.min()), int(C.max()), E, C


def boltzmann(energies, beta):
    """Exact Boltzmann weights exp(-beta E)/Z over an enumerated state space."""
    e = np.asarray(energies, dtype=np.float64)
    a = -beta * (e - e.min())
    p = np.exp(a)
    return p / p.sum()


# --------------------------------------------------------------------------
# Campaign statistics: Eq. 3 (repetitions), Eq. 4 (STT), Eq. 5 (TTT)
# --------------------------------------------------------------------------
def repetitions(Ps):
    """Eq. 3: r = max(1, log(1 - 0.99) / log(1 - P_s)).

    P_s = 1 gives r = 1; P_s = 0 gives inf (target not reached).
    """
    Ps = float(Ps)
    if Ps >= 1.0:
        return 1.0
    if Ps <= 0.0:
        return math.inf
    return max(1.0, math.log(1.0 - 0.99) / math.log(1.0 - Ps))


def sweeps_to_target(S_trial, Ps):
    """Eq. 4: STT = S_trial * r."""
    return S_trial * repetitions(Ps)


def time_to_target(t_trial, Ps):
    """Eq. 5: TTT = t_trial * r, t_trial the average time per trial."""
    return t_trial * repetitions(Ps)


def success_probability(cuts, target):
    """Fraction of trials whose cut reaches the target (Section III)."""
    c = np.asarray(cuts)
    return float((c >= target).sum()) / float(max(1, c.size))


def target_cut(best, quality=0.999):
    """Smallest integer cut at or above quality * best (Table I writes the
    99.9% targets as real thresholds, e.g. >= 14045.94 for best 14060)."""
    return int(math.ceil(quality * best - 1e-9))
