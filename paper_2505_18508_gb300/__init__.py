"""GB300 toroidal Ising / Max-Cut annealer: Python binding of include/ising.h.

Every step of the annealing path runs in the CUDA kernels of libising.so;
this module only marshals arguments.  PyTorch provides device memory and the
current CUDA stream.  Output tensors (and contiguous copies of inputs) are
allocated on the current stream; a caller that passes another `stream`
orders the two streams itself (for example with `stream.wait_stream`) and
keeps the tensors alive until that stream's work is done.

    import paper_2505_18508_gb300 as ia
    prob = ia.Problem.from_csr(n, row_ptr, col, J, X, Y)
    spins, cuts = ia.anneal(prob, trials=1024, betas=betas, seed=1002)

The method (Zick 2025, Sections II-III): independent trials of sweeps on the
Ising form of a toroidal Max-Cut instance (J = -w, h = 0), read out at the
end of each trial, with the exact cut of Eq. 1.  Each sweep is a Metropolis
sweep over the two checkerboard colours with Philox4x32-10 draws.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import IsingError, check, lib

__all__ = ["Problem", "anneal", "anneal_trace", "cut", "energy", "greedy_colouring", "anneal_batched", "BatchPlan",
           "IsingError", "lib", "spins_to_hex", "hex_to_spins", "philox", "anneal_pt", "thresholds"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _device_tensor(t, dtype, shape, name, write=False):
    """The C ABI takes raw device pointers: check that `t` is a tensor on the
    current CUDA device with this dtype and shape (None: any), before any
    pointer reaches a kernel.  Inputs are made contiguous; tensors the call
    writes into (write=True) must already be.  Raises ValueError."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be on the current CUDA device, got {t.device}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: must be on the current CUDA device (cuda:{torch.cuda.current_device()}), "
                         f"got {t.device}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if shape is not None and tuple(t.shape) != tuple(int(v) for v in shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(int(v) for v in shape)}")
    if not t.is_contiguous():
        if write:
            raise ValueError(f"{name}: written in place, so it must be contiguous")
        t = t.contiguous()
    return t


def _rows(t, name):
    """Row count of a 2-D tensor argument (checked before use)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dim() != 2:
        raise ValueError(f"{name}: expected a 2-D tensor [rows, sites]")
    return int(t.shape[0])


class Problem:
    """A validated instance packed on the current CUDA device: a torus
    (from_csr / from_instance) or a general sparse graph (from_graph)."""

    def __init__(self, handle, X, Y, n=None):
        self._h = handle
        self.X, self.Y = X, Y
        self.n = X * Y if n is None else int(n)

    @classmethod
    def from_graph(cls, g):
        """From a dict with n, row_ptr, col, J and optional h (e.g. synth.random_graph)."""
        row_ptr = np.ascontiguousarray(g["row_ptr"], dtype=np.int64)
        col = np.ascontiguousarray(g["col"], dtype=np.int32)
        J = np.ascontiguousarray(g["J"], dtype=np.int8)
        h = g.get("h")
        hp = None
        if h is not None:
            h = np.ascontiguousarray(h, dtype=np.int8)
            hp = h.ctypes.data_as(ctypes.c_void_p)
        out = ctypes.c_void_p()
        rc = lib().ising_graph_create(int(g["n"]), row_ptr.ctypes.data_as(ctypes.c_void_p),
                                      col.ctypes.data_as(ctypes.c_void_p), J.ctypes.data_as(ctypes.c_void_p),
                                      hp, ctypes.byref(out))
        check(rc, "ising_graph_create")
        return cls(out, 0, 0, n=int(g["n"]))

    def graph_info(self):
        n, k, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().ising_graph_info(self.handle, ctypes.byref(n), ctypes.byref(k), ctypes.byref(d)),
              "ising_graph_info")
        return {"n": n.value, "colours": k.value, "Dmax": d.value}

    @classmethod
    def from_csr(cls, n, row_ptr, col, J, X, Y, h=None):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        J = np.ascontiguousarray(J, dtype=np.int8)
        hp = None
        if h is not None:
            h = np.ascontiguousarray(h, dtype=np.int8)
            hp = h.ctypes.data_as(ctypes.c_void_p)
        out = ctypes.c_void_p()
        rc = lib().ising_create(int(n), row_ptr.ctypes.data_as(ctypes.c_void_p),
                                col.ctypes.data_as(ctypes.c_void_p), J.ctypes.data_as(ctypes.c_void_p),
                                hp, int(X), int(Y), ctypes.byref(out))
        check(rc, "ising_create")
        return cls(out, int(X), int(Y))

    @classmethod
    def from_instance(cls, inst):
        """From a dict with n, row_ptr, col, J, X, Y (e.g. synth.torus_instance)."""
        return cls.from_csr(inst["n"], inst["row_ptr"], inst["col"], inst["J"], inst["X"], inst["Y"])

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("problem already destroyed")
        return self._h

    def info(self):
        X, Y, W = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().ising_problem_info(self.handle, ctypes.byref(X), ctypes.byref(Y), ctypes.byref(W)),
              "ising_problem_info")
        return {"X": X.value, "Y": Y.value, "weight_sum": W.value}

    def set_launch(self, group_trials=0, strips=0, threads=0):
        check(lib().ising_set_launch(self.handle, int(group_trials), int(strips), int(threads)),
              "ising_set_launch")

    def set_draw_bits(self, bits):
        """32 (default decision stream) or 16 (one Philox block per eight trials)."""
        check(lib().ising_set_draw_bits(self.handle, int(bits)), "ising_set_draw_bits")

    def set_kernel(self, kind):
        """0 automatic, 1 cluster-strip kernel, 2 persistent kernel."""
        check(lib().ising_set_kernel(self.handle, int(kind)), "ising_set_kernel")

    def set_graph_threads_per_site(self, tpw):
        """General graphs: threads that share one site word's update (1, 4 or
        8; 0 automatic)."""
        check(lib().ising_set_graph_threads_per_site(self.handle, int(tpw)), "ising_set_graph_threads_per_site")

    def last_kernel(self):
        v = ctypes.c_int32()
        check(lib().ising_last_kernel(self.handle, ctypes.byref(v)), "ising_last_kernel")
        return v.value

    def get_status(self, stream=None):
        """Wait for the stream, then read and clear the device status word."""
        v = ctypes.c_int32()
        check(lib().ising_get_status(self.handle, _stream_ptr(stream), ctypes.byref(v)), "ising_get_status")
        return v.value

    def set_wait_limit(self, cycles=0, stall_test=0):
        check(lib().ising_set_wait_limit(self.handle, int(cycles), int(stall_test)), "ising_set_wait_limit")

    def last_launch(self):
        v = [ctypes.c_int32() for _ in range(4)]
        check(lib().ising_last_launch(self.handle, *[ctypes.byref(x) for x in v]), "ising_last_launch")
        return {"group_trials": v[0].value, "strips": v[1].value, "threads": v[2].value,
                "grid_ctas": v[3].value}

    def destroy(self):
        if self._h is not None:
            lib().ising_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def anneal(prob, trials, betas, seed, sweep_offset=0, init=None, out_spins=None, out_cuts=None,
           want_spins=True, stream=None):
    """Queue ``trials`` trials of len(betas) sweeps; returns (spins, cuts) CUDA tensors.

    init: optional int8 CUDA tensor [trials, n] of starting spins.
    out_spins / out_cuts: optional preallocated CUDA tensors to write into.
    """
    torch = _torch()
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    dev = torch.device("cuda", torch.cuda.current_device())
    if want_spins and out_spins is None:
        out_spins = torch.empty((trials, prob.n), dtype=torch.int8, device=dev)
    elif want_spins:
        out_spins = _device_tensor(out_spins, torch.int8, (trials, prob.n), "out_spins", write=True)
    if out_cuts is None:
        out_cuts = torch.empty((trials,), dtype=torch.int32, device=dev)
    else:
        out_cuts = _device_tensor(out_cuts, torch.int32, (trials,), "out_cuts", write=True)
    if init is not None:
        init = _device_tensor(init, torch.int8, (trials, prob.n), "init")
    rc = lib().ising_anneal(prob.handle, int(trials), betas.ctypes.data_as(ctypes.c_void_p),
                            int(betas.shape[0]), int(seed) & 0xFFFFFFFFFFFFFFFF,
                            int(sweep_offset) & 0xFFFFFFFF, _dptr(init),
                            _dptr(out_spins) if want_spins else None, _dptr(out_cuts), _stream_ptr(stream))
    check(rc, "ising_anneal")
    return out_spins, out_cuts


def anneal_trace(prob, trials, betas, seed, trace_every, sweep_offset=0, init=None, want_best_spins=True,
                 stream=None):
    """ising_anneal with read-out along the trajectory: returns (spins, cuts,
    trace [points, trials], best [trials], best_spins [trials, n] or None) as
    CUDA tensors; trace row p holds every trial's cut after sweep
    min((p + 1) * trace_every, S) of the call."""
    torch = _torch()
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    S = int(betas.shape[0])
    points = (S + int(trace_every) - 1) // int(trace_every) if trace_every > 0 else 0
    dev = torch.device("cuda", torch.cuda.current_device())
    spins = torch.empty((trials, prob.n), dtype=torch.int8, device=dev)
    cuts = torch.empty((trials,), dtype=torch.int32, device=dev)
    trace = torch.empty((max(points, 0), trials), dtype=torch.int32, device=dev)
    best = torch.empty((trials,), dtype=torch.int32, device=dev)
    best_spins = torch.empty((trials, prob.n), dtype=torch.int8, device=dev) if want_best_spins else None
    if init is not None:
        init = _device_tensor(init, torch.int8, (trials, prob.n), "init")
    rc = lib().ising_anneal_trace(prob.handle, int(trials), betas.ctypes.data_as(ctypes.c_void_p), S,
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(sweep_offset) & 0xFFFFFFFF, _dptr(init),
                                  _dptr(spins), _dptr(cuts), int(trace_every), _dptr(trace) if points else None,
                                  _dptr(best), _dptr(best_spins), _stream_ptr(stream))
    check(rc, "ising_anneal_trace")
    return spins, cuts, trace, best, best_spins


def greedy_colouring(g):
    """The first-fit colouring the general-graph sweep uses (host only)."""
    row_ptr = np.ascontiguousarray(g["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(g["col"], dtype=np.int32)
    colour = np.zeros(int(g["n"]), dtype=np.int32)
    k = ctypes.c_int32()
    check(lib().ising_greedy_colouring(int(g["n"]), row_ptr.ctypes.data_as(ctypes.c_void_p),
                                       col.ctypes.data_as(ctypes.c_void_p), colour.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(k)), "ising_greedy_colouring")
    return colour, k.value


def anneal_pt(prob, betas, chains, rounds, sweeps_per_round, seed, stream=None):
    """Replica exchange: returns (spins [R*C, n], cuts [R*C], swaps [1]) CUDA
    tensors; slot r * chains + c is chain c at temperature betas[r]."""
    torch = _torch()
    b = np.ascontiguousarray(betas, dtype=np.float64)
    R, T = int(b.shape[0]), int(b.shape[0]) * int(chains)
    dev = torch.device("cuda", torch.cuda.current_device())
    spins = torch.empty((T, prob.n), dtype=torch.int8, device=dev)
    cuts = torch.empty((T,), dtype=torch.int32, device=dev)
    swaps = torch.zeros((1,), dtype=torch.int32, device=dev)
    check(lib().ising_anneal_pt(prob.handle, R, b.ctypes.data_as(ctypes.c_void_p), int(chains), int(rounds),
                                int(sweeps_per_round), int(seed) & 0xFFFFFFFFFFFFFFFF, _dptr(spins), _dptr(cuts),
                                _dptr(swaps), _stream_ptr(stream)), "ising_anneal_pt")
    return spins, cuts, swaps


def spins_to_hex(spins):
    """A configuration (int8 [n], host) as hex digits (the paper's App. C-E form;
    the first spin of each digit in its most significant bit, +1 -> 1)."""
    s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
    buf = ctypes.create_string_buffer((s.shape[0] + 3) // 4 + 1)
    check(lib().ising_spins_to_hex(s.ctypes.data_as(ctypes.c_void_p), int(s.shape[0]), buf, len(buf)),
          "ising_spins_to_hex")
    return buf.value.decode()


def hex_to_spins(hexstr, n):
    """The inverse of spins_to_hex: int8 [n] in {-1, +1}."""
    out = np.zeros(int(n), dtype=np.int8)
    check(lib().ising_hex_to_spins(hexstr.encode(), int(n), out.ctypes.data_as(ctypes.c_void_p)),
          "ising_hex_to_spins")
    return out


def flow_split(Y, X, trials, group_trials=32, draw_bits=32, sms=152, weighted=True):
    """The persistent kernel's division of the stacked site words over its
    CTAs (host only): returns (split int32 [ctas + 1], most local rows of a
    CTA, most trial groups a CTA touches)."""
    cap = int(sms) + 1
    out = np.zeros(cap, dtype=np.int32)
    ctas, lr, seg = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(lib().ising_flow_split(int(Y), int(X) // 2, int(trials), int(group_trials), int(draw_bits), int(sms),
                                 1 if weighted else 0, out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(ctas),
                                 ctypes.byref(lr), ctypes.byref(seg)), "ising_flow_split")
    return out[:ctas.value + 1].copy(), lr.value, seg.value


def batch_schedule(shapes, trials, sweeps, draw_bits=32, group_trials=0, ctas_per_sm=0, sms=152,
                   smem_per_cta_max=0):
    """The batched launch's schedule (host only) for tori shapes [(X, Y)]:
    returns (CTAs per SM, threads per CTA, trials per unit [m], units
    int32 [k, 2] of (instance, group) in the order the CTAs take them)."""
    m = len(shapes)
    X = np.ascontiguousarray([s[0] for s in shapes], dtype=np.int32)
    Y = np.ascontiguousarray([s[1] for s in shapes], dtype=np.int32)
    T = np.ascontiguousarray(trials, dtype=np.int32)
    S = np.ascontiguousarray(sweeps, dtype=np.int32)
    G = np.zeros(m, dtype=np.int32)
    cap = int(sum((int(t) + 3) // 4 for t in T)) + 1
    units = np.zeros((cap, 2), dtype=np.int32)
    per_sm, threads, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
    check(lib().ising_batch_schedule(m, vp(X), vp(Y), vp(T), vp(S), int(draw_bits), int(group_trials),
                                     int(ctas_per_sm), int(sms), int(smem_per_cta_max), ctypes.byref(per_sm),
                                     ctypes.byref(threads), vp(G), vp(units), cap, ctypes.byref(k)),
          "ising_batch_schedule")
    return per_sm.value, threads.value, G, units[:k.value].copy()


def thresholds(betas, draw_bits=32):
    """The library's acceptance thresholds for a schedule (ising_thresholds,
    host only): uint32 [S, 2] of (T_4, T_8) per sweep; in the 16-bit mode
    shifted left by 16 bits, as the kernels compare them."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    out = np.zeros((b.shape[0], 2), dtype=np.uint32)
    check(lib().ising_thresholds(b.ctypes.data_as(ctypes.c_void_p), int(b.shape[0]), int(draw_bits),
                                 out.ctypes.data_as(ctypes.c_void_p)), "ising_thresholds")
    return out


def philox(counters, seed, stream=None):
    """The library's Philox4x32-10 blocks for uint32 counters [k, 4] (CUDA tensor or array)."""
    torch = _torch()
    c = counters if isinstance(counters, torch.Tensor) else torch.as_tensor(
        np.ascontiguousarray(counters, dtype=np.uint32).view(np.int32))
    c = c.to(device="cuda", dtype=torch.int32).contiguous()
    out = torch.empty_like(c)
    check(lib().ising_philox(_dptr(c), int(seed) & 0xFFFFFFFFFFFFFFFF, int(c.shape[0]), _dptr(out),
                             _stream_ptr(stream)), "ising_philox")
    return out


def energy(prob, spins, out=None, stream=None):
    """Eq. 2 (with fields) of each row of an int8 CUDA tensor [k, n] -> int64."""
    torch = _torch()
    k = _rows(spins, "spins")
    spins = _device_tensor(spins, torch.int8, (k, prob.n), "spins")
    if out is None:
        out = torch.empty((k,), dtype=torch.int64, device=spins.device)
    else:
        out = _device_tensor(out, torch.int64, (k,), "out", write=True)
    check(lib().ising_energy(prob.handle, _dptr(spins), int(k), _dptr(out), _stream_ptr(stream)), "ising_energy")
    return out


def cut(prob, spins, out=None, stream=None):
    """Exact Eq. 1 cut of each row of an int8 CUDA tensor [k, n]."""
    torch = _torch()
    k = _rows(spins, "spins")
    spins = _device_tensor(spins, torch.int8, (k, prob.n), "spins")
    if out is None:
        out = torch.empty((k,), dtype=torch.int32, device=spins.device)
    else:
        out = _device_tensor(out, torch.int32, (k,), "out", write=True)
    check(lib().ising_cut(prob.handle, _dptr(spins), int(k), _dptr(out), _stream_ptr(stream)), "ising_cut")
    return out


def _batch_arrays(probs, trials, sweeps, betas, seeds, out_spins, out_cuts):
    m = len(probs)
    P = (ctypes.c_void_p * m)(*[p.handle.value for p in probs])
    Tn = (ctypes.c_int32 * m)(*[int(t) for t in trials])
    Sn = (ctypes.c_int32 * m)(*[int(s) for s in sweeps])
    barrs = [np.ascontiguousarray(b, dtype=np.float64) for b in betas]
    B = (ctypes.c_void_p * m)(*[b.ctypes.data for b in barrs])
    Sd = (ctypes.c_uint64 * m)(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
    Os = (ctypes.c_void_p * m)(*[(o.data_ptr() if o is not None else None) for o in out_spins])
    Oc = (ctypes.c_void_p * m)(*[(o.data_ptr() if o is not None else None) for o in out_cuts])
    return m, P, Tn, Sn, B, Sd, Os, Oc, barrs


def _alloc_outputs(probs, trials, want_spins):
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    spins = [torch.empty((t, p.n), dtype=torch.int8, device=dev) if want_spins else None
             for p, t in zip(probs, trials)]
    cuts = [torch.empty((t,), dtype=torch.int32, device=dev) for t in trials]
    return spins, cuts


def anneal_batched(probs, trials, sweeps, betas, seeds, want_spins=True, stream=None):
    """One persistent launch over uneven instances; returns (spins list, cuts list)."""
    spins, cuts = _alloc_outputs(probs, trials, want_spins)
    m, P, Tn, Sn, B, Sd, Os, Oc, keep = _batch_arrays(probs, trials, sweeps, betas, seeds, spins, cuts)
    rc = lib().ising_anneal_batched(P, m, Tn, Sn, B, Sd, Os, Oc, _stream_ptr(stream))
    check(rc, "ising_anneal_batched")
    return spins, cuts


class BatchPlan:
    """A prepared batch replayed as a CUDA graph (ising_batch_create / _launch)."""

    def __init__(self, probs, trials, sweeps, betas, seeds, want_spins=True, group_trials=0,
                 ctas_per_sm=0, stream=None):
        self.probs = list(probs)
        self.spins, self.cuts = _alloc_outputs(self.probs, trials, want_spins)
        m, P, Tn, Sn, B, Sd, Os, Oc, keep = _batch_arrays(self.probs, trials, sweeps, betas, seeds,
                                                          self.spins, self.cuts)
        out = ctypes.c_void_p()
        rc = lib().ising_batch_create(P, m, Tn, Sn, B, Sd, Os, Oc, int(group_trials), int(ctas_per_sm),
                                      _stream_ptr(stream), ctypes.byref(out))
        check(rc, "ising_batch_create")
        self._h = out

    def launch(self, stream=None):
        check(lib().ising_batch_launch(self._h, _stream_ptr(stream)), "ising_batch_launch")
        return self.spins, self.cuts

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            lib().ising_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------------------------------------------------------- learned proposals
CNN_PARAMS = 19681


class CNN:
    """The proposal network on the device (ising_cnn_*); params: float array of CNN_PARAMS."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.shape == (CNN_PARAMS,)
        out = ctypes.c_void_p()
        check(lib().ising_cnn_create(p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)), "ising_cnn_create")
        self._h = out
        self._ws = {}

    @property
    def handle(self):
        return self._h

    def params(self):
        out = np.zeros(CNN_PARAMS, dtype=np.float32)
        check(lib().ising_cnn_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)), "ising_cnn_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(lib().ising_cnn_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)), "ising_cnn_set_params")

    def _workspace(self, B, n, train):
        torch = _torch()
        need = int(lib().ising_cnn_workspace_bytes(int(B), int(n), int(train)))
        key = bool(train)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
            self._ws[key] = ws
        return ws, need

    def forward(self, prob, spins, out=None, stream=None):
        torch = _torch()
        B = _rows(spins, "spins")
        spins = _device_tensor(spins, torch.int8, (B, prob.n), "spins")
        if out is None:
            out = torch.empty((B, prob.n), dtype=torch.float32, device=spins.device)
        else:
            out = _device_tensor(out, torch.float32, (B, prob.n), "out", write=True)
        ws, need = self._workspace(B, prob.n, 0)
        check(lib().ising_cnn_forward(self._h, prob.handle, _dptr(spins), int(B), _dptr(out), _dptr(ws),
                                      ctypes.c_size_t(ws.numel()), _stream_ptr(stream)), "ising_cnn_forward")
        return out

    def grad(self, prob, spins, targets, stream=None):
        torch = _torch()
        B = _rows(spins, "spins")
        spins = _device_tensor(spins, torch.int8, (B, prob.n), "spins")
        targets = _device_tensor(targets, torch.uint8, (B, prob.n), "targets")
        g = torch.empty(CNN_PARAMS, dtype=torch.float32, device=spins.device)
        loss = torch.empty(1, dtype=torch.float32, device=spins.device)
        ws, need = self._workspace(B, prob.n, 1)
        check(lib().ising_cnn_grad(self._h, prob.handle, _dptr(spins), _dptr(targets), int(B), _dptr(g), _dptr(loss),
                                   _dptr(ws), ctypes.c_size_t(ws.numel()), _stream_ptr(stream)), "ising_cnn_grad")
        return loss, g

    def set_wait_limit(self, cycles=0, stall_test=0):
        check(lib().ising_cnn_set_wait_limit(self._h, int(cycles), int(stall_test)), "ising_cnn_set_wait_limit")

    def adam_step(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        grad = _device_tensor(grad, _torch().float32, (CNN_PARAMS,), "grad")
        check(lib().ising_cnn_adam_step(self._h, _dptr(grad), ctypes.c_float(lr), ctypes.c_float(beta1),
                                        ctypes.c_float(beta2), ctypes.c_float(eps), _stream_ptr(stream)),
              "ising_cnn_adam_step")

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            lib().ising_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def propose(prob, spins, logits, tile, accepted=None, stream=None):
    """Exact-acceptance proposals in place on spins (see ising_propose); returns accepted [B]."""
    torch = _torch()
    B = _rows(spins, "spins")
    spins = _device_tensor(spins, torch.int8, (B, prob.n), "spins", write=True)
    logits = _device_tensor(logits, torch.float32, (B, prob.n), "logits")
    if accepted is None:
        accepted = torch.zeros(B, dtype=torch.int32, device=spins.device)
    else:
        accepted = _device_tensor(accepted, torch.int32, (B,), "accepted", write=True)
    check(lib().ising_propose(prob.handle, _dptr(spins), int(B), _dptr(logits), int(tile),
                              _dptr(accepted), _stream_ptr(stream)), "ising_propose")
    return accepted


class LearnedPlan:
    """The learned form of the annealer for m same-shape problems, prepared
    once and replayed as one CUDA graph (ising_learned_create / _launch):
    sweeps [0, k_first) batched from the Philox start (after the network's
    warm start with warm=True), then for every chunk of `every` sweeps the
    chunk batched and resumed, the network's cluster block flips (net not
    None) and partner moves (partner_period > 0); then the cuts.  The
    state, cuts, accepted counts, logits and the network's workspace are
    device tensors owned here."""

    def __init__(self, probs, net, trials, betas, seeds, k_first, every=100, partner_period=0, warm=False,
                 stream=None):
        torch = _torch()
        self.probs = list(probs)
        m, n = len(self.probs), self.probs[0].n
        self.trials = int(trials)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.spins = torch.empty((m * self.trials, n), dtype=torch.int8, device=dev)
        self.cuts = torch.empty((m * self.trials,), dtype=torch.int32, device=dev)
        self.accepted = torch.zeros((m * self.trials,), dtype=torch.int32, device=dev)
        self.logits = self.ws = None
        if net is not None:
            self.logits = torch.empty((m * self.trials, n), dtype=torch.float32, device=dev)
            need = int(lib().ising_cnn_workspace_bytes(self.trials, int(n), 0))
            self.ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        self._betas = np.ascontiguousarray(betas, dtype=np.float64)
        self._seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        assert self._seeds.shape == (m,)
        handles = (ctypes.c_void_p * m)(*[p.handle for p in self.probs])
        out = ctypes.c_void_p()
        self.net = net
        check(lib().ising_learned_create(handles, int(m), self.trials,
                                         self._betas.ctypes.data_as(ctypes.c_void_p), int(self._betas.shape[0]),
                                         self._seeds.ctypes.data_as(ctypes.c_void_p), int(k_first), int(every),
                                         net.handle if net is not None else None, int(partner_period), int(bool(warm)),
                                         _dptr(self.spins), _dptr(self.cuts), _dptr(self.accepted),
                                         _dptr(self.logits) if self.logits is not None else None,
                                         _dptr(self.ws) if self.ws is not None else None,
                                         ctypes.c_size_t(self.ws.numel() if self.ws is not None else 0),
                                         _stream_ptr(stream), ctypes.byref(out)), "ising_learned_create")
        self._h = out

    def launch(self, stream=None):
        """Enqueue one learned anneal; returns (spins, cuts, accepted) views."""
        check(lib().ising_learned_launch(self._h, _stream_ptr(stream)), "ising_learned_launch")
        return self.spins, self.cuts, self.accepted

    def destroy(self):
        """Free the plan after the device has finished its queued launches
        (ising_learned_destroy itself does not wait)."""
        if getattr(self, "_h", None) is not None:
            torch = _torch()
            if not torch.cuda.is_current_stream_capturing():
                torch.cuda.synchronize()
            lib().ising_learned_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def propose_clusters(probs, spins, logits, accepted=None, stream=None):
    """Cluster block flips in place (ising_propose_clusters).  probs: one
    Problem, or a list of m Problems of one shape whose configurations are
    stacked in spins [m * B, n]; returns accepted components [m * B]."""
    torch = _torch()
    probs = list(probs) if isinstance(probs, (list, tuple)) else [probs]
    rows = _rows(spins, "spins")
    m = len(probs)
    if rows % m:
        raise ValueError("spins rows must be a multiple of the number of problems")
    n = probs[0].n
    spins = _device_tensor(spins, torch.int8, (rows, n), "spins", write=True)
    logits = _device_tensor(logits, torch.float32, (rows, n), "logits")
    if accepted is None:
        accepted = torch.zeros(rows, dtype=torch.int32, device=spins.device)
    else:
        accepted = _device_tensor(accepted, torch.int32, (rows,), "accepted", write=True)
    handles = (ctypes.c_void_p * m)(*[p.handle for p in probs])
    check(lib().ising_propose_clusters(handles, int(m), _dptr(spins), int(rows // m), _dptr(logits),
                                       _dptr(accepted), _stream_ptr(stream)), "ising_propose_clusters")
    return accepted


def transcribe(probs, spins, shift, out=None, accepted=None, stream=None):
    """Partner moves (ising_transcribe): returns (new spins [m * B, n],
    flipped components [m * B]); probs as in propose_clusters."""
    torch = _torch()
    probs = list(probs) if isinstance(probs, (list, tuple)) else [probs]
    rows = _rows(spins, "spins")
    m = len(probs)
    if rows % m:
        raise ValueError("spins rows must be a multiple of the number of problems")
    n = probs[0].n
    spins = _device_tensor(spins, torch.int8, (rows, n), "spins")
    if out is None:
        out = torch.empty_like(spins)
    else:
        out = _device_tensor(out, torch.int8, (rows, n), "out", write=True)
    if accepted is None:
        accepted = torch.zeros(rows, dtype=torch.int32, device=spins.device)
    else:
        accepted = _device_tensor(accepted, torch.int32, (rows,), "accepted", write=True)
    handles = (ctypes.c_void_p * m)(*[p.handle for p in probs])
    check(lib().ising_transcribe(handles, int(m), _dptr(spins), _dptr(out), int(rows // m), int(shift),
                                 _dptr(accepted), _stream_ptr(stream)), "ising_transcribe")
    return out, accepted


def droplet_targets(prob, spins, ref, out=None, stream=None):
    """Droplet training targets (ising_droplet_targets): uint8 [B, n]."""
    torch = _torch()
    B = _rows(spins, "spins")
    spins = _device_tensor(spins, torch.int8, (B, prob.n), "spins")
    ref = _device_tensor(ref, torch.int8, (B, prob.n), "ref")
    if out is None:
        out = torch.empty((B, prob.n), dtype=torch.uint8, device=spins.device)
    else:
        out = _device_tensor(out, torch.uint8, (B, prob.n), "out", write=True)
    check(lib().ising_droplet_targets(prob.handle, _dptr(spins), _dptr(ref), int(B), _dptr(out), _stream_ptr(stream)),
          "ising_droplet_targets")
    return out


def flip_targets(spins, ref, out=None, stream=None):
    """Gauge-aligned flip targets (ising_flip_targets): uint8 [B, n]."""
    torch = _torch()
    B = _rows(spins, "spins")
    n = int(spins.shape[1])
    spins = _device_tensor(spins, torch.int8, (B, n), "spins")
    ref = _device_tensor(ref, torch.int8, (B, n), "ref")
    if out is None:
        out = torch.empty((B, n), dtype=torch.uint8, device=spins.device)
    else:
        out = _device_tensor(out, torch.uint8, (B, n), "out", write=True)
    check(lib().ising_flip_targets(_dptr(spins), _dptr(ref), int(B), int(n), _dptr(out), _stream_ptr(stream)),
          "ising_flip_targets")
    return out
