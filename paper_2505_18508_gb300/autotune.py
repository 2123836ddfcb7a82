"""Autotuner for the launch shape of ising_anneal and of batch plans.

It times short probe runs of candidate shapes on the current GPU and keeps
the fastest.  Results do not depend on the shape (the random stream is keyed
by site, sweep and trial), so only time is compared.  Winners are cached in a
JSON file keyed by GPU name, torus shape and trial count:
$ISING_AUTOTUNE_CACHE, else ~/.cache/paper_2505_18508_gb300/autotune.json.

Candidates for one instance:
  * the persistent kernel with 32, 28, 24 or 16 trials per group;
  * the cluster-strip kernel with 32 trials per group, 1..8 strips and the
    thread counts that leave the fewest idle item slots.
For a batch: trials per work unit (0 = automatic, 32, 16, 8) times 1 or 2
CTAs per SM.
"""
from __future__ import annotations

import json
import os

import numpy as np


def cache_path():
    p = os.environ.get("ISING_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2505_18508_gb300", "autotune.json")


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(key, value, path=None):
    path = path or cache_path()
    data = load_cache(path)
    data[key] = value
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def anneal_key(gpu, X, Y, trials):
    return f"anneal|{gpu}|{X}x{Y}|T={trials}"


def batch_key(gpu, shapes):
    """shapes: list of (X, Y, trials, sweeps)."""
    h = 0
    for s in shapes:
        for v in s:
            h = (h * 1000003 + int(v)) & 0xFFFFFFFFFFFF
    return f"batch|{gpu}|m={len(shapes)}|{h:012x}"


def anneal_candidates(X, Y, trials):
    out = []
    for G in (32, 28, 24, 16):
        if G <= max(4, trials):
            out.append({"kernel": 2, "group_trials": G, "strips": 0, "threads": 0})
    H = X // 2
    for C in (1, 2, 4, 8):
        if C > Y // 2 and C != 1:
            continue
        rows = -(-Y // C)
        items = rows * H
        for th in sorted({_best_threads(items), 1024, 512}):
            out.append({"kernel": 1, "group_trials": 32, "strips": C, "threads": th})
    return out


def _best_threads(items):
    if items <= 768:
        return max(64, -(-items // 32) * 32)
    best, be = 1024, -1.0
    for t in range(768, 1025, 32):
        it = -(-items // t)
        e = items / (it * t)
        if e > be + 1e-9:
            best, be = t, e
    return best


def _apply(prob, c):
    prob.set_kernel(c["kernel"])
    prob.set_launch(c["group_trials"], c["strips"], c["threads"])


def tune_anneal(prob, trials, probe_sweeps=200, reps=2, use_cache=True, candidates=None):
    """Time the candidates on `prob` and apply the fastest; returns it."""
    import torch
    from . import IsingError, anneal
    gpu = torch.cuda.get_device_name()
    key = anneal_key(gpu, prob.X, prob.Y, trials)
    if use_cache and candidates is None:
        hit = load_cache().get(key)
        if hit:
            _apply(prob, hit)
            return hit
    betas = np.linspace(0.1, 3.0, probe_sweeps)
    cuts = torch.empty(trials, dtype=torch.int32, device="cuda")
    best, best_ms = None, float("inf")
    for c in candidates or anneal_candidates(prob.X, prob.Y, trials):
        try:
            _apply(prob, c)
            anneal(prob, trials, betas, 1, want_spins=False, out_cuts=cuts)
            torch.cuda.synchronize()
        except IsingError:
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            anneal(prob, trials, betas, 1, want_spins=False, out_cuts=cuts)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if ms < best_ms:
            best, best_ms = dict(c), ms
    if best is None:
        _apply(prob, {"kernel": 0, "group_trials": 0, "strips": 0, "threads": 0})
        return None
    best["probe_ms"] = best_ms
    best["probe_sweeps"] = probe_sweeps
    _apply(prob, best)
    if use_cache:
        store_cache(key, best)
    return best


def tune_batched(probs, trials, sweeps, probe_fraction=0.05, use_cache=True):
    """Pick (group_trials, ctas_per_sm) for a batch by timing plan replays on
    schedules shortened to `probe_fraction` of each instance's sweeps."""
    import torch
    from . import BatchPlan, IsingError
    gpu = torch.cuda.get_device_name()
    key = batch_key(gpu, [(p.X, p.Y, t, s) for p, t, s in zip(probs, trials, sweeps)])
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            return hit
    short = [max(1, int(s * probe_fraction)) for s in sweeps]
    betas = [np.linspace(0.1, 3.0, s) for s in short]
    seeds = list(range(len(probs)))
    best, best_ms = None, float("inf")
    for G in (0, 32, 16, 8):
        for per_sm in (1, 2):
            try:
                plan = BatchPlan(probs, trials, short, betas, seeds, want_spins=False, group_trials=G,
                                 ctas_per_sm=per_sm)
            except IsingError:
                continue
            plan.launch()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.launch()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            plan.destroy()
            if ms < best_ms:
                best, best_ms = {"group_trials": G, "ctas_per_sm": per_sm, "probe_ms": ms}, ms
    if best is not None and use_cache:
        store_cache(key, best)
    return best
