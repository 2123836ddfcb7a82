"""Sweep-budget campaigns on one instance (the shape of the paper's Fig. 1:
highest and average cut against sweeps per trial; Fig. 3: the distribution
of final cuts at one budget).

Every budget S of the ladder is an independent batch of trials, each a full
anneal with its own linear schedule beta 0.1 -> 3.0 over S sweeps (Section
III: the sweeps per trial is the campaign's knob).  Each budget is one
ising_anneal call, so the persistent kernel spreads its trial groups' rows
over every SM; a batched launch would give each trial group of the longest
budget a single CTA and leave the rest of the GPU idle.

    python -m paper_2505_18508_gb300.campaign --X 200 --Y 100 --trials 256 \\
        --budgets 1000,3000,10000,30000,100000

Orchestration only: the anneals and cuts run in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def linear_schedule(beta0, beta1, S):
    """beta_k = beta0 + (beta1 - beta0) k / (S - 1), k = 0 .. S-1 (S = 1: beta0)."""
    if S <= 1:
        return np.full(max(S, 0), float(beta0))
    k = np.arange(S, dtype=np.float64)
    return beta0 + (beta1 - beta0) * k / float(S - 1)


def run_campaign(prob, budgets, trials, seed, beta0=0.1, beta1=3.0, hist_bins=None):
    """Anneal `trials` trials at every budget of `budgets`; returns a dict with,
    per budget, the highest, mean and lowest final cut and the histogram of
    final cuts (integer bins), plus the wall time of the whole ladder."""
    import torch
    from . import anneal

    budgets = [int(S) for S in budgets]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cuts = [anneal(prob, trials, linear_schedule(beta0, beta1, S), seed + 7919 * j, want_spins=False)[1]
            for j, S in enumerate(budgets)]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    rows = []
    for S, c in zip(budgets, cuts):
        v = c.cpu().numpy().astype(np.int64)
        lo, hi = int(v.min()), int(v.max())
        edges = np.arange(lo, hi + 2) if hist_bins is None else np.linspace(lo, hi + 1, hist_bins + 1)
        counts, _ = np.histogram(v, bins=edges)
        rows.append({"sweeps": S, "highest": hi, "mean": float(v.mean()), "lowest": lo,
                     "histogram": {"first_cut": lo, "counts": [int(x) for x in counts]}})
    updates = sum(budgets) * trials * prob.n
    return {"budgets": rows, "trials_per_budget": trials, "wall_s": wall, "updates": updates,
            "updates_per_s": updates / wall}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--X", type=int, default=200)
    ap.add_argument("--Y", type=int, default=100)
    ap.add_argument("--inst-seed", type=int, default=2)
    ap.add_argument("--trials", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--budgets", default="1000,3000,10000,30000,100000")
    args = ap.parse_args(argv)
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    from . import Problem
    torch.cuda.set_device(0)
    prob = Problem.from_instance(synth.torus_instance(args.X, args.Y, args.inst_seed))
    out = run_campaign(prob, [int(s) for s in args.budgets.split(",")], args.trials, args.seed)
    prob.destroy()
    out["workload"] = f"{args.X}x{args.Y} torus, instance seed {args.inst_seed}"
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
