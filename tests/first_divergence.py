"""Debugging aid: find the first (sweep, site, trial) where the CUDA path and
the oracle part ways.

The random stream is keyed by (site, sweep, trial), so a run of S sweeps
equals S one-sweep calls chained through `init` and `sweep_offset`.  This
tool advances both sides one sweep at a time from the same start and stops
at the first sweep after which their states differ, printing the differing
sites (with their checkerboard colour) and trials.

    python tests/first_divergence.py --X 8 --Y 6 --trials 37 --sweeps 25 [--kernel 0|1|2] [--draw-bits 32|16]

Test infrastructure (it runs the oracle); exit status 0 iff no divergence.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402


def first_divergence(X, Y, inst_seed, trials, sweeps, seed, kernel=0, draw_bits=32, beta0=0.1, beta1=3.0):
    """Returns None if both sides agree after every sweep, else a dict with
    the sweep index and the first differing (site, colour, trial) triples."""
    import torch
    import oracle
    import paper_2505_18508_gb300 as ia
    inst = synth.torus_instance(X, Y, inst_seed)
    betas = synth.linear_betas(beta0, beta1, sweeps)
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(kernel)
    prob.set_draw_bits(draw_bits)
    g_state = None
    o_state = None
    try:
        # the start (no sweeps)
        g_state, _ = ia.anneal(prob, trials, betas[:0], seed)
        o_state, _ = oracle.anneal(inst, betas[:0], seed, t_count=trials, draw_bits=draw_bits)
        for k in range(sweeps + 1):
            torch.cuda.synchronize()
            g = g_state.cpu().numpy()
            if not np.array_equal(g, o_state):
                t_idx, i_idx = np.nonzero(g != o_state)
                pairs = sorted(zip(i_idx.tolist(), t_idx.tolist()))[:16]
                return {"after_sweeps": k, "differing_entries": int(t_idx.size),
                        "first": [{"site": i, "x": i % X, "y": i // X, "colour": (i % X + i // X) & 1, "trial": t}
                                  for i, t in pairs]}
            if k == sweeps:
                break
            g_state, _ = ia.anneal(prob, trials, betas[k:k + 1], seed, sweep_offset=k, init=g_state)
            o_state, _ = oracle.anneal(inst, betas[k:k + 1], seed, t_count=trials, sweep_offset=k, init=o_state,
                                       draw_bits=draw_bits)
        return None
    finally:
        prob.destroy()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--X", type=int, default=8)
    ap.add_argument("--Y", type=int, default=6)
    ap.add_argument("--inst-seed", type=int, default=1)
    ap.add_argument("--trials", type=int, default=37)
    ap.add_argument("--sweeps", type=int, default=25)
    ap.add_argument("--seed", type=int, default=1001)
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--draw-bits", type=int, default=32)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    d = first_divergence(args.X, args.Y, args.inst_seed, args.trials, args.sweeps, args.seed, args.kernel,
                         args.draw_bits)
    print(json.dumps({"divergence": d}))
    return 0 if d is None else 1


if __name__ == "__main__":
    sys.exit(main())
