"""One full-parity run of the 200x100, 1,024-trial, 10,000-sweep workload:
every trial's final spins and cut from the CUDA path against the CPU oracle.

Not collected by pytest (it needs ~4,000 core-seconds of oracle time); run it
on a machine with a GPU and many host cores:

    python tests/full_parity_200x100_1024trials.py [--procs N] [--kernel 0|1|2] [--draw-bits 32|16]

The GPU result is computed first; the oracle then runs in N spawned
processes (default: every host core), each on a contiguous slice of trials.
Prints one JSON line: trials compared, trials that differ, wall times.
Exit status 0 iff every trial matches bit for bit.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

X, Y, INST_SEED, TRIALS, SWEEPS, SEED = 200, 100, 2, 1024, 10000, 1002


def _oracle_slice(job):
    import oracle
    t_begin, t_count, draw_bits = job
    inst = synth.torus_instance(X, Y, INST_SEED)
    betas = synth.linear_betas(0.1, 3.0, SWEEPS)
    spins, cuts = oracle.anneal(inst, betas, SEED, t_begin=t_begin, t_count=t_count, draw_bits=draw_bits)
    return t_begin, spins, cuts


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--draw-bits", type=int, default=32)
    args = ap.parse_args(argv)
    ctx = mp.get_context("spawn")   # the pool starts by spawn, never by fork after CUDA is up
    import oracle
    oracle.lib()                    # build the C oracle before the workers load it

    import torch
    import paper_2505_18508_gb300 as ia
    torch.cuda.set_device(0)
    inst = synth.torus_instance(X, Y, INST_SEED)
    betas = synth.linear_betas(0.1, 3.0, SWEEPS)
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(args.kernel)
    prob.set_draw_bits(args.draw_bits)
    t0 = time.perf_counter()
    spins, cuts = ia.anneal(prob, TRIALS, betas, SEED)
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    kernel = prob.last_kernel()
    g_spins, g_cuts = spins.cpu().numpy(), cuts.cpu().numpy()
    prob.destroy()

    per = (TRIALS + args.procs - 1) // args.procs
    jobs = [(b, min(per, TRIALS - b), args.draw_bits) for b in range(0, TRIALS, per)]
    t0 = time.perf_counter()
    bad = []
    with ctx.Pool(args.procs) as pool:
        for t_begin, rs, rc in pool.imap_unordered(_oracle_slice, jobs):
            for j in range(rs.shape[0]):
                t = t_begin + j
                if g_cuts[t] != rc[j] or not np.array_equal(g_spins[t], rs[j]):
                    bad.append(t)
    t_cpu = time.perf_counter() - t0
    out = {"workload": f"{X}x{Y} torus, instance seed {INST_SEED}, {TRIALS} trials x {SWEEPS} sweeps, seed {SEED}",
           "kernel": kernel, "draw_bits": args.draw_bits, "trials_compared": TRIALS, "trials_differing": len(bad),
           "first_differing": sorted(bad)[:8], "gpu_s": round(t_gpu, 3), "oracle_s": round(t_cpu, 1),
           "oracle_procs": args.procs, "best_cut": int(g_cuts.max())}
    print(json.dumps(out))
    return 0 if not bad else 1


if __name__ == "__main__":
    sys.exit(main())
