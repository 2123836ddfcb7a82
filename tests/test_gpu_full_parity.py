"""Full parity of the 200x100, 1,024-trial, 10,000-sweep workload: every
trial's final spins and cut from the CUDA path against the CPU oracle.

It needs ~4,000 core-seconds of oracle time, so it runs only when
ISING_FULL_PARITY=1 is set (on a GPU machine with many host cores); the
sampled parity of the same workload (one trial per 32-trial group) runs in
every GPU test run (test_gpu_anneal.py, test_gpu_draw16.py).

    ISING_FULL_PARITY=1 python -m pytest tests/test_gpu_full_parity.py -m gpu -s

The GPU result is computed first; the oracle then runs in one spawned
process per host core, each on a contiguous slice of trials.
"""
import json
import multiprocessing as mp
import os
import time

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("ISING_FULL_PARITY") != "1",
                                 reason="full parity runs only with ISING_FULL_PARITY=1 (~4,000 core-seconds)")]

X, Y, INST_SEED, TRIALS, SWEEPS, SEED = 200, 100, 2, 1024, 10000, 1002


def _oracle_slice(job):
    import oracle
    t_begin, t_count, draw_bits = job
    inst = synth.torus_instance(X, Y, INST_SEED)
    betas = synth.linear_betas(0.1, 3.0, SWEEPS)
    spins, cuts = oracle.anneal(inst, betas, SEED, t_begin=t_begin, t_count=t_count, draw_bits=draw_bits)
    return t_begin, spins, cuts


@pytest.mark.parametrize("kernel,draw_bits", [(2, 32), (1, 32), (2, 16)])
def test_full_parity_200x100_1024_trials(kernel, draw_bits):
    ctx = mp.get_context("spawn")   # the pool starts by spawn, never by fork after CUDA is up
    import oracle
    oracle.lib()
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    torch.cuda.set_device(0)
    inst = synth.torus_instance(X, Y, INST_SEED)
    betas = synth.linear_betas(0.1, 3.0, SWEEPS)
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(kernel)
    prob.set_draw_bits(draw_bits)
    spins, cuts = ia.anneal(prob, TRIALS, betas, SEED)
    torch.cuda.synchronize()
    assert prob.last_kernel() == kernel
    g_spins, g_cuts = spins.cpu().numpy(), cuts.cpu().numpy()
    prob.destroy()
    procs = os.cpu_count() or 1
    per = (TRIALS + procs - 1) // procs
    jobs = [(b, min(per, TRIALS - b), draw_bits) for b in range(0, TRIALS, per)]
    t0 = time.perf_counter()
    bad = []
    with ctx.Pool(procs) as pool:
        for t_begin, rs, rc in pool.imap_unordered(_oracle_slice, jobs):
            for j in range(rs.shape[0]):
                if g_cuts[t_begin + j] != rc[j] or not np.array_equal(g_spins[t_begin + j], rs[j]):
                    bad.append(t_begin + j)
    print(json.dumps({"kernel": kernel, "draw_bits": draw_bits, "trials_compared": TRIALS,
                      "trials_differing": len(bad), "oracle_s": round(time.perf_counter() - t0, 1),
                      "oracle_procs": procs, "best_cut": int(g_cuts.max())}))
    assert not bad, f"trials differing: {sorted(bad)[:8]}"
