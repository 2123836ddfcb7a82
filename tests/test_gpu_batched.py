"""GPU parity for the persistent batched launch and its CUDA-graph plans.

Each instance of a batch must equal the CPU oracle (and the single-instance
entry point) bit for bit, whatever the work-unit width and grid."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ia():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    torch.cuda.set_device(0)
    return ia


SMALL = [  # X, Y, inst_seed, trials, sweeps, seed
    (4, 4, 1, 7, 30, 11),
    (12, 8, 2, 64, 40, 12),
    (50, 50, 3, 33, 25, 13),
    (20, 6, 4, 0, 10, 14),       # no trials
    (10, 10, 5, 5, 0, 15),       # no sweeps
    (140, 100, 6, 40, 6, 16),
    (16, 12, 7, 100, 35, 17),
]


def _run_small(ia, **plan_kw):
    import torch
    insts = [synth.torus_instance(X, Y, s) for (X, Y, s, _, _, _) in SMALL]
    probs = [ia.Problem.from_instance(i) for i in insts]
    trials = [c[3] for c in SMALL]
    sweeps = [c[4] for c in SMALL]
    betas = [synth.linear_betas(0.1, 3.0, S) for S in sweeps]
    seeds = [c[5] for c in SMALL]
    if plan_kw:
        plan = ia.BatchPlan(probs, trials, sweeps, betas, seeds, **plan_kw)
        spins, cuts = plan.launch()
        torch.cuda.synchronize()
        first = ([s.clone() for s in spins], [c.clone() for c in cuts])
        for s in spins:
            s.fill_(0)
        spins, cuts = plan.launch()          # a replay must give the same results
        torch.cuda.synchronize()
        for a, b in zip(first[0], spins):
            assert torch.equal(a, b)
        for a, b in zip(first[1], cuts):
            assert torch.equal(a, b)
        plan.destroy()
    else:
        spins, cuts = ia.anneal_batched(probs, trials, sweeps, betas, seeds)
        torch.cuda.synchronize()
    return insts, probs, trials, betas, seeds, spins, cuts


@pytest.mark.parametrize("plan_kw", [{}, {"group_trials": 0}, {"group_trials": 8, "ctas_per_sm": 1},
                                     {"group_trials": 20, "ctas_per_sm": 2}, {"group_trials": 4, "ctas_per_sm": 1}])
def test_batched_small_against_oracle(ia, plan_kw):
    insts, probs, trials, betas, seeds, spins, cuts = _run_small(ia, **plan_kw)
    for q, inst in enumerate(insts):
        rs, rc = oracle.anneal(inst, betas[q], seeds[q], t_count=trials[q])
        np.testing.assert_array_equal(spins[q].cpu().numpy(), rs)
        np.testing.assert_array_equal(cuts[q].cpu().numpy(), rc)
    for p in probs:
        p.destroy()


def test_batched_equals_single_entry_point(ia):
    import torch
    insts, probs, trials, betas, seeds, spins, cuts = _run_small(ia)
    for q in range(len(insts)):
        s1, c1 = ia.anneal(probs[q], trials[q], betas[q], seeds[q])
        torch.cuda.synchronize()
        assert torch.equal(s1, spins[q]) and torch.equal(c1, cuts[q])
    for p in probs:
        p.destroy()


def test_batched_argument_errors(ia):
    p = ia.Problem.from_instance(synth.torus_instance(8, 8, 1))
    with pytest.raises(ia.IsingError):
        ia.anneal_batched([p], [4], [3], [np.array([1.0, 0.0, 1.0])], [1])
    with pytest.raises(ia.IsingError):
        ia.BatchPlan([p], [4], [3], [np.ones(3)], [1], group_trials=6)
    p.destroy()


def test_batched_96_instances_sampled(ia):
    """The 96-instance uneven batch (50/100/140/200 x 100, 32-512 trials,
    2k-20k sweeps) in one graph-captured persistent launch: every instance's
    fused cuts against the cut kernel, the first and the last trial of every
    instance against the oracle (one oracle call per trial, in a thread pool:
    the C oracle runs without the interpreter lock), and two instances against
    the single entry point."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    import torch
    cfg = synth.batched_config()
    insts = [synth.torus_instance(c["X"], c["Y"], c["inst_seed"]) for c in cfg]
    probs = [ia.Problem.from_instance(i) for i in insts]
    trials = [c["trials"] for c in cfg]
    sweeps = [c["sweeps"] for c in cfg]
    betas = [synth.linear_betas(0.1, 3.0, S) for S in sweeps]
    seeds = [c["seed"] for c in cfg]
    plan = ia.BatchPlan(probs, trials, sweeps, betas, seeds)
    spins, cuts = plan.launch()
    torch.cuda.synchronize()
    for q in range(len(cfg)):
        assert torch.equal(ia.cut(probs[q], spins[q]), cuts[q])
    work = [insts[q]["n"] * sweeps[q] for q in range(len(cfg))]
    jobs = sorted(((q, t) for q in range(len(cfg)) for t in (0, trials[q] - 1)), key=lambda j: -work[j[0]])
    oracle.lib()   # built once, before the pool

    def run(job):
        q, t = job
        rs, rc = oracle.anneal(insts[q], betas[q], seeds[q], t_begin=t, t_count=1)
        return q, t, rs[0], rc[0]

    checked = 0
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for q, t, rs, rc in ex.map(run, jobs):
            np.testing.assert_array_equal(spins[q][t].cpu().numpy(), rs)
            assert cuts[q][t].item() == rc
            checked += 1
    assert checked == 2 * len(cfg)
    for q in (1, 94):
        s1, c1 = ia.anneal(probs[q], trials[q], betas[q], seeds[q])
        torch.cuda.synchronize()
        assert torch.equal(s1, spins[q]) and torch.equal(c1, cuts[q])
    plan.destroy()
    for p in probs:
        p.destroy()
