"""GPU parity of the 16-bit draw mode (one Philox4x32-10 block per eight
trials, 16-bit thresholds) against the oracle's 16-bit mode, bit for bit, on
both annealing kernels, the batched launch and the no-allocation entry point.
"""
import ctypes

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


def _run(ia, inst, trials, betas, seed, kernel=0, shape=None, **kw):
    import torch
    prob = ia.Problem.from_instance(inst)
    prob.set_draw_bits(16)
    prob.set_kernel(kernel)
    if shape is not None:
        prob.set_launch(*shape)
    spins, cuts = ia.anneal(prob, trials, betas, seed, **kw)
    torch.cuda.synchronize()
    used = prob.last_kernel()
    assert prob.get_status() == 0
    prob.destroy()
    return spins.cpu().numpy(), cuts.cpu().numpy(), used


STRIP_CASES = [
    # X, Y, inst_seed, trials, sweeps, (group_trials, strips, threads)
    (4, 4, 1, 1, 30, None),
    (4, 4, 2, 37, 30, None),          # ragged: 37 = 4 x 8 + 5
    (6, 4, 3, 32, 20, (32, 1, 64)),
    (8, 8, 5, 100, 25, (16, 4, 64)),
    (10, 6, 6, 13, 25, (8, 3, 96)),
    (12, 10, 7, 70, 25, (24, 5, 128)),
    (50, 50, 9, 96, 40, None),
    (50, 50, 11, 64, 30, (32, 8, 128)),
    (200, 100, 13, 36, 8, (8, 7, 448)),
]


@pytest.mark.parametrize("X,Y,iseed,trials,S,shape", STRIP_CASES)
def test_strip_kernel_parity(ia, X, Y, iseed, trials, S, shape):
    inst = synth.torus_instance(X, Y, iseed)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0xABCD0000 + iseed
    gs, gc, used = _run(ia, inst, trials, betas, seed, kernel=1, shape=shape)
    assert used == 1
    rs, rc = oracle.anneal(inst, betas, seed, t_count=trials, draw_bits=16)
    np.testing.assert_array_equal(gs, rs)
    np.testing.assert_array_equal(gc, rc)


FLOW_CASES = [
    # X, Y, inst_seed, trials, sweeps, group_trials (0 = auto)
    (4, 4, 71, 64, 20, 0),
    (8, 6, 72, 37, 25, 0),
    (50, 50, 74, 1000, 12, 0),
    (100, 100, 75, 512, 10, 16),
    (200, 100, 77, 100, 8, 24),      # ragged last group
    (140, 100, 78, 7, 20, 0),
    (24, 16, 79, 3000, 5, 8),
]


@pytest.mark.parametrize("X,Y,iseed,trials,S,G", FLOW_CASES)
def test_flow_kernel_parity(ia, X, Y, iseed, trials, S, G):
    inst = synth.torus_instance(X, Y, iseed)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0x5EED1600 + iseed
    gs, gc, used = _run(ia, inst, trials, betas, seed, kernel=2, shape=(G, 0, 0) if G else None)
    assert used == 2
    if trials <= 128 or X * Y <= 2500:
        rs, rc = oracle.anneal(inst, betas, seed, t_count=trials, draw_bits=16)
        np.testing.assert_array_equal(gs, rs)
        np.testing.assert_array_equal(gc, rc)
    else:
        for t in (0, trials // 2, trials - 1):
            rs, rc = oracle.anneal(inst, betas, seed, t_begin=t, t_count=1, draw_bits=16)
            np.testing.assert_array_equal(gs[t], rs[0])
            assert gc[t] == rc[0]


def test_full_size_sampled_and_modes_differ(ia):
    """200x100, 1,024 trials x 10,000 sweeps in the default launch: trial 33g
    of every 32-trial group g against the oracle (every group, every bit
    position, the first and the last trial; a thread pool runs the C oracle
    without the interpreter lock); the fused cuts against the cut kernel;
    the 16-bit stream is not the 32-bit one, but the starting spins are."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    import torch
    inst = synth.torus_instance(200, 100, 2)
    betas = synth.linear_betas(0.1, 3.0, 10000)
    prob = ia.Problem.from_instance(inst)
    prob.set_draw_bits(16)
    spins, cuts = ia.anneal(prob, 1024, betas, 1002)
    recut = ia.cut(prob, spins)
    s0_16, _ = ia.anneal(prob, 64, np.zeros(0), 1002)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cuts.cpu().numpy(), recut.cpu().numpy())
    s = spins.cpu().numpy()
    c = cuts.cpu().numpy()
    sample = [33 * g for g in range(32)]
    oracle.lib()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        runs = list(ex.map(lambda t: oracle.anneal(inst, betas, 1002, t_begin=t, t_count=1, draw_bits=16), sample))
    for t, (rs, rc) in zip(sample, runs):
        np.testing.assert_array_equal(s[t], rs[0])
        assert c[t] == rc[0]
    prob.set_draw_bits(32)
    s32, _ = ia.anneal(prob, 64, betas[:50], 1002)
    s16_50 = ia.anneal(prob, 64, np.zeros(0), 1002)[0]
    prob.set_draw_bits(16)
    t16, _ = ia.anneal(prob, 64, betas[:50], 1002)
    torch.cuda.synchronize()
    assert torch.equal(s0_16, s16_50)                # same starting spins
    assert not torch.equal(s32, t16)                 # different decision streams
    prob.destroy()


def test_batched_and_noalloc_equal_single_call(ia):
    import torch
    cases = [(12, 8, 2, 64, 40, 12), (50, 50, 3, 33, 25, 13), (140, 100, 6, 40, 6, 16)]
    insts = [synth.torus_instance(X, Y, s) for (X, Y, s, _, _, _) in cases]
    probs = [ia.Problem.from_instance(i) for i in insts]
    for p in probs:
        p.set_draw_bits(16)
    trials = [c[3] for c in cases]
    sweeps = [c[4] for c in cases]
    betas = [synth.linear_betas(0.1, 3.0, S) for S in sweeps]
    seeds = [c[5] for c in cases]
    for kw in ({}, {"group_trials": 8, "ctas_per_sm": 1}, {"group_trials": 24, "ctas_per_sm": 2}):
        plan = ia.BatchPlan(probs, trials, sweeps, betas, seeds, **kw)
        bs, bc = plan.launch()
        torch.cuda.synchronize()
        for q, inst in enumerate(insts):
            rs, rc = oracle.anneal(inst, betas[q], seeds[q], t_count=trials[q], draw_bits=16)
            np.testing.assert_array_equal(bs[q].cpu().numpy(), rs)
            np.testing.assert_array_equal(bc[q].cpu().numpy(), rc)
        plan.destroy()
    # the no-allocation entry point in the 16-bit mode
    L = ia.lib()
    p, T = probs[1], trials[1]
    sp = torch.empty((T, p.n), dtype=torch.int8, device="cuda")
    ct = torch.empty((T,), dtype=torch.int32, device="cuda")
    b = np.ascontiguousarray(betas[1], dtype=np.float64)
    rc = L.ising_anneal_noalloc(p.handle, T, b.ctypes.data_as(ctypes.c_void_p), b.shape[0], seeds[1], 0, None,
                                ctypes.c_void_p(sp.data_ptr()), ctypes.c_void_p(ct.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    ref_s, ref_c = ia.anneal(p, T, betas[1], seeds[1])
    torch.cuda.synchronize()
    assert torch.equal(sp, ref_s) and torch.equal(ct, ref_c)
    for p in probs:
        p.destroy()


def test_mode_arguments(ia):
    inst = synth.torus_instance(8, 8, 1)
    prob = ia.Problem.from_instance(inst)
    for bad in (0, 8, 24, 64):
        with pytest.raises(ia.IsingError):
            prob.set_draw_bits(bad)
    prob.set_draw_bits(16)
    prob.set_launch(12, 0, 0)           # not a multiple of 8
    with pytest.raises(ia.IsingError):
        ia.anneal(prob, 24, synth.linear_betas(0.1, 3.0, 5), 1)
    prob.set_launch(16, 0, 0)
    ia.anneal(prob, 24, synth.linear_betas(0.1, 3.0, 5), 1)
    prob.destroy()
