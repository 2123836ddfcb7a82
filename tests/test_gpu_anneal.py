"""GPU parity: the CUDA annealer through the C ABI against the CPU oracle.

Bit-exact on spins and cuts (integer and bit work; the only floating point is
the host threshold table, computed with FP64 exp on both sides).
"""
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


def _gpu(ia, inst, trials, betas, seed, shape=None, kernel=0, **kw):
    import torch
    prob = ia.Problem.from_instance(inst)
    if shape is not None:
        prob.set_launch(*shape)
    prob.set_kernel(kernel)
    spins, cuts = ia.anneal(prob, trials, betas, seed, **kw)
    torch.cuda.synchronize()
    last = prob.last_launch()
    prob.destroy()
    return spins.cpu().numpy(), cuts.cpu().numpy(), last


CASES = [
    # X, Y, inst_seed, trials, sweeps, (group_trials, strips, threads)
    (4, 4, 1, 1, 30, None),
    (4, 4, 2, 37, 30, None),
    (6, 4, 3, 32, 20, (32, 1, 64)),
    (4, 6, 4, 64, 20, (32, 2, 64)),
    (8, 8, 5, 100, 25, (16, 4, 64)),
    (10, 6, 6, 33, 25, (4, 3, 96)),
    (12, 10, 7, 70, 25, (12, 5, 128)),
    (14, 8, 8, 29, 25, (28, 8, 64)),
    (50, 50, 9, 96, 40, None),
    (50, 50, 10, 64, 30, (32, 1, 1024)),
    (50, 50, 11, 64, 30, (32, 8, 128)),
    (140, 100, 12, 40, 10, None),
    (200, 100, 13, 36, 8, (8, 7, 448)),
]


@pytest.mark.parametrize("X,Y,iseed,trials,S,shape", CASES)
def test_parity_small(ia, X, Y, iseed, trials, S, shape):
    inst = synth.torus_instance(X, Y, iseed)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0xDEADBEEF00000000 + iseed
    gs, gc, last = _gpu(ia, inst, trials, betas, seed, shape)
    rs, rc = oracle.anneal(inst, betas, seed, t_count=trials)
    np.testing.assert_array_equal(gs, rs)
    np.testing.assert_array_equal(gc, rc)
    if shape is not None:
        assert (last["group_trials"], last["strips"], last["threads"]) == shape


def test_config1_full_parity(ia):
    """50x50 torus, 64 trials x 1,000 sweeps, beta linear 0.1 -> 3.0."""
    inst = synth.torus_instance(50, 50, 1)
    betas = synth.linear_betas(0.1, 3.0, 1000)
    gs, gc, _ = _gpu(ia, inst, 64, betas, 1001)
    rs, rc = oracle.anneal(inst, betas, 1001, t_count=64)
    np.testing.assert_array_equal(gs, rs)
    np.testing.assert_array_equal(gc, rc)


def test_brute_force_4x4_on_gpu(ia):
    inst = synth.torus_instance(4, 4, 11)
    edges = oracle.torus_edges(4, 4, inst["w_right"], inst["w_down"])
    _, Cmax, _, _ = oracle.brute_force(edges, 16)
    gs, gc, _ = _gpu(ia, inst, 256, synth.linear_betas(0.1, 3.0, 300), 5)
    assert gc.max() == Cmax and (gc == Cmax).mean() > 0.5
    for s, c in zip(gs, gc):
        assert int(oracle.cut_eq1(edges, s)) == c


def test_warm_start_and_resume(ia):
    import torch
    inst = synth.torus_instance(20, 12, 21)
    betas = synth.linear_betas(0.1, 3.0, 60)
    init = synth.random_spins(45, inst["n"], 4)
    prob = ia.Problem.from_instance(inst)
    s1, _ = ia.anneal(prob, 45, betas[:25], 9, init=torch.from_numpy(init).cuda())
    s2, c2 = ia.anneal(prob, 45, betas[25:], 9, sweep_offset=25, init=s1)
    torch.cuda.synchronize()
    rs, rc = oracle.anneal(inst, betas, 9, t_count=45, init=init)
    np.testing.assert_array_equal(s2.cpu().numpy(), rs)
    np.testing.assert_array_equal(c2.cpu().numpy(), rc)
    prob.destroy()


def test_zero_sweeps_zero_trials_and_infinite_beta(ia):
    import torch
    inst = synth.torus_instance(8, 6, 31)
    gs, gc, _ = _gpu(ia, inst, 10, np.zeros(0), 3)
    rs, rc = oracle.anneal(inst, np.zeros(0), 3, t_count=10)
    np.testing.assert_array_equal(gs, rs)
    np.testing.assert_array_equal(gc, rc)
    prob = ia.Problem.from_instance(inst)
    s, c = ia.anneal(prob, 0, np.zeros(3) + 1.0, 3)
    assert s.shape == (0, 48) and c.shape == (0,)
    prob.destroy()
    b = np.array([np.inf] * 5)
    gs, gc, _ = _gpu(ia, inst, 12, b, 8)
    rs, rc = oracle.anneal(inst, b, 8, t_count=12)
    np.testing.assert_array_equal(gs, rs)
    torch.cuda.synchronize()


def test_bad_betas_are_rejected(ia):
    inst = synth.torus_instance(8, 6, 31)
    prob = ia.Problem.from_instance(inst)
    for bad in (np.array([0.5, 0.0]), np.array([np.nan]), np.array([-1.0])):
        with pytest.raises(ia.IsingError) as e:
            ia.anneal(prob, 4, bad, 1)
        assert e.value.code == -1
    prob.destroy()


def test_cut_kernel_against_oracle(ia):
    import torch
    inst = synth.torus_instance(30, 20, 41)
    S = synth.random_spins(300, inst["n"], 5)
    prob = ia.Problem.from_instance(inst)
    got = ia.cut(prob, torch.from_numpy(S).cuda()).cpu().numpy()
    ref = np.array([oracle.cut_csr(inst, s) for s in S])
    np.testing.assert_array_equal(got, ref)
    # int8 values other than +-1 read as sign (>0 -> +1)
    S2 = (S * 3).astype(np.int8)
    S2[S2 < 0] = 0
    got2 = ia.cut(prob, torch.from_numpy(S2).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got2, ref)
    prob.destroy()


def test_gauge_invariance_on_gpu(ia):
    import torch
    X, Y = 16, 12
    inst = synth.torus_instance(X, Y, 51)
    tau = (2 * np.random.default_rng(3).integers(0, 2, size=(Y, X)) - 1).astype(np.int8)
    wr = inst["w_right"] * tau * np.roll(tau, -1, axis=1)
    wd = inst["w_down"] * tau * np.roll(tau, -1, axis=0)
    rp, col, J = synth.torus_csr(X, Y, wr, wd)
    inst2 = dict(inst, w_right=wr, w_down=wd, row_ptr=rp, col=col, J=J)
    init = synth.random_spins(64, X * Y, 6)
    betas = synth.linear_betas(0.1, 3.0, 80)
    p1, p2 = ia.Problem.from_instance(inst), ia.Problem.from_instance(inst2)
    a, _ = ia.anneal(p1, 64, betas, 4, init=torch.from_numpy(init).cuda())
    b, _ = ia.anneal(p2, 64, betas, 4, init=torch.from_numpy(init * tau.reshape(-1)).cuda())
    np.testing.assert_array_equal(b.cpu().numpy(), a.cpu().numpy() * tau.reshape(-1))
    p1.destroy(); p2.destroy()


def test_launch_shape_does_not_change_results(ia):
    inst = synth.torus_instance(24, 16, 61)
    betas = synth.linear_betas(0.1, 3.0, 50)
    ref = None
    for shape in [(32, 1, 1024), (32, 2, 128), (16, 4, 64), (8, 8, 64), (4, 8, 64), (20, 3, 96)]:
        gs, gc, _ = _gpu(ia, inst, 77, betas, 123, shape)
        if ref is None:
            ref = (gs, gc)
        else:
            np.testing.assert_array_equal(gs, ref[0])
            np.testing.assert_array_equal(gc, ref[1])


def test_config2_full_size_sampled(ia):
    """200x100, 1,024 trials x 10,000 sweeps in the benchmark's launch shape:
    one trial of every 32-trial group against the oracle (trial 33g of group g,
    so the sample also walks through every bit position of a word, from the
    first trial to the last), run in a thread pool (the C oracle runs without
    the interpreter lock); every trial's fused cut against the separate cut
    kernel."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    import torch
    inst = synth.torus_instance(200, 100, 2)
    betas = synth.linear_betas(0.1, 3.0, 10000)
    prob = ia.Problem.from_instance(inst)
    spins, cuts = ia.anneal(prob, 1024, betas, 1002)
    recut = ia.cut(prob, spins)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cuts.cpu().numpy(), recut.cpu().numpy())
    s = spins.cpu().numpy()
    c = cuts.cpu().numpy()
    sample = [33 * g for g in range(32)]
    assert sample[0] == 0 and sample[-1] == 1023
    oracle.lib()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        runs = list(ex.map(lambda t: oracle.anneal(inst, betas, 1002, t_begin=t, t_count=1), sample))
    for t, (rs, rc) in zip(sample, runs):
        np.testing.assert_array_equal(s[t], rs[0])
        assert c[t] == rc[0]
    prob.destroy()


# ---------------------------------------------------------------- persistent kernel
FLOW_CASES = [
    # X, Y, inst_seed, trials, sweeps, group_trials (0 = auto)
    (4, 4, 71, 64, 20, 0),
    (8, 6, 72, 37, 25, 0),
    (50, 50, 73, 64, 40, 0),
    (50, 50, 74, 1000, 12, 0),     # many groups: CTAs span several groups
    (100, 100, 75, 512, 10, 16),
    (200, 100, 76, 1024, 6, 0),
    (200, 100, 77, 100, 8, 28),    # ragged last group
    (140, 100, 78, 7, 20, 0),      # a single partial group over many CTAs
    (24, 16, 79, 3000, 5, 8),
]


@pytest.mark.parametrize("X,Y,iseed,trials,S,G", FLOW_CASES)
def test_flow_kernel_parity(ia, X, Y, iseed, trials, S, G):
    inst = synth.torus_instance(X, Y, iseed)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0x5EED0000 + iseed
    import torch
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(2)
    if G:
        prob.set_launch(G, 0, 0)
    spins, cuts = ia.anneal(prob, trials, betas, seed)
    torch.cuda.synchronize()
    assert prob.last_kernel() == 2
    assert prob.get_status() == 0
    gs, gc = spins.cpu().numpy(), cuts.cpu().numpy()
    prob.destroy()
    if trials <= 128 or X * Y <= 2500:
        rs, rc = oracle.anneal(inst, betas, seed, t_count=trials)
        np.testing.assert_array_equal(gs, rs)
        np.testing.assert_array_equal(gc, rc)
    else:   # first, middle and last trial
        for t in (0, trials // 2, trials - 1):
            rs, rc = oracle.anneal(inst, betas, seed, t_begin=t, t_count=1)
            np.testing.assert_array_equal(gs[t], rs[0])
            assert gc[t] == rc[0]


def test_flow_equals_strip_kernel_and_resume(ia):
    import torch
    inst = synth.torus_instance(200, 100, 80)
    betas = synth.linear_betas(0.1, 3.0, 60)
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(1)
    a_s, a_c = ia.anneal(prob, 1024, betas, 9)
    prob.set_kernel(2)
    b_s, b_c = ia.anneal(prob, 1024, betas, 9)
    half, _ = ia.anneal(prob, 1024, betas[:25], 9)
    c_s, c_c = ia.anneal(prob, 1024, betas[25:], 9, sweep_offset=25, init=half)
    torch.cuda.synchronize()
    assert torch.equal(a_s, b_s) and torch.equal(a_c, b_c)
    assert torch.equal(a_s, c_s) and torch.equal(a_c, c_c)
    # cuts only, no spins
    _, d_c = ia.anneal(prob, 1024, betas, 9, want_spins=False)
    torch.cuda.synchronize()
    assert torch.equal(a_c, d_c)
    prob.destroy()


def test_flow_wait_timeout_is_reported_and_context_survives(ia):
    """A wait that nothing satisfies (test switch) must give up after its
    limit, report ISING_ERR_TIMEOUT through the status word, and leave the
    context usable for the next, normal call."""
    import torch
    inst = synth.torus_instance(100, 100, 81)
    betas = synth.linear_betas(0.1, 3.0, 20)
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(2)
    prob.set_wait_limit(2_000_000, stall_test=1)       # about 1 ms of cycles
    ia.anneal(prob, 256, betas, 3)
    assert prob.get_status() == -7                      # ISING_ERR_TIMEOUT
    assert prob.get_status() == 0                       # read-and-clear
    prob.set_wait_limit(0, 0)
    s, c = ia.anneal(prob, 64, betas, 3)
    torch.cuda.synchronize()
    assert prob.get_status() == 0
    rs, rc = oracle.anneal(inst, betas, 3, t_count=64)
    np.testing.assert_array_equal(s.cpu().numpy(), rs)
    np.testing.assert_array_equal(c.cpu().numpy(), rc)
    prob.destroy()
