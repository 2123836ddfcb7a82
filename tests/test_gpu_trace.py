"""GPU parity of the read-out along the trajectory (ising_anneal_trace): the
cut after every traced sweep, the best-so-far cut and its configuration,
against the oracle's trajectory read-out, bit for bit; and the final state
equal to one plain ising_anneal call."""
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


CASES = [
    # X, Y, inst_seed, trials, sweeps, trace_every, kernel, draw_bits
    (4, 4, 1, 9, 30, 10, 1, 32),
    (8, 6, 2, 37, 31, 10, 1, 32),       # ragged last chunk
    (12, 10, 3, 40, 7, 1, 1, 32),       # a point after every sweep
    (10, 8, 4, 20, 5, 9, 1, 32),        # one chunk shorter than trace_every
    (50, 50, 5, 64, 60, 25, 2, 32),     # persistent kernel
    (50, 50, 6, 48, 40, 15, 2, 16),     # 16-bit draw mode
    (100, 100, 7, 512, 12, 5, 2, 32),   # many trial groups
]


@pytest.mark.parametrize("X,Y,iseed,trials,S,every,kernel,bits", CASES)
def test_trace_against_oracle(ia, X, Y, iseed, trials, S, every, kernel, bits):
    import torch
    inst = synth.torus_instance(X, Y, iseed)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0x7AC30000 + iseed
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(kernel)
    prob.set_draw_bits(bits)
    spins, cuts, trace, best, bspins = ia.anneal_trace(prob, trials, betas, seed, every)
    plain_s, plain_c = ia.anneal(prob, trials, betas, seed)
    torch.cuda.synchronize()
    assert torch.equal(spins, plain_s) and torch.equal(cuts, plain_c)
    prob.destroy()
    sub = slice(None) if trials <= 64 else slice(0, 64)
    rs, rc, rtr, rb, rbs = oracle.anneal_trace(inst, betas, seed, every, t_count=trials if trials <= 64 else 64,
                                               draw_bits=bits)
    np.testing.assert_array_equal(spins.cpu().numpy()[sub], rs)
    np.testing.assert_array_equal(cuts.cpu().numpy()[sub], rc)
    np.testing.assert_array_equal(trace.cpu().numpy()[:, sub], rtr)
    np.testing.assert_array_equal(best.cpu().numpy()[sub], rb)
    np.testing.assert_array_equal(bspins.cpu().numpy()[sub], rbs)


def test_trace_resume_and_zero_sweeps(ia):
    import torch
    inst = synth.torus_instance(16, 12, 9)
    betas = synth.linear_betas(0.1, 3.0, 40)
    prob = ia.Problem.from_instance(inst)
    half, _ = ia.anneal(prob, 24, betas[:15], 3)
    s, c, tr, b, bs = ia.anneal_trace(prob, 24, betas[15:], 3, 10, sweep_offset=15, init=half)
    full_s, full_c = ia.anneal(prob, 24, betas, 3)
    s0, c0, tr0, b0, bs0 = ia.anneal_trace(prob, 24, np.zeros(0), 3, 4)
    torch.cuda.synchronize()
    assert torch.equal(s, full_s) and torch.equal(c, full_c)
    assert tr.shape == (3, 24) and torch.equal(tr[-1], c)
    assert tr0.shape == (0, 24) and torch.equal(b0, c0) and torch.equal(bs0, s0)
    rs, rc, rtr, rb, rbs = oracle.anneal_trace(inst, betas[15:], 3, 10, t_count=24, sweep_offset=15,
                                               init=half.cpu().numpy())
    np.testing.assert_array_equal(tr.cpu().numpy(), rtr)
    np.testing.assert_array_equal(b.cpu().numpy(), rb)
    np.testing.assert_array_equal(bs.cpu().numpy(), rbs)
    with pytest.raises(ia.IsingError):
        ia.anneal_trace(prob, 24, betas, 3, 0)
    prob.destroy()
