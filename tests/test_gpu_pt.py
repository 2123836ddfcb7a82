"""GPU parity of replica exchange (ising_anneal_pt) against the oracle's
definition, bit for bit: spins, cuts and the number of swaps taken."""
import numpy as np
import pytest

import synth
from oracle import pt

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
    # X, Y, inst_seed, betas, chains, rounds, sweeps per round
    (20, 12, 1, [0.2, 0.5, 1.0, 2.0], 32, 6, 5),
    (50, 50, 2, [0.4, 0.7, 1.3], 64, 5, 4),
    (16, 8, 3, [0.9], 32, 3, 7),                 # one temperature: no swaps
    (12, 10, 4, [0.5, 0.5, 0.5], 32, 4, 2),      # equal temperatures: every swap taken
    (40, 30, 5, [0.3, 0.8], 32, 0, 5),           # no rounds: the start
    # large enough for the persistent kernel (per-group threshold tables)
    (64, 48, 7, [0.3, 0.6, 1.1, 2.0], 128, 4, 6),
    (64, 48, 8, [0.2, 0.35, 0.5, 0.7, 0.9, 1.2, 1.6, 2.4], 64, 5, 5),
]


@pytest.mark.parametrize("X,Y,iseed,betas,chains,rounds,L", CASES)
def test_pt_against_oracle(ia, X, Y, iseed, betas, chains, rounds, L):
    import torch
    inst = synth.torus_instance(X, Y, iseed)
    prob = ia.Problem.from_instance(inst)
    spins, cuts, swaps = ia.anneal_pt(prob, betas, chains, rounds, L, 0xBEEF + iseed)
    recut = ia.cut(prob, spins)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cuts.cpu().numpy(), recut.cpu().numpy())
    rs, rc, rsw = pt.anneal_pt(inst, betas, chains, rounds, L, 0xBEEF + iseed)
    np.testing.assert_array_equal(spins.cpu().numpy(), rs)
    np.testing.assert_array_equal(cuts.cpu().numpy(), rc)
    assert int(swaps.item()) == rsw
    prob.destroy()


def test_pt_arguments(ia):
    inst = synth.torus_instance(8, 8, 6)
    prob = ia.Problem.from_instance(inst)
    for bad in (dict(chains=16), dict(chains=33), dict(betas=[0.5, -1.0]), dict(betas=[0.5, float("inf")])):
        kw = dict(betas=[0.5, 1.0], chains=32)
        kw.update(bad)
        with pytest.raises(ia.IsingError):
            ia.anneal_pt(prob, kw["betas"], kw["chains"], 2, 2, 1)
    prob.destroy()


def test_pt_persistent_kernel_equals_strip_kernel(ia):
    """The headline-sized exchange (200 x 100, 8 temperatures x 128 chains)
    takes the persistent kernel; forcing the strip kernel gives the same
    spins, cuts and swap count."""
    import torch
    inst = synth.torus_instance(200, 100, 9)
    betas = list(np.geomspace(0.5, 3.0, 8))
    prob = ia.Problem.from_instance(inst)
    a = ia.anneal_pt(prob, betas, 128, 10, 20, 77)
    torch.cuda.synchronize()
    assert prob.last_kernel() == 2
    prob.set_kernel(1)
    b = ia.anneal_pt(prob, betas, 128, 10, 20, 77)
    torch.cuda.synchronize()
    assert prob.last_kernel() == 1
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and int(a[2].item()) == int(b[2].item())
    prob.destroy()
