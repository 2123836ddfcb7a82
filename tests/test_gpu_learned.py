"""The learned form end to end.

* parity: the GPU's learned loop (anneal chunks, network logits, tile
  proposals) against the CPU oracle fed with the same logits -- spins and cuts
  bit for bit;
* training on the plain annealer's own trajectories lowers the loss;
* gain: what the trained network's proposals add to the annealer at the
  proposal points (energy drop, which the plain method does not have there),
  compared with an untrained network of the same shape.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ia():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    torch.cuda.set_device(0)
    return ia


def test_learned_loop_matches_oracle(ia):
    import torch
    X, Y, T, S, every, tile, seed = 24, 12, 40, 300, 100, 2, 4242
    inst = synth.torus_instance(X, Y, 61)
    betas = synth.linear_betas(0.1, 3.0, S)
    prob = ia.Problem.from_instance(inst)
    params = ocnn.init_params(7, scale=0.8)
    params[ocnn.N_PARAMS - 1] = 0.0
    net = ia.CNN(params)
    s, _ = ia.anneal(prob, T, np.zeros(0), seed)
    logits_seen = []
    n_acc = 0
    for k0 in range(0, S, every):
        s, _ = ia.anneal(prob, T, betas[k0:k0 + every], seed, sweep_offset=k0, init=s)
        z = net.forward(prob, s)
        logits_seen.append(z.cpu().numpy())
        n_acc += int(ia.propose(prob, s, z, tile).sum().item())
    cuts = ia.cut(prob, s)
    torch.cuda.synchronize()
    assert n_acc > 0
    # oracle: same anneal chunks, proposals decided from the GPU's logits
    rs, _ = oracle.anneal(inst, np.zeros(0), seed, t_count=T)
    for j, k0 in enumerate(range(0, S, every)):
        rs, _ = oracle.anneal(inst, betas[k0:k0 + every], seed, t_count=T, sweep_offset=k0, init=rs)
        rs, _ = ocnn.propose_tiles(rs, logits_seen[j], inst["w_right"], inst["w_down"], tile)
    np.testing.assert_array_equal(s.cpu().numpy(), rs)
    np.testing.assert_array_equal(cuts.cpu().numpy(), np.array([oracle.cut_csr(inst, r) for r in rs]))
    # the logits themselves, against the FP64 forward on the same states
    ref = ocnn.forward(params, rs, inst["w_right"], inst["w_down"]).reshape(T, -1)
    got = net.forward(prob, s).cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-2
    net.destroy(); prob.destroy()


def test_training_and_gain_at_proposal_points(ia):
    import torch
    from paper_2505_18508_gb300 import learned
    S, every = 600, 100
    betas = synth.linear_betas(0.1, 3.0, S)
    train = [synth.torus_instance(50, 50, 10000 + k) for k in range(48)]
    data = learned.make_dataset(train, betas, every, snap_trials=4, target="future")
    net = ia.CNN(ocnn.init_params(3, scale=0.7))
    losses = learned.train(net, data, 1200, batch=16, lr=2e-3, log_every=100)
    first, last = losses[0][1], np.mean([l for _, l in losses[-3:]])
    assert last < 0.85 * first, losses
    untrained = ia.CNN(ocnn.init_params(3, scale=0.7))

    def gain(model):
        """Mean cut gained by the proposal rounds, summed over the rounds."""
        total = 0.0
        for q in range(3):
            inst = synth.torus_instance(50, 50, 20000 + q)
            prob = ia.Problem.from_instance(inst)
            s, _ = ia.anneal(prob, 256, np.zeros(0), 99 + q)
            for k0 in range(0, S, every):
                s, _ = ia.anneal(prob, 256, betas[k0:k0 + every], 99 + q, sweep_offset=k0, init=s)
                before = ia.cut(prob, s).double().mean().item()
                ia.propose(prob, s, model.forward(prob, s), 5)
                after = ia.cut(prob, s).double().mean().item()
                assert after >= before          # exact acceptance never loses energy
                total += after - before
            prob.destroy()
        return total / 3

    g_trained, g_untrained = gain(net), gain(untrained)
    assert g_trained > 0.0
    assert g_trained > g_untrained
    net.destroy(); untrained.destroy()
