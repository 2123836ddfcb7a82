"""GPU parity for the learned proposal stage against the FP64 CPU oracle.

* logits within 2e-2 absolute of the FP64 forward (BF16 weights/activations);
* gradients within 3e-2 of the FP64 gradient, per parameter tensor, in norm;
* Adam: the update of the device master weights equals the Adam formula;
* proposals: bit-exact against the oracle fed with the same logits.
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


def _params(seed, scale=0.7):
    p = ocnn.init_params(seed, scale=scale)
    p[ocnn.N_PARAMS - 1] = -0.3
    return p


@pytest.mark.parametrize("X,Y,B", [(20, 10, 3), (24, 8, 2), (100, 100, 2), (200, 100, 1), (6, 4, 4)])
def test_forward_against_fp64(ia, X, Y, B):
    import torch
    inst = synth.torus_instance(X, Y, 5)
    params = _params(1)
    s = synth.random_spins(B, X * Y, 7)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(params)
    z = net.forward(prob, torch.from_numpy(s).cuda())
    torch.cuda.synchronize()
    ref = ocnn.forward(params, s, inst["w_right"], inst["w_down"]).reshape(B, -1)
    err = np.abs(z.cpu().numpy() - ref).max()
    assert err <= 2e-2, (err, np.abs(ref).max())
    net.destroy(); prob.destroy()


def _tensor_slices():
    out, o = [], 0
    for name, shp in ocnn.SHAPES:
        k = int(np.prod(shp))
        out.append((name, slice(o, o + k)))
        o += k
    return out


@pytest.mark.parametrize("X,Y,B", [(20, 10, 4), (50, 50, 2)])
def test_gradient_against_fp64(ia, X, Y, B):
    import torch
    inst = synth.torus_instance(X, Y, 9)
    params = _params(2)
    s = synth.random_spins(B, X * Y, 3)
    ref_state = synth.random_spins(B, X * Y, 4)
    y = ocnn.flip_targets(s, ref_state)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(params)
    loss, g = net.grad(prob, torch.from_numpy(s).cuda(), torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    rl, rg = ocnn.loss_and_grad(params, s, y, inst["w_right"], inst["w_down"])
    assert abs(loss.item() - rl) <= 1e-2 * abs(rl)
    gg = g.cpu().numpy().astype(np.float64)
    # layer-1 gradients pass through three BF16 forward and three BF16 backward
    # tensors and the ReLU masks of all three hidden layers (a pre-activation
    # within rounding of zero flips its mask): 6e-2 there, 3e-2 elsewhere
    errs = {name: np.linalg.norm(gg[sl] - rg[sl]) / (np.linalg.norm(rg[sl]) + 1e-12)
            for name, sl in _tensor_slices()}
    for name, e in errs.items():
        assert e <= (6e-2 if name in ("W1", "b1") else 3e-2), errs
    net.destroy(); prob.destroy()


def test_gradient_is_reproducible(ia):
    """Every reduction of the backward pass runs in a fixed order: the same
    batch gives the same gradient, bit for bit (so training is reproducible),
    on a batch large enough to spread over many CTAs."""
    import torch
    inst = synth.torus_instance(100, 100, 19)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(_params(5))
    s = torch.from_numpy(synth.random_spins(16, prob.n, 5)).cuda()
    y = torch.from_numpy(ocnn.flip_targets(synth.random_spins(16, prob.n, 5),
                                           synth.random_spins(16, prob.n, 6))).cuda()
    grads = [net.grad(prob, s, y)[1].clone() for _ in range(3)]
    torch.cuda.synchronize()
    assert all(torch.equal(grads[0], g) for g in grads[1:])
    net.destroy(); prob.destroy()


def test_adam_step_matches_formula(ia):
    import torch
    params = _params(3).astype(np.float32)
    net = ia.CNN(params)
    g = torch.from_numpy(np.random.default_rng(1).normal(size=ocnn.N_PARAMS).astype(np.float32)).cuda()
    net.adam_step(g, lr=1e-2)
    net.adam_step(g * 0.5, lr=1e-2)
    torch.cuda.synchronize()
    got = net.params().astype(np.float64)
    gh = g.cpu().numpy().astype(np.float64)
    m = np.zeros_like(gh); v = np.zeros_like(gh); w = params.astype(np.float64).copy()
    for t, gt in ((1, gh), (2, 0.5 * gh)):
        m = 0.9 * m + 0.1 * gt
        v = 0.999 * v + 0.001 * gt * gt
        w -= 1e-2 * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    np.testing.assert_allclose(got, w, rtol=1e-5, atol=1e-6)
    net.destroy()


def test_training_steps_reduce_loss(ia):
    import torch
    inst = synth.torus_instance(30, 20, 13)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(_params(4))
    s = torch.from_numpy(synth.random_spins(8, 600, 1)).cuda()
    y = torch.from_numpy(ocnn.flip_targets(synth.random_spins(8, 600, 1), synth.random_spins(8, 600, 2))).cuda()
    # target: a fixed pattern learnable from the inputs (flip where w_right = -1)
    y = torch.from_numpy(np.tile((inst["w_right"].reshape(-1) < 0).astype(np.uint8), (8, 1))).cuda()
    first = None
    for it in range(60):
        loss, g = net.grad(prob, s, y)
        net.adam_step(g, lr=3e-3)
        if first is None:
            first = loss.item()
    torch.cuda.synchronize()
    assert loss.item() < 0.5 * first
    net.destroy(); prob.destroy()


@pytest.mark.parametrize("X,Y,tile", [(20, 8, 5), (16, 8, 4), (26, 12, 7), (12, 8, 12), (100, 100, 10)])
def test_tile_proposals_against_oracle(ia, X, Y, tile):
    import torch
    inst = synth.torus_instance(X, Y, 17)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(_params(5))
    s = synth.random_spins(5, X * Y, 8)
    sd = torch.from_numpy(s).cuda()
    z = net.forward(prob, sd)
    acc = ia.propose(prob, sd, z, tile)
    torch.cuda.synchronize()
    rs, racc = ocnn.propose_tiles(s, z.cpu().numpy(), inst["w_right"], inst["w_down"], tile)
    np.testing.assert_array_equal(sd.cpu().numpy(), rs)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    for b in range(5):
        assert oracle.energy_csr(inst, rs[b]) <= oracle.energy_csr(inst, s[b])
    net.destroy(); prob.destroy()


def test_global_proposal_against_oracle(ia):
    import torch
    X, Y = 40, 30
    inst = synth.torus_instance(X, Y, 19)
    prob = ia.Problem.from_instance(inst)
    s = synth.random_spins(16, X * Y, 2)
    z = np.random.default_rng(6).normal(size=(16, X * Y)).astype(np.float32)
    z[3] = -1.0                      # empty proposal
    sd = torch.from_numpy(s).cuda()
    acc = ia.propose(prob, sd, torch.from_numpy(z).cuda(), 0)
    torch.cuda.synchronize()
    rs, racc = ocnn.propose_global(s, z, inst["w_right"], inst["w_down"])
    np.testing.assert_array_equal(sd.cpu().numpy(), rs)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    prob.destroy()


def test_bad_tile_counts_are_rejected(ia):
    import torch
    inst = synth.torus_instance(12, 8, 1)
    prob = ia.Problem.from_instance(inst)
    s = torch.from_numpy(synth.random_spins(1, 96, 1)).cuda()
    with pytest.raises(ia.IsingError):
        ia.propose(prob, s, torch.zeros((1, 96), device="cuda"), 4)
    prob.destroy()
