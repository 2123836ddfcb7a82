"""GPU parity for the learned proposal stage against the FP64 CPU oracle.

* logits within 2e-2 absolute of the FP64 forward (BF16 weights/activations);
* gradients element by element against the FP64 gradient, on parameters
  built so that every hidden ReLU mask is unambiguous (see
  _unambiguous_params), and within 3e-2 per parameter tensor in norm on
  random parameters;
* flip targets (ising_flip_targets) equal to the oracle's, ties included;
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


# widths up to 512: three and four 128-pixel tiles per row (the accumulator
# ring of the convolution then fills all 512 tensor-memory columns)
@pytest.mark.parametrize("X,Y,B", [(20, 10, 3), (24, 8, 2), (100, 100, 2), (200, 100, 1), (6, 4, 4), (300, 6, 2),
                                   (512, 4, 1)])
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


def test_forward_refuses_widths_above_512(ia):
    import torch
    inst = synth.torus_instance(520, 4, 5)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(_params(1))
    with pytest.raises(ia.IsingError) as ei:
        net.forward(prob, torch.from_numpy(synth.random_spins(1, 520 * 4, 7)).cuda())
    assert ei.value.code == -8          # ISING_ERR_UNSUPPORTED
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


def _bf16_exact(a):
    a32 = np.asarray(a, dtype=np.float32)
    return np.array_equal(a32.view(np.uint32) & 0xFFFF, np.zeros(a32.shape, np.uint32))


def _abs_conv(h, W):
    """(|W| conv |h|) on the torus: per element the sum of |w| |a| over the
    terms of a pre-activation."""
    import torch
    F = torch.nn.functional
    t = torch.from_numpy(np.abs(h))
    return F.conv2d(F.pad(t, (1, 1, 1, 1), mode="circular"), torch.from_numpy(np.abs(W))).numpy()


def _unambiguous_params(inst, s, seed):
    """Parameters whose hidden ReLU masks are the same on the GPU as in FP64,
    asserted on the oracle's side.

    Layers 1 and 2 compute exactly on the GPU: the features are +-1, W1 holds
    multiples of 1/8 (|W1| <= 1/2) and b1 odd multiples of 1/16, so every
    layer-1 pre-activation is an odd multiple of 1/16 (|p1| >= 1/16) and every
    h1 = j/16 with j < 256 is exact in BF16; W2 holds multiples of 1/32
    (|W2| <= 1/4), so p2 - b2 is a multiple of 1/512 and its FP32 sums are
    exact, and b2 is an odd multiple of 1/1024 placed at the median of its
    channel (|p2| >= 1/1024, both signs occur).  h2 is rounded to BF16 (at
    most 2^-8 relative), so layer 3's pre-activations carry an error of at
    most e3 = 2^-8 (|W3| conv |h2|); each layer-3 channel is put entirely on
    or off with |p3| >= 2 e3 everywhere.  W3, W4 hold multiples of 1/64."""
    rng = np.random.default_rng(seed)
    P = {"W1": rng.integers(-4, 5, (32, 3, 3, 3)) / 8.0,
         "b1": (2 * rng.integers(-8, 8, 32) + 1) / 16.0,
         "W2": rng.integers(-8, 9, (32, 32, 3, 3)) / 32.0, "b2": np.zeros(32),
         "W3": rng.integers(-8, 9, (32, 32, 3, 3)) / 64.0, "b3": np.zeros(32),
         "W4": rng.integers(-8, 9, (1, 32, 3, 3)) / 64.0, "b4": np.array([-0.25])}

    def flat():
        return np.concatenate([P[name].reshape(-1) for name, _ in ocnn.SHAPES])

    def fwd():
        return ocnn.forward(flat(), s, inst["w_right"], inst["w_down"], return_all=True)

    v = fwd()["p2"]                       # b2 = 0: p2 - b2
    for o in range(32):
        med = np.median(v[:, o])
        P["b2"][o] = (2 * np.floor(-med * 512.0) + 1) / 1024.0
    f = fwd()
    v, e3 = f["p3"], 2.0 ** -8 * _abs_conv(f["h2"], P["W3"])
    for o in range(32):
        m = 2 * e3[:, o].max() + 2 ** -6
        P["b3"][o] = (-v[:, o].min() + m) if o % 2 == 0 else (-v[:, o].max() - m)
    P["b3"] = P["b3"].astype(np.float32).astype(np.float64)
    f = fwd()
    # the margins, on the oracle's side
    p1 = f["p1"]
    assert np.all(np.abs(p1) >= 1.0 / 16) and np.all((p1 * 16) % 2 == 1)
    assert np.all(f["h1"] * 16 < 256) and _bf16_exact(f["h1"])
    p2 = f["p2"]
    assert np.all(np.abs(p2) >= 1.0 / 1024) and np.all((p2 * 1024) % 2 == 1) and np.all(np.abs(p2) < 2 ** 14)
    for o in range(32):                    # both signs in every layer-2 channel
        assert (p2[:, o] > 0).any() and (p2[:, o] < 0).any()
    e3 = 2.0 ** -8 * _abs_conv(f["h2"], P["W3"])
    assert np.all(np.abs(f["p3"]) >= 2 * e3)
    params = flat()
    assert _bf16_exact(np.concatenate([P[k].reshape(-1) for k in ("W1", "W2", "W3", "W4")]))
    assert np.array_equal(params.astype(np.float32).astype(np.float64), params)
    return params


@pytest.mark.parametrize("X,Y,B,seed", [(12, 8, 3, 1), (20, 10, 2, 2), (34, 6, 2, 3)])
def test_gradient_elementwise_against_fp64(ia, X, Y, B, seed):
    """Every gradient element against FP64 autograd, with all ReLU masks
    fixed (above).  What remains is BF16 storage of h2, h3 and of the three
    backward activation gradients, each at most 2^-8 relative: a term passing
    six such roundings moves by < 6 * 2^-8 = 2.3e-2 of itself, hence
    |g - g64| <= 3e-2 |g64| + 1e-2 max|g64 of the tensor| (the absolute part
    covers elements whose terms cancel)."""
    import torch
    inst = synth.torus_instance(X, Y, 40 + seed)
    s = synth.random_spins(B, X * Y, 60 + seed)
    y = ocnn.flip_targets(s, synth.random_spins(B, X * Y, 80 + seed))
    params = _unambiguous_params(inst, s, seed)
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(params)
    loss, g = net.grad(prob, torch.from_numpy(s).cuda(), torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    rl, rg = ocnn.loss_and_grad(params, s, y, inst["w_right"], inst["w_down"])
    assert abs(loss.item() - rl) <= 1e-2 * abs(rl)
    gg = g.cpu().numpy().astype(np.float64)
    worst = {}
    for name, sl in _tensor_slices():
        d = np.abs(gg[sl] - rg[sl])
        tol = 3e-2 * np.abs(rg[sl]) + 1e-2 * np.abs(rg[sl]).max()
        worst[name] = float((d / tol).max())
        bad = np.nonzero(d > tol)[0]
        assert bad.size == 0, (name, bad[:8], gg[sl][bad[:8]], rg[sl][bad[:8]])
    print(worst)
    net.destroy(); prob.destroy()


def test_flip_targets_against_oracle_with_ties(ia):
    """ising_flip_targets equals the oracle's flip_targets, including rows with
    exactly n/2 differing sites, with site 0 equal and with site 0 different."""
    import torch
    rng = np.random.default_rng(12)
    n = 200
    s = synth.random_spins(12, n, 13)
    r = synth.random_spins(12, n, 14)
    for row in range(4, 12):                 # exact ties
        idx = rng.permutation(n)[: n // 2]
        if row % 2 == 0:
            idx = idx[idx != 0]
            idx = np.concatenate([idx, [next(i for i in range(1, n) if i not in set(idx))]])
        elif 0 not in idx:
            idx[0] = 0
        r[row] = s[row]
        r[row, idx] = -s[row, idx]
        assert (r[row] != s[row]).sum() == n // 2
        assert (r[row, 0] != s[row, 0]) == (row % 2 == 1)
    got = ia.flip_targets(torch.from_numpy(s).cuda(), torch.from_numpy(r).cuda())
    torch.cuda.synchronize()
    ref = ocnn.flip_targets(s, r)
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    assert (ref[4:, 0] == 0).all()
    # odd n and a single site
    for nn in (7, 1):
        s1 = synth.random_spins(5, nn, 15)
        r1 = synth.random_spins(5, nn, 16)
        got = ia.flip_targets(torch.from_numpy(s1).cuda(), torch.from_numpy(r1).cuda())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ocnn.flip_targets(s1, r1))


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


def test_tensor_core_wait_timeout_is_reported_and_next_call_is_exact(ia):
    """The test switch makes CTA 0 of every tensor-core launch wait on an
    mbarrier nothing arrives at, with a ~1 ms limit: the wait must run out,
    the kernel must still await its committed MMAs before freeing tensor
    memory, the status word must read ISING_ERR_TIMEOUT, and the next calls
    (forward and gradient) on the same context must be exact again."""
    import torch
    X, Y, B = 20, 10, 3
    inst = synth.torus_instance(X, Y, 5)
    params = _params(1)
    s = synth.random_spins(B, X * Y, 7)
    y = ocnn.flip_targets(s, synth.random_spins(B, X * Y, 8))
    prob = ia.Problem.from_instance(inst)
    net = ia.CNN(params)
    sd, yd = torch.from_numpy(s).cuda(), torch.from_numpy(y).cuda()
    ref_z = net.forward(prob, sd).clone()
    ref_loss, ref_g = net.grad(prob, sd, yd)
    ref_g = ref_g.clone()
    torch.cuda.synchronize()
    assert prob.get_status() == 0
    net.set_wait_limit(2_000_000, stall_test=1)            # about 1 ms of cycles
    net.forward(prob, sd)
    assert prob.get_status() == -7                          # ISING_ERR_TIMEOUT
    assert prob.get_status() == 0                           # read-and-clear
    net.grad(prob, sd, yd)
    assert prob.get_status() == -7
    net.set_wait_limit(0, 0)
    z = net.forward(prob, sd)
    loss, g = net.grad(prob, sd, yd)
    torch.cuda.synchronize()
    assert prob.get_status() == 0
    assert torch.equal(z, ref_z)                             # the same kernels, the same bits
    assert torch.equal(g, ref_g)                             # fixed-order reductions
    assert abs(loss.item() - ref_loss.item()) <= 1e-6 * abs(ref_loss.item())
    err = np.abs(z.cpu().numpy() - ocnn.forward(params, s, inst["w_right"], inst["w_down"]).reshape(B, -1)).max()
    assert err <= 2e-2
    net.destroy(); prob.destroy()
