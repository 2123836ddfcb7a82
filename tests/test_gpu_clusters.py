"""Cluster moves (ising_propose_clusters, ising_droplet_targets) against the
CPU oracle, bit for bit: components of the logit > 0 sites flipped iff
dE <= 0, and droplet targets (improving components of the disagreement with
a gauge-aligned better state), on ragged and full-size tori, stacked
problems, and the degenerate masks (empty, everything, a tie in the gauge)."""
import numpy as np
import pytest

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


def _flipped(s, frac, seed):
    r = s.copy()
    m = np.random.default_rng(seed).random(s.shape) < frac
    r[m] = -r[m]
    return r


@pytest.mark.parametrize("X,Y,B", [(12, 8, 4), (20, 10, 3), (34, 6, 2), (50, 50, 2), (200, 100, 1)])
def test_droplet_targets_match_oracle(ia, X, Y, B):
    import torch
    inst = synth.torus_instance(X, Y, 70 + X)
    prob = ia.Problem.from_instance(inst)
    s = synth.random_spins(B, X * Y, 3 + X)
    for frac in (0.05, 0.3, 0.55):
        r = _flipped(s, frac, int(frac * 100) + X)
        got = ia.droplet_targets(prob, torch.from_numpy(s).cuda(), torch.from_numpy(r).cuda())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ocnn.droplet_targets(s, r, inst["w_right"], inst["w_down"]))
    prob.destroy()


def test_droplet_targets_on_annealed_states_and_ties(ia):
    import torch
    X, Y, T = 24, 12, 16
    inst = synth.torus_instance(X, Y, 5)
    prob = ia.Problem.from_instance(inst)
    s, c = ia.anneal(prob, T, synth.linear_betas(0.1, 3.0, 300), 9)
    best = s[int(c.argmax().item())].expand(T, -1).contiguous()
    got = ia.droplet_targets(prob, s, best)
    torch.cuda.synchronize()
    sn, bn = s.cpu().numpy(), best.cpu().numpy()
    ref = ocnn.droplet_targets(sn, bn, inst["w_right"], inst["w_down"])
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    # an exact gauge tie (n/2 sites differ) with site 0 equal and different
    n = X * Y
    s2 = synth.random_spins(2, n, 1)
    r2 = s2.copy()
    idx = np.arange(1, n // 2 + 1)
    r2[0, idx] = -r2[0, idx]                 # site 0 equal
    r2[1, :n // 2] = -r2[1, :n // 2]         # site 0 different
    got = ia.droplet_targets(prob, torch.from_numpy(s2).cuda(), torch.from_numpy(r2).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), ocnn.droplet_targets(s2, r2, inst["w_right"], inst["w_down"]))
    prob.destroy()


@pytest.mark.parametrize("X,Y,B", [(12, 8, 4), (20, 10, 3), (50, 50, 2), (200, 100, 1)])
def test_cluster_proposals_match_oracle(ia, X, Y, B):
    import torch
    inst = synth.torus_instance(X, Y, 90 + X)
    prob = ia.Problem.from_instance(inst)
    s = synth.random_spins(B, X * Y, 11 + X)
    rng = np.random.default_rng(X)
    for bias in (-1.0, 0.0, 0.6):
        z = (rng.normal(size=(B, X * Y)) + bias).astype(np.float32)
        sd = torch.from_numpy(s).cuda()
        acc = ia.propose_clusters(prob, sd, torch.from_numpy(z).cuda())
        torch.cuda.synchronize()
        rs, racc = ocnn.propose_clusters(s, z, inst["w_right"], inst["w_down"])
        np.testing.assert_array_equal(sd.cpu().numpy(), rs)
        np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    prob.destroy()


def test_cluster_proposals_stacked_problems_and_degenerate_masks(ia):
    import torch
    X, Y, B = 16, 10, 3
    insts = [synth.torus_instance(X, Y, 200 + q) for q in range(3)]
    probs = [ia.Problem.from_instance(i) for i in insts]
    s = synth.random_spins(3 * B, X * Y, 5)
    z = np.random.default_rng(1).normal(size=(3 * B, X * Y)).astype(np.float32)
    z[0] = -1.0                              # nothing proposed
    z[1] = 1.0                               # the whole torus: one component with no boundary, dE = 0
    sd = torch.from_numpy(s).cuda()
    acc = ia.propose_clusters(probs, sd, torch.from_numpy(z).cuda())
    torch.cuda.synchronize()
    got = sd.cpu().numpy()
    for q, inst in enumerate(insts):
        rs, racc = ocnn.propose_clusters(s[q * B:(q + 1) * B], z[q * B:(q + 1) * B], inst["w_right"], inst["w_down"])
        np.testing.assert_array_equal(got[q * B:(q + 1) * B], rs)
        np.testing.assert_array_equal(acc.cpu().numpy()[q * B:(q + 1) * B], racc)
    assert (got[0] == s[0]).all() and (got[1] == -s[1]).all()
    # limits: mixed shapes and an instance too large for one CTA's shared memory
    other = ia.Problem.from_instance(synth.torus_instance(X + 2, Y, 1))
    with pytest.raises(ia.IsingError):
        ia.propose_clusters([probs[0], other], torch.zeros((2, X * Y), dtype=torch.int8, device="cuda"),
                            torch.zeros((2, X * Y), device="cuda"))
    big = ia.Problem.from_instance(synth.torus_instance(200, 200, 1))
    with pytest.raises(ia.IsingError) as e:
        ia.propose_clusters(big, torch.zeros((1, 40000), dtype=torch.int8, device="cuda"),
                            torch.zeros((1, 40000), device="cuda"))
    assert e.value.code == -8
    for p in probs + [other, big]:
        p.destroy()


@pytest.mark.parametrize("X,Y,B,shift", [(12, 8, 5, 1), (12, 8, 5, 2), (50, 50, 3, 1), (200, 100, 2, 1), (16, 10, 4, 4)])
def test_partner_moves_match_oracle(ia, X, Y, B, shift):
    import torch
    inst = synth.torus_instance(X, Y, 400 + X)
    prob = ia.Problem.from_instance(inst)
    s = synth.random_spins(B, X * Y, 40 + X)
    sd = torch.from_numpy(s).cuda()
    out, acc = ia.transcribe(prob, sd, shift)
    torch.cuda.synchronize()
    rs, racc = ocnn.transcribe(s, shift, inst["w_right"], inst["w_down"])
    np.testing.assert_array_equal(out.cpu().numpy(), rs)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    assert (sd.cpu().numpy() == s).all()                      # the input is not modified
    prob.destroy()


def test_partner_moves_on_annealed_states_of_stacked_problems(ia):
    import torch
    X, Y, T = 24, 12, 8
    insts = [synth.torus_instance(X, Y, 500 + q) for q in range(2)]
    probs = [ia.Problem.from_instance(i) for i in insts]
    betas = synth.linear_betas(0.1, 3.0, 200)
    s = torch.cat([ia.anneal(p, T, betas, 31 + q)[0] for q, p in enumerate(probs)]).contiguous()
    out, acc = ia.transcribe(probs, s, 3)
    torch.cuda.synchronize()
    sn = s.cpu().numpy()
    for q, inst in enumerate(insts):
        rs, racc = ocnn.transcribe(sn[q * T:(q + 1) * T], 3, inst["w_right"], inst["w_down"])
        np.testing.assert_array_equal(out.cpu().numpy()[q * T:(q + 1) * T], rs)
        np.testing.assert_array_equal(acc.cpu().numpy()[q * T:(q + 1) * T], racc)
    with pytest.raises(ia.IsingError):
        ia.transcribe(probs, s, 1, out=s)                      # out may not alias the input
    for p in probs:
        p.destroy()


@pytest.mark.parametrize("X,Y", [(160, 132), (4, 6452)])
def test_cluster_moves_at_the_shared_memory_limit(ia, X, Y):
    """Sizes at the per-block shared-memory limit (227 KiB), which the kernel's
    static arrays share with its 9 bytes per site (and the 2-byte list of
    masked sites when that fits): 160x132 (21,120 sites) has room for the
    per-site arrays but not for the list beside the static arrays; 4x6452
    (25,808 sites) is the largest size that fits at all.  Proposals and
    partner moves equal the oracle's; 4x6454 is refused as unsupported and
    the next call is exact."""
    import torch
    inst = synth.torus_instance(X, Y, 600 + X)
    prob = ia.Problem.from_instance(inst)
    n, B = X * Y, 2
    s = synth.random_spins(B, n, 60 + X)
    z = (np.random.default_rng(X).normal(size=(B, n)) + 0.3).astype(np.float32)
    sd = torch.from_numpy(s).cuda()
    acc = ia.propose_clusters(prob, sd, torch.from_numpy(z).cuda())
    torch.cuda.synchronize()
    rs, racc = ocnn.propose_clusters(s, z, inst["w_right"], inst["w_down"])
    np.testing.assert_array_equal(sd.cpu().numpy(), rs)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    out, acc = ia.transcribe(prob, torch.from_numpy(s).cuda(), 1)
    torch.cuda.synchronize()
    rs, racc = ocnn.transcribe(s, 1, inst["w_right"], inst["w_down"])
    np.testing.assert_array_equal(out.cpu().numpy(), rs)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc)
    if X == 4:
        big = ia.Problem.from_instance(synth.torus_instance(4, Y + 2, 1))
        with pytest.raises(ia.IsingError) as e:
            ia.transcribe(big, torch.zeros((B, 4 * (Y + 2)), dtype=torch.int8, device="cuda"), 1)
        assert e.value.code == -8
        big.destroy()
        out2, _ = ia.transcribe(prob, torch.from_numpy(s).cuda(), 1)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out2.cpu().numpy(), rs)
    prob.destroy()
