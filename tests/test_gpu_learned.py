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


def test_window_and_batched_forms_equal_the_chunked_loop(ia):
    """The learned form with a proposal window: the sweeps before the window
    in one call (anneal_learned), or in one persistent launch over all
    instances (anneal_learned_batched), give the spins and cuts of the loop
    that runs every chunk on its own and proposes after the chunks that end
    past `start`."""
    import torch
    from paper_2505_18508_gb300 import learned
    S, every, tile, T, start = 400, 100, 2, 40, 250     # tiles per side: even (or one)
    insts = [synth.torus_instance(20, 12, 81), synth.torus_instance(24, 16, 82)]
    probs = [ia.Problem.from_instance(i) for i in insts]
    betas = synth.linear_betas(0.1, 3.0, S)
    seeds = [501, 502]
    net = ia.CNN(ocnn.init_params(9, scale=0.8))
    ref, n_acc = [], 0
    for p, sd in zip(probs, seeds):
        s = learned.initial_state(p, T, sd)
        for k0 in range(0, S, every):
            s, _ = ia.anneal(p, T, betas[k0:k0 + every], sd, sweep_offset=k0, init=s)
            if k0 + every > start:
                n_acc += int(ia.propose(p, s, net.forward(p, s), tile).sum().item())
        ref.append((s, ia.cut(p, s)))
    assert n_acc > 0
    assert learned.first_proposal_sweep(S, every, start) == 200
    for q, (p, sd) in enumerate(zip(probs, seeds)):
        st = {}
        s1, c1 = learned.anneal_learned(p, net, T, betas, sd, every=every, tile=tile, start=start, stats=st)
        torch.cuda.synchronize()
        assert torch.equal(s1, ref[q][0]) and torch.equal(c1, ref[q][1])
    sb, cb = learned.anneal_learned_batched(probs, net, T, betas, seeds, every=every, tile=tile, start=start)
    torch.cuda.synchronize()
    for q in range(len(probs)):
        assert torch.equal(sb[q], ref[q][0]) and torch.equal(cb[q], ref[q][1])
    # no window at all: the batched form is the plain batched annealer
    sp, cp = learned.anneal_learned_batched(probs, net, T, betas, seeds, every=every, tile=tile, start=S)
    for q, (p, sd) in enumerate(zip(probs, seeds)):
        s0, c0 = ia.anneal(p, T, betas, sd)
        torch.cuda.synchronize()
        assert torch.equal(sp[q], s0) and torch.equal(cp[q], c0)
    net.destroy()
    for p in probs:
        p.destroy()


def _host_loop(ia, probs, net, T, betas, seeds, k_first, every, partner_period=0, warm=False):
    """The learned form step by step through the single-call ABI: per problem
    the sweeps before the window (after the warm start), then per chunk each
    problem's sweeps (resumed), the network's logits and one cluster-proposal
    call over all problems, then the partner moves."""
    import torch
    states = []
    for p, sd in zip(probs, seeds):
        if warm:
            s0, _ = ia.anneal(p, T, np.zeros(0), sd)
            ia.propose(p, s0, net.forward(p, s0), 0)
            s, _ = ia.anneal(p, T, betas[:k_first], sd, init=s0)
        else:
            s, _ = ia.anneal(p, T, betas[:k_first], sd)
        states.append(s)
    s = torch.cat(states, 0).contiguous()
    logits_seen = []
    for j, k0 in enumerate(range(k_first, len(betas), every)):
        parts = []
        for q, (p, sd) in enumerate(zip(probs, seeds)):
            sq, _ = ia.anneal(p, T, betas[k0:k0 + every], sd, sweep_offset=k0, init=s[q * T:(q + 1) * T].contiguous())
            parts.append(sq)
        s = torch.cat(parts, 0).contiguous()
        if net is not None:
            z = torch.cat([net.forward(p, s[q * T:(q + 1) * T].contiguous()) for q, p in enumerate(probs)]).contiguous()
            logits_seen.append(z.cpu().numpy())
            ia.propose_clusters(probs, s, z)
        if partner_period:
            s, _ = ia.transcribe(probs, s, 1 + j % partner_period)
    cuts = torch.cat([ia.cut(p, s[q * T:(q + 1) * T].contiguous()) for q, p in enumerate(probs)])
    return s, cuts, logits_seen


def test_learned_plan_equals_plain_without_chunks_and_the_host_loop_with_them(ia):
    import torch
    X, Y, T, S, every = 24, 12, 40, 300, 100
    insts = [synth.torus_instance(X, Y, 300 + q) for q in range(3)]
    probs = [ia.Problem.from_instance(i) for i in insts]
    betas = synth.linear_betas(0.1, 3.0, S)
    seeds = [901, 902, 903]
    params = ocnn.init_params(7, scale=0.8)
    params[ocnn.N_PARAMS - 1] = 0.0
    net = ia.CNN(params)
    # no chunk: exactly the plain annealer
    plan = ia.LearnedPlan(probs, net, T, betas, seeds, k_first=S, every=every)
    s, c, acc = plan.launch()
    torch.cuda.synchronize()
    for q, (p, sd) in enumerate(zip(probs, seeds)):
        rs, rc = ia.anneal(p, T, betas, sd)
        assert torch.equal(s[q * T:(q + 1) * T], rs) and torch.equal(c[q * T:(q + 1) * T], rc)
    assert int(acc.sum().item()) == 0
    plan.destroy()
    # chunks from sweep 100: the graph equals the host loop, launch after launch
    plan = ia.LearnedPlan(probs, net, T, betas, seeds, k_first=100, every=every)
    hs, hc, logits_seen = _host_loop(ia, probs, net, T, betas, seeds, 100, every)
    for _ in range(2):
        s, c, acc = plan.launch()
        torch.cuda.synchronize()
        assert torch.equal(s, hs) and torch.equal(c, hc)
    assert int(acc.sum().item()) > 0
    # and the host loop equals the oracle fed the same logits
    for q, inst in enumerate(insts):
        rs, _ = oracle.anneal(inst, betas[:100], seeds[q], t_count=T)
        for j, k0 in enumerate(range(100, S, every)):
            rs, _ = oracle.anneal(inst, betas[k0:k0 + every], seeds[q], t_count=T, sweep_offset=k0, init=rs)
            rs, _ = ocnn.propose_clusters(rs, logits_seen[j][q * T:(q + 1) * T], inst["w_right"], inst["w_down"])
        np.testing.assert_array_equal(hs[q * T:(q + 1) * T].cpu().numpy(), rs)
        np.testing.assert_array_equal(hc[q * T:(q + 1) * T].cpu().numpy(),
                                      np.array([oracle.cut_csr(inst, r) for r in rs]))
    plan.destroy()
    # the window from sweep 0 (every chunk proposes)
    plan = ia.LearnedPlan(probs, net, T, betas, seeds, k_first=0, every=every)
    hs, hc, _ = _host_loop(ia, probs, net, T, betas, seeds, 0, every)
    s, c, _ = plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(s, hs) and torch.equal(c, hc)
    plan.destroy()
    net.destroy()
    for p in probs:
        p.destroy()


def test_learned_plan_partner_moves_and_warm_start(ia):
    import torch
    X, Y, T, S, every = 20, 10, 24, 400, 100
    insts = [synth.torus_instance(X, Y, 320 + q) for q in range(2)]
    probs = [ia.Problem.from_instance(i) for i in insts]
    betas = synth.linear_betas(0.1, 3.0, S)
    seeds = [77, 78]
    params = ocnn.init_params(9, scale=0.8)
    params[ocnn.N_PARAMS - 1] = -0.5
    net = ia.CNN(params)
    cases = [dict(net=None, partner_period=3, warm=False, k_first=100),
             dict(net=net, partner_period=2, warm=False, k_first=200),
             dict(net=net, partner_period=0, warm=True, k_first=100),
             dict(net=net, partner_period=1, warm=True, k_first=0)]
    for cs in cases:
        plan = ia.LearnedPlan(probs, cs["net"], T, betas, seeds, k_first=cs["k_first"], every=every,
                              partner_period=cs["partner_period"], warm=cs["warm"])
        hs, hc, logits_seen = _host_loop(ia, probs, cs["net"], T, betas, seeds, cs["k_first"], every,
                                         cs["partner_period"], cs["warm"])
        for _ in range(2):
            s, c, acc = plan.launch()
            torch.cuda.synchronize()
            assert torch.equal(s, hs) and torch.equal(c, hc), cs
        plan.destroy()
        if cs["warm"]:
            continue
        # the oracle fed the same logits: chunks, network block flips, partner moves
        rs_all = [oracle.anneal(inst, betas[:cs["k_first"]], seeds[q], t_count=T)[0] for q, inst in enumerate(insts)]
        for j, k0 in enumerate(range(cs["k_first"], S, every)):
            rs_all = [oracle.anneal(inst, betas[k0:k0 + every], seeds[q], t_count=T, sweep_offset=k0,
                                    init=rs_all[q])[0] for q, inst in enumerate(insts)]
            if cs["net"] is not None:
                rs_all = [ocnn.propose_clusters(rs_all[q], logits_seen[j][q * T:(q + 1) * T], inst["w_right"],
                                                inst["w_down"])[0] for q, inst in enumerate(insts)]
            if cs["partner_period"]:
                rs_all = [ocnn.transcribe(rs_all[q], 1 + j % cs["partner_period"], inst["w_right"], inst["w_down"])[0]
                          for q, inst in enumerate(insts)]
        for q, inst in enumerate(insts):
            np.testing.assert_array_equal(hs[q * T:(q + 1) * T].cpu().numpy(), rs_all[q])
            np.testing.assert_array_equal(hc[q * T:(q + 1) * T].cpu().numpy(),
                                          np.array([oracle.cut_csr(inst, r) for r in rs_all[q]]))
    net.destroy()
    for p in probs:
        p.destroy()


def test_config4_100x100_warm_start_block_flips_and_partner_gain(ia):
    """Config 4's shape (100x100, warm start plus block flips): a network
    trained briefly on droplet targets drives the plan, which equals the
    step-by-step host loop bit for bit; partner moves in the last window
    raise the mean cut over the plain annealer on the same instances and
    decision streams (every move is an exact energy decrease; the gain is
    large, tens of units of cut per trial)."""
    import torch
    from paper_2505_18508_gb300 import learned
    X, Y, T, S, every, window = 100, 100, 64, 2000, 100, 1000
    train = [ia.Problem.from_instance(synth.torus_instance(X, Y, 10000 + k)) for k in range(8)]
    data = learned.droplet_dataset(train, 8, synth.linear_betas(0.1, 3.0, 1000))
    net = ia.CNN(ocnn.init_params(5, scale=0.7))
    learned.train(net, data, 60, batch=8)
    for p in train:
        p.destroy()
    probs = [ia.Problem.from_instance(synth.torus_instance(X, Y, 20000 + q)) for q in range(2)]
    betas = synth.linear_betas(0.1, 3.0, S)
    seeds = [20000 + q for q in range(2)]
    kf = S - window
    plan = ia.LearnedPlan(probs, net, T, betas, seeds, k_first=kf, every=every, warm=True)
    s, c, _ = plan.launch()
    torch.cuda.synchronize()
    hs, hc, _ = _host_loop(ia, probs, net, T, betas, seeds, kf, every, 0, True)
    assert torch.equal(s, hs) and torch.equal(c, hc)
    plan.destroy()
    plain = ia.BatchPlan(probs, [T] * 2, [S] * 2, [betas] * 2, seeds, want_spins=False)
    _, pc = plain.launch()
    partner = ia.LearnedPlan(probs, None, T, betas, seeds, k_first=kf, every=every, partner_period=7)
    _, xc, xacc = partner.launch()
    torch.cuda.synchronize()
    plain_mean = torch.cat(pc).double().mean().item()
    partner_mean = xc.double().mean().item()
    assert int(xacc.sum().item()) > 0
    assert partner_mean > plain_mean + 10.0, (plain_mean, partner_mean)
    plain.destroy(); partner.destroy(); net.destroy()
    for p in probs:
        p.destroy()
