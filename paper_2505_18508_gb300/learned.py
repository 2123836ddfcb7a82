"""The learned form of the annealer: training data, training, and annealing
with network proposals.  Orchestration only: every numeric step runs in the
library's kernels (ising_anneal, ising_cnn_*, ising_propose,
ising_flip_targets, ising_cut), called through the C ABI.

Learned anneal (per instance, T trials, schedule of S sweeps):
    s <- the Philox starting state (ising_anneal with no sweeps)
    optional warm start: logits = CNN(s); whole-lattice proposal
    the sweeps before the first chunk that ends past `start`: one ising_anneal
    for every later chunk of `every` sweeps:
        s <- ising_anneal(the chunk's betas, sweep_offset = chunk start, init = s)
        logits = CNN(s); tile proposals (exact dE <= 0 acceptance)
    cuts <- ising_cut(s)
The batched form runs the sweeps before the proposal window for all
instances in one persistent launch (ising_anneal_batched), then the window
instance by instance; its results equal the per-instance form's, since the
random stream is keyed by site, sweep and trial and a resumed run continues
exactly.
Every proposal is judged by its exact integer energy change, so the plain
annealer's moves are never undone by a bad proposal; with the proposals
removed the loop is exactly the plain annealer (resume is bit-exact).

Training data (held-out instances): the plain annealer's best state r of each
instance (best cut over `ref_trials` trials of the full schedule) and
snapshots s of other trials at the end of each chunk; targets are the
gauge-aligned flip targets [s != +-r].

The cluster form (LearnedPlan, one CUDA graph over several instances) uses
connected-component block flips instead of tiles, trained on droplet
targets (droplet_dataset): the improving components of each final state's
disagreement with its instance's best state.  Its proposals can also take
their blocks from a partner trial instead of the network (partner moves).
"""
from __future__ import annotations

import numpy as np

from . import CNN, Problem, anneal, anneal_batched, cut, droplet_targets, flip_targets, propose  # noqa: F401


def _torch():
    import torch
    return torch


def initial_state(prob, trials, seed):
    """The Philox starting configuration (no sweeps)."""
    s, _ = anneal(prob, trials, np.zeros(0), seed)
    return s


def best_state(prob, trials, betas, seed):
    """Best (highest-cut) final state of `trials` plain trials: int8 [n] device."""
    s, c = anneal(prob, trials, betas, seed)
    i = int(c.argmax().item())
    return s[i].clone(), int(c[i].item())


def snapshots(prob, trials, betas, seed, every):
    """States of `trials` plain trials at the end of every chunk: int8 [chunks*trials, n]."""
    torch = _torch()
    S = len(betas)
    s = initial_state(prob, trials, seed)
    out = []
    for k0 in range(0, S, every):
        s, _ = anneal(prob, trials, betas[k0:k0 + every], seed, sweep_offset=k0, init=s)
        out.append(s.clone())
    return torch.cat(out, 0)


def make_dataset(instances, betas, every, snap_trials=4, ref_trials=32, seed=77, target="future"):
    """[(Problem, spins int8 [m, n], targets uint8 [m, n], best cut)] on the device.

    target "future": each snapshot against the final state of the same trial
    (where will the anneal still change this state); target "best": against
    the instance's best state over `ref_trials` full trials.
    """
    torch = _torch()
    data = []
    for q, inst in enumerate(instances):
        prob = Problem.from_instance(inst)
        s = snapshots(prob, snap_trials, betas, seed + 1000 * q + 1, every)
        if target == "best":
            ref, best = best_state(prob, ref_trials, betas, seed + 1000 * q)
            refs = ref.expand(s.shape[0], -1).contiguous()
        else:
            final = s[-snap_trials:]
            refs = final.repeat(s.shape[0] // snap_trials, 1)
            best = int(cut(prob, final).max().item())
        y = flip_targets(s, refs)
        keep = torch.ones(s.shape[0], dtype=torch.bool, device=s.device)
        if target != "best":
            keep[-snap_trials:] = False       # the final states themselves have empty targets
        data.append((prob, s[keep].contiguous(), y[keep].contiguous(), best))
    return data


def train(net, data, steps, batch=16, lr=2e-3, seed=0, log_every=0):
    """Adam on mini-batches drawn from one instance at a time; returns losses."""
    torch = _torch()
    rng = np.random.Generator(np.random.PCG64(seed))
    losses = []
    for it in range(steps):
        prob, s, y, _ = data[it % len(data)]
        idx = torch.from_numpy(rng.choice(s.shape[0], size=min(batch, s.shape[0]), replace=False)).cuda()
        loss, g = net.grad(prob, s.index_select(0, idx), y.index_select(0, idx))
        net.adam_step(g, lr=lr)
        if log_every and (it % log_every == 0 or it == steps - 1):
            losses.append((it, float(loss.item())))
    return losses


def first_proposal_sweep(S, every, start):
    """Start of the first `every`-sweep chunk that ends past sweep `start`
    (chunks begin at multiples of `every`); S if there is none."""
    k = max(0, -(-(start - every + 1) // every) * every)
    return min(k, S)


def _proposal_window(prob, net, s, trials, betas, seed, k_first, every, tile, acc_total, logits):
    for k0 in range(k_first, len(betas), every):
        s, _ = anneal(prob, trials, betas[k0:k0 + every], seed, sweep_offset=k0, init=s)
        net.forward(prob, s, out=logits)
        acc_total += propose(prob, s, logits, tile).to(acc_total.dtype)
    return s


def anneal_learned(prob, net, trials, betas, seed, every=100, tile=10, warm=False, stats=None, start=0):
    """The learned form; returns (spins, cuts) on the device.  Proposal rounds
    run after every chunk that ends past sweep `start`; the sweeps before the
    first such chunk run in one call."""
    torch = _torch()
    S = len(betas)
    s = initial_state(prob, trials, seed)
    acc_total = torch.zeros(trials, dtype=torch.int64, device=s.device)
    logits = torch.empty((trials, prob.n), dtype=torch.float32, device=s.device)
    if warm:
        net.forward(prob, s, out=logits)
        acc_total += propose(prob, s, logits, 0).to(torch.int64)
    k_first = first_proposal_sweep(S, every, start)
    if k_first > 0:
        s, _ = anneal(prob, trials, betas[:k_first], seed, init=s)
    s = _proposal_window(prob, net, s, trials, betas, seed, k_first, every, tile, acc_total, logits)
    cuts = cut(prob, s)
    if stats is not None:
        stats["accepted_per_trial"] = float(acc_total.double().mean().item())
    return s, cuts


def anneal_learned_batched(probs, net, trials, betas, seeds, every=100, tile=10, start=0):
    """The learned form over several instances (the same trial count and
    schedule, one seed each): the sweeps before the proposal window in one
    persistent launch over all instances, then each instance's window.
    Returns ([spins], [cuts]); instance q's results equal
    anneal_learned(probs[q], net, trials, betas, seeds[q], every, tile,
    start=start)."""
    torch = _torch()
    S = len(betas)
    m = len(probs)
    k_first = first_proposal_sweep(S, every, start)
    if k_first > 0:
        states, _ = anneal_batched(probs, [trials] * m, [k_first] * m, [betas[:k_first]] * m, list(seeds))
    else:
        states = [initial_state(p, trials, sd) for p, sd in zip(probs, seeds)]
    spins, cuts = [], []
    for p, sd, s in zip(probs, seeds, states):
        acc_total = torch.zeros(trials, dtype=torch.int64, device=s.device)
        logits = torch.empty((trials, p.n), dtype=torch.float32, device=s.device)
        s = _proposal_window(p, net, s, trials, betas, sd, k_first, every, tile, acc_total, logits)
        spins.append(s)
        cuts.append(cut(p, s))
    return spins, cuts


def droplet_dataset(probs, trials, betas, seed=50000):
    """[(Problem, final states int8 [trials, n], droplet targets uint8
    [trials, n], best cut)] for each problem: `trials` plain anneals of the
    full schedule (all problems in batched launches of up to 8), targets
    against the best final state of the problem (ising_droplet_targets)."""
    data = []
    for g0 in range(0, len(probs), 8):
        group = probs[g0:g0 + 8]
        spins, cuts = anneal_batched(group, [trials] * len(group), [len(betas)] * len(group), [betas] * len(group),
                                     [seed + g0 + q for q in range(len(group))])
        for p, s, c in zip(group, spins, cuts):
            best = s[int(c.argmax().item())]
            y = droplet_targets(p, s, best.expand(s.shape[0], -1).contiguous())
            data.append((p, s, y, int(c.max().item())))
    return data
