"""Parallel tempering (replica exchange) on the torus: the oracle's
definition.  TEST INFRASTRUCTURE ONLY -- only the tests, the smoke run and the
benchmark's CPU-baseline leg may use it.

The paper's update rule is unpublished (Section III); replica exchange is a
variant of this project built on the same Metropolis sweep.  Definition:

* R temperatures beta_0 < ... < beta_{R-1}, C chains; trial slot
  t = r * C + c holds chain c's replica at temperature r.  A slot keeps its
  random stream (the sweep draws of trial index t) whatever configuration a
  swap moves into it.
* Start: the annealer's start spins of every slot (trial index t).
* Round q = 0 .. Q-1: every slot runs L sweeps at its constant beta_r,
  global sweeps q L .. q L + L - 1 (oracle.anneal with t_begin = r C).  Then
  the pairs (r, r+1) with r = q mod 2, q mod 2 + 2, ... exchange, for every
  chain c: with d = E_{r,c} - E_{r+1,c} (Eq. 2 energies, E = W - 2 cut) the
  swap is accepted iff d <= 0 or u < T, where
  T = min(floor(exp(-(beta_{r+1} - beta_r) d) 2^32), 2^32 - 1) and u is word 0
  of Philox4x32-10 at counter (c, q, r, 0xFFFFFFFD) under the run's key
  (Metropolis acceptance min(1, exp((beta_r - beta_{r+1})(E_r - E_{r+1})))).
  An accepted swap exchanges the two slots' configurations.
"""
from __future__ import annotations

import math

import numpy as np

from . import anneal, philox4x32_10, torus_edges


def swap_threshold(dbeta, d):
    """T = min(floor(exp(-dbeta d) 2^32), 2^32 - 1) for d > 0."""
    v = math.floor(math.exp(-(dbeta * d)) * 4294967296.0)
    return min(v, 4294967295)


def anneal_pt(inst, betas, chains, rounds, sweeps_per_round, seed):
    """Returns (spins int8 [R*C, n], cuts int32 [R*C], accepted swaps int)."""
    R, C, L = len(betas), int(chains), int(sweeps_per_round)
    T = R * C
    n = int(inst["n"])
    edges = torus_edges(inst["X"], inst["Y"], inst["w_right"], inst["w_down"])
    W = int(edges[2].sum())
    spins, cuts = anneal(inst, np.zeros(0), seed, t_count=T)
    key = (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    swaps = 0
    for q in range(rounds):
        for r in range(R):
            sl = slice(r * C, (r + 1) * C)
            spins[sl], cuts[sl] = anneal(inst, np.full(L, float(betas[r])), seed, t_begin=r * C, t_count=C,
                                         sweep_offset=q * L, init=spins[sl])
        E = W - 2 * cuts.astype(np.int64)
        for r in range(q % 2, R - 1, 2):
            dbeta = float(betas[r + 1]) - float(betas[r])
            for c in range(C):
                a, b = r * C + c, (r + 1) * C + c
                d = int(E[a] - E[b])
                take = d <= 0
                if not take:
                    u = philox4x32_10((c, q, r, 0xFFFFFFFD), key)[0]
                    take = u < swap_threshold(dbeta, d)
                if take:
                    spins[[a, b]] = spins[[b, a]]
                    cuts[[a, b]] = cuts[[b, a]]
                    E[[a, b]] = E[[b, a]]
                    swaps += 1
    return spins, cuts, swaps
