"""Pins for the oracle's general-graph annealer (integer couplings, fields),
each against something other than that code itself:

* the greedy colouring is proper and first-fit (checked by brute force), and
  on an even torus it is the checkerboard;
* on a torus the general annealer equals the torus annealer bit for bit;
* on tiny graphs it equals a pure-Python restatement that takes every dE as a
  difference of whole-graph energies (Eq. 2 with fields);
* at low temperature it reaches the brute-force ground state; at fixed beta
  its samples follow the exact Boltzmann distribution;
* Eq. 1 / Eq. 2 identities with h = 0.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import _pyref


def _edges(g):
    i, j, Jv = [], [], []
    rp, col, J = g["row_ptr"], g["col"], g["J"]
    for a in range(g["n"]):
        for e in range(rp[a], rp[a + 1]):
            if col[e] > a:
                i.append(a)
                j.append(int(col[e]))
                Jv.append(int(J[e]))
    return np.array(i), np.array(j), np.array(Jv)


def _adj(g):
    return [list(g["col"][g["row_ptr"][a]:g["row_ptr"][a + 1]]) for a in range(g["n"])]


@pytest.mark.parametrize("n,m,seed", [(30, 60, 1), (200, 900, 2), (60, 400, 3), (12, 0, 4)])
def test_colouring_is_proper_first_fit(n, m, seed):
    g = synth.random_graph(n, m, seed)
    colour, k = oracle.greedy_colouring(g)
    adj = _adj(g)
    assert list(colour) == _pyref.first_fit_colouring(n, adj)
    for a in range(n):
        assert all(colour[b] != colour[a] for b in adj[a])
    assert k == (int(colour.max()) + 1 if n else 0)


@pytest.mark.parametrize("X,Y,seed", [(4, 4, 1), (8, 6, 2), (20, 10, 3)])
def test_torus_as_graph_equals_torus_annealer(X, Y, seed):
    inst = synth.torus_instance(X, Y, seed)
    g = {"n": inst["n"], "row_ptr": inst["row_ptr"], "col": inst["col"], "J": inst["J"], "h": None}
    colour, k = oracle.greedy_colouring(g)
    y, x = np.divmod(np.arange(X * Y), X)
    np.testing.assert_array_equal(colour, (x + y) & 1)
    assert k == 2
    betas = synth.linear_betas(0.1, 3.0, 40)
    a_s, a_c = oracle.anneal(inst, betas, 77, t_count=11, sweep_offset=3)
    b_s, b_c = oracle.anneal_graph(g, betas, 77, 11, sweep_offset=3)
    np.testing.assert_array_equal(a_s, b_s)
    np.testing.assert_array_equal(a_c, b_c)


@pytest.mark.parametrize("n,m,seed,weights,hmax", [(7, 10, 5, "pm1", 0), (8, 12, 6, "int", 2),
                                                   (6, 15, 7, "one", 1), (9, 9, 8, "int", 3)])
def test_graph_annealer_equals_full_energy_restatement(n, m, seed, weights, hmax):
    g = synth.random_graph(n, m, seed, weights=weights, hmax=hmax)
    colour, _ = oracle.greedy_colouring(g)
    betas = synth.linear_betas(0.2, 1.5, 6)
    ref = _pyref.anneal_graph_full_energy(n, _edges(g), g["h"], list(colour), betas, 0xC0FFEE, 5, sweep_offset=2)
    got, cuts = oracle.anneal_graph(g, betas, 0xC0FFEE, 5, sweep_offset=2, check_fields=True)
    np.testing.assert_array_equal(got, ref)
    w_edges = _edges(g)
    for s, c in zip(got, cuts):
        assert c == sum(-int(Jv) for a, b, Jv in zip(*w_edges) if s[a] != s[b])


def _all_states(n):
    return (((np.arange(2 ** n)[:, None] >> np.arange(n)) & 1) * 2 - 1).astype(np.int8)


def test_low_temperature_reaches_ground_state():
    g = synth.random_graph(14, 30, 9, weights="int", hmax=2)
    states = _all_states(14)
    E = np.array([oracle.energy_h(g, s) for s in states])
    spins, _ = oracle.anneal_graph(g, synth.linear_betas(0.1, 3.0, 300), 5, 48)
    got = np.array([oracle.energy_h(g, s) for s in spins])
    assert got.min() == E.min()
    assert (got == E.min()).mean() > 0.3


def test_fixed_beta_samples_follow_boltzmann_with_fields():
    g = synth.random_graph(10, 18, 10, weights="int", hmax=2)
    states = _all_states(10)
    E = np.array([oracle.energy_h(g, s) for s in states], dtype=np.float64)
    beta = 0.3
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    levels, inv = np.unique(E, return_inverse=True)
    p_level = np.bincount(inv, weights=p)
    trials = 6000
    spins, _ = oracle.anneal_graph(g, np.full(60, beta), 99, trials)
    got = np.array([oracle.energy_h(g, s) for s in spins], dtype=np.float64)
    obs = np.array([(got == L).sum() for L in levels], dtype=np.float64)
    exp = p_level * trials
    keep = exp >= 5
    chi2 = (((obs[keep] - exp[keep]) ** 2) / exp[keep]).sum()
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)
    assert abs(got.mean() - (p * E).sum()) < 0.3


def test_energy_identities_without_fields():
    g = synth.random_graph(40, 120, 11)
    W = int(g["w"].sum()) // 2
    for s in synth.random_spins(10, 40, 12):
        H = oracle.energy_h(g, s)
        _, c = oracle.anneal_graph(g, np.zeros(0), 1, 1, init=s[None, :])
        assert 2 * int(c[0]) == W - H


def test_improper_colouring_is_rejected():
    g = synth.random_graph(10, 20, 13)
    with pytest.raises(ValueError):
        oracle.anneal_graph(g, np.ones(2), 1, 1, colour=np.zeros(10, dtype=np.int32))
