"""Pins for the oracle's replica exchange (parallel tempering):
* one temperature is the plain annealer at constant beta;
* with equal temperatures every swap is taken (exp(0) = 1);
* on a 4x4 torus the energies of two exchanging temperatures follow the
  product of the two exact Boltzmann distributions (exchange keeps it), and
  the exchange does take place;
* the swap threshold against a 60-digit evaluation."""
import math
from decimal import Decimal, getcontext

import numpy as np

import oracle
import synth
from oracle import pt


def test_one_temperature_is_plain_annealing():
    inst = synth.torus_instance(8, 6, 3)
    s, c, sw = pt.anneal_pt(inst, [0.7], 8, 4, 5, 21)
    rs, rc = oracle.anneal(inst, np.full(20, 0.7), 21, t_count=8)
    np.testing.assert_array_equal(s, rs)
    np.testing.assert_array_equal(c, rc)
    assert sw == 0


def test_equal_temperatures_always_swap():
    inst = synth.torus_instance(6, 4, 4)
    R, C, Q = 3, 4, 6
    _, _, sw = pt.anneal_pt(inst, [0.5] * R, C, Q, 2, 9)
    # one pair per round ((0,1) on even rounds, (1,2) on odd ones): every attempt is taken
    assert sw == Q * C


def test_exchange_keeps_the_boltzmann_product():
    inst = synth.torus_instance(4, 4, 21)
    edges = oracle.torus_edges(4, 4, inst["w_right"], inst["w_down"])
    _, _, E, _ = oracle.brute_force(edges, 16)
    betas = [0.3, 0.6]
    C = 3000
    s, c, sw = pt.anneal_pt(inst, betas, C, 12, 5, 77)
    assert sw > C                                   # the two temperatures do exchange
    W = int(edges[2].sum())
    for r, beta in enumerate(betas):
        got = W - 2 * c[r * C:(r + 1) * C].astype(np.int64)
        p = oracle.boltzmann(E, beta)
        levels, inv = np.unique(E, return_inverse=True)
        pl = np.bincount(inv, weights=p)
        obs = np.array([(got == L).sum() for L in levels], dtype=np.float64)
        exp = pl * C
        keep = exp >= 5
        chi2 = (((obs[keep] - exp[keep]) ** 2) / exp[keep]).sum()
        dof = keep.sum() - 1
        assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (r, chi2, dof)


def test_swap_threshold_high_precision():
    getcontext().prec = 60
    for dbeta in (0.01, 0.3, 1.7):
        for d in (4, 8, 12, 100, 4000):
            v = (-(Decimal(dbeta) * d)).exp() * (Decimal(2) ** 32)
            exact = min(int(v), 2 ** 32 - 1)
            if abs(v - int(v)) > Decimal("1e-5"):
                assert pt.swap_threshold(dbeta, d) == exact
