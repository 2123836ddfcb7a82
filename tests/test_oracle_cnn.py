"""Pins for the FP64 CNN oracle and the exact proposal step.

* forward: a direct numpy loop over taps, channels and torus positions;
* gradient: central finite differences in FP64;
* loss: exact values (zero logits give ln 2);
* targets: gauge invariance;
* proposals: acceptance re-derived from whole-lattice energy differences;
* torus components: networkx's periodic grid graph on random masks.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import cnn

torch = pytest.importorskip("torch")


def _direct_conv(x, W, b):
    """out[o, y, x] = b[o] + sum W[o, c, ky, kx] in[c, (y+ky-1)%Y, (x+kx-1)%X]."""
    C, Y, X = x.shape
    O = W.shape[0]
    out = np.zeros((O, Y, X))
    for o in range(O):
        for y in range(Y):
            for xx in range(X):
                acc = b[o]
                for c in range(C):
                    for ky in range(3):
                        for kx in range(3):
                            acc += W[o, c, ky, kx] * x[c, (y + ky - 1) % Y, (xx + kx - 1) % X]
                out[o, y, xx] = acc
    return out


def test_forward_matches_direct_loop():
    X, Y = 5, 4
    inst = synth.torus_instance(6, 4, 3)     # weights only; use a 6x4 torus
    wr, wd = inst["w_right"], inst["w_down"]
    X = 6
    params = cnn.init_params(11) + 0.05 * np.random.default_rng(2).normal(size=cnn.N_PARAMS)
    s = synth.random_spins(2, X * Y, 5)
    got = cnn.forward(params, s, wr, wd, return_all=True)
    p = cnn.unflatten(params)
    for b in range(2):
        x = cnn.features(s[b:b + 1], wr, wd)[0]
        h1 = np.maximum(_direct_conv(x, p["W1"], p["b1"]), 0)
        h2 = np.maximum(_direct_conv(h1, p["W2"], p["b2"]), 0)
        h3 = np.maximum(_direct_conv(h2, p["W3"], p["b3"]), 0)
        z = _direct_conv(h3, p["W4"], p["b4"])[0]
        np.testing.assert_allclose(got["h1"][b], h1, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got["z"][b], z, rtol=1e-11, atol=1e-11)


def test_zero_network_loss_is_ln2():
    params = np.zeros(cnn.N_PARAMS)
    inst = synth.torus_instance(8, 6, 1)
    s = synth.random_spins(3, 48, 1)
    y = np.random.default_rng(0).integers(0, 2, size=(3, 48)).astype(np.uint8)
    loss, g = cnn.loss_and_grad(params, s, y, inst["w_right"], inst["w_down"])
    assert abs(loss - math.log(2.0)) < 1e-15
    # with all weights zero, only the last bias gets a gradient: mean(sigmoid(0) - y)
    b4 = cnn.N_PARAMS - 1
    assert abs(g[b4] - (0.5 - y.mean())) < 1e-15
    assert np.abs(np.delete(g, b4)).max() == 0.0


def test_gradient_matches_finite_differences():
    inst = synth.torus_instance(6, 4, 7)
    s = synth.random_spins(2, 24, 3)
    y = np.random.default_rng(4).integers(0, 2, size=(2, 24)).astype(np.uint8)
    params = cnn.init_params(5) + 0.1 * np.random.default_rng(6).normal(size=cnn.N_PARAMS)
    loss, g = cnn.loss_and_grad(params, s, y, inst["w_right"], inst["w_down"])
    rng = np.random.default_rng(8)
    idx = list(rng.choice(cnn.N_PARAMS, size=40, replace=False)) + [cnn.N_PARAMS - 1, 864, 864 + 32 + 9216]
    h = 1e-6
    for i in idx:
        pp = params.copy(); pp[i] += h
        pm = params.copy(); pm[i] -= h
        lp, _ = cnn.loss_and_grad(pp, s, y, inst["w_right"], inst["w_down"])
        lm, _ = cnn.loss_and_grad(pm, s, y, inst["w_right"], inst["w_down"])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_flip_targets_are_gauge_invariant():
    s = synth.random_spins(4, 50, 1)
    r = synth.random_spins(4, 50, 2)
    a = cnn.flip_targets(s, r)
    b = cnn.flip_targets(s, -r)
    np.testing.assert_array_equal(a, b)
    assert (cnn.flip_targets(s, s) == 0).all() and (cnn.flip_targets(s, -s) == 0).all()
    assert (a.sum(axis=1) <= 25).all()


def test_flip_target_tie_rule_on_hand_built_states():
    """Exactly n/2 sites differ: r and -r are equally close to s, and the
    reading keeps the aligned reference that agrees with s at site 0, so the
    target never asks to flip site 0 on a tie, and r and -r give the same
    targets.  Hand-built: n = 4 and n = 6, site 0 equal and different."""
    s = np.array([[1, 1, 1, 1]], dtype=np.int8)
    r_keep = np.array([[1, 1, -1, -1]], dtype=np.int8)      # site 0 equal: r itself is used
    r_flip = np.array([[-1, -1, 1, 1]], dtype=np.int8)      # site 0 differs: -r is used
    np.testing.assert_array_equal(cnn.flip_targets(s, r_keep), [[0, 0, 1, 1]])
    np.testing.assert_array_equal(cnn.flip_targets(s, r_flip), [[0, 0, 1, 1]])
    np.testing.assert_array_equal(cnn.flip_targets(s, -r_keep), [[0, 0, 1, 1]])
    np.testing.assert_array_equal(cnn.flip_targets(s, -r_flip), [[0, 0, 1, 1]])
    s6 = np.array([[1, -1, 1, -1, 1, -1], [-1, -1, 1, 1, -1, 1]], dtype=np.int8)
    r6 = np.array([[-1, 1, 1, -1, -1, -1], [-1, 1, -1, 1, -1, 1]], dtype=np.int8)
    # row 0: sites 0, 1, 4 differ (a tie, site 0 differs) -> flip r: targets = sites 2, 3, 5
    # row 1: sites 1, 2 differ (2 < 3, no tie) -> keep r: targets = sites 1, 2
    np.testing.assert_array_equal(cnn.flip_targets(s6, r6), [[0, 0, 1, 1, 0, 1], [0, 1, 1, 0, 0, 0]])
    # away from ties the targets are the Hamming-nearer gauge copy's differences
    assert cnn.flip_targets(np.ones((1, 5), np.int8), np.array([[1, -1, -1, -1, 1]], np.int8)).tolist() == \
        [[1, 0, 0, 0, 1]]


def _energy(inst, s):
    return oracle.energy_csr(inst, s)


@pytest.mark.parametrize("X,Y,tile", [(16, 8, 2), (16, 8, 4), (16, 8, 8), (18, 8, 5), (12, 4, 6)])
def test_tile_proposals_are_exact(X, Y, tile):
    inst = synth.torus_instance(X, Y, 21)
    wr, wd = inst["w_right"], inst["w_down"]
    s = synth.random_spins(6, X * Y, 9)
    z = np.random.default_rng(3).normal(size=(6, Y, X))
    new, acc = cnn.propose_tiles(s, z, wr, wd, tile)
    # re-derive every decision from whole-lattice energies, tile by tile
    ntx, nty = -(-X // tile), -(-Y // tile)
    for b in range(6):
        cur = s[b].copy()
        n_acc = 0
        for phase in (0, 1):
            for ty in range(nty):
                for tx in range(ntx):
                    if (tx + ty) % 2 != phase:
                        continue
                    m = np.zeros((Y, X), dtype=bool)
                    m[ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile] = \
                        z[b, ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile] > 0
                    if not m.any():
                        continue
                    cand = cur.copy()
                    cand[m.reshape(-1)] *= -1
                    if _energy(inst, cand) <= _energy(inst, cur):
                        cur = cand
                        n_acc += 1
        np.testing.assert_array_equal(new[b], cur)
        assert acc[b] == n_acc
        assert _energy(inst, new[b]) <= _energy(inst, s[b])


def test_odd_tile_counts_are_rejected():
    inst = synth.torus_instance(12, 8, 1)
    with pytest.raises(ValueError):
        cnn.propose_tiles(synth.random_spins(1, 96, 1), np.zeros((1, 8, 12)), inst["w_right"], inst["w_down"], 4)


def test_global_proposal_is_exact():
    X, Y = 10, 6
    inst = synth.torus_instance(X, Y, 31)
    s = synth.random_spins(8, X * Y, 4)
    z = np.random.default_rng(5).normal(size=(8, Y, X))
    new, acc = cnn.propose_global(s, z, inst["w_right"], inst["w_down"])
    for b in range(8):
        cand = s[b] * np.where(z[b].reshape(-1) > 0, -1, 1).astype(np.int8)
        take = _energy(inst, cand) <= _energy(inst, s[b])
        np.testing.assert_array_equal(new[b], cand if take else s[b])
        assert acc[b] == int(take)


# ---------------------------------------------------------------- clusters
def _grid_instance(X, Y, seed):
    inst = synth.torus_instance(X, Y, seed)
    return inst, inst["w_right"], inst["w_down"]


def test_torus_components_hand_built():
    m = np.zeros((4, 6), dtype=bool)
    m[0, 0] = m[0, 5] = True          # joined across the left/right wrap
    m[3, 0] = True                    # joined to (0, 0) across the top/bottom wrap
    m[2, 2] = m[2, 3] = True          # a separate pair
    m[1, 4] = True                    # diagonal to nothing, alone
    comps = sorted(sorted(c) for c in cnn.torus_components(m))
    assert comps == [[(0, 0), (0, 5), (3, 0)], [(1, 4)], [(2, 2), (2, 3)]]


@pytest.mark.parametrize("Y, X, p", [(4, 4, 0.5), (6, 10, 0.3), (8, 6, 0.55), (10, 12, 0.45)])
def test_torus_components_equal_periodic_grid_graph_components(Y, X, p):
    """On random masks, the components are those of the masked sites' subgraph
    of networkx's periodic 2-D grid (a library routine, not the search)."""
    nx = pytest.importorskip("networkx")
    grid = nx.grid_2d_graph(Y, X, periodic=True)
    rng = np.random.default_rng(Y * 100 + X)
    for _ in range(20):
        m = rng.random((Y, X)) < p
        ours = sorted(sorted(c) for c in cnn.torus_components(m))
        lib = sorted(sorted(c) for c in nx.connected_components(grid.subgraph(zip(*np.nonzero(m)))))
        assert ours == [[(int(y), int(x)) for y, x in c] for c in lib]


def test_component_energy_changes_add_up_to_the_state_difference():
    """Components of the disagreement set are never adjacent, so their flip
    energies add up exactly to E(r') - E(s) (flipping all of them turns s into
    r'); and the targets are gauge invariant."""
    X, Y = 12, 8
    inst, wr, wd = _grid_instance(X, Y, 5)
    rng = np.random.default_rng(3)
    for trial in range(6):
        s = synth.random_spins(1, X * Y, 10 + trial)
        r = s.copy()
        flip = rng.random(X * Y) < 0.3
        r[0, flip] = -r[0, flip]
        d = cnn.flip_targets(s, r).reshape(Y, X).astype(bool)
        sg = s.reshape(Y, X)
        total = sum(cnn.component_dE(sg, c, wr, wd) for c in cnn.torus_components(d))
        rp = np.where(d, -sg, sg)
        assert total == cnn._energy_grid(rp, wr, wd) - cnn._energy_grid(sg, wr, wd)
        # Eq. 2 on the CSR gives the same energies
        assert cnn._energy_grid(sg, wr, wd) == oracle.energy_csr(inst, s[0])
        y = cnn.droplet_targets(s, r, wr, wd)
        np.testing.assert_array_equal(y, cnn.droplet_targets(s, -r, wr, wd))
        # flipping exactly the target sites lowers the energy by the sum of
        # the improving components' changes, each negative
        imp = [cnn.component_dE(sg, c, wr, wd) for c in cnn.torus_components(d)]
        after = np.where(y.reshape(Y, X).astype(bool), -sg, sg)
        assert cnn._energy_grid(after, wr, wd) - cnn._energy_grid(sg, wr, wd) == sum(v for v in imp if v < 0)
    assert (cnn.droplet_targets(s, s, wr, wd) == 0).all() and (cnn.droplet_targets(s, -s, wr, wd) == 0).all()


def test_single_site_droplet_is_a_metropolis_move():
    """A one-site component lowers the energy iff its single-spin flip has
    dE = -2 s_i sum_j w_ij s_j < 0 (the sweep's own energy change)."""
    X, Y = 6, 4
    inst, wr, wd = _grid_instance(X, Y, 9)
    s = synth.random_spins(1, X * Y, 4)
    sg = s.reshape(Y, X).astype(np.int64)
    for i in range(X * Y):
        y, x = divmod(i, X)
        f = (wr[y, x] * sg[y, (x + 1) % X] + wr[y, (x - 1) % X] * sg[y, (x - 1) % X]
             + wd[y, x] * sg[(y + 1) % Y, x] + wd[(y - 1) % Y, x] * sg[(y - 1) % Y, x])
        assert cnn.component_dE(sg, [(y, x)], wr, wd) == -2 * sg[y, x] * f


def test_cluster_proposals_never_raise_the_energy():
    X, Y = 10, 6
    inst, wr, wd = _grid_instance(X, Y, 11)
    s = synth.random_spins(5, X * Y, 21)
    z = np.random.default_rng(2).normal(size=(5, X * Y))
    new, acc = cnn.propose_clusters(s, z, wr, wd)
    for b in range(5):
        sg, ng = s[b].reshape(Y, X), new[b].reshape(Y, X)
        comps = cnn.torus_components(z[b].reshape(Y, X) > 0)
        gains = [cnn.component_dE(sg, c, wr, wd) for c in comps]
        assert acc[b] == sum(g <= 0 for g in gains)
        assert cnn._energy_grid(ng, wr, wd) - cnn._energy_grid(sg, wr, wd) == sum(g for g in gains if g <= 0)
        changed = (sg != ng)
        assert not (changed & (z[b].reshape(Y, X) <= 0)).any()      # only proposed sites move


def test_transcription_lowers_each_energy_by_its_improving_components():
    """Each configuration ends exactly lower by the sum of its improving
    components' changes (never higher), and with a partner identical to it
    (shift = B) nothing moves."""
    X, Y, B = 10, 8, 5
    inst, wr, wd = _grid_instance(X, Y, 13)
    s = synth.random_spins(B, X * Y, 30)
    new, comps = cnn.transcribe(s, 2, wr, wd)
    for b in range(B):
        sg = s[b].reshape(Y, X)
        d = cnn.flip_targets(s[b:b + 1], s[(b + 2) % B][None]).reshape(Y, X).astype(bool)
        gains = [cnn.component_dE(sg, c, wr, wd) for c in cnn.torus_components(d)]
        assert comps[b] == sum(g < 0 for g in gains)
        assert cnn._energy_grid(new[b].reshape(Y, X), wr, wd) - cnn._energy_grid(sg, wr, wd) == sum(g for g in gains if g < 0)
    same, c0 = cnn.transcribe(s, B, wr, wd)
    assert (same == s).all() and (c0 == 0).all()
