"""GPU parity of the general-graph annealer (integer couplings, fields)
against the oracle's general-graph annealer, bit for bit; a torus given as a
graph against the torus kernels; cut and energy; launch shapes; errors."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ia():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    torch.cuda.set_device(0)
    return ia


CASES = [
    # n, m, graph seed, weights, hmax, trials, sweeps, strips (0 = auto)
    (30, 60, 1, "pm1", 0, 37, 30, 0),
    (100, 400, 2, "int", 2, 64, 25, 0),
    (800, 4000, 3, "pm1", 0, 100, 20, 0),
    (800, 19176, 4, "one", 0, 32, 10, 0),     # dense-ish (average degree 48)
    (2000, 6000, 5, "int", 3, 70, 15, 4),
    (5000, 10000, 6, "pm1", 1, 33, 12, 8),
    (7, 10, 7, "int", 2, 1, 40, 1),
    (300, 900, 8, "one", 0, 1024, 6, 0),
]


@pytest.mark.parametrize("n,m,gseed,weights,hmax,trials,S,C", CASES)
def test_graph_parity(ia, n, m, gseed, weights, hmax, trials, S, C):
    import torch
    g = synth.random_graph(n, m, gseed, weights=weights, hmax=hmax)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0x6A0000 + gseed
    prob = ia.Problem.from_graph(g)
    if C:
        prob.set_launch(0, C, 0)
    spins, cuts = ia.anneal(prob, trials, betas, seed)
    recut = ia.cut(prob, spins)
    en = ia.energy(prob, spins)
    torch.cuda.synchronize()
    assert prob.last_kernel() == 3
    np.testing.assert_array_equal(cuts.cpu().numpy(), recut.cpu().numpy())
    sub = min(trials, 64)
    rs, rc = oracle.anneal_graph(g, betas, seed, sub)
    np.testing.assert_array_equal(spins.cpu().numpy()[:sub], rs)
    np.testing.assert_array_equal(cuts.cpu().numpy()[:sub], rc)
    e = en.cpu().numpy()
    for t in range(min(sub, 8)):
        assert e[t] == oracle.energy_h(g, rs[t])
    prob.destroy()


def test_torus_as_graph_equals_torus_kernels(ia):
    import torch
    inst = synth.torus_instance(200, 100, 2)
    betas = synth.linear_betas(0.1, 3.0, 200)
    torus = ia.Problem.from_instance(inst)
    graph = ia.Problem.from_graph({"n": inst["n"], "row_ptr": inst["row_ptr"], "col": inst["col"],
                                   "J": inst["J"], "h": None})
    assert graph.graph_info()["colours"] == 2 and graph.graph_info()["Dmax"] == 4
    a_s, a_c = ia.anneal(torus, 96, betas, 1002)
    b_s, b_c = ia.anneal(graph, 96, betas, 1002)
    ea, eb = ia.energy(torus, a_s), ia.energy(graph, b_s)
    torch.cuda.synchronize()
    assert torch.equal(a_s, b_s) and torch.equal(a_c, b_c) and torch.equal(ea, eb)
    torus.destroy()
    graph.destroy()


def test_cluster_sizes_resume_and_warm_start(ia):
    import torch
    g = synth.random_graph(1500, 6000, 11, weights="int", hmax=2)
    betas = synth.linear_betas(0.1, 3.0, 40)
    prob = ia.Problem.from_graph(g)
    ref_s, ref_c = None, None
    for C in (1, 2, 4, 8):
        prob.set_launch(0, C, 0)
        s, c = ia.anneal(prob, 64, betas, 5)
        torch.cuda.synchronize()
        if ref_s is None:
            ref_s, ref_c = s, c
        assert torch.equal(s, ref_s) and torch.equal(c, ref_c)
    prob.set_launch(0, 0, 0)
    half, _ = ia.anneal(prob, 64, betas[:17], 5)
    s2, c2 = ia.anneal(prob, 64, betas[17:], 5, sweep_offset=17, init=half)
    tr = ia.anneal_trace(prob, 64, betas, 5, 10)
    torch.cuda.synchronize()
    assert torch.equal(s2, ref_s) and torch.equal(c2, ref_c)
    assert torch.equal(tr[0], ref_s) and torch.equal(tr[2][-1], ref_c)
    assert torch.equal(tr[3], tr[2].max(dim=0).values)
    prob.destroy()


def test_graph_errors(ia):
    g = synth.random_graph(20, 40, 12)
    # asymmetric coupling
    J = g["J"].copy()
    J[0] = -J[0]
    with pytest.raises(ia.IsingError):
        ia.Problem.from_graph(dict(g, J=J))
    # a self loop
    col = g["col"].copy()
    col[0] = 0 if g["row_ptr"][1] > 0 else col[0]
    with pytest.raises(ia.IsingError):
        ia.Problem.from_graph(dict(g, col=col))
    # sum |J| + |h| above 255 at one site
    star = synth.graph_from_edges(3, [0, 0], [1, 2], [100, 100], h=np.array([100, 0, 0]))
    with pytest.raises(ia.IsingError):
        ia.Problem.from_graph(star)
    prob = ia.Problem.from_graph(g)
    prob.set_draw_bits(16)
    with pytest.raises(ia.IsingError):
        ia.anneal(prob, 8, np.ones(3), 1)
    prob.set_draw_bits(32)
    with pytest.raises(ia.IsingError):
        ia.anneal_batched([prob], [8], [3], [np.ones(3)], [1])
    # the learned stage needs the torus layout
    import torch
    from oracle import cnn as ocnn
    net = ia.CNN(ocnn.init_params(1))
    s = torch.ones((2, g["n"]), dtype=torch.int8, device="cuda")
    with pytest.raises(ia.IsingError) as ei:
        net.forward(prob, s)
    assert ei.value.code == -8          # ISING_ERR_UNSUPPORTED
    with pytest.raises(ia.IsingError):
        ia.propose(prob, s, torch.zeros((2, g["n"]), device="cuda"), 0)
    net.destroy()
    prob.destroy()


TEAM_CASES = [
    # n, m, graph seed, weights, hmax, trials, sweeps, strips
    (2000, 19990, 22, "one", 0, 96, 12, 0),    # G22-like: small colour classes
    (600, 3000, 31, "int", 3, 70, 15, 2),      # fields, integer weights, ragged trials
    (3000, 9000, 32, "pm1", 1, 33, 10, 8),
]


@pytest.mark.parametrize("tpw", [1, 4, 8])
@pytest.mark.parametrize("n,m,gseed,weights,hmax,trials,S,C", TEAM_CASES)
def test_graph_threads_per_site_parity(ia, n, m, gseed, weights, hmax, trials, S, C, tpw):
    """A site word's update split over 1, 4 or 8 threads (neighbour counts
    summed with shuffles, Philox blocks shared out) gives the oracle's
    trajectory bit for bit."""
    import torch
    g = synth.random_graph(n, m, gseed, weights=weights, hmax=hmax)
    betas = synth.linear_betas(0.1, 3.0, S)
    seed = 0x7B0000 + gseed
    prob = ia.Problem.from_graph(g)
    if C:
        prob.set_launch(0, C, 0)
    prob.set_graph_threads_per_site(tpw)
    spins, cuts = ia.anneal(prob, trials, betas, seed)
    torch.cuda.synchronize()
    sub = min(trials, 40)
    rs, rc = oracle.anneal_graph(g, betas, seed, sub)
    np.testing.assert_array_equal(spins.cpu().numpy()[:sub], rs)
    np.testing.assert_array_equal(cuts.cpu().numpy()[:sub], rc)
    prob.destroy()


def test_graph_threads_per_site_arguments(ia):
    g = synth.random_graph(50, 100, 33, weights="pm1")
    prob = ia.Problem.from_graph(g)
    for bad in (2, 3, 16, -1):
        with pytest.raises(ia.IsingError):
            prob.set_graph_threads_per_site(bad)
    prob.destroy()
