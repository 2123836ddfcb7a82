"""Edge cases of the annealer against the oracle, bit for bit: a torus of a
million spins, extreme inverse temperatures, a sweep counter that wraps past
2^32, and ragged trial counts at size; and a torus beyond the shared-memory
limits, which is refused cleanly."""
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


def test_a_million_spins(ia):
    import torch
    inst = synth.torus_instance(1024, 1024, 5)
    betas = synth.linear_betas(0.3, 2.0, 3)
    prob = ia.Problem.from_instance(inst)
    spins, cuts = ia.anneal(prob, 33, betas, 77)
    recut = ia.cut(prob, spins)
    torch.cuda.synchronize()
    assert prob.get_status() == 0
    np.testing.assert_array_equal(cuts.cpu().numpy(), recut.cpu().numpy())
    s = spins.cpu().numpy()
    for t in (0, 32):
        rs, rc = oracle.anneal(inst, betas, 77, t_begin=t, t_count=1)
        np.testing.assert_array_equal(s[t], rs[0])
        assert cuts[t].item() == rc[0]
    prob.destroy()


def test_beyond_shared_memory_is_refused(ia):
    # 2048 x 1024 with two trial groups: neither a persistent CTA's rows nor a
    # 16-strip cluster's rows fit in shared memory
    inst = synth.torus_instance(2048, 1024, 5)
    prob = ia.Problem.from_instance(inst)
    with pytest.raises(ia.IsingError) as ei:
        ia.anneal(prob, 33, np.ones(2), 1)
    assert ei.value.code == -8          # ISING_ERR_UNSUPPORTED
    prob.destroy()


@pytest.mark.parametrize("kernel", [1, 2])
def test_extreme_betas(ia, kernel):
    import torch
    inst = synth.torus_instance(64, 48, 6)
    betas = np.array([1e-300, 1e-12, 0.5, 1e3, 1e300, np.inf, 2.0, 1e-300, 40.0])
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(kernel)
    spins, cuts = ia.anneal(prob, 70, betas, 5)
    torch.cuda.synchronize()
    rs, rc = oracle.anneal(inst, betas, 5, t_count=70)
    np.testing.assert_array_equal(spins.cpu().numpy(), rs)
    np.testing.assert_array_equal(cuts.cpu().numpy(), rc)
    prob.destroy()


@pytest.mark.parametrize("kernel", [1, 2])
def test_sweep_counter_wraps(ia, kernel):
    import torch
    inst = synth.torus_instance(40, 30, 7)
    betas = synth.linear_betas(0.1, 3.0, 24)
    off = 0xFFFFFFF0                      # sweeps 2^32 - 16 .. 2^32 + 7 (mod 2^32)
    prob = ia.Problem.from_instance(inst)
    prob.set_kernel(kernel)
    spins, cuts = ia.anneal(prob, 40, betas, 9, sweep_offset=off)
    torch.cuda.synchronize()
    rs, rc = oracle.anneal(inst, betas, 9, t_count=40, sweep_offset=off)
    np.testing.assert_array_equal(spins.cpu().numpy(), rs)
    np.testing.assert_array_equal(cuts.cpu().numpy(), rc)
    prob.destroy()


@pytest.mark.parametrize("trials", [1, 31, 33, 257, 1023])
def test_ragged_trials_at_size(ia, trials):
    import torch
    inst = synth.torus_instance(200, 100, 8)
    betas = synth.linear_betas(0.1, 3.0, 30)
    prob = ia.Problem.from_instance(inst)
    spins, cuts = ia.anneal(prob, trials, betas, 11)
    torch.cuda.synchronize()
    s = spins.cpu().numpy()
    for t in sorted({0, trials // 2, trials - 1}):
        rs, rc = oracle.anneal(inst, betas, 11, t_begin=t, t_count=1)
        np.testing.assert_array_equal(s[t], rs[0])
        assert cuts[t].item() == rc[0]
    prob.destroy()


@pytest.mark.parametrize("kernel,bits", [(1, 32), (2, 32), (2, 16)])
def test_sweep_by_sweep_no_divergence(ia, kernel, bits):
    """The debugging aid that steps both sides one sweep at a time finds no
    divergent sweep (and the chained one-sweep calls are themselves the
    resume property, sweep by sweep)."""
    from tests import first_divergence
    X, Y, T = (64, 48, 96) if kernel == 2 else (8, 6, 37)
    assert first_divergence.first_divergence(X, Y, 3, T, 6, 4242, kernel=kernel, draw_bits=bits) is None
