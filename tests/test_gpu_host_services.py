"""GPU checks of the library's host services: its Philox4x32-10 against the
oracle's and against cuRAND's device Philox4_32_10 (called, not read); the
allocation-failure hook (ISING_ERR_OOM, then normal service, no leak); the
ISING_LOG launch line."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
OOM = -5   # ISING_ERR_OOM
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ia():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    torch.cuda.set_device(0)
    return ia


def test_philox_matches_oracle(ia):
    rng = np.random.default_rng(31)
    ctr = rng.integers(0, 2 ** 32, size=(500, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x0123_4567_89AB_CDEF
    got = ia.philox(ctr, seed).cpu().numpy().view(np.uint32)
    for j in range(0, 500, 7):
        assert list(got[j]) == oracle.philox4x32_10(ctr[j], (seed & 0xFFFFFFFF, seed >> 32))


def test_philox_matches_curand(ia):
    import __graft_entry__
    from paper_2505_18508_gb300.build import build_program
    exe = build_program(__graft_entry__.CURAND_CHECK_SRC, __graft_entry__.CURAND_CHECK_EXE, ("-O2",))
    for seed, sub in ((0x1234_5678_9ABC_DEF0, 7), (42, 0x1_0000_0003), (0, 0)):
        out = subprocess.run([exe, hex(seed), hex(sub), "6"], capture_output=True, text=True, check=True).stdout
        cur = [[int(w, 16) for w in line.split()] for line in out.strip().splitlines()]
        # output i of subsequence s is the block at counter (i, 0, s mod 2^32, s / 2^32)
        ctr = np.array([[i, 0, sub & 0xFFFFFFFF, sub >> 32] for i in range(6)], dtype=np.uint32)
        lib = ia.philox(ctr, seed).cpu().numpy().view(np.uint32)
        for i in range(6):
            assert list(lib[i]) == cur[i], (seed, sub, i)


def test_allocation_failures_are_reported_and_recovered(ia):
    import torch
    inst = synth.torus_instance(50, 50, 3)
    betas = synth.linear_betas(0.1, 3.0, 20)
    L = ia.lib()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):                         # creation: its first allocation fails
        L.ising_debug_fail_allocs(1)
        with pytest.raises(ia.IsingError) as ei:
            ia.Problem.from_instance(inst)
        assert ei.value.code == OOM
    L.ising_debug_fail_allocs(0)
    prob = ia.Problem.from_instance(inst)
    for kernel in (1, 2):                      # the per-call allocation of both kernels' paths
        prob.set_kernel(kernel)
        L.ising_debug_fail_allocs(1)
        with pytest.raises(ia.IsingError) as ei:
            ia.anneal(prob, 64, betas, 1)
        assert ei.value.code == OOM
        L.ising_debug_fail_allocs(0)
        s, c = ia.anneal(prob, 64, betas, 1)
        torch.cuda.synchronize()
        rs, rc = oracle.anneal(inst, betas, 1, t_count=64)
        np.testing.assert_array_equal(s.cpu().numpy(), rs)
        np.testing.assert_array_equal(c.cpu().numpy(), rc)
    prob.destroy()
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 64 << 20     # nothing of size leaked


def test_log_line(ia):
    code = ("import sys; sys.path.insert(0, %r); import numpy as np, torch, synth; "
            "import paper_2505_18508_gb300 as ia; p = ia.Problem.from_instance(synth.torus_instance(8, 8, 1)); "
            "ia.anneal(p, 32, np.ones(3), 1); torch.cuda.synchronize()" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, ISING_LOG="1"), capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "ising: anneal n=64 trials=32 sweeps=3 kernel=" in r.stderr


def test_staging_calls_refuse_stream_capture(ia):
    """The calls that copy per-call tables from host memory (or wait on the
    stream) return ISING_ERR_UNSUPPORTED while the stream captures a graph,
    before queuing anything: the capture stays valid, records the work around
    them and replays it; outside the capture the same calls run exactly."""
    import torch
    X, Y, T, S = 16, 8, 40, 30
    inst = synth.torus_instance(X, Y, 3)
    prob = ia.Problem.from_instance(inst)
    betas = synth.linear_betas(0.2, 2.0, S)
    x = torch.zeros(4, device="cuda")
    calls = {
        "anneal": lambda: ia.anneal(prob, T, betas, 5),
        "anneal_trace": lambda: ia.anneal_trace(prob, T, betas, 5, 10),
        "anneal_batched": lambda: ia.anneal_batched([prob], [T], [S], [betas], [5]),
        "batch_create": lambda: ia.BatchPlan([prob], [T], [S], [betas], [5]),
        "anneal_pt": lambda: ia.anneal_pt(prob, betas[:2], 32, 2, 5, 5),
        "learned_create": lambda: ia.LearnedPlan([prob], None, T, betas, [5], 20, every=5, partner_period=3),
        "get_status": lambda: prob.get_status(),
    }
    codes = {}
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        x.add_(1.0)
        for name, call in calls.items():
            with pytest.raises(ia.IsingError) as e:
                call()
            codes[name] = e.value.code
        x.add_(1.0)
    assert codes == {name: -8 for name in calls}     # ISING_ERR_UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert x.tolist() == [2.0] * 4
    spins, cuts = ia.anneal(prob, T, betas, 5)
    torch.cuda.synchronize()
    rs, rc = oracle.anneal(inst, betas, 5, t_begin=0, t_count=T)
    np.testing.assert_array_equal(spins.cpu().numpy(), rs)
    np.testing.assert_array_equal(cuts.cpu().numpy(), rc)
    assert prob.get_status() == 0
    del g
    prob.destroy()
