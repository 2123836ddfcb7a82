"""Autotuner: cache logic on the CPU; tuning on the GPU keeps results exact."""
import numpy as np
import pytest

import oracle
import synth
from paper_2505_18508_gb300 import autotune


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "at.json"
    monkeypatch.setenv("ISING_AUTOTUNE_CACHE", str(path))
    assert autotune.load_cache() == {}
    autotune.store_cache("a", {"kernel": 2})
    autotune.store_cache("b", {"kernel": 1, "strips": 4})
    assert autotune.load_cache() == {"a": {"kernel": 2}, "b": {"kernel": 1, "strips": 4}}
    path.write_text("not json")
    assert autotune.load_cache() == {}


def test_keys_and_candidates():
    k1 = autotune.batch_key("gpu", [(50, 100, 32, 2000), (100, 100, 64, 3000)])
    k2 = autotune.batch_key("gpu", [(50, 100, 32, 2000), (100, 100, 64, 3001)])
    assert k1 != k2 and k1.startswith("batch|gpu|m=2|")
    assert autotune.anneal_key("g", 200, 100, 1024) == "anneal|g|200x100|T=1024"
    for X, Y, T in ((200, 100, 1024), (50, 50, 64), (8, 6, 7)):
        cands = autotune.anneal_candidates(X, Y, T)
        assert cands and all(c["kernel"] in (1, 2) for c in cands)
        for c in cands:
            assert c["group_trials"] % 4 == 0 and 4 <= c["group_trials"] <= 32
            if c["kernel"] == 1:
                assert 1 <= c["strips"] <= 8 and 64 <= c["threads"] <= 1024 and c["threads"] % 32 == 0


@pytest.mark.gpu
def test_tuned_shape_keeps_results_exact(tmp_path, monkeypatch):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    monkeypatch.setenv("ISING_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    inst = synth.torus_instance(50, 50, 1)
    prob = ia.Problem.from_instance(inst)
    best = autotune.tune_anneal(prob, 64, probe_sweeps=100)
    assert best is not None and best["probe_ms"] > 0
    again = autotune.tune_anneal(prob, 64)          # served from the cache
    assert {k: again[k] for k in ("kernel", "group_trials", "strips", "threads")} == \
        {k: best[k] for k in ("kernel", "group_trials", "strips", "threads")}
    betas = synth.linear_betas(0.1, 3.0, 150)
    s, c = ia.anneal(prob, 64, betas, 1001)
    torch.cuda.synchronize()
    rs, rc = oracle.anneal(inst, betas, 1001, t_count=64)
    np.testing.assert_array_equal(s.cpu().numpy(), rs)
    np.testing.assert_array_equal(c.cpu().numpy(), rc)
    probs = [ia.Problem.from_instance(synth.torus_instance(x, 20, 5 + x)) for x in (20, 40)]
    b = autotune.tune_batched(probs, [64, 100], [400, 300])
    assert b is not None and b["ctas_per_sm"] in (1, 2)
    for p in probs:
        p.destroy()
    prob.destroy()
