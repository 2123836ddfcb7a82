"""The sweep-budget campaign (Fig. 1: highest and average cut against sweeps
per trial; Fig. 3: the distribution of final cuts) against statistics the
test computes itself from oracle runs of the same budgets, schedules and
seeds: highest, mean, lowest cut and the integer histogram, per budget."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("X,Y,trials,budgets", [(16, 12, 48, (1, 40, 150, 500)), (30, 10, 70, (200, 900))])
def test_campaign_statistics_equal_the_oracle(X, Y, trials, budgets):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_18508_gb300 as ia
    from paper_2505_18508_gb300 import campaign
    torch.cuda.set_device(0)
    inst = synth.torus_instance(X, Y, 31)
    prob = ia.Problem.from_instance(inst)
    seed = 900
    out = campaign.run_campaign(prob, budgets, trials, seed)
    prob.destroy()
    assert [r["sweeps"] for r in out["budgets"]] == list(budgets)
    assert out["updates"] == sum(budgets) * trials * X * Y
    for j, (S, row) in enumerate(zip(budgets, out["budgets"])):
        # budget j: its own linear schedule 0.1 -> 3.0 over S sweeps and seed
        # seed + 7919 j
        _, c = oracle.anneal(inst, synth.linear_betas(0.1, 3.0, S), seed + 7919 * j, t_count=trials)
        c = c.astype(np.int64)
        assert row["highest"] == c.max() and row["lowest"] == c.min()
        assert row["mean"] == pytest.approx(c.mean(), rel=0, abs=1e-9)
        counts = np.bincount(c - c.min())
        assert row["histogram"]["first_cut"] == c.min()
        assert row["histogram"]["counts"] == counts.tolist()
        assert sum(row["histogram"]["counts"]) == trials
