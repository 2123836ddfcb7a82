"""The package's time-to-target statistics (Eq. 3-5, host side) against the
oracle's, and against values fixed by the equations."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_18508_gb300 import stats


def test_target_matches_oracle_and_is_the_smallest_integer_at_or_above():
    for best in list(range(0, 3000)) + [14060, 9027, 20000, 39999, 40000]:
        t = stats.target_cut(best)
        assert t == oracle.target_cut(best)
        assert 1000 * t >= 999 * best and 1000 * (t - 1) < 999 * best


def test_table1_target_threshold():
    # the 99.9% row of a best cut of 14060 is the real threshold 14045.94
    assert stats.target_cut(14060) == 14046


def test_success_probability_matches_oracle():
    rng = np.random.default_rng(3)
    for _ in range(200):
        cuts = rng.integers(900, 1000, size=int(rng.integers(1, 600)))
        tgt = int(rng.integers(900, 1001))
        assert stats.success_probability(cuts, tgt) == oracle.success_probability(cuts, tgt)
    assert stats.success_probability(np.zeros(0, dtype=np.int32), 1) == 0.0


@pytest.mark.parametrize("ps", [1e-6, 1e-3, 0.01, 0.1, 0.25, 0.5, 0.9, 0.99, 0.999999])
def test_repetitions_match_oracle_and_eq3(ps):
    r = stats.repetitions(ps)
    assert math.isclose(r, oracle.repetitions(ps), rel_tol=1e-9)
    # Eq. 3: (1 - P_s)^r = 0.01 whenever r > 1
    if r > 1.0:
        assert math.isclose((1.0 - ps) ** r, 0.01, rel_tol=1e-9)


def test_repetition_edge_cases():
    assert stats.repetitions(1.0) == 1.0
    assert stats.repetitions(0.0) == math.inf
    assert stats.time_to_target(2.0, 0.0) == math.inf
    assert stats.sweeps_to_target(1000, 1.0) == 1000
