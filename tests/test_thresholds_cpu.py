"""The library's acceptance-threshold table (ising_thresholds, host only)
against the oracle's own computation of T_d = min(floor(exp(-beta d) 2^B),
2^B - 1): equal, word for word, on the schedules the path uses and at the
clamps.  The oracle's table is itself pinned against high-precision values
(test_oracle_pins)."""
import math

import numpy as np
import pytest

import oracle
import synth

SCHEDULES = {
    "linear 0.1..3.0, 10,000 sweeps": synth.linear_betas(0.1, 3.0, 10000),
    "replica ladder 0.5..3.0": np.geomspace(0.5, 3.0, 8),
    "clamps and extremes": np.array([1e-300, 1e-12, 1e-9, 1e-3, 0.0866, 0.5 * math.log(2.0), 5.0, 30.0, 1e3,
                                     math.inf]),
    "random": np.random.default_rng(7).uniform(1e-4, 4.0, size=5000),
}


@pytest.fixture(scope="module")
def ia():
    from paper_2505_18508_gb300 import build
    build.build()
    import paper_2505_18508_gb300 as ia
    return ia


@pytest.mark.parametrize("name", list(SCHEDULES))
def test_library_table_equals_oracle_32(ia, name):
    b = SCHEDULES[name]
    got = ia.thresholds(b)
    T4, T8 = oracle.thresholds(b)
    np.testing.assert_array_equal(got[:, 0], T4)
    np.testing.assert_array_equal(got[:, 1], T8)
    assert np.all(got[:, 1] <= got[:, 0])            # exp(-8 beta) <= exp(-4 beta)


@pytest.mark.parametrize("name", list(SCHEDULES))
def test_library_table_equals_oracle_16(ia, name):
    b = SCHEDULES[name]
    got = ia.thresholds(b, draw_bits=16)
    T4, T8 = oracle.thresholds(b, draw_bits=16)
    assert np.all((got & 0xFFFF) == 0)                # stored shifted left by 16
    np.testing.assert_array_equal(got[:, 0] >> 16, T4)
    np.testing.assert_array_equal(got[:, 1] >> 16, T8)


def test_clamps(ia):
    got = ia.thresholds(np.array([1e-300, math.inf]))
    assert got[0].tolist() == [0xFFFFFFFF, 0xFFFFFFFF]   # exp(-0) 2^32 clamps to 2^32 - 1
    assert got[1].tolist() == [0, 0]                     # beta = inf: never uphill
    got16 = ia.thresholds(np.array([1e-300]), draw_bits=16)
    assert got16[0].tolist() == [0xFFFF0000, 0xFFFF0000]


def test_bad_arguments(ia):
    for bad in ([0.0], [-1.0], [math.nan], [1.0, 0.0]):
        with pytest.raises(ia.IsingError) as e:
            ia.thresholds(np.array(bad))
        assert e.value.code == -1
    with pytest.raises(ia.IsingError):
        ia.thresholds(np.array([1.0]), draw_bits=8)
    assert ia.thresholds(np.zeros(0)).shape == (0, 2)
