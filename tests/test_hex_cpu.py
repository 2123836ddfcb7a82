"""Hex import/export of configurations (the form of the paper's App. C-E
bitstrings), through the library's host functions; no GPU needed."""
import numpy as np
import pytest

import synth


def test_known_digits():
    from paper_2505_18508_gb300 import hex_to_spins, spins_to_hex
    s = np.array([1, -1, -1, 1, 1, 1, 1, 1, -1, 1], dtype=np.int8)
    # 1001 -> 9, 1111 -> F, 01(00 padding) -> 4
    assert spins_to_hex(s) == "9F4"
    np.testing.assert_array_equal(hex_to_spins("9F4", 10), s)
    np.testing.assert_array_equal(hex_to_spins(" 9f\n4 ", 10), s)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 8, 33, 2500, 20000])
def test_round_trip(n):
    from paper_2505_18508_gb300 import hex_to_spins, spins_to_hex
    s = synth.random_spins(1, n, n)[0]
    h = spins_to_hex(s)
    assert len(h) == (n + 3) // 4
    np.testing.assert_array_equal(hex_to_spins(h, n), s)


def test_rejects_bad_strings():
    from paper_2505_18508_gb300 import IsingError, hex_to_spins
    for bad, n in (("9G", 8), ("9F", 12), ("9F4", 8), ("7", 3)):   # bad digit, too few, too many, padding bit set
        with pytest.raises(IsingError):
            hex_to_spins(bad, n)
