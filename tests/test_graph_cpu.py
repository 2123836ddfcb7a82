"""Host-side pieces of the general-graph path that need no GPU: the
library's first-fit colouring against the oracle's."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n,m,seed", [(30, 60, 1), (500, 3000, 2), (2000, 19990, 3), (9, 0, 4), (64, 2016, 5)])
def test_library_colouring_equals_oracle(n, m, seed):
    from paper_2505_18508_gb300 import greedy_colouring
    g = synth.random_graph(n, m, seed)
    a, ka = greedy_colouring(g)
    b, kb = oracle.greedy_colouring(g)
    np.testing.assert_array_equal(a, b)
    assert ka == kb


def test_library_colouring_of_torus_is_checkerboard():
    from paper_2505_18508_gb300 import greedy_colouring
    inst = synth.torus_instance(200, 100, 2)
    c, k = greedy_colouring(inst)
    y, x = np.divmod(np.arange(20000), 200)
    np.testing.assert_array_equal(c, (x + y) & 1)
    assert k == 2
