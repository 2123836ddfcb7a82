"""The Python binding refuses tensors the C ABI cannot take (no GPU needed):
a host tensor, a wrong dtype or shape, a non-contiguous buffer that a call
writes into.  Each is a ValueError raised before any pointer reaches the
library."""
import types

import pytest


@pytest.fixture(scope="module")
def ia():
    import paper_2505_18508_gb300 as ia
    return ia


def _fake_problem(n=16):
    return types.SimpleNamespace(n=n, handle=None)


def test_host_tensors_are_refused(ia):
    import torch
    prob = _fake_problem()
    s = torch.ones((2, 16), dtype=torch.int8)
    for call in (lambda: ia.cut(prob, s), lambda: ia.energy(prob, s),
                 lambda: ia.propose(prob, s, torch.zeros((2, 16)), 4),
                 lambda: ia.flip_targets(s, s)):
        with pytest.raises(ValueError, match="CUDA device"):
            call()


def test_shapes_and_kinds_are_checked_first(ia):
    import torch
    prob = _fake_problem()
    with pytest.raises(ValueError, match="2-D"):
        ia.cut(prob, torch.ones(16, dtype=torch.int8))
    with pytest.raises(ValueError, match="2-D"):
        ia.propose(prob, [[1] * 16], torch.zeros((1, 16)), 4)
    with pytest.raises(ValueError, match="torch.Tensor"):
        ia._device_tensor([1, 2], torch.int8, None, "x")


def test_validation_helper_rules(ia):
    import torch
    # the rules that do not need a device: a host tensor fails before dtype
    # and shape are looked at; a non-tensor fails first of all
    t = torch.zeros((3, 4), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA device"):
        ia._device_tensor(t, torch.int8, (3, 4), "t")
    with pytest.raises(ValueError, match="torch.Tensor"):
        ia._device_tensor(None, torch.int8, (3, 4), "t")
