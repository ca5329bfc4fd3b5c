"""The Cauchy tensor generator (Sec. 5.3): entries from the closed form,
symmetry in the indices, and the device generator's values (run on the CPU
device here)."""

import numpy as np

from synth import cauchy_tensor, cauchy_tensor_device


def test_entries_from_the_closed_form():
    x = cauchy_tensor(6, 4, 2.0)
    for idx in [(0, 0, 0, 0), (5, 1, 3, 2), (2, 2, 5, 0)]:
        i = np.array(idx) + 1.0
        assert abs(x[idx] - 1.0 / np.sqrt(np.sum(i * i))) <= 1e-15
    assert x[0, 0, 0, 0] == 0.5
    assert np.allclose(x, np.transpose(x, (2, 0, 3, 1)))
    x3 = cauchy_tensor(5, 3, 1.0)
    assert abs(x3[1, 2, 4] - 1.0 / (2 + 3 + 5)) <= 1e-15


def test_device_generator_matches_host():
    import torch
    x = cauchy_tensor(7, 4, 2.0)
    t = cauchy_tensor_device(7, 4, 2.0, device="cpu", dtype=torch.float64, slabs_per_chunk=3)
    assert np.allclose(t.numpy(), np.ascontiguousarray(x), rtol=4e-16, atol=0)
