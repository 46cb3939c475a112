"""The bench line's error measure against the serial fine solution (Sec. 4.1: the
relative error of each field at the slice boundaries, Frobenius norm), on CPU
tensors with known answers."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_rel_errors_per_field_and_boundary():
    N, nodes = 4, 7
    rng = np.random.default_rng(5)
    ref = torch.tensor(rng.uniform(-1, 1, (N + 1, nodes * 5)), dtype=torch.float64)
    got = ref.clone()
    got[0] += 1.0                                   # the initial state is not a boundary of the metric
    assert all(v == 0.0 for v in bench.rel_errors(got, ref, N).values())
    v = got.view(N + 1, nodes, 5)
    v[2, :, 2:4] *= 1.0 + 3e-7                      # displacement at boundary 2 off by 3e-7 relative
    v[3, 1, 4] += 1e-5 * ref.view(N + 1, nodes, 5)[3, :, 4].norm()   # one pressure entry at boundary 3
    e = bench.rel_errors(got, ref, N)
    assert e["v"] == 0.0
    assert e["u"] == pytest.approx(3e-7, rel=1e-6)
    assert e["p"] == pytest.approx(1e-5, rel=1e-9)


def test_rel_errors_take_the_largest_boundary():
    N, nodes = 3, 5
    ref = torch.ones((N + 1, nodes * 5), dtype=torch.float64)
    got = ref.clone()
    for n, f in ((1, 1e-3), (2, 4e-3), (3, 2e-3)):
        got.view(N + 1, nodes, 5)[n, :, 0:2] *= 1.0 + f
    assert bench.rel_errors(got, ref, N)["v"] == pytest.approx(4e-3, rel=1e-9)
