"""The input both CPU legs of the benchmark time (bench.cpu_sample), on every
workload: at most 2^10 rows per mode, coordinates inside the sample's
dimensions and distinct, at most half of its cells (skewed shapes such as the
Netflix-shaped one would otherwise ask for more nonzeros than the sample has
cells), values and start factors of the right shapes, and a description that
states what was drawn."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402


@pytest.mark.parametrize("name", sorted(synth.WORKLOADS))
def test_cpu_sample_is_a_valid_scaled_tensor(name):
    import bench
    w = synth.WORKLOADS[name]
    dims, idx, t, start, desc = bench.cpu_sample(w)
    n = len(idx[0])
    assert all(1 <= I <= 1024 for I in dims) and n > 0
    for d in range(3):
        assert len(idx[d]) == n and idx[d].min() >= 0 and idx[d].max() < dims[d]
    key = (idx[0].astype(np.int64) * dims[1] + idx[1]) * dims[2] + idx[2]
    assert len(np.unique(key)) == n
    assert n <= dims[0] * dims[1] * dims[2] // 2 or w.coords == "feistel"
    assert t.shape == (n,) and np.isfinite(t).all()
    assert [a.shape for a in start] == [(I, w.rank) for I in dims]
    assert f"{n} nonzeros" in desc
    if w.coords != "feistel" and round(w.nnz * min(1.0, 1024.0 / max(w.dims))) > n:
        assert "capped at half the sample's cells" in desc
