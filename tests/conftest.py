import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def small_problem(dims, nnz, R, seed, dist=("uniform",) * 3, factor="normal", noise=0.0,
                  recipe="noise"):
    """A seeded small tensor: coordinates in draw order, planted factors and
    values made from the oracle's own model entries."""
    import oracle
    import synth
    idx = synth.distinct_coords(dims, nnz, dist, seed)
    planted = synth.factor_matrices(dims, R, factor, seed)
    model = oracle.model_entries(dims, idx, planted)
    t = synth.observe(model, recipe, seed, noise)
    return idx, planted, t


@pytest.fixture
def rng():
    return np.random.default_rng(12345)
