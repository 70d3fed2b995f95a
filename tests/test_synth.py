"""The keyed-permutation coordinate generator used for the 4e9-nonzero
workload: a bijection of the 3b-bit index space (so coordinates are distinct
without a dedup pass), uniform per mode and across mode pairs, and identical
on numpy arrays and torch tensors."""
import numpy as np
import pytest
import torch

import synth


@pytest.mark.parametrize("bits", [2, 4, 6])
def test_feistel_is_a_bijection(bits):
    keys = synth.feistel_keys(11)
    e = np.arange(1 << (3 * bits), dtype=np.int64)
    c = synth.feistel_coords(e, bits, keys)
    for x in c:
        assert x.min() >= 0 and x.max() < (1 << bits)
    key = (c[0] << (2 * bits)) | (c[1] << bits) | c[2]
    assert np.array_equal(np.sort(key), e)


def test_feistel_distinct_and_uniform_at_22_bits():
    keys = synth.feistel_keys(synth.WORKLOADS["cp3_4M_m4B_r16"].seed)
    n = 1 << 21
    c = synth.feistel_coords(np.arange(n, dtype=np.int64), 22, keys)
    key = (c[0] << 44) | (c[1] << 22) | c[2]
    assert np.unique(key).size == n
    # chi-square over 64 bins per mode and over 16 x 16 bins of each mode pair
    def chi2(counts):
        exp = counts.sum() / counts.size
        return float(((counts - exp) ** 2 / exp).sum())
    for x in c:
        h = np.bincount(x >> 16, minlength=64)
        assert chi2(h) < 130          # 63 degrees of freedom: p ~ 1e-6
    for a, b in ((0, 1), (0, 2), (1, 2)):
        h = np.bincount((c[a] >> 18) * 16 + (c[b] >> 18), minlength=256)
        assert chi2(h) < 370          # 255 degrees of freedom: p ~ 1e-5


def test_feistel_numpy_and_torch_agree():
    keys = synth.feistel_keys(3)
    e = np.arange(5_000_000_000 - 100_000, 5_000_000_000, dtype=np.int64)
    a = synth.feistel_coords(e, 22, keys)
    b = synth.feistel_coords(torch.as_tensor(e), 22, keys)
    for x, y in zip(a, b):
        assert np.array_equal(x, y.numpy())


def test_feistel_rejects_odd_bits():
    with pytest.raises(ValueError):
        synth.feistel_coords(np.arange(4, dtype=np.int64), 3, synth.feistel_keys(1))
