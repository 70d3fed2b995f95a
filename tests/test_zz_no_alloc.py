"""The allocation-free sort entry point against the oracle and the allocating one.

tc_sort_mode_noalloc exists for callers that may not allocate device memory
(a process whose memory belongs to another allocator's pool, a server that
forbids allocation while serving, a thread that must not stall on the implicit
synchronization an allocation can cause).  It keeps its work space in a fixed
array inside the library, so consecutive calls reuse whatever the previous one
left there.  These tests call it through the C ABI:
* twice in a row with inputs of different sizes (the second smaller, so stale
  work space from the first would show), requiring the oracle's stable
  counting sort (Sec. 3.4) bit for bit, and the same as tc_build_pattern's
  sorted views of the same tensors;
* on the edge cases: a mode of dimension 1 (no digit pass), no nonzeros, no
  status word (the library's own), and a key outside [0, I) (TC_ERR_RANGE
  reported, perm still a permutation);
* at the size limit's boundary.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


def _views(tc, idx, dims):
    p = tc.build_pattern([torch.as_tensor(c).cuda() for c in idx], dims)
    return [tuple(v.cpu().numpy() for v in p.view(d)[:2]) for d in range(3)]


def _noalloc(tc, key, I, with_status=True, expect=None):
    n = key.shape[0]
    key_d = torch.as_tensor(key).cuda() if n else None
    perm = torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda")
    row_ptr = torch.full((I + 1,), -7, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda") if with_status else None
    rc = tc._lib.tc_sort_mode_noalloc(
        n, ctypes.c_void_p(key_d.data_ptr() if n else None), I, ctypes.c_void_p(perm.data_ptr()),
        ctypes.c_void_p(row_ptr.data_ptr()),
        ctypes.c_void_p(status.data_ptr()) if with_status else None,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tc.OK
    torch.cuda.synchronize()
    if with_status:
        assert status.item() == (tc.OK if expect is None else expect)
    return perm.cpu().numpy()[:n], row_ptr.cpu().numpy()


def test_noalloc_sort_matches_oracle_twice(tc):
    # first call: near the size limit, skewed rows; second call: smaller, uniform
    dims_a = (3000, 700, 5)
    idx_a = synth.distinct_coords(dims_a, 900_000, ("zipf", "zipf", "uniform"), 31)
    dims_b = (10_000, 123, 4000)
    idx_b = synth.distinct_coords(dims_b, 70_001, ("uniform",) * 3, 32)
    views_a = _views(tc, idx_a, dims_a)
    views_b = _views(tc, idx_b, dims_b)
    for key, I, view in ((idx_a[0], dims_a[0], views_a[0]), (idx_b[1], dims_b[1], views_b[1])):
        perm, row_ptr = _noalloc(tc, key, I)
        perm_o, row_ptr_o = oracle.counting_sort(key, I)
        assert np.array_equal(perm, perm_o)
        assert np.array_equal(row_ptr, row_ptr_o)
        assert np.array_equal(perm, view[1]) and np.array_equal(row_ptr, view[0])


def test_noalloc_sort_edge_cases(tc):
    rng = np.random.default_rng(7)
    # a mode of dimension 1: every key is 0, no digit pass
    key = np.zeros(5000, np.int32)
    perm, row_ptr = _noalloc(tc, key, 1)
    assert np.array_equal(perm, np.arange(5000)) and list(row_ptr) == [0, 5000]
    # no nonzeros: every row offset is 0
    perm, row_ptr = _noalloc(tc, np.zeros(0, np.int32), 37)
    assert perm.size == 0 and np.array_equal(row_ptr, np.zeros(38, np.int64))
    # no status word given: the library's own is used; same result
    key = rng.integers(0, 1000, 123_457).astype(np.int32)
    perm, row_ptr = _noalloc(tc, key, 1000, with_status=False)
    perm_o, row_ptr_o = oracle.counting_sort(key, 1000)
    assert np.array_equal(perm, perm_o) and np.array_equal(row_ptr, row_ptr_o)
    # a key outside [0, I): TC_ERR_RANGE, and perm is still a permutation
    key = rng.integers(0, 300, 40_000).astype(np.int32)
    key[123] = 300
    key[4567] = 2_000_000_000
    key[9999] = -5
    perm, row_ptr = _noalloc(tc, key, 300, expect=tc.ERR_RANGE)
    assert np.array_equal(np.sort(perm), np.arange(key.shape[0]))
    assert row_ptr[0] >= 0 and row_ptr[-1] <= key.shape[0] and np.all(np.diff(row_ptr) >= 0)


def test_noalloc_sort_size_limit(tc):
    n = tc.SORT_NOALLOC_MAX_NNZ
    key = np.random.default_rng(8).integers(0, 1 << 20, n).astype(np.int32)
    perm, row_ptr = _noalloc(tc, key, 1 << 20)
    perm_o, row_ptr_o = oracle.counting_sort(key, 1 << 20)
    assert np.array_equal(perm, perm_o) and np.array_equal(row_ptr, row_ptr_o)
    n += 1
    key = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int64, device="cuda")
    row_ptr = torch.empty(2, dtype=torch.int64, device="cuda")
    rc = tc._lib.tc_sort_mode_noalloc(n, ctypes.c_void_p(key.data_ptr()), 1,
                                      ctypes.c_void_p(perm.data_ptr()),
                                      ctypes.c_void_p(row_ptr.data_ptr()), None,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tc.ERR_UNSUPPORTED
