"""The allocation-free sort entry point against the allocating one.

tc_sort_mode_noalloc exists for callers that may not allocate device memory
(a process whose memory belongs to another allocator's pool, a server that
forbids allocation while serving, a thread that must not stall on the implicit
synchronization an allocation can cause).  It keeps its work space in a fixed
array inside the library, so consecutive calls reuse whatever the previous one
left there.  This test calls it twice in a row, through the C ABI, with inputs
of different sizes (the second smaller, so stale work space from the first
would show), and requires the same permutation and row offsets -- index work,
so bit for bit -- as tc_build_pattern's sorted views of the same tensors.  It
also checks the size limit.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

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


def _noalloc(tc, key, I):
    key_d = torch.as_tensor(key).cuda()
    perm = torch.full((key.shape[0],), -7, dtype=torch.int64, device="cuda")
    row_ptr = torch.full((I + 1,), -7, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    rc = tc._lib.tc_sort_mode_noalloc(key.shape[0], ctypes.c_void_p(key_d.data_ptr()), I,
                                      ctypes.c_void_p(perm.data_ptr()),
                                      ctypes.c_void_p(row_ptr.data_ptr()),
                                      ctypes.c_void_p(status.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tc.OK
    torch.cuda.synchronize()
    assert status.item() == tc.OK
    return perm.cpu().numpy(), row_ptr.cpu().numpy()


def test_noalloc_sort_matches_build_pattern_twice(tc):
    # first call: near the size limit, skewed rows; second call: smaller, uniform
    dims_a = (3000, 700, 5)
    idx_a = synth.distinct_coords(dims_a, 900_000, ("zipf", "zipf", "uniform"), 31)
    dims_b = (10_000, 123, 4000)
    idx_b = synth.distinct_coords(dims_b, 70_001, ("uniform",) * 3, 32)
    views_a = _views(tc, idx_a, dims_a)
    views_b = _views(tc, idx_b, dims_b)
    perm, row_ptr = _noalloc(tc, idx_a[0], dims_a[0])
    assert np.array_equal(perm, views_a[0][1])
    assert np.array_equal(row_ptr, views_a[0][0])
    perm, row_ptr = _noalloc(tc, idx_b[1], dims_b[1])
    assert np.array_equal(perm, views_b[1][1])
    assert np.array_equal(row_ptr, views_b[1][0])


def test_noalloc_sort_rejects_oversize(tc):
    n = tc.SORT_NOALLOC_MAX_NNZ + 1
    key = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int64, device="cuda")
    row_ptr = torch.empty(2, dtype=torch.int64, device="cuda")
    rc = tc._lib.tc_sort_mode_noalloc(n, ctypes.c_void_p(key.data_ptr()), 1,
                                      ctypes.c_void_p(perm.data_ptr()),
                                      ctypes.c_void_p(row_ptr.data_ptr()), None,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tc.ERR_UNSUPPORTED
