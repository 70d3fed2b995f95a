"""CCD++ sweeps on the GPU (tc_ccd_sweep) against the FP64 oracle's ccd_sweep,
FP32 and FP64, ranks that do and do not fill their tier, and the rank-1
identity with the ALS sweep."""
import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

# a sweep is 3R dependent rank-1 solves: FP32 carries their rounding
SWEEP_TOL = {"f32": 1e-4, "f64": 1e-11}


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


@pytest.mark.parametrize("dtype,R", [("f32", 16), ("f64", 16), ("f32", 5), ("f64", 3)])
def test_ccd_sweep_matches_oracle(tc, dtype, R):
    prob = make_problem("ccd%s%d" % (dtype, R), (60, 50, 40), 15000, R, dtype, seed=R + 50,
                        noise=0.1, init="random")
    p = build(prob)
    A = [to_dev(a, dtype) for a in prob.factors]
    tc.ccd_sweep(p, A, 0.2)
    ref = oracle.ccd_sweep(prob.dims, prob.idx, prob.t, prob.factors, 0.2)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= SWEEP_TOL[dtype], (dtype, R, d)
    assert tc.last_error(p) == tc.OK


def test_ccd_rank1_equals_als(tc):
    from paper_1910_02371_gb300 import drivers
    prob = make_problem("ccd1", (40, 30, 20), 6000, 1, "f64", seed=61, noise=0.1, init="random")
    p = build(prob)
    A = [to_dev(a, "f64") for a in prob.factors]
    B = [a.clone() for a in A]
    tc.ccd_sweep(p, A, 0.3)
    drivers.als_sweep(p, B, 0.3)
    for d in range(3):
        assert rel(host(A[d]), host(B[d])) <= 1e-11
