"""General-loss ALS on the GPU (tc_newton_als_mode) against the FP64 oracle's
newton_als_sweep: the Poisson log link on count data (FP32 and FP64), the
identity link, least squares (where one Newton step is the ALS solve, so it
must agree with the ALS sweep), the stop test, and argument errors."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

# after a fixed number of Newton steps the FP32 path carries the FP32 solve
# error of each step (kappa u, refined away by the later steps); one decade
# above the kernel tolerance
SWEEP_TOL = {"f32": 1e-4, "f64": 1e-10}


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


def poisson_problem(dtype, dims=(60, 50, 40), nnz=12000, R=8, seed=17):
    prob = make_problem("pois%s" % dtype, dims, nnz, R, dtype, seed, factor="uniform01",
                        recipe="poisson")
    # start below the planted factors: exp(m) stays moderate
    A = [0.8 * a for a in prob.factors]
    if dtype == "f32":
        A = [a.astype(np.float32).astype(np.float64) for a in A]
    return prob, A


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_newton_als_sweep_matches_oracle(tc, dtype):
    from paper_1910_02371_gb300 import drivers
    loss = "poisson_log"
    prob, A = poisson_problem(dtype)
    p = build(prob)
    Ad = [to_dev(a, dtype) for a in A]
    steps = drivers.newton_als_sweep(p, Ad, loss, 0.1, inner_iters=4, tol=0.0)
    assert steps == [4, 4, 4]
    ref = oracle.newton_als_sweep(prob.dims, prob.idx, prob.t, A, loss, 0.1, inner_iters=4, tol=0.0)
    for d in range(3):
        assert rel(host(Ad[d]), ref[d]) <= SWEEP_TOL[dtype], (loss, d)
    assert tc.last_error(p) == tc.OK
    f0 = oracle.objective(prob.dims, prob.idx, prob.t, A, loss, 0.1)
    f1 = oracle.objective(prob.dims, prob.idx, prob.t, [host(a) for a in Ad], loss, 0.1)
    assert f1 < f0


def test_newton_ls_one_step_is_als(tc):
    from paper_1910_02371_gb300 import drivers
    prob = make_problem("nls", (50, 40, 30), 8000, 6, "f64", 23)
    p = build(prob)
    A = [to_dev(a, "f64") for a in prob.factors]
    B = [a.clone() for a in A]
    steps = drivers.newton_als_sweep(p, A, "ls", 0.2, inner_iters=1, tol=0.0)
    assert steps == [1, 1, 1]
    drivers.als_sweep(p, B, 0.2)
    for d in range(3):
        assert rel(host(A[d]), host(B[d])) <= 1e-11
    ref = oracle.als_sweep(prob.dims, prob.idx, prob.t, prob.factors, 0.2)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= TOL["f64"]


def test_newton_stop_test_and_errors(tc):
    prob, A = poisson_problem("f64", seed=29)
    p = build(prob)
    Ad = [to_dev(a, "f64") for a in A]
    steps = tc.newton_als_mode(p, Ad, 0, "poisson_log", 0.1, inner_iters=30, tol=1e-9)
    o, taken = oracle.newton_als_mode(prob.dims, prob.idx, prob.t, A, 0, "poisson_log", 0.1,
                                      inner_iters=30, tol=1e-9)
    assert 1 < steps < 30 and abs(steps - taken) <= 1
    assert rel(host(Ad[0]), o[0]) <= 1e-9
    with pytest.raises(tc.TcError):
        tc.newton_als_mode(p, Ad, 0, "poisson_log", 0.1, inner_iters=0)
    with pytest.raises(tc.TcError):
        tc.newton_als_mode(p, Ad, 3, "poisson_log", 0.1)


def test_newton_identity_link_leaves_domain_like_the_oracle(tc):
    """With the identity link phi'' = t / m^2 vanishes at zero counts, so full
    Newton steps on count data overshoot to m <= 0: the device reports the
    domain error exactly where the oracle raises it."""
    from paper_1910_02371_gb300 import drivers
    prob, _ = poisson_problem("f64")
    A = list(prob.factors)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.newton_als_sweep(prob.dims, prob.idx, prob.t, A, "poisson_id", 0.1, inner_iters=2,
                                tol=0.0)
    assert ei.value.rc == oracle.ERR_DOMAIN
    p = build(prob)
    Ad = [to_dev(a, "f64") for a in A]
    drivers.newton_als_sweep(p, Ad, "poisson_id", 0.1, inner_iters=2, tol=0.0)
    assert tc.last_error(p) == tc.ERR_DOMAIN
