"""Coordinate minimization for a general loss on the GPU (tc_ccd_newton_sweep)
against the FP64 oracle's ccd_newton_sweep: the Poisson log link on count data
(FP32 and FP64, ranks that do and do not fill their tier), least squares
(where one step per column is the CCD++ update, so it must agree with
tc_ccd_sweep), the stop test, the identity link's domain error, and argument
errors."""
import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

# a sweep is 3R dependent columns of several Newton steps each, and the model
# entries are updated incrementally: FP32 carries that rounding
SWEEP_TOL = {"f32": 1e-4, "f64": 1e-10}


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


def poisson_problem(dtype, R, dims=(50, 40, 30), nnz=9000, seed=71):
    prob = make_problem("ccdn%s%d" % (dtype, R), dims, nnz, R, dtype, seed, factor="uniform01",
                        recipe="poisson")
    A = [0.8 * a for a in prob.factors]
    if dtype == "f32":
        A = [a.astype(np.float32).astype(np.float64) for a in A]
    return prob, A


@pytest.mark.parametrize("dtype,R", [("f32", 8), ("f64", 8), ("f32", 5), ("f64", 3)])
def test_ccd_newton_poisson_matches_oracle(tc, dtype, R):
    prob, A = poisson_problem(dtype, R, seed=71 + R)
    p = build(prob)
    Ad = [to_dev(a, dtype) for a in A]
    # a fixed step count (tol 0) so both sides take the same steps
    steps = tc.ccd_newton_sweep(p, Ad, "poisson_log", 1.0, inner_iters=3, tol=0.0)
    assert steps == [[3, 3, 3]] * R
    ref, osteps = oracle.ccd_newton_sweep(prob.dims, prob.idx, prob.t, A, "poisson_log", 1.0,
                                          inner_iters=3, tol=0.0)
    assert (osteps == 3).all()
    for d in range(3):
        assert rel(host(Ad[d]), ref[d]) <= SWEEP_TOL[dtype], (dtype, R, d)
    assert tc.last_error(p) == tc.OK
    f0 = oracle.objective(prob.dims, prob.idx, prob.t, A, "poisson_log", 1.0)
    f1 = oracle.objective(prob.dims, prob.idx, prob.t, [host(a) for a in Ad], "poisson_log", 1.0)
    assert f1 < f0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ccd_newton_ls_one_step_is_ccd(tc, dtype):
    prob = make_problem("ccdnls%s" % dtype, (40, 35, 30), 8000, 6, dtype, seed=73, noise=0.1,
                        init="random")
    p = build(prob)
    A = [to_dev(a, dtype) for a in prob.factors]
    B = [a.clone() for a in A]
    steps = tc.ccd_newton_sweep(p, A, "ls", 0.2, inner_iters=1, tol=0.0)
    assert steps == [[1, 1, 1]] * 6
    tc.ccd_sweep(p, B, 0.2)
    ref = oracle.ccd_sweep(prob.dims, prob.idx, prob.t, prob.factors, 0.2)
    for d in range(3):
        assert rel(host(A[d]), host(B[d])) <= (1e-5 if dtype == "f32" else 1e-11)
        assert rel(host(A[d]), ref[d]) <= SWEEP_TOL[dtype]
    assert tc.last_error(p) == tc.OK


def test_ccd_newton_stop_test(tc):
    """FP64: with a tolerance the step counts per column follow the oracle's
    (within one where a norm ratio sits at the threshold) and the factors
    agree."""
    prob, A = poisson_problem("f64", 4, seed=79)
    p = build(prob)
    Ad = [to_dev(a, "f64") for a in A]
    steps = np.array(tc.ccd_newton_sweep(p, Ad, "poisson_log", 1.0, inner_iters=20, tol=1e-6))
    ref, osteps = oracle.ccd_newton_sweep(prob.dims, prob.idx, prob.t, A, "poisson_log", 1.0,
                                          inner_iters=20, tol=1e-6)
    assert steps.max() < 20 and steps.min() >= 2
    assert np.abs(steps - osteps).max() <= 1
    for d in range(3):
        assert rel(host(Ad[d]), ref[d]) <= 1e-7
    assert tc.last_error(p) == tc.OK


def test_ccd_newton_identity_link_domain(tc):
    """Identity link: the device records the domain error when (and only when)
    the oracle raises it on the same sweep."""
    prob, A = poisson_problem("f64", 3, seed=83)
    raised = False
    try:
        oracle.ccd_newton_sweep(prob.dims, prob.idx, prob.t, A, "poisson_id", 0.1, inner_iters=3,
                                tol=0.0)
    except oracle.OracleError as e:
        assert e.rc == oracle.ERR_DOMAIN
        raised = True
    p = build(prob)
    Ad = [to_dev(a, "f64") for a in A]
    tc.ccd_newton_sweep(p, Ad, "poisson_id", 0.1, inner_iters=3, tol=0.0)
    assert tc.last_error(p) == (tc.ERR_DOMAIN if raised else tc.OK)


def test_ccd_newton_errors(tc):
    prob, A = poisson_problem("f32", 3, seed=89)
    p = build(prob)
    Ad = [to_dev(a, "f32") for a in A]
    for kw in (dict(inner_iters=0), dict(tol=-1.0), dict(lam=-0.1)):
        args = dict(inner_iters=2, tol=1e-3, lam=0.5)
        args.update(kw)
        with pytest.raises(tc.TcError) as e:
            tc.ccd_newton_sweep(p, Ad, "poisson_log", args["lam"], inner_iters=args["inner_iters"],
                                tol=args["tol"])
        assert e.value.status == tc.ERR_ARG
    novals = build(prob, with_vals=False)
    with pytest.raises(tc.TcError) as e:
        tc.ccd_newton_sweep(novals, Ad, "poisson_log", 0.5)
    assert e.value.status == tc.ERR_ARG
