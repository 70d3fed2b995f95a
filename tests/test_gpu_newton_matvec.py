"""Full Newton Hessian-vector product (tc_newton_matvec) against the FP64
oracle for every loss and dtype, on the plain and on the interleaved (PCG)
layout, and Newton-CG through the solver with the full Hessian selected."""
import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

LOSS_CASES = [("ls", "f32", 16), ("ls", "f64", 16), ("poisson_log", "f32", 8),
              ("poisson_log", "f64", 5), ("poisson_id", "f64", 8), ("ls", "f32", 12)]


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


def problem(loss, dtype, R):
    if loss == "ls":
        return make_problem("nm" + dtype + str(R), (40, 35, 30), 6000, R, dtype, seed=R + 3, noise=0.3,
                            init="random")
    prob = make_problem("nmp" + dtype + str(R), (40, 35, 30), 6000, R, dtype, seed=R + 4,
                        factor="uniform01", recipe="poisson")
    return prob


@pytest.mark.parametrize("loss,dtype,R", LOSS_CASES)
def test_newton_matvec_matches_oracle(tc, loss, dtype, R):
    prob = problem(loss, dtype, R)
    p = build(prob)
    A = [to_dev(a, dtype) for a in prob.factors]
    rng = np.random.default_rng(R)
    x = [rng.standard_normal((I, R)) for I in prob.dims]
    if dtype == "f32":
        x = [v.astype(np.float32).astype(np.float64) for v in x]
    y = tc.newton_matvec(p, A, [to_dev(v, dtype) for v in x], loss, 0.1)
    yo = oracle.newton_matvec(prob.dims, prob.idx, prob.t, prob.factors, loss, 0.1, x)
    for d in range(3):
        assert rel(host(y[d]), yo[d]) <= TOL[dtype], (loss, dtype, d)
    # the solver's product (interleaved layout on the vector path) agrees
    cg = tc.CG(p, A, loss, 0.1)
    cg.set_hessian(True)
    y2 = cg.matvec([to_dev(v, dtype) for v in x])
    for d in range(3):
        assert rel(host(y2[d]), yo[d]) <= TOL[dtype], (loss, dtype, d, "cg")
    assert tc.last_error(p) == tc.OK


def test_newton_cg_solve_matches_oracle_pcg(tc):
    """Least squares away from the fit: PCG with the full Hessian from the
    solver against CG on the oracle's full Hessian (same iteration, same
    block-diagonal preconditioner)."""
    prob = problem("ls", "f64", 16)
    p = build(prob)
    A = [to_dev(a, "f64") for a in prob.factors]
    cg = tc.CG(p, A, "ls", 0.5)
    cg.set_hessian(True)
    cg.setup()
    _, g = oracle.loss_grad(prob.dims, prob.idx, prob.t, prob.factors, "ls", 0.5)
    b = [-v for v in g]
    dx = [host(v) for v in cg.solve([to_dev(v, "f64") for v in b], 6)]
    rc = tc.last_error(p)
    # oracle PCG with the full Hessian (composition of pinned routines)
    H = lambda v: oracle.newton_matvec(prob.dims, prob.idx, prob.t, prob.factors, "ls", 0.5, v)
    P = lambda v: oracle.precond_apply(prob.dims, prob.idx, prob.t, prob.factors, "ls", 0.5, v)
    dot = lambda a, c: sum(np.vdot(u, w) for u, w in zip(a, c))
    x = [np.zeros_like(v) for v in b]
    r = [v.copy() for v in b]
    z = P(r)
    pv = [v.copy() for v in z]
    rz = dot(r, z)
    stopped = False
    for _ in range(6):
        Hp = H(pv)
        pHp = dot(pv, Hp)
        if pHp <= 0:
            stopped = True
            break
        al = rz / pHp
        x = [a + al * c for a, c in zip(x, pv)]
        r = [a - al * c for a, c in zip(r, Hp)]
        z = P(r)
        rzn = dot(r, z)
        pv = [a + (rzn / rz) * c for a, c in zip(z, pv)]
        rz = rzn
    assert (rc == tc.ERR_BREAKDOWN) == stopped
    for d in range(3):
        assert rel(dx[d], x[d]) <= 1e-9


def test_hessian_selector_switches_back(tc):
    prob = problem("ls", "f64", 16)
    p = build(prob)
    A = [to_dev(a, "f64") for a in prob.factors]
    rng = np.random.default_rng(1)
    x = [to_dev(rng.standard_normal((I, 16)), "f64") for I in prob.dims]
    cg = tc.CG(p, A, "ls", 0.1)
    g1 = [host(v) for v in cg.matvec(x)]
    cg.set_hessian(True)
    n1 = [host(v) for v in cg.matvec(x)]
    cg.set_hessian(False)
    g2 = [host(v) for v in cg.matvec(x)]
    gg = [host(v) for v in tc.ggn_matvec(p, A, x, "ls", 0.1)]
    for d in range(3):
        assert rel(g1[d], gg[d]) <= 1e-12 and rel(g2[d], gg[d]) <= 1e-12
    assert sum(rel(a, b) for a, b in zip(n1, gg)) > 1e-6
    with pytest.raises(tc.TcError):
        tc._check(tc._lib.tc_cg_set_hessian(cg.handle, 2), "set")
