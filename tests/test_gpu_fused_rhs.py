"""Right-hand sides formed in Solve Factor's Gram pass.

tc_als_update -- the MTTKRP of the values and Solve Factor of one mode in one
call, the right-hand side formed in the Gram pass where the Gram kernel
supports it -- against the FP64 oracle's Solve Factor on the oracle's MTTKRP,
on Zipf and uniform rows, rows split over many chunks (their right-hand sides
summed in FP64 slots), rows beyond the last nonzero (empty), every rank tier
and both dtypes; and a whole fused ALS sweep against the oracle's sweep.

tc_ggn_step, whose preconditioner passes also form the gradient's
MTTKRP(phi') and the loss (FP32, R <= 32): the objective it reports and the
step it takes against the oracle's, for every loss, with rows cut across
chunks."""
import zlib

import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "zipf_f32_r16": dict(dims=(5000, 800, 60), nnz=80000, R=16, dtype="f32",
                         dist=("zipf", "zipf", "uniform")),
    "zipf_f32_r7": dict(dims=(3000, 400, 30), nnz=40000, R=7, dtype="f32",
                        dist=("zipf", "zipf", "uniform")),
    "f32_r32": dict(dims=(800, 300, 90), nnz=40000, R=32, dtype="f32"),
    "f32_r24": dict(dims=(700, 500, 80), nnz=30000, R=24, dtype="f32"),
    "zipf_f32_r64": dict(dims=(4000, 600, 50), nnz=60000, R=64, dtype="f32",
                         dist=("zipf", "zipf", "uniform")),
    "zipf_f64_r16": dict(dims=(2000, 300, 40), nnz=30000, R=16, dtype="f64",
                         dist=("zipf", "zipf", "uniform")),
    "zipf_f64_r24": dict(dims=(1500, 300, 40), nnz=25000, R=24, dtype="f64",
                         dist=("zipf", "zipf", "uniform")),
    # more rows than the coordinates reach: empty rows solve lambda a_i = 0
    "sparse_f32_r16": dict(dims=(20000, 3000, 50), nnz=20000, R=16, dtype="f32"),
}
# (chunk_nnz, batch_bytes, chol_rows_per_warp): automatic, tiny chunks (nearly
# every row cut), odd chunks with one warp's rows per batch
TUNINGS = [(0, 0, 0), (16, 0, 0), (37, 1, 0)]

_cache = {}


def problem(name):
    if name not in _cache:
        c = dict(CASES[name])
        _cache[name] = make_problem(name, c.pop("dims"), c.pop("nnz"), c.pop("R"), c.pop("dtype"),
                                    seed=zlib.crc32(name.encode()) % 10_000 + 17, **c)
    return _cache[name]


@pytest.fixture(scope="module")
def tc():
    import torch
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    yield t
    t.set_solve_tuning(torch.float32, 0, reset=True)
    t.set_solve_tuning(torch.float64, 0, reset=True)


def _tune(tc, prob, tuning):
    import torch
    dt = torch.float32 if prob.dtype == "f32" else torch.float64
    tc.set_solve_tuning(dt, 0, reset=True)
    if tuning != (0, 0, 0):
        tc.set_solve_tuning(dt, prob.R, chunk_nnz=tuning[0], batch_bytes=tuning[1],
                            chol_rows_per_warp=tuning[2])


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tuning", TUNINGS)
def test_als_update_matches_oracle(tc, name, tuning):
    import torch
    prob = problem(name)
    _tune(tc, prob, tuning)
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    lam = 0.5
    for mode in range(3):
        rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
        ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, lam)
        assert rc == 0
        status = torch.full((prob.dims[mode],), 5, dtype=torch.int8, device="cuda")
        out = torch.empty_like(A[mode])
        tc.als_update(p, A, mode, lam, out=out, row_status=status)
        assert not status.any().item()
        assert rel(host(out), ref) <= TOL[prob.dtype], (name, tuning, mode, rel(host(out), ref))
    assert tc.last_error(p) == tc.OK


def rhs_rounding_bound(prob, mode, lam):
    """Normwise bound, relative to the exact solution's norm, on what an FP32
    right-hand side alone moves the solution (numpy, FP64): rhs_i[r] is a sum
    of n_i FP32 products, off by at most gamma(n_i) sum_e |t_e h_e[r]|
    (gamma(n) = n u / (1 - n u), u = 2^-24, any summation order), and the
    solve maps it through (G_i + lam I)^-1.  Refinement removes the Gram's
    rounding, not this."""
    o1, o2 = [d for d in range(3) if d != mode]
    A, idx, t = prob.factors, prob.idx, prob.t
    order = np.argsort(idx[mode], kind="stable")
    rows = idx[mode][order]
    H = A[o1][idx[o1][order]] * A[o2][idx[o2][order]]
    tH = np.abs(t[order])[:, None] * np.abs(H)
    bounds = np.searchsorted(rows, np.arange(prob.dims[mode] + 1))
    u = 2.0 ** -24
    err2 = 0.0
    sol2 = 0.0
    for i in range(prob.dims[mode]):
        a, b = bounds[i], bounds[i + 1]
        n = b - a
        if n == 0:
            continue
        Hi = H[a:b]
        M = Hi.T @ Hi + lam * np.eye(prob.R)
        gamma = n * u / (1 - n * u)
        d_rhs = gamma * tH[a:b].sum(axis=0)
        err2 += (np.linalg.norm(d_rhs) / np.linalg.eigvalsh(M)[0]) ** 2
        sol2 += np.linalg.norm(np.linalg.solve(M, Hi.T @ t[order][a:b])) ** 2
    return np.sqrt(err2 / sol2)


@pytest.mark.parametrize("prec,lam", [("fp32_refine", 0.5), ("tf32_refine2", 0.5),
                                      ("fp32_refine", 0.05)])
@pytest.mark.parametrize("name", ["zipf_f32_r16", "f32_r32", "zipf_f32_r64"])
def test_als_update_refined_forms(tc, name, prec, lam):
    """The refinement residual and correction read the right-hand side the
    Gram pass formed.  At lambda = 0.5 the refined forms reach the oracle's
    solve within the FP32 tolerance.  At lambda = 0.05 the short Zipf rows are
    ill-conditioned (kappa ~ 10^3) and the FP32 right-hand side limits the
    solution (about 1e-5 on zipf_f32_r16, 5.5e-5 on zipf_f32_r64, measured):
    the error must stay within the FP32 tolerance plus rhs_rounding_bound, and
    within twice the error of the two-call path (tc_mttkrp, then
    tc_solve_factor), whose right-hand side is an FP32 sum too."""
    prob = problem(name)
    _tune(tc, prob, (16, 0, 0))
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    for mode in range(3):
        rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
        ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, lam)
        assert rc == 0
        out = host(tc.als_update(p, A, mode, lam, out=A[mode].clone(), prec=prec))
        err = rel(out, ref)
        if lam >= 0.5:
            assert err <= TOL["f32"], (name, prec, mode, err)
            continue
        tol = TOL["f32"] + rhs_rounding_bound(prob, mode, lam)
        b = tc.mttkrp(p, A, mode)
        two_call = rel(host(tc.solve_factor(p, A, mode, b, lam, prec=prec)), ref)
        assert err <= tol and err <= max(TOL["f32"], 2 * two_call), (name, prec, mode, err, tol,
                                                                     two_call)
    assert tc.last_error(p) == tc.OK


@pytest.mark.parametrize("name", ["zipf_f32_r16", "zipf_f64_r16", "f32_r32"])
def test_fused_sweep_matches_oracle_and_two_call_sweep(tc, name):
    """A fused ALS sweep (in place, each mode seeing the modes updated before
    it) against the oracle's sweep, and against the two-call sweep."""
    from paper_1910_02371_gb300 import drivers
    prob = problem(name)
    _tune(tc, prob, (0, 0, 0))
    p = build(prob)
    lam = 0.5
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    drivers.als_sweep(p, A, lam)
    B = [to_dev(a, prob.dtype) for a in prob.factors]
    drivers.als_sweep(p, B, lam, fused=False)
    ref = oracle.als_sweep(prob.dims, prob.idx, prob.t, prob.factors, lam)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= 3 * TOL[prob.dtype], (name, d)
        assert rel(host(A[d]), host(B[d])) <= 3 * TOL[prob.dtype], (name, d)
    assert tc.last_error(p) == tc.OK


def test_als_update_rejects_a_pattern_without_values(tc):
    prob = problem("f32_r32")
    p = build(prob, with_vals=False)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    with pytest.raises(tc.TcError) as ei:
        tc.als_update(p, A, 0, 0.5)
    assert ei.value.status == tc.ERR_ARG


def positive_problem(R):
    key = ("pos", R)
    if key not in _cache:
        _cache[key] = make_problem("pos%d" % R, (400, 300, 50), 30000, R, "f32", seed=77 + R,
                                   factor="uniform01", recipe="poisson",
                                   dist=("zipf", "uniform", "uniform"))
    return _cache[key]


# A Gauss-Newton step chains the gradient, the preconditioner and 10 PCG
# iterations; as for the library's other CG tests, 10x the FP32 kernel
# tolerance.
CG_TOL_F32 = 10 * TOL["f32"]


@pytest.mark.parametrize("R", [7, 16, 32])
@pytest.mark.parametrize("loss", ["ls", "poisson_log", "poisson_id"])
@pytest.mark.parametrize("chunk", [0, 16])
def test_ggn_step_with_the_gradient_in_the_preconditioner_pass(tc, R, loss, chunk):
    import torch
    prob = positive_problem(R)
    tc.set_solve_tuning(torch.float32, 0, reset=True)
    if chunk:
        tc.set_solve_tuning(torch.float32, R, chunk_nnz=chunk)
    lam = 0.1
    A0 = [0.5 * a for a in prob.factors]
    p = build(prob)
    A = [to_dev(a, "f32") for a in A0]
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    tc.CG(p, A, loss, lam).ggn_step(10, loss_out=f)
    fo = oracle.objective(prob.dims, prob.idx, prob.t, A0, loss, lam)
    assert abs(f.item() - fo) <= TOL["f32"] * abs(fo), (loss, R, f.item(), fo)
    ref = oracle.ggn_step(prob.dims, prob.idx, prob.t, A0, loss, lam, 10)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= CG_TOL_F32, (loss, R, d, rel(host(A[d]), ref[d]))
    assert tc.last_error(p) == tc.OK
    tc.set_solve_tuning(torch.float32, 0, reset=True)
