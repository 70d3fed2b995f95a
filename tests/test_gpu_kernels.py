"""GPU parity: every kernel of the hot path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.  Index work must match bit for bit;
floating-point outputs within the normwise relative tolerance of their dtype
(1e-5 for FP32, 1e-12 for FP64).  Cases span many warps and chunks, ragged
tails, non-vector ranks, skewed (Zipf) rows with empty rows, and a mode of
dimension 1."""
import zlib

import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, idx_dev, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "tiny_f64_r3": dict(dims=(5, 6, 4), nnz=60, R=3, dtype="f64"),
    "f32_r16": dict(dims=(60, 50, 40), nnz=20000, R=16, dtype="f32"),
    "f32_r5": dict(dims=(70, 30, 90), nnz=9000, R=5, dtype="f32"),
    "f64_r5_200cube": dict(dims=(200, 200, 200), nnz=40000, R=5, dtype="f64"),
    "zipf_f32_r32": dict(dims=(3000, 500, 100), nnz=50000, R=32, dtype="f32",
                         dist=("zipf", "zipf", "uniform")),
    "f32_r64": dict(dims=(100, 80, 60), nnz=20000, R=64, dtype="f32"),
    "f32_r1": dict(dims=(50, 40, 30), nnz=5000, R=1, dtype="f32"),
    "f64_dim1_r8": dict(dims=(1, 7, 300), nnz=1000, R=8, dtype="f64"),
    "f32_r12": dict(dims=(40, 45, 50), nnz=8000, R=12, dtype="f32"),
    "f64_r16": dict(dims=(30, 40, 50), nnz=10000, R=16, dtype="f64"),
}

_cache = {}


def problem(name):
    if name not in _cache:
        c = dict(CASES[name])
        _cache[name] = make_problem(name, c.pop("dims"), c.pop("nnz"), c.pop("R"), c.pop("dtype"),
                                    seed=zlib.crc32(name.encode()) % 10_000 + 1, **c)
    return _cache[name]


def dev_factors(prob, fs=None):
    return [to_dev(a, prob.dtype) for a in (fs if fs is not None else prob.factors)]


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


# ------------------------------------------------------------------ pattern (bit-exact)
@pytest.mark.parametrize("name", list(CASES))
def test_pattern_bit_exact(tc, name):
    prob = problem(name)
    p = build(prob)
    for d in range(3):
        row_ptr, perm, nz = p.view(d)
        operm, orow, onz = oracle.pattern(prob.dims, prob.idx, d)
        assert np.array_equal(perm.cpu().numpy(), operm)
        assert np.array_equal(row_ptr.cpu().numpy(), orow)
        assert np.array_equal(nz.cpu().numpy(), onz)
        assert row_ptr[-1].item() == prob.nnz


def test_pattern_rejects_range_and_duplicates(tc):
    import torch
    idx = [np.array([0, 1, 2], np.int32), np.array([0, 1, 1], np.int32), np.array([0, 0, 3], np.int32)]
    with pytest.raises(tc.TcError) as e:
        tc.build_pattern(idx_dev(idx), (3, 2, 3))
    assert e.value.status == tc.ERR_RANGE
    dup = [np.array([0, 1, 0], np.int32), np.array([1, 1, 1], np.int32), np.array([2, 0, 2], np.int32)]
    tc.build_pattern(idx_dev(dup), (3, 2, 3))                      # unchecked: accepted
    with pytest.raises(tc.TcError) as e:
        tc.build_pattern(idx_dev(dup), (3, 2, 3), check_duplicates=True)
    assert e.value.status == tc.ERR_DUPLICATE
    prob = problem("f32_r16")
    tc.build_pattern(idx_dev(prob.idx), prob.dims, check_duplicates=True)   # distinct: accepted
    torch.cuda.synchronize()


def test_empty_tensor(tc):
    import torch
    idx = [torch.zeros(0, dtype=torch.int32, device="cuda") for _ in range(3)]
    vals = torch.zeros(0, dtype=torch.float32, device="cuda")
    p = tc.build_pattern(idx, (4, 5, 6), vals)
    A = [torch.randn(I, 8, device="cuda") for I in (4, 5, 6)]
    x = tc.tttp(p, A)
    assert x.numel() == 0
    out = tc.mttkrp(p, A, 1)
    assert torch.count_nonzero(out).item() == 0
    rhs = torch.randn(4, 8, device="cuda")
    a = tc.solve_factor(p, A, 0, rhs, 0.5)
    torch.testing.assert_close(a, rhs / 0.5)
    loss, g = tc.loss_grad(p, A, "ls", 0.25)
    np.testing.assert_allclose(loss.item(), 0.25 * sum(float((f.double() ** 2).sum()) for f in A),
                               rtol=1e-6)
    for gi, f in zip(g, A):
        torch.testing.assert_close(gi, 0.5 * f)
    assert tc.last_error(p) == tc.OK


# ------------------------------------------------------------------ TTTP
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("weights", ["one", "values", "array"])
def test_tttp(tc, name, weights):
    prob = problem(name)
    p = build(prob)
    perm0 = oracle.pattern(prob.dims, prob.idx, 0)[0]
    rng = np.random.default_rng(7)
    s_in = None if weights == "one" else (prob.t if weights == "values" else rng.standard_normal(prob.nnz))
    if prob.dtype == "f32" and s_in is not None:
        s_in = s_in.astype(np.float32).astype(np.float64)
    w = None if weights == "one" else ("values" if weights == "values" else to_dev(s_in[perm0], prob.dtype))
    x = host(tc.tttp(p, dev_factors(prob), weights=w))
    ref = oracle.tttp(prob.dims, prob.idx, s_in, prob.factors)[perm0]
    assert rel(x, ref) <= TOL[prob.dtype]


@pytest.mark.parametrize("name", ["f32_r16", "f64_r5_200cube", "f32_r5"])
@pytest.mark.parametrize("skip", [0, 1, 2])
def test_tttp_skipped_mode(tc, name, skip):
    prob = problem(name)
    p = build(prob)
    perm0 = oracle.pattern(prob.dims, prob.idx, 0)[0]
    fs = [None if n == skip else f for n, f in enumerate(prob.factors)]
    x = host(tc.tttp(p, [None if f is None else to_dev(f, prob.dtype) for f in fs], weights="values"))
    ref = oracle.tttp(prob.dims, prob.idx, prob.t, fs)[perm0]
    assert rel(x, ref) <= TOL[prob.dtype]


# ------------------------------------------------------------------ MTTKRP
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mttkrp(tc, name, mode):
    prob = problem(name)
    p = build(prob)
    out = host(tc.mttkrp(p, dev_factors(prob), mode, weights="values"))
    ref = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
    assert rel(out, ref) <= TOL[prob.dtype]


@pytest.mark.parametrize("name", ["f32_r16", "zipf_f32_r32", "f64_r16"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mttkrp_weights_and_accumulate(tc, name, mode):
    prob = problem(name)
    p = build(prob)
    A = dev_factors(prob)
    perm0 = oracle.pattern(prob.dims, prob.idx, 0)[0]
    # unit weights (Omega-hat)
    out = host(tc.mttkrp(p, A, mode, weights="one"))
    assert rel(out, oracle.mttkrp(prob.dims, prob.idx, None, prob.factors, mode)) <= TOL[prob.dtype]
    # caller array in pattern order, accumulated onto a start value
    s_in = np.random.default_rng(3).standard_normal(prob.nnz)
    if prob.dtype == "f32":
        s_in = s_in.astype(np.float32).astype(np.float64)
    start = np.random.default_rng(4).standard_normal((prob.dims[mode], prob.R))
    o = to_dev(start, prob.dtype)
    tc.mttkrp(p, A, mode, weights=to_dev(s_in[perm0], prob.dtype), out=o, accumulate=True)
    ref = start + oracle.mttkrp(prob.dims, prob.idx, s_in, prob.factors, mode)
    assert rel(host(o), ref) <= TOL[prob.dtype]


# ------------------------------------------------------------------ Solve Factor
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_solve_factor(tc, name, mode):
    prob = problem(name)
    p = build(prob)
    A = dev_factors(prob)
    lam = 0.5
    rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, mode)
    if prob.dtype == "f32":
        rhs = rhs.astype(np.float32).astype(np.float64)
    status = __import__("torch").zeros(prob.dims[mode], dtype=__import__("torch").int8, device="cuda")
    out = host(tc.solve_factor(p, A, mode, to_dev(rhs, prob.dtype), lam, row_status=status))
    ref, ost, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, lam)
    assert rc == 0 and not status.any().item()
    assert rel(out, ref) <= TOL[prob.dtype]
    assert tc.last_error(p) == tc.OK


@pytest.mark.parametrize("name", ["f32_r16", "f64_r16", "zipf_f32_r32"])
def test_solve_factor_weighted(tc, name):
    prob = problem(name)
    p = build(prob)
    perm0 = oracle.pattern(prob.dims, prob.idx, 0)[0]
    w_in = np.abs(np.random.default_rng(9).standard_normal(prob.nnz)) + 0.1
    if prob.dtype == "f32":
        w_in = w_in.astype(np.float32).astype(np.float64)
    for mode in range(3):
        rhs = np.random.default_rng(mode).standard_normal((prob.dims[mode], prob.R))
        out = host(tc.solve_factor(p, dev_factors(prob), mode, to_dev(rhs, prob.dtype), 0.3,
                                   weights=to_dev(w_in[perm0], prob.dtype)))
        ref, _, _ = oracle.solve_factor(prob.dims, prob.idx, w_in, prob.factors, mode, rhs, 0.3)
        assert rel(out, ref) <= TOL[prob.dtype]


def test_solve_factor_not_spd_rows_untouched(tc):
    import torch
    prob = problem("zipf_f32_r32")
    p = build(prob)
    mode = 0
    rhs = np.random.default_rng(1).standard_normal((prob.dims[mode], prob.R))
    prev = np.full((prob.dims[mode], prob.R), 7.0)
    out = to_dev(prev, "f32")
    status = torch.zeros(prob.dims[mode], dtype=torch.int8, device="cuda")
    tc.solve_factor(p, dev_factors(prob), mode, to_dev(rhs, "f32"), -0.1, out=out, row_status=status)
    assert tc.last_error(p) == tc.ERR_NOT_SPD
    ref, ost, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, mode, rhs, -0.1, out=prev)
    assert rc == oracle.ERR_NOT_SPD
    st = status.cpu().numpy()
    assert np.array_equal(st, ost)          # rows with fewer than R nonzeros are indefinite
    got = host(out)
    np.testing.assert_array_equal(got[st == 1], prev[st == 1])
    # the rows that factored are barely definite (lambda < 0), hence badly
    # conditioned: their solutions carry the FP32 Gram error times a large
    # condition number, so only a loose agreement is meaningful here
    ok_rows = np.nonzero(st == 0)[0]
    if ok_rows.size:
        assert np.all(np.isfinite(got[ok_rows]))
        assert rel(got[ok_rows], ref[ok_rows]) <= 1e-2
    assert tc.last_error(p) == tc.OK        # cleared


# ------------------------------------------------------------------ loss and gradient
LOSS_CASES = [("f32_r16", "ls"), ("f64_r16", "ls"), ("zipf_f32_r32", "ls"), ("f32_r5", "ls"),
              ("f64_r5_200cube", "ls"), ("f32_r64", "ls")]


def positive_problem(name, dtype, R=8):
    key = ("pos", name, dtype, R)
    if key not in _cache:
        _cache[key] = make_problem(key, (40, 30, 50), 12000, R, dtype, seed=77, factor="uniform01",
                                   recipe="poisson")
    return _cache[key]


@pytest.mark.parametrize("name,loss", LOSS_CASES)
def test_loss_grad(tc, name, loss):
    prob = problem(name)
    p = build(prob)
    lam = 0.05
    f, g = tc.loss_grad(p, dev_factors(prob), loss, lam)
    fo, go = oracle.loss_grad(prob.dims, prob.idx, prob.t, prob.factors, loss, lam)
    assert abs(f.item() - fo) <= TOL[prob.dtype] * abs(fo)
    for d in range(3):
        assert rel(host(g[d]), go[d]) <= TOL[prob.dtype]


@pytest.mark.parametrize("loss", ["poisson_log", "poisson_id"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_loss_grad_poisson(tc, loss, dtype):
    prob = positive_problem("p", dtype)
    p = build(prob)
    A = prob.factors if loss == "poisson_id" else [0.5 * a for a in prob.factors]
    f, g = tc.loss_grad(p, dev_factors(prob, A), loss, 0.1)
    fo, go = oracle.loss_grad(prob.dims, prob.idx, prob.t, A, loss, 0.1)
    assert abs(f.item() - fo) <= TOL[dtype] * abs(fo)
    for d in range(3):
        assert rel(host(g[d]), go[d]) <= TOL[dtype]


def test_loss_poisson_identity_domain_error(tc):
    prob = positive_problem("p", "f32")
    p = build(prob)
    A = [-a for a in prob.factors[:1]] + prob.factors[1:]     # every model entry < 0
    tc.loss_grad(p, dev_factors(prob, A), "poisson_id", 0.1)
    assert tc.last_error(p) == tc.ERR_DOMAIN


# ------------------------------------------------------------------ Gauss-Newton matvec
@pytest.mark.parametrize("name,loss", LOSS_CASES)
def test_ggn_matvec(tc, name, loss):
    prob = problem(name)
    p = build(prob)
    rng = np.random.default_rng(11)
    x = [rng.standard_normal((I, prob.R)) for I in prob.dims]
    if prob.dtype == "f32":
        x = [v.astype(np.float32).astype(np.float64) for v in x]
    y = tc.ggn_matvec(p, dev_factors(prob), [to_dev(v, prob.dtype) for v in x], loss, 0.05)
    yo = oracle.ggn_matvec(prob.dims, prob.idx, prob.t, prob.factors, loss, 0.05, x)
    for d in range(3):
        assert rel(host(y[d]), yo[d]) <= TOL[prob.dtype]


@pytest.mark.parametrize("loss", ["poisson_log", "poisson_id"])
def test_ggn_matvec_poisson(tc, loss):
    prob = positive_problem("p", "f64")
    p = build(prob)
    A = prob.factors if loss == "poisson_id" else [0.5 * a for a in prob.factors]
    rng = np.random.default_rng(12)
    x = [rng.standard_normal((I, prob.R)) for I in prob.dims]
    y = tc.ggn_matvec(p, dev_factors(prob, A), [to_dev(v, "f64") for v in x], loss, 0.1)
    yo = oracle.ggn_matvec(prob.dims, prob.idx, prob.t, A, loss, 0.1, x)
    for d in range(3):
        assert rel(host(y[d]), yo[d]) <= TOL["f64"]


# ------------------------------------------------------------------ preconditioner, PCG, GGN step
@pytest.mark.parametrize("name", ["f32_r16", "f64_r16", "f64_r5_200cube"])
def test_precond_apply(tc, name):
    prob = problem(name)
    p = build(prob)
    A = dev_factors(prob)
    cg = tc.CG(p, A, "ls", 0.05)
    cg.setup()
    rng = np.random.default_rng(13)
    r = [rng.standard_normal((I, prob.R)) for I in prob.dims]
    if prob.dtype == "f32":
        r = [v.astype(np.float32).astype(np.float64) for v in r]
    z = cg.precond_apply([to_dev(v, prob.dtype) for v in r])
    zo = oracle.precond_apply(prob.dims, prob.idx, prob.t, prob.factors, "ls", 0.05, r)
    for d in range(3):
        assert rel(host(z[d]), zo[d]) <= TOL[prob.dtype]


# After k CG iterations the iterate depends on every earlier rounding; the
# FP32 bound is the kernel tolerance times the iteration count.
CG_TOL = {"f32": 10 * TOL["f32"], "f64": 1e-10}


@pytest.mark.parametrize("name,precond", [("f64_r16", True), ("f64_r16", False),
                                          ("f32_r16", True), ("f64_r5_200cube", True)])
def test_cg_solve(tc, name, precond):
    import torch
    prob = problem(name)
    p = build(prob)
    A = dev_factors(prob)
    lam = 0.05
    _, g = oracle.loss_grad(prob.dims, prob.idx, prob.t, prob.factors, "ls", lam)
    b = [-v for v in g]
    if prob.dtype == "f32":
        b = [v.astype(np.float32).astype(np.float64) for v in b]
    cg = tc.CG(p, A, "ls", lam, precondition=precond)
    cg.setup()
    rz = torch.zeros(11, dtype=torch.float64, device="cuda")
    bd = [to_dev(v, prob.dtype) for v in b]
    dx = cg.solve(bd, 10, rz=rz)
    first = [host(v).copy() for v in dx]
    dx2 = cg.solve(bd, 10, dx=dx, rz=rz)        # replay of the captured graph
    xo = oracle.pcg(prob.dims, prob.idx, prob.t, prob.factors, "ls", lam, b, 10, precond)
    for d in range(3):
        assert rel(first[d], xo[d]) <= CG_TOL[prob.dtype]
        # FP64 atomics make the summation order (not the result) vary run to run
        assert rel(host(dx2[d]), first[d]) <= CG_TOL[prob.dtype]
    assert (rz.cpu().numpy() >= 0).all()
    assert tc.last_error(p) == tc.OK


@pytest.mark.parametrize("name", ["f32_r16", "f64_r16", "f32_r5", "f64_r5_200cube"])
def test_cg_matvec(tc, name):
    prob = problem(name)
    p = build(prob)
    cg = tc.CG(p, dev_factors(prob), "ls", 0.05)
    rng = np.random.default_rng(21)
    x = [rng.standard_normal((I, prob.R)) for I in prob.dims]
    if prob.dtype == "f32":
        x = [v.astype(np.float32).astype(np.float64) for v in x]
    y = cg.matvec([to_dev(v, prob.dtype) for v in x])
    yo = oracle.ggn_matvec(prob.dims, prob.idx, prob.t, prob.factors, "ls", 0.05, x)
    for d in range(3):
        assert rel(host(y[d]), yo[d]) <= TOL[prob.dtype]


@pytest.mark.parametrize("name,loss", [("f64_r16", "ls"), ("f32_r16", "ls")])
def test_ggn_step(tc, name, loss):
    import torch
    prob = problem(name)
    p = build(prob)
    A = dev_factors(prob)
    lam = 0.05
    cg = tc.CG(p, A, loss, lam)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    cg.ggn_step(10, loss_out=f)
    ref = oracle.ggn_step(prob.dims, prob.idx, prob.t, prob.factors, loss, lam, 10)
    fo = oracle.objective(prob.dims, prob.idx, prob.t, prob.factors, loss, lam)
    assert abs(f.item() - fo) <= TOL[prob.dtype] * abs(fo)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= CG_TOL[prob.dtype]
    # the step decreases the objective like the oracle's
    f_new = oracle.objective(prob.dims, prob.idx, prob.t, [host(a) for a in A], loss, lam)
    f_ref = oracle.objective(prob.dims, prob.idx, prob.t, ref, loss, lam)
    assert f_new < fo and abs(f_new - f_ref) <= 1e-4 * abs(fo)


@pytest.mark.parametrize("loss", ["poisson_log"])
def test_ggn_step_poisson(tc, loss):
    prob = positive_problem("p", "f64")
    p = build(prob)
    A0 = [0.5 * a for a in prob.factors]
    A = dev_factors(prob, A0)
    cg = tc.CG(p, A, loss, 0.1)
    cg.ggn_step(8)
    ref = oracle.ggn_step(prob.dims, prob.idx, prob.t, A0, loss, 0.1, 8)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= CG_TOL["f64"]


# ------------------------------------------------------------------ ALS sweep
@pytest.mark.parametrize("name", ["f64_r5_200cube", "f32_r16", "zipf_f32_r32"])
def test_als_sweep(tc, name):
    from paper_1910_02371_gb300 import drivers
    prob = problem(name)
    p = build(prob)
    A = dev_factors(prob)
    lam = 1e-3 if prob.dtype == "f64" else 0.5
    drivers.als_sweep(p, A, lam)
    ref = oracle.als_sweep(prob.dims, prob.idx, prob.t, prob.factors, lam)
    # a sweep chains three MTTKRP + Solve Factor pairs, each feeding the next
    tol = TOL[prob.dtype] * (1 if prob.dtype == "f64" else 3)
    for d in range(3):
        assert rel(host(A[d]), ref[d]) <= tol
    assert tc.last_error(p) == tc.OK


# ------------------------------------------------------------------ refill
def test_pattern_refill(tc):
    import torch
    a = problem("f32_r16")
    b = make_problem("refill_b", a.dims, a.nnz, a.R, "f32", seed=4242)
    p = tc.build_pattern(idx_dev(a.idx), a.dims, to_dev(a.t, "f32"), refillable=True)
    A = dev_factors(b)
    x_before = tc.tttp(p, A, weights="values").clone()
    tc.refill_pattern(p, idx_dev(b.idx), to_dev(b.t, "f32"))
    for d in range(3):
        row_ptr, perm, nz = p.view(d)
        operm, orow, onz = oracle.pattern(b.dims, b.idx, d)
        assert np.array_equal(perm.cpu().numpy(), operm)
        assert np.array_equal(row_ptr.cpu().numpy(), orow)
        assert np.array_equal(nz.cpu().numpy(), onz)
    perm0 = oracle.pattern(b.dims, b.idx, 0)[0]
    x = host(tc.tttp(p, A, weights="values"))
    assert rel(x, oracle.tttp(b.dims, b.idx, b.t, b.factors)[perm0]) <= TOL["f32"]
    assert not np.allclose(x, host(x_before))
    out = host(tc.mttkrp(p, A, 2))
    assert rel(out, oracle.mttkrp(b.dims, b.idx, b.t, b.factors, 2)) <= TOL["f32"]
    assert tc.last_error(p) == tc.OK
    # a pattern built without the flag cannot be refilled
    q = build(a)
    with pytest.raises(tc.TcError):
        tc.refill_pattern(q, idx_dev(b.idx), to_dev(b.t, "f32"))
    torch.cuda.synchronize()


def test_pattern_refill_range_error_is_recorded(tc):
    a = problem("f32_r5")
    p = tc.build_pattern(idx_dev(a.idx), a.dims, to_dev(a.t, "f32"), refillable=True)
    bad = [c.copy() for c in a.idx]
    bad[1][17] = a.dims[1] + 3          # one index past its mode
    tc.refill_pattern(p, idx_dev(bad), to_dev(a.t, "f32"))
    assert tc.last_error(p) == tc.ERR_RANGE
    tc.refill_pattern(p, idx_dev(a.idx), to_dev(a.t, "f32"))
    assert tc.last_error(p) == tc.OK


def test_refill_keeps_captured_cg_graph_valid(tc):
    import torch
    a = problem("f64_r16")
    b = make_problem("refill_cg", a.dims, a.nnz, a.R, "f64", seed=515)
    p = tc.build_pattern(idx_dev(a.idx), a.dims, to_dev(a.t, "f64"), dtype=torch.float64,
                         refillable=True)
    A = dev_factors(b)
    lam = 0.05
    cg = tc.CG(p, A, "ls", lam)
    _, g = oracle.loss_grad(b.dims, b.idx, b.t, b.factors, "ls", lam)
    bd = [to_dev(-v, "f64") for v in g]
    cg.setup()
    dx = cg.solve(bd, 6)                    # captured against the first tensor
    tc.refill_pattern(p, idx_dev(b.idx), to_dev(b.t, "f64"))
    cg.setup()
    dx = cg.solve(bd, 6, dx=dx)             # replayed against the refilled one
    xo = oracle.pcg(b.dims, b.idx, b.t, b.factors, "ls", lam, [-v for v in g], 6)
    for d in range(3):
        assert rel(host(dx[d]), xo[d]) <= CG_TOL["f64"]
