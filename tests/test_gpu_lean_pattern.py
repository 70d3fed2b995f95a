"""Lean patterns: no stored positions, and a build that borrows its sort work
space from the arrays of modes not yet built and, when allowed, from the
consumed input (the layout that lets a 4e9-nonzero tensor fit one GPU).

* The sorted copies (row offsets, nonempty rows, other-mode indices, values)
  equal the oracle's stable sort bit for bit, for modes sorted in zero, one,
  two (an even count: one extra identity pass brings the result back) and
  three digit passes, with and without values, FP32 and FP64.
* Every computation on a lean pattern matches the one on a full pattern of the
  same tensor (the kernels read the same sorted arrays; only the order of the
  atomic additions at chunk boundaries and in the FP64 sums may differ, so
  within 1e-6 / 1e-13 normwise for FP32 / FP64), and the oracle within the
  dtype tolerance.
* Calls that need the mode-0 maps report TC_ERR_UNSUPPORTED; invalid flag
  combinations TC_ERR_ARG."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, host, idx_dev, make_problem, rel, to_dev, torch_dtype

pytestmark = pytest.mark.gpu

CASES = {
    # dims < 256: one digit pass per mode
    "one_pass_f32": dict(dims=(200, 150, 250), nnz=30000, R=16, dtype="f32"),
    # 12-, 16- and 10-bit modes: two passes each (the consumed-input schedule
    # adds a third)
    "two_pass_f64": dict(dims=(3000, 40000, 700), nnz=50000, R=5, dtype="f64"),
    # 17 bits, 9 bits, 22 bits: three, two, three passes
    "three_pass_f32": dict(dims=(70000, 300, 1 << 22), nnz=60000, R=8, dtype="f32"),
    # a mode of dimension 1: no digit pass (plain copy)
    "dim1_f32": dict(dims=(1, 60, 5000), nnz=4000, R=4, dtype="f32"),
    "zipf_f32": dict(dims=(5000, 800, 90), nnz=40000, R=32, dtype="f32",
                     dist=("zipf", "zipf", "uniform")),
}

_cache = {}


def problem(name):
    if name not in _cache:
        c = dict(CASES[name])
        _cache[name] = make_problem(name, c.pop("dims"), c.pop("nnz"), c.pop("R"), c.pop("dtype"),
                                    seed=sum(map(ord, name)) + 7, **c)
    return _cache[name]


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


def lean_build(tc, prob, consume, with_vals=True):
    vals = to_dev(prob.t, prob.dtype) if with_vals else None
    return tc.build_pattern(idx_dev(prob.idx), prob.dims, vals, dtype=torch_dtype(prob.dtype),
                            lean=True, consume_input=consume)


@pytest.mark.parametrize("consume", [False, True])
@pytest.mark.parametrize("name", list(CASES))
def test_lean_sorted_copies_bit_exact(tc, name, consume):
    prob = problem(name)
    for with_vals in ((True, False) if name == "two_pass_f64" else (True,)):
        p = lean_build(tc, prob, consume, with_vals)
        vdt = np.float32 if prob.dtype == "f32" else np.float64
        for d in range(3):
            o1, o2 = [m for m in range(3) if m != d]
            row_ptr, perm, nz = p.view(d)
            assert perm is None
            operm, orow, onz = oracle.pattern(prob.dims, prob.idx, d)
            assert np.array_equal(row_ptr.cpu().numpy(), orow), (name, d)
            assert np.array_equal(nz.cpu().numpy(), onz), (name, d)
            c1, c2, v = p.columns(d)
            assert np.array_equal(c1.cpu().numpy(), prob.idx[o1][operm]), (name, d)
            assert np.array_equal(c2.cpu().numpy(), prob.idx[o2][operm]), (name, d)
            if with_vals:
                assert np.array_equal(v.cpu().numpy(), prob.t.astype(vdt)[operm]), (name, d)
            else:
                assert v is None
        assert tc.last_error(p) == tc.OK


@pytest.mark.parametrize("consume", [False, True])
@pytest.mark.parametrize("name", ["one_pass_f32", "two_pass_f64", "zipf_f32"])
def test_lean_computations_equal_full(tc, name, consume):
    prob = problem(name)
    full = tc.build_pattern(idx_dev(prob.idx), prob.dims, to_dev(prob.t, prob.dtype),
                            dtype=torch_dtype(prob.dtype))
    lean = lean_build(tc, prob, consume)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    rng = np.random.default_rng(5)
    x = [to_dev(rng.standard_normal(a.shape), prob.dtype) for a in prob.factors]
    tol = TOL[prob.dtype]
    spread = 1e-6 if prob.dtype == "f32" else 1e-13

    def same(a, b, bound=spread):
        assert rel(host(b), host(a)) <= bound

    same(tc.tttp(full, A, weights="values"), tc.tttp(lean, A, weights="values"))
    for d in range(3):
        m_full = tc.mttkrp(full, A, d)
        same(m_full, tc.mttkrp(lean, A, d))
        assert rel(host(m_full), oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, d)) <= tol
        for prec in (("fp32", "fp32_refine") if prob.dtype == "f32" else ("fp32",)):
            same(tc.solve_factor(full, A, d, m_full, 0.1, prec=prec),
                 tc.solve_factor(lean, A, d, m_full, 0.1, prec=prec))
    for loss in ("ls", "poisson_log"):
        f1, g1 = tc.loss_grad(full, A, loss, 0.05)
        f2, g2 = tc.loss_grad(lean, A, loss, 0.05)
        same(f1, f2)
        for a, b in zip(g1, g2):
            same(a, b)
        for a, b in zip(tc.ggn_matvec(full, A, x, loss, 0.05), tc.ggn_matvec(lean, A, x, loss, 0.05)):
            same(a, b)
    # a Gauss-Newton step (CG graph, preconditioner) on each: CG carries the
    # atomic-order differences of its products through its iterations (the
    # Zipf case's ill-conditioned rows amplify them to a few 1e-6 in FP32)
    B1 = [a.clone() for a in A]
    B2 = [a.clone() for a in A]
    tc.CG(full, B1, "ls", 0.05).ggn_step(4)
    tc.CG(lean, B2, "ls", 0.05).ggn_step(4)
    for a, b in zip(B1, B2):
        same(a, b, 1e-4 if prob.dtype == "f32" else 1e-10)
    assert tc.last_error(full) == tc.OK and tc.last_error(lean) == tc.OK


def test_lean_rejects_what_needs_positions(tc):
    prob = problem("one_pass_f32")
    p = lean_build(tc, prob, False)
    A = [to_dev(a, prob.dtype) for a in prob.factors]
    w = torch.ones(prob.nnz, device="cuda", dtype=torch.float32)
    # mode 0 needs no map; modes 1 and 2 do
    tc.mttkrp(p, A, 0, weights=w)
    for d in (1, 2):
        with pytest.raises(tc.TcError) as e:
            tc.mttkrp(p, A, d, weights=w)
        assert e.value.status == tc.ERR_UNSUPPORTED
    rhs = torch.zeros_like(A[1])
    with pytest.raises(tc.TcError) as e:
        tc.solve_factor(p, A, 1, rhs, 0.1, weights=w)
    assert e.value.status == tc.ERR_UNSUPPORTED
    with pytest.raises(tc.TcError) as e:
        tc.ccd_sweep(p, [a.clone() for a in A], 0.1)
    assert e.value.status == tc.ERR_UNSUPPORTED
    assert tc.last_error(p) == tc.OK


def test_lean_flag_combinations(tc):
    prob = problem("dim1_f32")
    dt = torch_dtype(prob.dtype)
    for kw in (dict(consume_input=True), dict(lean=True, refillable=True),
               dict(lean=True, check_duplicates=True)):
        with pytest.raises(tc.TcError) as e:
            tc.build_pattern(idx_dev(prob.idx), prob.dims, to_dev(prob.t, prob.dtype), dtype=dt, **kw)
        assert e.value.status == tc.ERR_ARG, kw
    # empty tensor
    e0 = [torch.zeros(0, dtype=torch.int32, device="cuda") for _ in range(3)]
    p = tc.build_pattern(e0, (4, 5, 6), torch.zeros(0, device="cuda"), lean=True, consume_input=True)
    row_ptr, perm, nz = p.view(2)
    assert perm is None and row_ptr.cpu().tolist() == [0] * 7 and nz.numel() == 0
