"""The row-sharded driver with the libtc kernels on one GPU, as one process
(no process group): its ALS sweep must equal drivers.als_sweep bit for bit
(the same kernels on the same sorted blocks), its objective the library's,
and its Gauss-Newton step -- PCG run on the host with tc_axpby / tc_dot and
the per-mode preconditioners -- the solver's own tc_ggn_step and the FP64
oracle's step within the FP32 tolerance of the composite path.  The
multi-process exchange itself is tested on the CPU (test_sharded_gloo.py)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import host, idx_dev, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    return t


def test_sharded_one_process_matches_library(tc):
    from paper_1910_02371_gb300 import drivers
    from paper_1910_02371_gb300.sharded import LibtcOps, ShardedCP
    prob = make_problem("sharded", (300, 250, 200), 60_000, 16, "f32", 4242,
                        dist=("zipf", "uniform", "uniform"))
    lam = 0.05
    idx = idx_dev(prob.idx)
    t = to_dev(prob.t, "f32")
    sh = ShardedCP(LibtcOps(), idx, t, prob.dims, "ls", lam)
    assert sh.world == 1 and all(sh.ranges[d] == [(0, prob.dims[d])] for d in range(3))
    p = tc.build_pattern(idx, prob.dims, t)
    A0 = [to_dev(a, "f32") for a in prob.factors]

    A = [a.clone() for a in A0]
    B = [a.clone() for a in A0]
    f_sh = sh.objective(A)
    f_tc, _ = tc.loss_grad(p, B, "ls", lam, want_grad=False)
    # (FP64 sums whose partial-sum order is not fixed)
    assert f_sh == pytest.approx(f_tc.item(), rel=1e-12)
    sh.als_sweep(A)
    drivers.als_sweep(p, B, lam)
    for d in range(3):
        # the same kernels; only the order of the chunk-boundary atomics differs
        assert rel(host(A[d]), host(B[d])) <= 1e-6, d

    # Gauss-Newton step from the swept factors: host-driven sharded PCG vs
    # the graph-captured solver, and vs the oracle
    start = [host(a) for a in A]
    hist = sh.ggn_step(A, 10)
    assert len(hist) == 11 and all(np.isfinite(hist))
    cg = tc.CG(p, B, "ls", lam)
    cg.ggn_step(10)
    ref = oracle.ggn_step(prob.dims, prob.idx, prob.t, start, "ls", lam, 10)
    for d in range(3):
        assert rel(host(A[d]), host(B[d])) <= 1e-4, d
        assert rel(host(A[d]), ref[d]) <= 1e-4, d
    assert tc.last_error(p) == tc.OK


def test_vector_steps(tc):
    rng = np.random.default_rng(9)
    for dt, tol in ((torch.float32, 1e-6), (torch.float64, 1e-14)):
        x = torch.as_tensor(rng.standard_normal(100_003), dtype=dt, device="cuda")
        y = torch.as_tensor(rng.standard_normal(100_003), dtype=dt, device="cuda")
        xd, yd = x.double().cpu().numpy(), y.double().cpu().numpy()
        d = tc.dot(x, y)
        assert d.item() == pytest.approx(float(np.dot(xd, yd)), rel=tol, abs=tol)
        tc.dot(x, x, out=d, accumulate=True)
        assert d.item() == pytest.approx(float(np.dot(xd, yd) + np.dot(xd, xd)), rel=tol)
        tc.axpby(0.5, x, -2.0, y)
        assert np.allclose(y.double().cpu().numpy(), 0.5 * xd - 2.0 * yd, rtol=tol, atol=tol)
        e = torch.empty(0, dtype=dt, device="cuda")
        assert tc.dot(e, e).item() == 0.0
