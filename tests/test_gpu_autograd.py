"""The autograd wrapper of the objective (eq. obj): its hand-written backward
(the fused gradient kernel, model entries recomputed) against FP64 central
differences of the oracle objective and against the oracle's analytic
gradient, at relative 1e-4, on a 1,000-nonzero tensor drawn with the Poisson
workload's recipe (dims 5e4 x 5e4 x 5e3, rank 32, Uniform(0,1) planted
factors, Poisson counts, lambda 0.1, evaluated at the planted factors times
Uniform(0.9, 1.1))."""
import numpy as np
import pytest

import oracle
import synth
from helpers import host, idx_dev, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import autograd, tc
    w = synth.WORKLOADS["cp3_50k_m50M_r32"]
    dims, R = w.dims, w.rank
    idx = synth.distinct_coords(dims, 1000, w.coord_dist, w.seed)
    planted = synth.factor_matrices(dims, R, w.factor_dist, w.seed)
    t = synth.observe(oracle.model_entries(dims, idx, planted), "poisson", w.seed)
    A = [a.astype(np.float32).astype(np.float64) for a in synth.perturb(planted, w.seed)]
    p = tc.build_pattern(idx_dev(idx), dims, to_dev(t, "f32"))
    return torch, autograd, tc, w, dims, idx, t, A, p


@pytest.mark.parametrize("loss,scale", [("poisson_log", 0.05), ("poisson_id", 1.0), ("ls", 1.0)])
def test_backward_matches_fd_and_oracle(setup, loss, scale):
    torch, autograd, tc, w, dims, idx, t, A, p = setup
    # the log link exponentiates the model: evaluate at smaller factors
    As = [a * scale for a in A]
    As = [a.astype(np.float32).astype(np.float64) for a in As]
    Ad = [to_dev(a, "f32").requires_grad_(True) for a in As]
    f = autograd.cp_completion_loss(p, Ad, loss, w.lam)
    f.backward()
    g = [host(a.grad) for a in Ad]
    fo, go = oracle.loss_grad(dims, idx, t, As, loss, w.lam)
    assert abs(f.item() - fo) <= 1e-5 * abs(fo)
    for d in range(3):
        assert rel(g[d], go[d]) <= 1e-4
    # central differences of the FP64 oracle objective on sampled entries
    rng = np.random.default_rng(3)
    fd, an = [], []
    for d in range(3):
        rows = np.unique(idx[d])                      # entries that the data touch
        for _ in range(12):
            i = int(rng.choice(rows))
            r = int(rng.integers(0, w.rank))
            h = 1e-4 * max(1.0, abs(As[d][i, r]))
            Ap = [a.copy() for a in As]
            Am = [a.copy() for a in As]
            Ap[d][i, r] += h
            Am[d][i, r] -= h
            fd.append((oracle.objective(dims, idx, t, Ap, loss, w.lam)
                       - oracle.objective(dims, idx, t, Am, loss, w.lam)) / (2 * h))
            an.append(g[d][i, r])
    assert rel(np.array(an), np.array(fd)) <= 1e-4


def test_chain_rule_scaling_and_descent(setup):
    torch, autograd, tc, w, dims, idx, t, A, p = setup
    Ad = [to_dev(a, "f32").requires_grad_(True) for a in A]
    f = autograd.cp_completion_loss(p, Ad, "poisson_id", w.lam)
    (3.0 * f).backward()
    g3 = [a.grad.clone() for a in Ad]
    for a in Ad:
        a.grad = None
    autograd.cp_completion_loss(p, Ad, "poisson_id", w.lam).backward()
    for a, b in zip(g3, Ad):
        torch.testing.assert_close(a, 3.0 * b.grad)
    # a small gradient step lowers the objective
    with torch.no_grad():
        step = [a - 1e-4 * a.grad for a in Ad]
    f1 = autograd.cp_completion_loss(p, step, "poisson_id", w.lam)
    assert f1.item() < f.item()
    assert tc.last_error(p) == tc.OK
