"""The Solve Factor autotuner on real patterns: it must pick one of its
candidates, install it, leave results unchanged (within the dtype's
tolerance of the FP64 oracle), and restore nothing else."""
import numpy as np
import pytest

import oracle
from helpers import TOL, build, host, make_problem, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    from paper_1910_02371_gb300 import build as b
    b.build()
    from paper_1910_02371_gb300 import tc as t
    yield t
    t.set_solve_tuning(torch.float32, 0, reset=True)


@pytest.mark.parametrize("R,dims,nnz", [(16, (3000, 400, 60), 60000), (32, (800, 300, 90), 40000),
                                        (64, (500, 200, 40), 30000)])
def test_autotune_picks_a_candidate_and_keeps_results(tc, R, dims, nnz):
    import torch
    from paper_1910_02371_gb300 import tuning
    prob = make_problem("tune%d" % R, dims, nnz, R, "f32", seed=R + 5, dist=("zipf", "zipf", "uniform"))
    p = build(prob)
    A = [to_dev(a, "f32") for a in prob.factors]
    tc.set_solve_tuning(torch.float32, 0, reset=True)
    rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, 0).astype(np.float32).astype(np.float64)
    key, rec = tuning.autotune(p, A, 0, to_dev(rhs, "f32"), 0.5)
    assert rec["chunk_nnz"] in (0, 256, 1024, 4096, 16384)
    rpws = (8, 16, 32) if R <= 16 else (4, 8, 16) if R <= 32 else (0,)
    assert rec["chol_rows_per_warp"] in rpws and rec["ms"] > 0
    assert rec["gram_kernel"] == 0
    assert tc.get_solve_tuning(torch.float32, R) == (rec["chunk_nnz"], rec["batch_bytes"],
                                                     rec["chol_rows_per_warp"], rec["gram_kernel"])
    out = host(tc.solve_factor(p, A, 0, to_dev(rhs, "f32"), 0.5))
    ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, 0, rhs, 0.5)
    assert rc == 0 and rel(out, ref) <= TOL["f32"]
    assert tc.last_error(p) == tc.OK


def test_autotune_times_both_gram_engines(tc):
    """At R = 64 with a tensor-core form the autotuner also chooses between the
    two Gram engines; the winner is installed and the refined solve stays
    within the form's error of the FP64 oracle."""
    import torch
    from paper_1910_02371_gb300 import tuning
    prob = make_problem("tune64e", (500, 200, 40), 30000, 64, "f32", seed=71,
                        dist=("zipf", "zipf", "uniform"))
    p = build(prob)
    A = [to_dev(a, "f32") for a in prob.factors]
    tc.set_solve_tuning(torch.float32, 0, reset=True)
    rhs = oracle.mttkrp(prob.dims, prob.idx, prob.t, prob.factors, 0).astype(np.float32).astype(np.float64)
    key, rec = tuning.autotune(p, A, 0, to_dev(rhs, "f32"), 0.5, prec="tf32_refine")
    assert rec["gram_kernel"] in (tc.GRAM_WARP_MMA, tc.GRAM_TCGEN05) and rec["ms"] > 0
    assert tc.get_solve_tuning(torch.float32, 64)[3] == rec["gram_kernel"]
    out = host(tc.solve_factor(p, A, 0, to_dev(rhs, "f32"), 0.5, prec="tf32_refine"))
    ref, _, rc = oracle.solve_factor(prob.dims, prob.idx, None, prob.factors, 0, rhs, 0.5)
    assert rc == 0 and rel(out, ref) <= 2e-5
    assert tc.last_error(p) == tc.OK
