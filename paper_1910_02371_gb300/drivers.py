"""Algorithms composed from the C-ABI calls (Sec. 2 and Sec. 4 of the paper).

* ``als_sweep`` -- alternating least squares (Sec. 2.2): for each mode, the
  right-hand sides are the MTTKRP of the observed tensor, then Solve Factor
  with the pattern and lambda overwrites that factor (block Gauss-Seidel order).
* ``newton_als_sweep`` -- ALS for a general loss (Sec. 2.2): Newton steps on
  each factor in turn with weights phi'' in Solve Factor.
* ``GaussNewton`` -- the generalized Gauss-Newton method with implicit
  preconditioned CG (Sec. 2.5), one ``tc_ggn_step`` per call.
Every arithmetic step runs in libtc kernels; this module only orders calls.
"""
from __future__ import annotations

from . import tc


def als_sweep(p: "tc.Pattern", factors, lam: float, rhs=None, row_status=None, prec="fp32",
              stream=None, fused=True):
    """One ALS sweep in place over modes 0, 1, 2; prec: the Solve Factor
    precision form (tc.PRECS).  fused: each mode in one tc_als_update (the
    right-hand side formed in the Gram pass); otherwise tc_mttkrp into rhs[d]
    (optional work buffers) and tc_solve_factor."""
    for d in range(len(factors)):
        rs = None if row_status is None else row_status[d]
        if fused:
            tc.als_update(p, factors, d, lam, out=factors[d], row_status=rs, prec=prec,
                          stream=stream)
            continue
        b = tc.mttkrp(p, factors, d, weights="values", out=None if rhs is None else rhs[d],
                      stream=stream)
        tc.solve_factor(p, factors, d, b, lam, weights=None, out=factors[d], row_status=rs,
                        prec=prec, stream=stream)
    return factors


def newton_als_sweep(p: "tc.Pattern", factors, loss: str, lam: float, inner_iters: int = 5,
                     tol: float = 1e-3, prec: str = "fp32", stream=None):
    """One general-loss ALS sweep in place (Sec. 2.2): Newton steps on each
    factor in turn (tc_newton_als_mode).  Returns the steps taken per mode."""
    return [tc.newton_als_mode(p, factors, d, loss, lam, inner_iters, tol, prec, stream)
            for d in range(len(factors))]


class GaussNewton:
    """Generalized Gauss-Newton steps for a loss in {"ls", "poisson_log",
    "poisson_id"}; the factors are updated in place."""

    def __init__(self, p: "tc.Pattern", factors, loss: str, lam: float, precondition=True):
        self.cg = tc.CG(p, factors, loss, lam, precondition)

    def step(self, cg_iters: int, loss_out=None, stream=None):
        self.cg.ggn_step(cg_iters, loss_out=loss_out, stream=stream)
