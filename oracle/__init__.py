"""FP64 CPU oracle for sparse CP tensor completion (arXiv:1910.02371).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path never does.  It shares no code with the CUDA
library.

The arithmetic lives in ``oracle.c`` (plain loops in double precision, see
``oracle.h``); this module only marshals numpy arrays and composes those
routines the way the paper composes its kernels:

* ALS sweep (Sec. 2.2; Sec. 4, "ALS solve for one factor matrix"): for each
  mode in turn, the right-hand side is the MTTKRP of the observed values, then
  Solve Factor with the pattern (unit weights) and lambda; the new factor is
  used at once (block Gauss-Seidel, Appendix A).
* General-loss ALS (Sec. 2.2, last paragraph; tolerances of Sec. 5.7): for each
  mode in turn, Newton steps on that factor with the others fixed -- gradient
  MTTKRP(phi') + 2 lambda A, the row Hessians sum phi'' h h^T + 2 lambda I
  solved through Solve Factor with weights phi'' -- until the step is small
  relative to the factor or an iteration cap is reached.
* Coordinate minimization, CCD++ order (Sec. 2.3): for each rank component r,
  the residual rho^(r) = t - m + u_r v_r w_r, then column r of each factor in
  turn set to MTTKRP(rho^(r)) / (lambda + sum of squared products), the
  residual updated in between.
* Coordinate minimization for a general loss (Sec. 2.3, last paragraph; the
  inner tolerances of Sec. 5.7): in the same order, Newton steps on each
  column with the rest fixed; the column's elements are decoupled, so a step
  is the gradient over the diagonal second derivative, element by element.
* Gauss-Newton step (Sec. 2.5): gradient, block-diagonal preconditioner (the
  diagonal blocks of the Gauss-Newton matrix, applied through Solve Factor with
  weights phi'' and regularization 2 lambda), preconditioned CG from zero for a
  fixed number of iterations, then the update.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

LOSSES = {"ls": 0, "poisson_log": 1, "poisson_id": 2}

OK, ERR_ARG, ERR_RANGE, ERR_NOT_SPD, ERR_DOMAIN = 0, 1, 2, 6, 7


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"oracle {what} returned {rc}")
        self.rc = rc


_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}
_parallel = False


def _compile(out, extra):
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(src),
                                                               os.path.getmtime(hdr)):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", *extra, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain, the parity checker) and
    liboracle_omp.so (the same loops split by OpenMP, the timed CPU baseline)
    with the host gcc."""
    if force:
        for f in (_SO, _SO_OMP):
            if os.path.exists(f):
                os.remove(f)
    _compile(_SO_OMP, ["-fopenmp"])
    return _compile(_SO, [])


def set_parallel(on: bool, threads: int = 0) -> int:
    """Route every oracle call through the OpenMP build (bit-identical results)
    or back through the plain one; returns the thread count in use."""
    global _parallel
    _parallel = bool(on)
    L = lib()
    if _parallel and threads > 0:
        L.orc_threads(int(threads))
    return int(L.orc_threads(0))


def lib():
    key = "omp" if _parallel else "plain"
    if key not in _libs:
        build()
        L = ctypes.CDLL(_SO_OMP if _parallel else _SO)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        for name, args in {
            "orc_threads": [ctypes.c_int],
            "orc_counting_sort": [i64, P, i64, P, P],
            "orc_tttp": [ctypes.c_int, P, i64, P, P, ctypes.c_int, P, P],
            "orc_mttkrp": [ctypes.c_int, P, i64, P, P, ctypes.c_int, P, ctypes.c_int, P],
            "orc_solve_factor": [ctypes.c_int, P, i64, P, P, ctypes.c_int, P, ctypes.c_int,
                                 P, ctypes.c_double, P, P],
            "orc_loss_terms": [ctypes.c_int, i64, P, P, P, P, P],
            "orc_loss_grad": [ctypes.c_int, P, i64, P, P, ctypes.c_int, P, ctypes.c_int,
                              ctypes.c_double, P, P],
            "orc_ggn_matvec": [ctypes.c_int, P, i64, P, P, ctypes.c_int, P, ctypes.c_int,
                               ctypes.c_double, P, P],
        }.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _libs[key] = L
    return _libs[key]


# ---------------------------------------------------------------- marshalling
def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Ptrs:
    """A C array of pointers plus the arrays it keeps alive.  The object must
    outlive the C call that reads `ptr` (hold it in a local variable): the
    arrays it keeps may be converted copies that die with it."""

    def __init__(self, arrays):
        self.keep = list(arrays)
        self.arr = (ctypes.c_void_p * max(1, len(self.keep)))(
            *[None if a is None else a.ctypes.data for a in self.keep])

    @property
    def ptr(self):
        return ctypes.cast(self.arr, ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray(dims, dtype=np.int64)


def _idx(idx):
    return _Ptrs([np.ascontiguousarray(c, dtype=np.int32) for c in idx])


def _check(rc, what, allow=()):
    if rc != OK and rc not in allow:
        raise OracleError(rc, what)
    return rc


# ---------------------------------------------------------------- kernels
def counting_sort(key, I):
    """Stable counting sort by key (Sec. 3.4): (perm, row_ptr)."""
    key = np.ascontiguousarray(key, dtype=np.int32)
    m = key.shape[0]
    perm = np.zeros(max(m, 1), np.int64)
    row_ptr = np.zeros(int(I) + 1, np.int64)
    _check(lib().orc_counting_sort(m, _p(key), int(I), _p(perm), _p(row_ptr)), "counting_sort")
    return perm[:m], row_ptr


def pattern(dims, idx, mode):
    """The mode-`mode` view of the pattern: perm, row_ptr, nonempty rows."""
    perm, row_ptr = counting_sort(idx[mode], dims[mode])
    nonempty = np.nonzero(np.diff(row_ptr) > 0)[0].astype(np.int32)
    return perm, row_ptr, nonempty


def tttp(dims, idx, s, factors):
    """Sec. 3.3: x_e = s_e sum_r prod_{provided n} A^(n)[i_n(e), r]."""
    N = len(dims)
    m = len(idx[0])
    R = next((a.shape[1] for a in factors if a is not None), 1)
    fs = [None if a is None else _f64(a) for a in factors]
    x = np.zeros(max(m, 1))
    ix = _idx(idx)
    sp = None if s is None else _f64(s)
    fp = _Ptrs(fs)
    _check(lib().orc_tttp(N, _p(_dims(dims)), m, ix.ptr, _p(sp), R, fp.ptr, _p(x)), "tttp")
    return x[:m]


def mttkrp(dims, idx, s, factors, mode):
    """Sec. 3.2: pattern-restricted MTTKRP into mode `mode`."""
    N = len(dims)
    m = len(idx[0])
    R = next(a.shape[1] for i, a in enumerate(factors) if a is not None and i != mode)
    fs = [None if a is None else _f64(a) for a in factors]
    out = np.zeros((int(dims[mode]), R))
    sp = None if s is None else _f64(s)
    ix, fp = _idx(idx), _Ptrs(fs)
    _check(lib().orc_mttkrp(N, _p(_dims(dims)), m, ix.ptr, _p(sp), R, fp.ptr, mode, _p(out)),
           "mttkrp")
    return out


def solve_factor(dims, idx, s, factors, mode, rhs, lam, out=None):
    """Sec. 3.4: per-row (G_i + lam I) a_i = rhs_i.  Returns (out, status, rc).
    Rows whose system is not positive definite keep the contents of `out`."""
    N = len(dims)
    m = len(idx[0])
    rhs = _f64(rhs)
    R = rhs.shape[1]
    fs = [None if a is None else _f64(a) for a in factors]
    out = np.zeros_like(rhs) if out is None else _f64(out).copy()
    status = np.zeros(int(dims[mode]), np.int8)
    sp = None if s is None else _f64(s)
    ix, fp = _idx(idx), _Ptrs(fs)
    rc = lib().orc_solve_factor(N, _p(_dims(dims)), m, ix.ptr, _p(sp), R, fp.ptr,
                                mode, _p(rhs), float(lam), _p(out), _p(status))
    _check(rc, "solve_factor", allow=(ERR_NOT_SPD,))
    return out, status, rc


def loss_terms(loss, t, model):
    """phi, phi', phi'' (Sec. 2.1, Table 1, Sec. 5.7)."""
    t = _f64(t)
    model = _f64(model)
    m = t.shape[0]
    phi, d1, d2 = (np.zeros(max(m, 1)) for _ in range(3))
    _check(lib().orc_loss_terms(LOSSES[loss], m, _p(t), _p(model), _p(phi), _p(d1), _p(d2)),
           "loss_terms")
    return phi[:m], d1[:m], d2[:m]


def loss_grad(dims, idx, t, factors, loss, lam, want_grad=True):
    """eq. obj and Table 1: (f, [grad^(d)])."""
    N = len(dims)
    m = len(idx[0])
    R = factors[0].shape[1]
    fs = [_f64(a) for a in factors]
    f = np.zeros(1)
    grads = [np.zeros((int(I), R)) for I in dims] if want_grad else None
    gh = _Ptrs(grads) if want_grad else None
    ix, fp = _idx(idx), _Ptrs(fs)
    _check(lib().orc_loss_grad(N, _p(_dims(dims)), m, ix.ptr, _p(_f64(t)), R, fp.ptr,
                               LOSSES[loss], float(lam), _p(f), gh.ptr if gh else None),
           "loss_grad")
    return float(f[0]), grads


def ggn_matvec(dims, idx, t, factors, loss, lam, x):
    """Sec. 2.5: y = (J^T diag(phi'') J + 2 lam I) x, block per mode."""
    N = len(dims)
    m = len(idx[0])
    R = factors[0].shape[1]
    fs = [_f64(a) for a in factors]
    xs = [_f64(a) for a in x]
    ys = [np.zeros((int(I), R)) for I in dims]
    ix, fp, xp, yp = _idx(idx), _Ptrs(fs), _Ptrs(xs), _Ptrs(ys)
    _check(lib().orc_ggn_matvec(N, _p(_dims(dims)), m, ix.ptr, _p(_f64(t)), R, fp.ptr,
                                LOSSES[loss], float(lam), xp.ptr, yp.ptr), "ggn_matvec")
    return ys


# ---------------------------------------------------------------- compositions
def model_entries(dims, idx, factors):
    """m_e = <u_i, v_j, w_k> at the observed coordinates (eq. 2), via TTTP."""
    return tttp(dims, idx, None, factors)


def als_sweep(dims, idx, t, factors, lam):
    """One ALS sweep for least squares (Sec. 2.2; Sec. 4 listing for one factor):
    rhs = MTTKRP(T, d); A^(d) = Solve_Factor(Omega, d, rhs, lam), modes in order."""
    A = [_f64(a).copy() for a in factors]
    for d in range(len(dims)):
        rhs = mttkrp(dims, idx, t, A, d)
        A[d], _, rc = solve_factor(dims, idx, None, A, d, rhs, lam, out=A[d])
        if rc != OK:
            raise OracleError(rc, "als_sweep")
    return A


def precond_apply(dims, idx, t, factors, loss, lam, r):
    """Block-diagonal preconditioner of the Gauss-Newton matrix (Sec. 2.5):
    per mode d and row k, (sum phi'' h h^T + 2 lam I)^-1 r^(d)_k -- Solve Factor
    with weights phi'' and regularization 2 lam."""
    model = model_entries(dims, idx, factors)
    _, _, d2 = loss_terms(loss, t, model)
    out = []
    for d in range(len(dims)):
        z, _, rc = solve_factor(dims, idx, d2, factors, d, r[d], 2.0 * lam)
        if rc != OK:
            raise OracleError(rc, "precond_apply")
        out.append(z)
    return out


def _dot(a, b):
    return float(sum(np.vdot(x.ravel(), y.ravel()) for x, y in zip(a, b)))


def pcg(dims, idx, t, factors, loss, lam, b, n_iter, precondition=True):
    """Preconditioned CG on the Gauss-Newton system from x0 = 0 for a fixed
    number of iterations (Hestenes-Stiefel recurrences)."""
    x = [np.zeros_like(_f64(v)) for v in b]
    r = [_f64(v).copy() for v in b]
    z = precond_apply(dims, idx, t, factors, loss, lam, r) if precondition else [v.copy() for v in r]
    p = [v.copy() for v in z]
    rz = _dot(r, z)
    for _ in range(n_iter):
        Ap = ggn_matvec(dims, idx, t, factors, loss, lam, p)
        alpha = rz / _dot(p, Ap)
        x = [xi + alpha * pi for xi, pi in zip(x, p)]
        r = [ri - alpha * api for ri, api in zip(r, Ap)]
        z = precond_apply(dims, idx, t, factors, loss, lam, r) if precondition else [v.copy() for v in r]
        rz_new = _dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = [zi + beta * pi for zi, pi in zip(z, p)]
    return x


def ggn_step(dims, idx, t, factors, loss, lam, n_iter, precondition=True):
    """One Gauss-Newton step (Sec. 2.5): solve H dx = -grad by PCG, A += dx."""
    _, g = loss_grad(dims, idx, t, factors, loss, lam)
    dx = pcg(dims, idx, t, factors, loss, lam, [-v for v in g], n_iter, precondition)
    return [_f64(a) + d for a, d in zip(factors, dx)]


def objective(dims, idx, t, factors, loss, lam):
    return loss_grad(dims, idx, t, factors, loss, lam, want_grad=False)[0]


def newton_matvec(dims, idx, t, factors, loss, lam, x):
    """Full Newton Hessian-vector product (Sec. 2.5 before the Gauss-Newton
    approximation; Appendix A): the Gauss-Newton product plus the phi' term.
    The second derivative of m_e with respect to rows of two different modes p,
    q is delta_rs prod_{n != p, q} a^(n) (zero within one mode), so the block of
    output mode d is, for each other mode p, MTTKRP(phi', d) of the factors with
    A^(p) replaced by x^(p)."""
    y = ggn_matvec(dims, idx, t, factors, loss, lam, x)
    d1, _ = loss_derivs(dims, idx, t, factors, loss)
    N = len(dims)
    for d in range(N):
        for q in range(N):
            if q == d:
                continue
            F = [_f64(a) for a in factors]
            F[q] = _f64(x[q])
            y[d] = y[d] + mttkrp(dims, idx, d1, F, d)
    return y


def loss_derivs(dims, idx, t, factors, loss):
    """phi' and phi'' at every observed entry (input order), at the model
    entries of `factors` (Table 1 notation, Sec. 2.1 / 5.7 losses)."""
    _, d1, d2 = loss_terms(loss, t, model_entries(dims, idx, factors))
    return d1, d2


def newton_als_mode(dims, idx, t, factors, mode, loss, lam, inner_iters=5, tol=1e-3):
    """Newton iterations on factor `mode` with the others fixed (Sec. 2.2: the
    per-row Newton step for a general loss, gradient and Hessian of Table 1):
      g = MTTKRP(phi', mode) + 2 lam A,   H_i = sum_e phi''_e h_e h_e^T + 2 lam I,
      A <- A - H^-1 g   (row by row, through Solve Factor with weights phi''),
    stopping when ||step||_F <= tol ||A||_F (a reading: one test for the whole
    factor) or after inner_iters steps.  Returns (factors, steps taken)."""
    A = [_f64(a).copy() for a in factors]
    taken = 0
    for _ in range(inner_iters):
        d1, d2 = loss_derivs(dims, idx, t, A, loss)
        g = mttkrp(dims, idx, d1, A, mode) + 2.0 * lam * A[mode]
        step, _, rc = solve_factor(dims, idx, d2, A, mode, -g, 2.0 * lam)
        if rc != OK:
            raise OracleError(rc, "newton_als_mode")
        A[mode] = A[mode] + step
        taken += 1
        if np.linalg.norm(step) <= tol * np.linalg.norm(A[mode]):
            break
    return A, taken


def newton_als_sweep(dims, idx, t, factors, loss, lam, inner_iters=5, tol=1e-3):
    """One general-loss ALS sweep: newton_als_mode for modes 0, 1, 2 in order."""
    A = [_f64(a).copy() for a in factors]
    for d in range(len(dims)):
        A, _ = newton_als_mode(dims, idx, t, A, d, loss, lam, inner_iters, tol)
    return A


def ccd_sweep(dims, idx, t, factors, lam):
    """One CCD++ sweep for least squares (Sec. 2.3): for r = 0 .. R-1, add the
    rank-r term back into the residual, update column r of each factor in turn
    (u_ir = sum_e v_jr w_kr rho_e / (lambda + sum_e v_jr^2 w_kr^2), the other
    columns fixed, the previously updated ones used at once), then subtract the
    updated rank-r term."""
    A = [_f64(a).copy() for a in factors]
    N = len(dims)
    R = A[0].shape[1]
    rho = _f64(t) - model_entries(dims, idx, A)
    for r in range(R):
        col = lambda n: A[n][:, r:r + 1].copy()
        rho = rho + tttp(dims, idx, None, [col(n) for n in range(N)])
        for d in range(N):
            cols = [col(n) for n in range(N)]
            num = mttkrp(dims, idx, rho, cols, d)[:, 0]
            den = lam + mttkrp(dims, idx, None, [c * c for c in cols], d)[:, 0]
            A[d][:, r] = num / den
        rho = rho - tttp(dims, idx, None, [col(n) for n in range(N)])
    return A


def ccd_newton_sweep(dims, idx, t, factors, loss, lam, inner_iters=5, tol=1e-3):
    """Coordinate minimization for a general loss (Sec. 2.3, last paragraph),
    CCD++ order: for r = 0 .. R-1 and each mode d in turn, Newton steps on
    column r of A^(d) with everything else fixed.  Each nonzero involves one
    row of A^(d), so the column's elements are decoupled and one step is, per
    row i (Table 1 scaling: f = sum phi + lam sum ||A||^2),
      delta_i = -(sum_e phi'_e h_e + 2 lam u_ir) / (sum_e phi''_e h_e^2 + 2 lam),
      h_e = prod_{n != d} A^(n)[i_n(e), r],
    with phi', phi'' at the current model entries.  A column stops after
    inner_iters steps or once ||delta||_2 <= tol ||column||_2 (after the step;
    one test per column, the reading used for general-loss ALS).  For least
    squares one step is the CCD++ update.  Returns (factors, steps), steps[r, d]
    the Newton steps taken on that column."""
    A = [_f64(a).copy() for a in factors]
    N = len(dims)
    R = A[0].shape[1]
    steps = np.zeros((R, N), dtype=np.int64)
    for r in range(R):
        for d in range(N):
            for _ in range(inner_iters):
                d1, d2 = loss_derivs(dims, idx, t, A, loss)
                cols = [A[n][:, r:r + 1].copy() for n in range(N)]
                g = mttkrp(dims, idx, d1, cols, d)[:, 0] + 2.0 * lam * A[d][:, r]
                h = mttkrp(dims, idx, d2, [c * c for c in cols], d)[:, 0] + 2.0 * lam
                if not np.all(h > 0.0):
                    raise OracleError(ERR_NOT_SPD, "ccd_newton_sweep")
                delta = -g / h
                A[d][:, r] = A[d][:, r] + delta
                steps[r, d] += 1
                if np.linalg.norm(delta) <= tol * np.linalg.norm(A[d][:, r]):
                    break
    return A, steps
