"""Thin Python binding of libtc (include/tc.h): argument marshalling only.

Every function here converts torch CUDA tensors to device pointers, passes the
current CUDA stream, calls the C entry point of the same name and raises
``TcError`` on a non-OK status.  There is no fallback: if ``libtc.so`` is not
built the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

OK, ERR_ARG, ERR_RANGE, ERR_DUPLICATE, ERR_OOM, ERR_CUDA, ERR_NOT_SPD, ERR_DOMAIN, \
    ERR_BREAKDOWN, ERR_UNSUPPORTED, ERR_TIMEOUT = range(11)
F32, F64 = 0, 1
LOSSES = {"ls": 0, "poisson_log": 1, "poisson_id": 2}
W_ONE, W_VALUES, W_ARRAY = 0, 1, 2
PRECS = {"fp32": 0, "tf32_refine": 1, "bf16_refine": 2, "fp32_refine": 3}
CHOL32 = 0x100
REFINE2 = 0x200
# the refined forms with two refinement steps, and with an FP32 factorization
PRECS.update({k + "2": v | REFINE2 for k, v in list(PRECS.items()) if k.endswith("_refine")})
PRECS.update({k + "_chol32": v | CHOL32 for k, v in list(PRECS.items()) if "_refine" in k})
CHECK_DUPLICATES = 1
REFILLABLE = 2
LEAN = 4
CONSUME_INPUT = 8

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run paper_1910_02371_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double

_SIGS = {
    "tc_build_pattern": [_I, _P, _I64, _P, _P, _I, ctypes.c_uint, _P, _P],
    "tc_pattern_refill": [_P, _P, _P, _P],
    "tc_pattern_destroy": [_P],
    "tc_pattern_view": [_P, _I, _P, _P, _P, _P],
    "tc_pattern_columns": [_P, _I, _P, _P, _P],
    "tc_pattern_info": [_P, _P, _P, _P, _P],
    "tc_last_error": [_P, _P],
    "tc_tttp": [_P, _I, _P, _I, _P, _P, _P],
    "tc_mttkrp": [_P, _I, _P, _I, _P, _I, _P, _I, _P],
    "tc_solve_factor": [_P, _I, _P, _I, _P, _I, _P, _D, _I, _P, _P, _P],
    "tc_als_update": [_P, _I, _P, _I, _D, _I, _P, _P, _P],
    "tc_loss_grad": [_P, _I, _I, _P, _D, _P, _P, _P],
    "tc_ggn_matvec": [_P, _I, _I, _P, _P, _D, _P, _P],
    "tc_cg_create": [_P, _I, _I, _P, _D, _I, _P],
    "tc_cg_destroy": [_P],
    "tc_cg_setup": [_P, _P],
    "tc_cg_precond_apply": [_P, _P, _P, _P],
    "tc_cg_solve": [_P, _P, _P, _I, _P, _P],
    "tc_ggn_step": [_P, _I, _P, _P],
    "tc_cg_matvec": [_P, _P, _P, _P],
    "tc_sort_mode_noalloc": [_I64, _P, _I64, _P, _P, _P, _P],
    "tc_set_solve_tuning": [_I, _I, _P],
    "tc_get_solve_tuning": [_I, _I, _P],
    "tc_autotune_solve": [_P, _I, _P, _I, _P, _I, _P, _D, _I, _P, _P, _P, _P],
    "tc_newton_als_mode": [_P, _I, _I, _P, _I, _D, _I, _D, _I, _P, _P],
    "tc_newton_matvec": [_P, _I, _I, _P, _P, _D, _P, _P],
    "tc_cg_set_hessian": [_P, _I],
    "tc_ccd_sweep": [_P, _I, _P, _D, _P],
    "tc_ccd_newton_sweep": [_P, _I, _I, _P, _D, _I, _D, _P, _P],
    "tc_axpby": [_I, _I64, _D, _P, _D, _P, _P],
    "tc_dot": [_I, _I64, _P, _P, _P, _I, _P],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _I
_lib.tc_launch_count.argtypes = []
_lib.tc_launch_count.restype = _I64
_lib.tc_status_string.argtypes = [_I]
_lib.tc_status_string.restype = ctypes.c_char_p


class TcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_lib.tc_status_string(status).decode()} ({status})")
        self.status = status


def _check(rc: int, what: str, allow=()):
    if rc != OK and rc not in allow:
        raise TcError(rc, what)
    return rc


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _ptrs(ts: Sequence) -> ctypes.Array:
    return (ctypes.c_void_p * len(ts))(*[_ptr(t) for t in ts])


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dtype_code(dt: torch.dtype) -> int:
    if dt == torch.float32:
        return F32
    if dt == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {dt}")


def launch_count() -> int:
    """tc_launch_count: kernels this library has launched in this process."""
    return int(_lib.tc_launch_count())


class Pattern:
    """Owner of a tc_pattern (tc_build_pattern / tc_pattern_destroy)."""

    def __init__(self, handle: int, dims, nnz: int, dtype: torch.dtype, device):
        self.handle = ctypes.c_void_p(handle)
        self.dims = tuple(int(d) for d in dims)
        self.nnz = int(nnz)
        self.dtype = dtype
        self.device = device

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.tc_pattern_destroy(h)
            self.handle = None

    def view(self, mode: int):
        """tc_pattern_view as tensors (copies): row_ptr, perm, nonempty_rows."""
        rp, pm, nz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        nne = ctypes.c_int64()
        _check(_lib.tc_pattern_view(self.handle, mode, ctypes.byref(rp), ctypes.byref(pm),
                                    ctypes.byref(nz), ctypes.byref(nne)), "tc_pattern_view")
        torch.cuda.current_stream().synchronize()
        I = self.dims[mode]

        def grab(ptr, n, dt):
            out = torch.empty(n, dtype=dt, device=self.device)
            if n:
                nbytes = n * out.element_size()
                _cuda_memcpy_d2d(out.data_ptr(), ptr.value, nbytes)
            return out

        perm = grab(pm, self.nnz, torch.int64) if pm.value else None   # None: lean pattern
        return grab(rp, I + 1, torch.int64), perm, grab(nz, nne.value, torch.int32)

    def columns(self, mode: int, lo: int = 0, hi: Optional[int] = None):
        """tc_pattern_columns as tensors (copies of sorted positions lo..hi-1):
        the other two modes' indices (ascending mode order) and the values
        (None if the pattern has none)."""
        hi = self.nnz if hi is None else hi
        if not 0 <= lo <= hi <= self.nnz:
            raise ValueError("0 <= lo <= hi <= nnz required")
        c1, c2, v = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(_lib.tc_pattern_columns(self.handle, mode, ctypes.byref(c1), ctypes.byref(c2),
                                       ctypes.byref(v)), "tc_pattern_columns")
        torch.cuda.current_stream().synchronize()
        n = hi - lo

        def grab(ptr, dt):
            out = torch.empty(n, dtype=dt, device=self.device)
            if n:
                es = out.element_size()
                _cuda_memcpy_d2d(out.data_ptr(), ptr.value + lo * es, n * es)
            return out

        return grab(c1, torch.int32), grab(c2, torch.int32), (grab(v, self.dtype) if v.value else None)


def _cuda_memcpy_d2d(dst: int, src: int, nbytes: int):
    # device-to-device copy of a raw pointer through torch (no extra runtime)
    st = torch.cuda.current_stream()
    src_t = _raw_tensor(src, nbytes)
    dst_t = _raw_tensor(dst, nbytes)
    dst_t.copy_(src_t)
    st.synchronize()


def _raw_tensor(ptr: int, nbytes: int):
    """A uint8 CUDA tensor view of raw device memory (no ownership)."""
    class _Holder:
        __cuda_array_interface__ = {
            "shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3,
            "strides": None,
        }
    return torch.as_tensor(_Holder(), device="cuda")


def build_pattern(idx: Sequence[torch.Tensor], dims: Sequence[int], vals: Optional[torch.Tensor] = None,
                  dtype: torch.dtype = torch.float32, check_duplicates: bool = False,
                  refillable: bool = False, lean: bool = False, consume_input: bool = False,
                  stream=None) -> Pattern:
    """tc_build_pattern.  idx: `order` int32 CUDA tensors of length nnz (input
    order); vals: nnz values of `dtype` or None.  lean: keep no positions
    (TC_PATTERN_LEAN); consume_input: the build may overwrite idx and vals
    (TC_PATTERN_CONSUME_INPUT, lean builds only)."""
    order = len(idx)
    nnz = int(idx[0].numel())
    for c in idx:
        if c.dtype != torch.int32 or not c.is_cuda or not c.is_contiguous() or c.numel() != nnz:
            raise ValueError("idx must be contiguous int32 CUDA tensors of equal length")
    if vals is not None and (vals.dtype != dtype or not vals.is_contiguous() or vals.numel() != nnz):
        raise ValueError("vals must be contiguous, of the pattern dtype and length nnz")
    dims_arr = (ctypes.c_int64 * order)(*[int(d) for d in dims])
    out = ctypes.c_void_p()
    flags = ((CHECK_DUPLICATES if check_duplicates else 0) | (REFILLABLE if refillable else 0) |
             (LEAN if lean else 0) | (CONSUME_INPUT if consume_input else 0))
    _check(_lib.tc_build_pattern(order, dims_arr, nnz, _ptrs(idx), _ptr(vals), _dtype_code(dtype),
                                 flags, _stream(stream), ctypes.byref(out)), "tc_build_pattern")
    return Pattern(out.value, dims, nnz, dtype, idx[0].device)


def refill_pattern(p: Pattern, idx: Sequence[torch.Tensor], vals: Optional[torch.Tensor] = None,
                   stream=None):
    """tc_pattern_refill: rebuild p in place from a same-shape tensor (async)."""
    _check(_lib.tc_pattern_refill(p.handle, _ptrs(idx), _ptr(vals), _stream(stream)),
           "tc_pattern_refill")


def last_error(p: Pattern, stream=None) -> int:
    """tc_last_error: synchronizes and returns (and clears) the device status."""
    return int(_lib.tc_last_error(p.handle, _stream(stream)))


def _wcode(w):
    if w is None or w == "one":
        return W_ONE, None
    if isinstance(w, str) and w == "values":
        return W_VALUES, None
    return W_ARRAY, w


def tttp(p: Pattern, factors, weights=None, out=None, R=None, stream=None):
    """tc_tttp.  weights: None/"one" (Omega-hat), "values" (the tensor) or a
    tensor of nnz weights in pattern order.  Returns x in pattern order."""
    R = R or next(f.shape[1] for f in factors if f is not None)
    wk, s = _wcode(weights)
    if out is None:
        out = torch.empty(p.nnz, dtype=p.dtype, device=p.device)
    _check(_lib.tc_tttp(p.handle, wk, _ptr(s), R, _ptrs(factors), _ptr(out), _stream(stream)),
           "tc_tttp")
    return out


def mttkrp(p: Pattern, factors, mode: int, weights="values", out=None, accumulate=False, R=None,
           stream=None):
    """tc_mttkrp into an I_mode x R tensor."""
    R = R or next(f.shape[1] for i, f in enumerate(factors) if f is not None and i != mode)
    wk, s = _wcode(weights)
    if out is None:
        out = torch.empty((p.dims[mode], R), dtype=p.dtype, device=p.device)
    _check(_lib.tc_mttkrp(p.handle, wk, _ptr(s), R, _ptrs(factors), mode, _ptr(out),
                          1 if accumulate else 0, _stream(stream)), "tc_mttkrp")
    return out


def solve_factor(p: Pattern, factors, mode: int, rhs: torch.Tensor, lam: float, weights=None,
                 out=None, row_status=None, prec: str = "fp32", stream=None):
    """tc_solve_factor: per-row (G_i + lam I) a_i = rhs_i.  prec: one of PRECS."""
    R = rhs.shape[1]
    wk, s = _wcode(weights)
    if out is None:
        out = torch.empty_like(rhs)
    _check(_lib.tc_solve_factor(p.handle, wk, _ptr(s), R, _ptrs(factors), mode, _ptr(rhs),
                                float(lam), PRECS[prec], _ptr(out), _ptr(row_status),
                                _stream(stream)),
           "tc_solve_factor")
    return out


def als_update(p: Pattern, factors, mode: int, lam: float, out=None, row_status=None,
               prec: str = "fp32", stream=None):
    """tc_als_update: one least-squares ALS update of factors[mode] -- the
    MTTKRP of the values and Solve Factor in one call.  out defaults to
    factors[mode] (in place)."""
    R = factors[0].shape[1]
    if out is None:
        out = factors[mode]
    _check(_lib.tc_als_update(p.handle, R, _ptrs(factors), mode, float(lam), PRECS[prec],
                              _ptr(out), _ptr(row_status), _stream(stream)), "tc_als_update")
    return out


def loss_grad(p: Pattern, factors, loss: str, lam: float, want_loss=True, want_grad=True,
              grads=None, stream=None):
    """tc_loss_grad: (loss as a 1-element float64 tensor or None, [grads] or None)."""
    R = factors[0].shape[1]
    loss_t = torch.empty(1, dtype=torch.float64, device=p.device) if want_loss else None
    if want_grad and grads is None:
        grads = [torch.empty_like(f) for f in factors]
    gp = _ptrs(grads) if want_grad else None
    _check(_lib.tc_loss_grad(p.handle, LOSSES[loss], R, _ptrs(factors), float(lam), _ptr(loss_t),
                             gp, _stream(stream)), "tc_loss_grad")
    return loss_t, (grads if want_grad else None)


def newton_matvec(p: Pattern, factors, x, loss: str, lam: float, y=None, stream=None):
    """tc_newton_matvec: y = (full Hessian) x, the Gauss-Newton product plus the phi' term."""
    R = factors[0].shape[1]
    if y is None:
        y = [torch.empty_like(v) for v in x]
    _check(_lib.tc_newton_matvec(p.handle, LOSSES[loss], R, _ptrs(factors), _ptrs(x), float(lam),
                                 _ptrs(y), _stream(stream)), "tc_newton_matvec")
    return y


def ggn_matvec(p: Pattern, factors, x, loss: str, lam: float, y=None, stream=None):
    """tc_ggn_matvec: y = (J^T diag(phi'') J + 2 lam I) x."""
    R = factors[0].shape[1]
    if y is None:
        y = [torch.empty_like(v) for v in x]
    _check(_lib.tc_ggn_matvec(p.handle, LOSSES[loss], R, _ptrs(factors), _ptrs(x), float(lam),
                              _ptrs(y), _stream(stream)), "tc_ggn_matvec")
    return y


class CG:
    """tc_cg_*: preconditioned CG on the Gauss-Newton system and GGN steps.
    The factor tensors are kept (and updated in place by ggn_step)."""

    def __init__(self, p: Pattern, factors, loss: str, lam: float, precondition=True):
        self.p = p
        self.factors = list(factors)
        self.R = factors[0].shape[1]
        h = ctypes.c_void_p()
        _check(_lib.tc_cg_create(p.handle, LOSSES[loss], self.R, _ptrs(self.factors), float(lam),
                                 1 if precondition else 0, ctypes.byref(h)), "tc_cg_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.tc_cg_destroy(h)
            self.handle = None

    def set_hessian(self, full_newton: bool):
        """tc_cg_set_hessian: iterate with the full Hessian (True) or the
        Gauss-Newton matrix (False, the default)."""
        _check(_lib.tc_cg_set_hessian(self.handle, 1 if full_newton else 0), "tc_cg_set_hessian")

    def setup(self, stream=None):
        _check(_lib.tc_cg_setup(self.handle, _stream(stream)), "tc_cg_setup")

    def precond_apply(self, r, z=None, stream=None):
        if z is None:
            z = [torch.empty_like(v) for v in r]
        _check(_lib.tc_cg_precond_apply(self.handle, _ptrs(r), _ptrs(z), _stream(stream)),
               "tc_cg_precond_apply")
        return z

    def solve(self, b, iters: int, dx=None, rz=None, stream=None):
        if dx is None:
            dx = [torch.empty_like(v) for v in b]
        _check(_lib.tc_cg_solve(self.handle, _ptrs(b), _ptrs(dx), int(iters), _ptr(rz),
                                _stream(stream)), "tc_cg_solve")
        return dx

    def matvec(self, x, y=None, stream=None):
        """tc_cg_matvec: y = H x at the solver's factors (its own layout)."""
        if y is None:
            y = [torch.empty_like(v) for v in x]
        _check(_lib.tc_cg_matvec(self.handle, _ptrs(x), _ptrs(y), _stream(stream)), "tc_cg_matvec")
        return y

    def ggn_step(self, iters: int, loss_out=None, stream=None):
        _check(_lib.tc_ggn_step(self.handle, int(iters), _ptr(loss_out), _stream(stream)),
               "tc_ggn_step")


SORT_NOALLOC_MAX_NNZ = 1 << 20


def sort_mode_noalloc(key: torch.Tensor, I: int, perm=None, row_ptr=None, status=None,
                      stream=None):
    """tc_sort_mode_noalloc: the stable per-mode sort without device
    allocations in the library (the output tensors are the caller's)."""
    n = int(key.numel())
    if perm is None:
        perm = torch.empty(n, dtype=torch.int64, device=key.device)
    if row_ptr is None:
        row_ptr = torch.empty(int(I) + 1, dtype=torch.int64, device=key.device)
    _check(_lib.tc_sort_mode_noalloc(n, _ptr(key), int(I), _ptr(perm), _ptr(row_ptr), _ptr(status),
                                     _stream(stream)), "tc_sort_mode_noalloc")
    return perm, row_ptr


class _SolveTuning(ctypes.Structure):
    _fields_ = [("chunk_nnz", _I64), ("batch_bytes", _I64), ("chol_rows_per_warp", ctypes.c_int32),
                ("gram_kernel", ctypes.c_int32)]


GRAM_AUTO, GRAM_WARP_MMA, GRAM_TCGEN05 = 0, 1, 2


def set_solve_tuning(dtype: torch.dtype, R: int = 0, chunk_nnz: int = 0, batch_bytes: int = 0,
                     chol_rows_per_warp: int = 0, gram_kernel: int = 0, reset: bool = False):
    """tc_set_solve_tuning: chunk size, batch budget, factorization rows per
    warp and Gram engine (GRAM_*) of Solve Factor for the rank tier of R
    (R = 0: every tier); reset=True restores the automatic choice."""
    t = None if reset else ctypes.byref(
        _SolveTuning(int(chunk_nnz), int(batch_bytes), int(chol_rows_per_warp), int(gram_kernel)))
    _check(_lib.tc_set_solve_tuning(_dtype_code(dtype), int(R), t), "tc_set_solve_tuning")


def get_solve_tuning(dtype: torch.dtype, R: int):
    """tc_get_solve_tuning: (chunk_nnz, batch_bytes, chol_rows_per_warp,
    gram_kernel), 0 meaning automatic."""
    t = _SolveTuning()
    _check(_lib.tc_get_solve_tuning(_dtype_code(dtype), int(R), ctypes.byref(t)),
           "tc_get_solve_tuning")
    return int(t.chunk_nnz), int(t.batch_bytes), int(t.chol_rows_per_warp), int(t.gram_kernel)


def autotune_solve(p: Pattern, factors, mode: int, rhs: torch.Tensor, lam: float, weights=None,
                   out=None, prec: str = "fp32", stream=None):
    """tc_autotune_solve: times Solve Factor at the candidate tunings, installs
    the fastest; returns ((chunk_nnz, batch_bytes, chol_rows_per_warp,
    gram_kernel), ms)."""
    R = rhs.shape[1]
    wk, s = _wcode(weights)
    if out is None:
        out = torch.empty_like(rhs)
    best = _SolveTuning()
    ms = ctypes.c_float()
    _check(_lib.tc_autotune_solve(p.handle, wk, _ptr(s), R, _ptrs(factors), mode, _ptr(rhs),
                                  float(lam), PRECS[prec], _ptr(out), ctypes.byref(best),
                                  ctypes.byref(ms), _stream(stream)), "tc_autotune_solve")
    return (int(best.chunk_nnz), int(best.batch_bytes), int(best.chol_rows_per_warp),
            int(best.gram_kernel)), float(ms.value)


def newton_als_mode(p: Pattern, factors, mode: int, loss: str, lam: float, inner_iters: int = 5,
                    tol: float = 1e-3, prec: str = "fp32", stream=None) -> int:
    """tc_newton_als_mode: Newton steps on factors[mode] in place; returns the
    number of steps taken."""
    R = factors[0].shape[1]
    steps = ctypes.c_int()
    _check(_lib.tc_newton_als_mode(p.handle, LOSSES[loss], R, _ptrs(factors), int(mode), float(lam),
                                   int(inner_iters), float(tol), PRECS[prec], ctypes.byref(steps),
                                   _stream(stream)), "tc_newton_als_mode")
    return int(steps.value)


def ccd_sweep(p: Pattern, factors, lam: float, stream=None):
    """tc_ccd_sweep: one CCD++ sweep (least squares) on the factors in place."""
    R = factors[0].shape[1]
    _check(_lib.tc_ccd_sweep(p.handle, R, _ptrs(factors), float(lam), _stream(stream)),
           "tc_ccd_sweep")
    return factors


def ccd_newton_sweep(p: Pattern, factors, loss: str, lam: float, inner_iters: int = 5,
                     tol: float = 1e-3, stream=None):
    """tc_ccd_newton_sweep: one coordinate-minimization sweep for a general loss
    on the factors in place.  Returns the Newton steps taken per column as a
    list of R lists (one entry per mode)."""
    R = factors[0].shape[1]
    steps = (ctypes.c_int * (R * len(factors)))()
    _check(_lib.tc_ccd_newton_sweep(p.handle, LOSSES[loss], R, _ptrs(factors), float(lam),
                                    int(inner_iters), float(tol), steps, _stream(stream)),
           "tc_ccd_newton_sweep")
    N = len(factors)
    return [[int(steps[r * N + d]) for d in range(N)] for r in range(R)]


def axpby(alpha: float, x: torch.Tensor, beta: float, y: torch.Tensor, stream=None):
    """tc_axpby: y = alpha x + beta y in place (same dtype and length)."""
    if x.numel() != y.numel() or x.dtype != y.dtype or not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x, y: contiguous tensors of one dtype and length")
    _check(_lib.tc_axpby(_dtype_code(y.dtype), y.numel(), float(alpha), _ptr(x), float(beta),
                         _ptr(y), _stream(stream)), "tc_axpby")
    return y


def dot(x: torch.Tensor, y: torch.Tensor, out=None, accumulate=False, stream=None):
    """tc_dot: FP64 sum of x_i y_i into a 1-element float64 device tensor."""
    if x.numel() != y.numel() or x.dtype != y.dtype or not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x, y: contiguous tensors of one dtype and length")
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=x.device)
    _check(_lib.tc_dot(_dtype_code(x.dtype), x.numel(), _ptr(x), _ptr(y), _ptr(out),
                       1 if accumulate else 0, _stream(stream)), "tc_dot")
    return out
