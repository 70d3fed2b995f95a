"""Sparse CP tensor-completion kernels for GB300 (sm_103a).

The library ``libtc.so`` (C ABI in ``include/tc.h``) holds every kernel of the
hot path: the per-mode pattern builder, TTTP, MTTKRP, Solve Factor, the loss
gradient, the Gauss-Newton matrix-vector product and the graph-captured PCG
driver.  ``tc`` is the thin Python binding (torch tensors in, C calls out);
``drivers`` composes those calls into ALS sweeps and Gauss-Newton steps.
"""
from . import build  # noqa: F401


def load():
    """Imports the binding (libtc.so must be built)."""
    from . import tc  # noqa: F401
    return tc
