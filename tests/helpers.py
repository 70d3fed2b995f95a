"""Shared helpers for the GPU parity tests: seeded problems whose values come
from the oracle, upload to the device, and the error measures."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle
import synth

# Tolerances: FP32 kernel outputs within 1e-5 relative (normwise per
# output array) of the FP64 oracle; FP64 kernels to 1e-12.
TOL = {"f32": 1e-5, "f64": 1e-12}


@dataclasses.dataclass
class Problem:
    dims: tuple
    idx: list            # int32 arrays, input order
    t: np.ndarray        # observed values (float64), input order
    factors: list        # float64 starting factors
    R: int
    dtype: str
    name: str = ""

    @property
    def nnz(self):
        return len(self.idx[0])


def make_problem(name, dims, nnz, R, dtype, seed, dist=("uniform",) * 3, factor="normal",
                 recipe="noise", noise=0.1, init="perturb"):
    idx = synth.distinct_coords(dims, nnz, dist, seed)
    planted = synth.factor_matrices(dims, R, factor, seed)
    model = oracle.model_entries(dims, idx, planted)
    t = synth.observe(model, recipe, seed, noise)
    if init == "perturb":
        A = synth.perturb(planted, seed)
    else:
        A = synth.init_factors(dims, R, seed)
    if dtype == "f32":
        # the device sees float32 inputs; the oracle gets exactly those values
        t = t.astype(np.float32).astype(np.float64)
        A = [a.astype(np.float32).astype(np.float64) for a in A]
    return Problem(tuple(dims), idx, t, A, R, dtype, name)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.linalg.norm(b)
    if den == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / den)


def torch_dtype(dtype):
    import torch
    return torch.float32 if dtype == "f32" else torch.float64


def to_dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch_dtype(dtype))


def idx_dev(idx):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(c, dtype=np.int32)).cuda() for c in idx]


def host(t):
    return t.detach().cpu().double().numpy()


def build(prob, with_vals=True, check_duplicates=False):
    from paper_1910_02371_gb300 import tc
    vals = to_dev(prob.t, prob.dtype) if with_vals else None
    return tc.build_pattern(idx_dev(prob.idx), prob.dims, vals, dtype=torch_dtype(prob.dtype),
                            check_duplicates=check_duplicates)
