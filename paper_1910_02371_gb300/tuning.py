"""Persisted Solve Factor tunings.

``autotune(p, factors, mode, rhs, lam)`` runs the library's autotuner
(tc_autotune_solve) on a real pattern and records the winner under a key of
the dtype, the rank tier and the mode's shape class (rows and nonzeros per
row, in powers of two); ``save(path)`` / ``load(path)`` write and read those
records as JSON (a record without ``gram_kernel`` means the automatic
engine), and ``apply(...)`` installs the record that matches a
workload.  Everything here is host bookkeeping; the timing runs in the
library.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Tuple

import torch

from . import tc

_records: Dict[str, dict] = {}


def _tier(R: int) -> int:
    return 8 if R <= 8 else 16 if R <= 16 else 32 if R <= 32 else 64


def shape_key(dtype: torch.dtype, R: int, rows: int, nnz: int, prec: str = "fp32") -> str:
    """dtype / rank tier / log2(rows) / log2(nonzeros per row) / precision form."""
    per_row = max(nnz, 1) / max(rows, 1)
    return "%s/r%d/rows2^%d/nnzrow2^%d/%s" % (
        "f32" if dtype == torch.float32 else "f64", _tier(R),
        int(math.log2(max(rows, 1))), int(math.log2(max(per_row, 1.0))), prec)


def autotune(p: "tc.Pattern", factors, mode: int, rhs: torch.Tensor, lam: float,
             prec: str = "fp32") -> Tuple[str, dict]:
    """Tunes Solve Factor for this pattern's mode, installs and records the winner."""
    R = rhs.shape[1]
    best, ms = tc.autotune_solve(p, factors, mode, rhs, lam, prec=prec)
    key = shape_key(p.dtype, R, p.dims[mode], p.nnz, prec)
    rec = {"chunk_nnz": best[0], "batch_bytes": best[1], "chol_rows_per_warp": best[2],
           "gram_kernel": best[3], "ms": ms}
    _records[key] = rec
    return key, rec


def records() -> Dict[str, dict]:
    return dict(_records)


def save(path: str):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(_records, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path: str) -> Dict[str, dict]:
    with open(path) as f:
        data = json.load(f)
    for k, v in data.items():
        if not isinstance(v, dict) or not {"chunk_nnz", "batch_bytes", "chol_rows_per_warp"} <= set(v):
            raise ValueError("bad tuning record %r" % k)
    _records.update(data)
    return data


def apply(dtype: torch.dtype, R: int, rows: int, nnz: int, prec: str = "fp32") -> bool:
    """Installs the recorded tuning for this workload's shape class, if any."""
    rec = _records.get(shape_key(dtype, R, rows, nnz, prec))
    if rec is None:
        return False
    tc.set_solve_tuning(dtype, R, chunk_nnz=rec["chunk_nnz"], batch_bytes=rec["batch_bytes"],
                        chol_rows_per_warp=rec["chol_rows_per_warp"],
                        gram_kernel=rec.get("gram_kernel", 0))
    return True
