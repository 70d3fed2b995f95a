"""Seeded synthetic inputs for sparse CP tensor completion.

This module is shared by the CUDA path's tests, the benchmark and the oracle's
tests.  It deliberately contains none of the method's arithmetic: it draws
coordinates, factor matrices and noise, and it turns model entries that the
*caller* computed (with the oracle, or on the device) into observed values by
adding noise, drawing Poisson counts or rounding.  It never evaluates the CP
model itself.

Randomness: numpy's counter-based Philox4x32-10 bit generator (Salmon et al.,
SC'11), one independent stream per (seed, purpose) pair, so every input is a
pure function of (seed, workload).

Workloads (the order-3 problems the method is benchmarked on):

* ``cp3_200_m40k_r5``    200x200x200, 4e4 uniform coordinates, rank 5, FP64,
                          planted N(0,1) factors + N(0, 0.01^2) noise, lambda 1e-3.
* ``cp3_10k_m10M_r16``   10^4 cubed, 10^7 uniform coordinates, rank 16, FP32,
                          planted N(0,1) factors + N(0, 0.1^2) noise, lambda 1e-2.
* ``cp3_50k_m50M_r32``   5e4 x 5e4 x 5e3, 5e7 coordinates, rank 32, FP32,
                          Uniform(0,1) factors, Poisson(model) counts, lambda 0.1.
* ``cp3_netflix_m100M_r64`` 480189 x 17770 x 2182, 1e8 coordinates with Zipf(1.1)
                          rows in modes 0 and 1, rank 64, values round(model)
                          clamped to 1..5, lambda 0.05 (a synthetic stand-in with
                          the shape of the Netflix ratings tensor).
* ``cp3_4M_m4B_r16``     2^22 cubed, 4e9 uniform coordinates, rank 16, FP32,
                          planted N(0,1) factors + N(0, 0.1^2) noise, lambda 1e-2
                          (the paper's 1e10-nonzero synthetic scaled to one GPU).
                          Too large for host generation: its coordinates come
                          from ``feistel_coords``, evaluated where they are used.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "stream", "distinct_coords", "zipf_ids",
    "factor_matrices", "observe", "make_coords", "scaled", "feistel_keys", "feistel_coords",
]

# Purposes of the independent random streams drawn from one seed.
_S_COORD = 1
_S_PLANT = 2
_S_NOISE = 3
_S_INIT = 4
_S_PERM = 5
_S_EXTRA = 6


def stream(seed: int, purpose: int) -> np.random.Generator:
    """An independent Philox4x32-10 stream keyed by (seed, purpose)."""
    key = (int(seed) & ((1 << 64) - 1)) | (int(purpose) << 64)
    return np.random.Generator(np.random.Philox(key=key))


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple
    nnz: int
    rank: int
    dtype: str            # "f32" | "f64"
    lam: float
    loss: str             # "ls" | "poisson_log" | "poisson_id"
    coord_dist: tuple     # per mode: "uniform" | "zipf"
    factor_dist: str      # "normal" | "uniform01" | "uniform_c"
    values: str           # "noise" | "poisson" | "round15"
    noise: float = 0.0
    zipf_s: float = 1.1
    seed: int = 1910023710
    coords: str = "draw"  # "draw": distinct_coords on the host; "feistel": feistel_coords

    @property
    def feistel_bits(self) -> int:
        """Bits per mode of a "feistel" workload (all dims 2^bits)."""
        return int(self.dims[0]).bit_length() - 1


WORKLOADS = {
    w.name: w for w in [
        Workload("cp3_200_m40k_r5", (200, 200, 200), 40_000, 5, "f64", 1e-3, "ls",
                 ("uniform",) * 3, "normal", "noise", noise=0.01, seed=1910023711),
        Workload("cp3_10k_m10M_r16", (10_000, 10_000, 10_000), 10_000_000, 16, "f32", 1e-2,
                 "ls", ("uniform",) * 3, "normal", "noise", noise=0.1, seed=1910023712),
        Workload("cp3_50k_m50M_r32", (50_000, 50_000, 5_000), 50_000_000, 32, "f32", 0.1,
                 "poisson_log", ("uniform",) * 3, "uniform01", "poisson", seed=1910023713),
        Workload("cp3_netflix_m100M_r64", (480_189, 17_770, 2_182), 100_000_000, 64, "f32",
                 0.05, "ls", ("zipf", "zipf", "uniform"), "uniform_c", "round15",
                 seed=1910023714),
        Workload("cp3_4M_m4B_r16", (1 << 22,) * 3, 4_000_000_000, 16, "f32", 1e-2, "ls",
                 ("uniform",) * 3, "normal", "noise", noise=0.1, seed=1910023715,
                 coords="feistel"),
    ]
}


# ------------------------------------------------------------------ keyed permutation
# Distinct uniform coordinates without a dedup pass, for tensors too large to
# draw on the host: entry e (e = 0, 1, ...) gets the image of e under a keyed
# permutation of the 3b-bit index space [0, 2^(3b)) (b bits per mode, all dims
# 2^b), so distinct entries get distinct coordinates and the coordinates look
# uniform.  The permutation is a balanced Feistel network (Luby & Rackoff,
# SIAM J. Comput. 17(2), 1988) of 4 rounds on two 3b/2-bit halves, with a
# multiply-xorshift round function.  Every intermediate stays below 2^63, so
# the same code runs on numpy int64 arrays and on torch int64 tensors (on any
# device) with identical results.
FEISTEL_ROUNDS = 4


def feistel_keys(seed: int):
    """Round keys: (xor key, odd multiplier, odd multiplier) per round, each
    below 2^30, from the coordinate stream of ``seed``."""
    rng = stream(seed, _S_COORD)
    k = rng.integers(1, 1 << 30, size=(FEISTEL_ROUNDS, 3), dtype=np.int64)
    k[:, 1:] |= 1
    return [tuple(int(v) for v in row) for row in k]


def _feistel_f(x, key, m1, m2, mask):
    y = (x ^ key) & mask
    y = (y * m1) & mask
    y = y ^ (y >> 16)
    y = (y * m2) & mask
    return y ^ (y >> 13)


def feistel_coords(e, bits: int, keys):
    """Coordinates (i_0, i_1, i_2) of entries e (int64 array or tensor, values
    in [0, 2^min(63, 3 bits))) for dims (2^bits,) * 3; bits even, 2..22.
    Returns three int64 arrays/tensors of e's type."""
    if bits % 2 or not 2 <= bits <= 22:
        raise ValueError("bits must be even, 2..22")
    h = 3 * bits // 2
    mask = (1 << h) - 1
    left, right = e >> h, e & mask
    for key, m1, m2 in keys:
        left, right = right, left ^ _feistel_f(right, key, m1, m2, mask)
    bmask = (1 << bits) - 1
    lo = bits // 2               # bits of i_1 held in `right`
    i0 = right & bmask
    i1 = (right >> bits) | ((left & ((1 << lo) - 1)) << (h - bits))
    i2 = left >> lo
    return i0, i1, i2


def scaled(w: Workload, nnz: int, dims: Optional[Sequence[int]] = None, **kw) -> Workload:
    """A smaller copy of a workload (same recipe, fewer coordinates)."""
    return dataclasses.replace(w, nnz=int(nnz), dims=tuple(dims) if dims else w.dims,
                               name=f"{w.name}@{nnz}", **kw)


def zipf_ids(n: int, dim: int, s: float, rng: np.random.Generator,
             perm: np.ndarray) -> np.ndarray:
    """n ids in [0, dim) with P(rank r) proportional to r^-s (r = 1..dim),
    drawn by inverting the truncated CDF, then relabelled through ``perm`` so
    that the heavy rows are spread over the id range."""
    w = np.arange(1, dim + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    r = np.searchsorted(cdf, u, side="right")
    np.minimum(r, dim - 1, out=r)
    return perm[r].astype(np.int32)


def _draw(dims, n, dists, s, rng, perms):
    cols = []
    for d, (I, dist) in enumerate(zip(dims, dists)):
        if dist == "uniform":
            cols.append(rng.integers(0, I, size=n, dtype=np.int64).astype(np.int32))
        elif dist == "zipf":
            cols.append(zipf_ids(n, I, s, rng, perms[d]))
        else:
            raise ValueError(dist)
    return cols


def _keys(cols, dims):
    total = 1
    for I in dims:
        total *= int(I)
    if total < (1 << 62):
        key = np.zeros(cols[0].shape[0], dtype=np.int64)
        for c, I in zip(cols, dims):
            key *= int(I)
            key += c.astype(np.int64)
        return key
    # wider than 62 bits: unique on the raw coordinate tuple
    stacked = np.ascontiguousarray(np.stack(cols, axis=1))
    return stacked.view(np.dtype((np.void, stacked.dtype.itemsize * stacked.shape[1]))).ravel()


def distinct_coords(dims, nnz, dists, seed, zipf_s=1.1):
    """``nnz`` distinct coordinates, in draw order (unsorted).

    Coordinates are drawn in rounds; of repeated draws the earliest is kept and
    the first ``nnz`` distinct coordinates in draw order form the tensor.
    Returns a list of int32 arrays, one per mode."""
    dims = tuple(int(x) for x in dims)
    total = math.prod(dims)
    if nnz > total:
        raise ValueError("more coordinates than cells")
    rng = stream(seed, _S_COORD)
    prng = stream(seed, _S_PERM)
    perms = [prng.permutation(I).astype(np.int64) for I in dims]
    cols = [np.zeros(0, np.int32) for _ in dims]
    parts = [[] for _ in dims]
    seen = None               # sorted keys kept so far (linear keys only)
    linear = total < (1 << 62)
    have = 0
    rounds = 0
    while have < nnz:
        need = nnz - have
        n = int(need * 1.05) + 1024
        if total - have < 4 * need:   # nearly full tensors: draw more per round
            n = max(n, 4 * need)
        new = _draw(dims, n, dists, zipf_s, rng, perms)
        if linear:
            # keep the first occurrence of every key not seen in earlier rounds,
            # in draw order: the same coordinates as deduplicating the whole
            # draw sequence at once, without re-sorting earlier rounds
            keys = _keys(new, dims)
            uk, first = np.unique(keys, return_index=True)
            if seen is not None and seen.size:
                pos = np.minimum(np.searchsorted(seen, uk), seen.size - 1)
                fresh = seen[pos] != uk
                uk, first = uk[fresh], first[fresh]
            first.sort()
            for d in range(len(dims)):
                parts[d].append(new[d][first])
            seen = uk if seen is None else np.sort(np.concatenate([seen, uk]), kind="stable")
            have += first.shape[0]
        else:
            cols = [np.concatenate([a, b]) for a, b in zip(cols, new)]
            _, first = np.unique(_keys(cols, dims), return_index=True)
            first.sort()
            cols = [c[first] for c in cols]
            have = cols[0].shape[0]
        rounds += 1
        if rounds > 200:
            raise RuntimeError("could not draw enough distinct coordinates")
    if linear:
        cols = [np.concatenate(pp) for pp in parts]
    return [np.ascontiguousarray(c[:nnz]) for c in cols]


def factor_matrices(dims, rank, dist, seed, purpose=_S_PLANT, dtype=np.float64):
    """One row-major I_n x R matrix per mode."""
    rng = stream(seed, purpose)
    out = []
    for I in dims:
        if dist == "normal":
            a = rng.standard_normal((I, rank))
        elif dist == "uniform01":
            a = rng.random((I, rank))
        elif dist == "uniform_c":
            # E[model entry] = R * (c/2)^3 = 3 for c = (24/R)^(1/3)
            c = (24.0 / rank) ** (1.0 / 3.0)
            a = c * rng.random((I, rank))
        else:
            raise ValueError(dist)
        out.append(np.ascontiguousarray(a.astype(dtype)))
    return out


def init_factors(dims, rank, seed, scale=1.0, dtype=np.float64):
    """Starting factors for an algorithm (a stream separate from the planted ones)."""
    rng = stream(seed, _S_INIT)
    return [np.ascontiguousarray((scale * rng.standard_normal((I, rank))).astype(dtype))
            for I in dims]


def perturb(factors, seed, lo=0.9, hi=1.1):
    """Multiply every factor entry by an independent Uniform(lo, hi) draw."""
    rng = stream(seed, _S_EXTRA)
    return [np.ascontiguousarray(a * rng.uniform(lo, hi, size=a.shape).astype(a.dtype))
            for a in factors]


def observe(model_entries: np.ndarray, recipe: str, seed: int, noise: float = 0.0) -> np.ndarray:
    """Observed values from model entries the caller computed.

    ``noise``: t = m + N(0, noise^2);  ``poisson``: t ~ Poisson(max(m, 0));
    ``round15``: t = clamp(round(m), 1, 5)."""
    m = np.asarray(model_entries, dtype=np.float64)
    rng = stream(seed, _S_NOISE)
    if recipe == "noise":
        return m + noise * rng.standard_normal(m.shape[0])
    if recipe == "poisson":
        return rng.poisson(np.maximum(m, 0.0)).astype(np.float64)
    if recipe == "round15":
        return np.clip(np.rint(m), 1.0, 5.0)
    if recipe == "exact":
        return m.copy()
    raise ValueError(recipe)


def make_coords(w: Workload):
    return distinct_coords(w.dims, w.nnz, w.coord_dist, w.seed, w.zipf_s)
