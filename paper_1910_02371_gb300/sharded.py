"""Row-sharded ALS and Gauss-Newton steps over several processes (one GPU each).

The paper distributes each factor over processes and, after every Solve
Factor, redistributes the updated rows to the processes that need them, and it
sums partial results across processes (Sec. 3.2 and Sec. 3.4; Sec. 2.5 for
the CG iteration).  Here every process holds the whole factors (they are small
next to the nonzeros) and owns, in every mode d, one contiguous range of rows
chosen so that the ranges carry about the same number of nonzeros.  For mode d
a process keeps exactly the nonzeros of its rows (its mode-d block), so

* MTTKRP and Solve Factor of mode d are local: the owned rows of the result
  need no nonzero of another process;
* after mode d's Solve Factor the owned row blocks are all-gathered, and every
  process continues with the whole new factor (the ALS sweep's Gauss-Seidel
  order is kept);
* the objective sums one block per process (the mode-0 blocks partition the
  nonzeros) with an all-reduce;
* the gradient, the Gauss-Newton product and the block-diagonal
  preconditioner of mode d are exact on the owned rows of the mode-d block;
* PCG keeps its vectors row-sharded: the search direction is all-gathered
  before each product (the product needs every mode's whole direction), and
  the two inner products per iteration are all-reduced in FP64.

Every arithmetic step runs in the `ops` object's kernels -- ``LibtcOps`` (the
libtc C ABI, one GPU per process) in production; the iteration's step
lengths are formed on the host from the all-reduced FP64 inner products.
Collectives go through torch.distributed (NCCL between GPUs, gloo on the
host); with no process group the object runs as one process.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np
import torch


def partition_rows(counts: np.ndarray, world: int) -> List[Tuple[int, int]]:
    """Contiguous row ranges [lo, hi) of one mode, one per process, cut where
    the running count of nonzeros first reaches k m / world (k = 1 .. world-1),
    so every range holds about m / world nonzeros (a row is never split)."""
    counts = np.asarray(counts, dtype=np.int64)
    cum = np.concatenate([[0], np.cumsum(counts)])
    m = int(cum[-1])
    cuts = [0]
    for k in range(1, world):
        c = int(np.searchsorted(cum, k * m / world, side="left"))
        cuts.append(min(max(c, cuts[-1]), len(counts)))
    cuts.append(len(counts))
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


class LibtcOps:
    """The per-process kernels of the sharded driver: libtc calls on this
    process's GPU (torch CUDA tensors in and out)."""

    def __init__(self, dtype=torch.float32):
        from . import tc     # the CUDA library; loading fails loudly if it is not built
        self.tc = tc
        self.dtype = dtype

    def build(self, idx, vals, dims):
        return self.tc.build_pattern(idx, dims, vals, dtype=self.dtype)

    def mttkrp(self, h, A, d, out):
        return self.tc.mttkrp(h, A, d, weights="values", out=out)

    def solve_factor(self, h, A, d, rhs, lam, out, prec="fp32"):
        return self.tc.solve_factor(h, A, d, rhs, lam, out=out, prec=prec)

    def als_update(self, h, A, d, lam, out, prec="fp32"):
        # the MTTKRP of the values and Solve Factor in one pass over the block
        return self.tc.als_update(h, A, d, lam, out=out, prec=prec)

    def loss(self, h, A, loss, lam):
        f, _ = self.tc.loss_grad(h, A, loss, lam, want_grad=False)
        return f

    def grad(self, h, A, loss, lam, d, out):
        grads = [None] * len(A)
        grads[d] = out
        self.tc.loss_grad(h, A, loss, lam, want_loss=False, grads=grads)
        return out

    def ggn_matvec(self, h, A, x, loss, lam, y):
        return self.tc.ggn_matvec(h, A, x, loss, lam, y=y)

    def precond(self, h, A, loss, lam):
        cg = self.tc.CG(h, A, loss, lam)
        cg.setup()
        return cg

    def precond_apply(self, pc, r, z):
        return pc.precond_apply(r, z)

    def axpby(self, alpha, x, beta, y):
        return self.tc.axpby(alpha, x, beta, y)

    def dot(self, x, y, out, accumulate):
        return self.tc.dot(x, y, out=out, accumulate=accumulate)

    def empty(self, shape, like):
        return torch.empty(shape, dtype=like.dtype, device=like.device)


class ShardedCP:
    """One process's share of a row-sharded order-3 CP completion problem.

    idx: the whole tensor's three int32 index tensors (input order), vals its
    values, on this process's device; each process passes the same tensor and
    keeps only its blocks.  A is the list of whole factors (updated in place)."""

    def __init__(self, ops, idx: Sequence[torch.Tensor], vals: torch.Tensor, dims, loss: str,
                 lam: float, group=None):
        import torch.distributed as dist
        self.ops = ops
        self.dims = tuple(int(x) for x in dims)
        self.loss = loss
        self.lam = float(lam)
        self.group = group
        self.dist = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if self.dist else 1
        self.rank = dist.get_rank(group) if self.dist else 0
        self.ranges = []          # per mode: every process's [lo, hi)
        self.block = []           # per mode: this process's block (pattern handle)
        for d, I in enumerate(self.dims):
            counts = torch.bincount(idx[d].long(), minlength=I).cpu().numpy()
            rg = partition_rows(counts, self.world)
            self.ranges.append(rg)
            lo, hi = rg[self.rank]
            keep = (idx[d] >= lo) & (idx[d] < hi)
            sub = [c[keep].contiguous() for c in idx]
            self.block.append(ops.build(sub, vals[keep].contiguous(), self.dims))

    # ---------------------------------------------------------------- collectives
    def own(self, d):
        return self.ranges[d][self.rank]

    def _allgather_rows(self, M: torch.Tensor, d: int):
        """Every process's owned rows of M (I_d x R) into every process's M."""
        if self.world == 1:
            return M
        import torch.distributed as dist
        rg = self.ranges[d]
        width = max(hi - lo for lo, hi in rg)
        lo, hi = rg[self.rank]
        send = torch.zeros((width, M.shape[1]), dtype=M.dtype, device=M.device)
        send[:hi - lo] = M[lo:hi]
        parts = [torch.empty_like(send) for _ in range(self.world)]
        dist.all_gather(parts, send, group=self.group)
        for (plo, phi), part in zip(rg, parts):
            M[plo:phi] = part[:phi - plo]
        return M

    def _allreduce_sum(self, v: torch.Tensor) -> float:
        """The FP64 sum of a one-element tensor over the processes (host value)."""
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(v, op=dist.ReduceOp.SUM, group=self.group)
        return float(v.item())

    def _dot_own(self, X, Y, out) -> float:
        """sum over modes of the owned rows' inner product, over all processes."""
        for d in range(3):
            lo, hi = self.own(d)
            self.ops.dot(X[d][lo:hi].reshape(-1), Y[d][lo:hi].reshape(-1), out, accumulate=d > 0)
        return self._allreduce_sum(out)

    # ---------------------------------------------------------------- algorithms
    def objective(self, A) -> float:
        """f = sum_e phi + lambda sum ||A||^2 (eq. obj): each process evaluates
        its mode-0 block with lambda / world, so the sum counts the regularizer once."""
        f = self.ops.loss(self.block[0], A, self.loss, self.lam / self.world)
        return self._allreduce_sum(f)

    def als_sweep(self, A, prec="fp32"):
        """One ALS sweep (Sec. 2.2) in place: for each mode the owned rows are
        solved locally from the mode's block (its MTTKRP and Solve Factor, one
        ops.als_update), then all-gathered."""
        for d in range(3):
            new = self.ops.empty(A[d].shape, A[d])
            self.ops.als_update(self.block[d], A, d, self.lam, new, prec)
            lo, hi = self.own(d)
            A[d][lo:hi] = new[lo:hi]
            self._allgather_rows(A[d], d)
        return A

    def gradient(self, A):
        """grad^(d) = MTTKRP(phi', d) + 2 lambda A^(d) (Table 1), exact on the
        owned rows of every mode (other rows are not meaningful)."""
        G = []
        for d in range(3):
            g = self.ops.empty(A[d].shape, A[d])
            self.ops.grad(self.block[d], A, self.loss, self.lam, d, g)
            G.append(g)
        return G

    def ggn_step(self, A, iters: int):
        """One Gauss-Newton step (Sec. 2.5) in place: PCG from zero for a fixed
        number of iterations on H dx = -grad with the block-diagonal
        preconditioner, vectors sharded by rows, then A += dx.  Returns the
        r^T z history (host floats)."""
        ops = self.ops
        dev0 = A[0]
        acc = torch.zeros(1, dtype=torch.float64, device=dev0.device)
        b = self.gradient(A)
        for v in b:
            ops.axpby(0.0, v.reshape(-1), -1.0, v.reshape(-1))
        pcs = [ops.precond(self.block[d], A, self.loss, self.lam) for d in range(3)]

        def precond(r, z):
            for d in range(3):
                zz = [ops.empty(v.shape, v) for v in r]
                ops.precond_apply(pcs[d], r, zz)
                lo, hi = self.own(d)
                z[d][lo:hi] = zz[d][lo:hi]

        x = [torch.zeros_like(v) for v in b]
        r = [v.clone() for v in b]
        z = [torch.zeros_like(v) for v in b]
        precond(r, z)
        p = [v.clone() for v in z]
        Ap = [torch.zeros_like(v) for v in b]
        rz = self._dot_own(r, z, acc)
        hist = [rz]
        for _ in range(iters):
            for d in range(3):
                self._allgather_rows(p[d], d)
            for d in range(3):
                y = [ops.empty(v.shape, v) for v in p]
                ops.ggn_matvec(self.block[d], A, p, self.loss, self.lam, y)
                lo, hi = self.own(d)
                Ap[d][lo:hi] = y[d][lo:hi]
            pap = self._dot_own(p, Ap, acc)
            if not (pap > 0.0 and np.isfinite(pap)) or rz == 0.0:
                break                      # breakdown (or converged): x stays as it is
            alpha = rz / pap
            for d in range(3):
                lo, hi = self.own(d)
                ops.axpby(alpha, p[d][lo:hi].reshape(-1), 1.0, x[d][lo:hi].reshape(-1))
                ops.axpby(-alpha, Ap[d][lo:hi].reshape(-1), 1.0, r[d][lo:hi].reshape(-1))
            precond(r, z)
            rz_new = self._dot_own(r, z, acc)
            beta = rz_new / rz
            rz = rz_new
            hist.append(rz)
            for d in range(3):
                lo, hi = self.own(d)
                ops.axpby(1.0, z[d][lo:hi].reshape(-1), beta, p[d][lo:hi].reshape(-1))
        for d in range(3):
            lo, hi = self.own(d)
            ops.axpby(1.0, x[d][lo:hi].reshape(-1), 1.0, A[d][lo:hi].reshape(-1))
            self._allgather_rows(A[d], d)
        return hist
