"""The row-sharded driver (paper_1910_02371_gb300.sharded) on two gloo
processes on the CPU.  The per-process kernels are the FP64 oracle's routines
(the test's stand-in for one GPU per process), so what is checked is the
sharding itself: the nonzero-balanced row ranges, each process's mode blocks,
the all-gather of the solved rows after every Solve Factor, the all-reduced
objective, and the row-sharded PCG with the direction all-gathered before each
product and its two inner products all-reduced (Sec. 3.2, 3.4, 2.5).  The
sharded ALS sweep must equal the single-process oracle sweep bit for bit (every
row is solved from the same nonzeros in the same order), and the sharded
Gauss-Newton step the single-process oracle step up to the order of the
inner products' partial sums."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleOps:
    """Per-process kernels of the sharded driver made of oracle routines (FP64,
    CPU torch tensors in and out)."""

    def __init__(self):
        import oracle
        self.o = oracle

    def build(self, idx, vals, dims):
        return dict(idx=[c.numpy().astype(np.int32) for c in idx], t=vals.numpy().astype(np.float64),
                    dims=tuple(dims))

    @staticmethod
    def _np(A):
        return [a.numpy() for a in A]

    def mttkrp(self, h, A, d, out):
        out.copy_(torch.from_numpy(self.o.mttkrp(h["dims"], h["idx"], h["t"], self._np(A), d)))

    def solve_factor(self, h, A, d, rhs, lam, out, prec="fp32"):
        res, _, rc = self.o.solve_factor(h["dims"], h["idx"], None, self._np(A), d, rhs.numpy(), lam)
        assert rc == 0
        out.copy_(torch.from_numpy(res))

    def als_update(self, h, A, d, lam, out, prec="fp32"):
        rhs = torch.from_numpy(self.o.mttkrp(h["dims"], h["idx"], h["t"], self._np(A), d))
        self.solve_factor(h, A, d, rhs, lam, out, prec)

    def loss(self, h, A, loss, lam):
        f, _ = self.o.loss_grad(h["dims"], h["idx"], h["t"], self._np(A), loss, lam, want_grad=False)
        return torch.tensor([f], dtype=torch.float64)

    def grad(self, h, A, loss, lam, d, out):
        _, g = self.o.loss_grad(h["dims"], h["idx"], h["t"], self._np(A), loss, lam)
        out.copy_(torch.from_numpy(g[d]))

    def ggn_matvec(self, h, A, x, loss, lam, y):
        ys = self.o.ggn_matvec(h["dims"], h["idx"], h["t"], self._np(A), loss, lam, self._np(x))
        for yd, v in zip(y, ys):
            yd.copy_(torch.from_numpy(v))

    def precond(self, h, A, loss, lam):
        return (h, [a.numpy().copy() for a in A], loss, lam)

    def precond_apply(self, pc, r, z):
        h, A, loss, lam = pc
        zs = self.o.precond_apply(h["dims"], h["idx"], h["t"], A, loss, lam, self._np(r))
        for zd, v in zip(z, zs):
            zd.copy_(torch.from_numpy(v))

    def axpby(self, alpha, x, beta, y):
        y.copy_(alpha * x + beta * y)

    def dot(self, x, y, out, accumulate):
        v = float(np.dot(x.numpy(), y.numpy()))
        out.fill_(v + (float(out.item()) if accumulate else 0.0))

    def empty(self, shape, like):
        return torch.empty(shape, dtype=like.dtype)


DIMS = (41, 37, 29)


def _problem():
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    idx = synth.distinct_coords(DIMS, 4000, ("zipf", "uniform", "uniform"), 77)
    planted = synth.factor_matrices(DIMS, 4, "normal", 77)
    t = synth.observe(oracle.model_entries(DIMS, idx, planted), "noise", 77, 0.1)
    start = synth.perturb(planted, 77)
    return idx, t, start


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1910_02371_gb300.sharded import ShardedCP
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx, t, start = _problem()
    sh = ShardedCP(OracleOps(), [torch.from_numpy(c) for c in idx], torch.from_numpy(t), DIMS,
                   "ls", 0.05)
    A = [torch.from_numpy(a.copy()) for a in start]
    f0 = sh.objective(A)
    sh.als_sweep(A)
    f_als = sh.objective(A)
    als = [a.numpy().tolist() for a in A]
    hist = sh.ggn_step(A, 6)
    f_gn = sh.objective(A)
    out = dict(ranges=sh.ranges, block_nnz=[int(len(b["t"])) for b in sh.block], f0=f0,
               f_als=f_als, als=als, gn=[a.numpy().tolist() for a in A], hist=hist, f_gn=f_gn)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(out, f)


def test_partition_rows_balances_nonzeros():
    from paper_1910_02371_gb300.sharded import partition_rows
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        counts = rng.zipf(1.5, size=500).clip(max=400)
        rg = partition_rows(counts, world)
        assert rg[0][0] == 0 and rg[-1][1] == 500
        assert all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
        share = [int(counts[lo:hi].sum()) for lo, hi in rg]
        assert sum(share) == counts.sum()
        # a range overshoots its even share by at most one row
        target = counts.sum() / world
        cum = np.cumsum(share)
        for k in range(world - 1):
            assert abs(cum[k] - (k + 1) * target) <= counts.max()
    # no nonzeros at all: the ranges still cover the rows
    assert partition_rows(np.zeros(7, np.int64), 2) == [(0, 0), (0, 7)]


def test_sharded_als_and_gauss_newton_two_processes(tmp_path):
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    idx, t, start = _problem()
    # the processes agree, and every mode's blocks partition the nonzeros
    for d in range(3):
        assert res[0]["ranges"][d] == res[1]["ranges"][d]
        assert res[0]["block_nnz"][d] + res[1]["block_nnz"][d] == len(t)
        assert 0 < res[0]["block_nnz"][d] < len(t)
    for key in ("f0", "f_als", "f_gn"):
        assert res[0][key] == pytest.approx(res[1][key], rel=1e-14)
    # objective: the all-reduced blocks equal the whole tensor's
    f0 = oracle.objective(DIMS, idx, t, start, "ls", 0.05)
    assert res[0]["f0"] == pytest.approx(f0, rel=1e-13)
    # ALS sweep: bit for bit the single-process oracle sweep
    als = oracle.als_sweep(DIMS, idx, t, start, 0.05)
    for d in range(3):
        for r in range(world):
            assert np.array_equal(np.array(res[r]["als"][d]), als[d])
    # Gauss-Newton step (6 PCG iterations) from the swept factors
    gn = oracle.ggn_step(DIMS, idx, t, als, "ls", 0.05, 6)
    for d in range(3):
        for r in range(world):
            got = np.array(res[r]["gn"][d])
            assert np.linalg.norm(got - gn[d]) <= 1e-11 * np.linalg.norm(gn[d])
    assert res[0]["f_gn"] < res[0]["f_als"]
