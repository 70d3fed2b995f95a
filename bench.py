"""Benchmark of the sparse CP-completion hot path on GB300.

Default workload: order-3 tensor 2^22 x 2^22 x 2^22 with 4e9 distinct uniform
coordinates (the paper's 1e10-nonzero synthetic problem of Sec. 5 scaled to one
GPU), values from a planted rank-16 CP model plus N(0, 0.1^2) noise, FP32
factors, int32 indices, R = 16, lambda = 1e-2, least squares.  The tensor is
generated on the device (keyed-permutation coordinates) and held in a lean
pattern built from the consumed input; the build is timed once and reported
beside the step (the consumed input cannot be sorted twice).

One step = one pass of every hot-path kernel over the tensor, all through the
C ABI of libtc:
  1. TTTP of the current model at the observed entries (tc_tttp),
  2. one ALS sweep: per mode the MTTKRP of the tensor and Solve Factor (Sec. 2.2),
     fused into one pass where the Gram kernel forms the right-hand side
     (tc_als_update),
  3. one generalized Gauss-Newton step: objective and gradient, block-diagonal
     preconditioner, 10 PCG iterations replayed from a CUDA graph, update (Sec. 2.5).
Workloads small enough to draw on the host (``--workload cp3_10k_m10M_r16``)
also rebuild the pattern in every step (tc_pattern_refill).
The headline value is observed entries per second through that step.

``e2e`` runs the same step end to end from host buffers: per step the host
coordinates and values are copied to the device, the pattern is rebuilt, the
step runs, and the factors and objective are copied back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference this method
has), OpenMP build on every host core, on the workload's CPU sample (the same
input as the ``cpu_baseline`` leg).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "cp3_4M_m4B_r16"
CG_ITERS = 10
GEN_CHUNK = 1 << 24


def metric_of(w):
    if w.coords == "feistel":
        return ("observed entries/s through one step (TTTP + ALS sweep + Gauss-Newton step with "
                "10 graph-captured PCG iterations) on the lean pattern, built once (build timed "
                "beside)")
    return ("observed entries/s through one full step (pattern rebuild + TTTP + ALS sweep + "
            "Gauss-Newton step with 10 graph-captured PCG iterations)")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel per workload, from ncu captures, keyed by the hash of the source file
# it was measured on; a stale hash reports null.  Each entry gives the bytes of
# one Gauss-Newton product (three launches of the sweep kernel, one per output
# mode) at the bench's full size, scaled from a smaller capture by the
# nonzero count (the capture size rule keeps multi-pass ncu runs off the full
# workload).
NCU_TRAFFIC = {
    # 4e6-nonzero capture (36.64 MB read per launch) scaled to 1e7
    ("cp3_10k_m10M_r16", "ggn_matvec"): {"bytes": 3 * 36.64e6 * 2.5,
                                         "file": ["paper_1910_02371_gb300/csrc/sweep.cu",
                                                  "paper_1910_02371_gb300/csrc/internal.cuh"],
                                         "src": "f6a6ccaa2cb4861c"},
    # 1e8-nonzero capture at the same 2^22 rows per mode (26.914 GB read +
    # 0.280 GB written per launch: every row gather misses L2 at both sizes)
    # scaled to 4e9
    ("cp3_4M_m4B_r16", "ggn_matvec"): {"bytes": 3 * (26.9144e9 + 0.2805e9) * 40,
                                       "file": ["paper_1910_02371_gb300/csrc/sweep.cu",
                                                "paper_1910_02371_gb300/csrc/internal.cuh"],
                                       "src": "f6a6ccaa2cb4861c"},
}


def src_hash(paths):
    """Hash of the kernel sources a capture was taken on (one path or a list)."""
    h = hashlib.sha256()
    for path in ([paths] if isinstance(paths, str) else paths):
        with open(os.path.join(ROOT, path), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ data
def make_inputs(w, seed_offset=0):
    """Host-drawn coordinates, planted and starting factors; values are made
    on the device by the caller from the planted model."""
    seed = w.seed + seed_offset
    idx = synth.distinct_coords(w.dims, w.nnz, w.coord_dist, seed, w.zipf_s)
    planted = synth.factor_matrices(w.dims, w.rank, w.factor_dist, seed, dtype=np.float64)
    start = synth.perturb(planted, seed)
    return seed, idx, planted, start


def make_device_inputs(w, seed, dev):
    """The tensor of a "feistel" workload generated on the device chunk by
    chunk: coordinates of entries 0 .. nnz-1 from synth.feistel_coords
    (distinct by construction), values = the planted CP model at them
    (plain torch FP64 ops) plus N(0, noise^2) from a seeded torch generator.
    Returns (idx, vals, start factors on the host)."""
    import torch
    planted = synth.factor_matrices(w.dims, w.rank, w.factor_dist, seed)
    start = [a.astype(np.float32).astype(np.float64) for a in synth.perturb(planted, seed)]
    pd = [torch.as_tensor(a, device=dev) for a in planted]
    del planted
    keys = synth.feistel_keys(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    idx = [torch.empty(w.nnz, dtype=torch.int32, device=dev) for _ in range(3)]
    vals = torch.empty(w.nnz, dtype=torch.float32, device=dev)
    for s in range(0, w.nnz, GEN_CHUNK):
        n = min(GEN_CHUNK, w.nnz - s)
        e = torch.arange(s, s + n, dtype=torch.int64, device=dev)
        c = synth.feistel_coords(e, w.feistel_bits, keys)
        m = pd[0][c[0]]
        m *= pd[1][c[1]]
        m *= pd[2][c[2]]
        t = m.sum(1)
        del m
        t += w.noise * torch.randn(n, dtype=torch.float64, device=dev, generator=gen)
        vals[s:s + n] = t.to(torch.float32)
        for d in range(3):
            idx[d][s:s + n] = c[d].to(torch.int32)
        del e, c, t
    del pd
    torch.cuda.synchronize()
    return idx, vals, start


# ------------------------------------------------------------------ CPU sample
def cpu_sample(w):
    """The input both oracle legs time (deterministic): the workload's recipe
    scaled to at most 2^10 rows per mode with the workload's nonzeros per row
    and its rank, so that the per-row and per-nonzero work keep their ratio.
    Returns (dims, idx, t, start factors, description)."""
    import oracle
    f = min(1.0, 1024.0 / max(w.dims))
    dims = tuple(max(1, int(round(I * f))) for I in w.dims)
    n = int(round(w.nnz * f))
    if w.coords == "feistel":
        bits = 10
        dims = (1 << bits,) * 3
        n = int(round(w.nnz / w.dims[0] * dims[0]))
        c = synth.feistel_coords(np.arange(n, dtype=np.int64), bits, synth.feistel_keys(w.seed))
        idx = [np.ascontiguousarray(x.astype(np.int32)) for x in c]
    capped = ""
    if w.coords != "feistel":
        # a skewed shape scaled this way can ask for more nonzeros than the
        # sample has cells: draw at most half of them
        cells = dims[0] * dims[1] * dims[2]
        if n > cells // 2:
            n = cells // 2
            capped = " (capped at half the sample's cells)"
        idx = synth.distinct_coords(dims, n, w.coord_dist, w.seed, w.zipf_s)
    planted = synth.factor_matrices(dims, w.rank, w.factor_dist, w.seed)
    t = synth.observe(oracle.model_entries(dims, idx, planted), w.values, w.seed, w.noise)
    start = synth.perturb(planted, w.seed)
    desc = (f"the workload's recipe scaled to {dims[0]}x{dims[1]}x{dims[2]} with its "
            f"{w.nnz / w.dims[0]:.0f} nonzeros per row{capped}: {n} nonzeros, rank {w.rank}; one "
            f"oracle step (3 counting sorts, TTTP, ALS sweep, GGN step with {CG_ITERS} PCG "
            f"iterations; the oracle's preconditioner re-solves its rows each iteration)")
    return dims, idx, t, start, desc


def oracle_step(dims, idx, t, A, lam, loss):
    """The same step on the FP64 oracle: patterns, TTTP, ALS sweep, GGN step."""
    import oracle
    for d in range(3):
        oracle.counting_sort(idx[d], dims[d])
    oracle.tttp(dims, idx, None, A)
    B = oracle.als_sweep(dims, idx, t, A, lam)
    return oracle.ggn_step(dims, idx, t, B, loss, lam, CG_ITERS)


def cpu_baseline(w, steps=1):
    """The OpenMP oracle on every host core, timed on the CPU sample."""
    import oracle
    oracle.build()
    cores = oracle.set_parallel(True, os.cpu_count() or 1)
    try:
        dims, idx, t, start, desc = cpu_sample(w)
        t0 = time.perf_counter()
        for _ in range(steps):
            oracle_step(dims, idx, t, start, w.lam, w.loss)
        dt = (time.perf_counter() - t0) / steps
    finally:
        oracle.set_parallel(False)
    return {"value": len(idx[0]) / dt, "unit": "nnz/s", "cores": cores, "kind": "oracle",
            "sample": f"subsample: {desc}; {dt:.1f} s per step, OpenMP build on {cores} cores "
                      f"(nproc {os.cpu_count()})"}


# ------------------------------------------------------------------ replicas
# Under torchrun every rank runs an independent replica on its own seeded batch
# of the same shape (no data-path collective); the job's time is the slowest
# rank's and its throughput counts every rank's nonzeros.
def job_time_ms(local_ms, world, device=None):
    """The maximum of the ranks' times (an all-reduce when world > 1)."""
    if world <= 1:
        return local_ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(world, nnz, steps, job_ms):
    """Whole-job throughput: the nonzeros all ranks processed over the job's time."""
    return world * nnz * steps / (job_ms / 1e3)


def algorithmic_bytes(kind, w, es=4):
    """Compulsory DRAM bytes of one call: every nonzero stream read once, factor
    matrices read once, outputs written once (random-gather reuse not credited)."""
    m = w.nnz
    I = w.dims
    R = w.rank
    sumI = sum(I)
    if kind == "tttp":           # j, k, value in, x out; row offsets; factors
        return m * (8 + 2 * es) + 8 * (I[0] + 1) + es * R * sumI
    if kind == "mttkrp":         # per mode, averaged: j, k, value; offsets; factors; out
        return m * (8 + es) + 8 * (sum(I) / 3 + 1) + es * R * (sumI + sumI / 3)
    if kind == "ggn_matvec":     # one pass: j, k (LS needs no value); factors, x, y
        return m * 8 + 8 * (I[0] + 1) + es * R * sumI * 3
    if kind == "solve_factor":   # per mode, averaged: j, k; offsets; other factors, rhs, out
        return m * 8 + 8 * (sum(I) / 3 + 1) + es * R * (sumI + sumI / 3)
    raise ValueError(kind)


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1910_02371_gb300 import build as tcbuild
    tcbuild.build()
    from paper_1910_02371_gb300 import drivers, tc

    w = synth.WORKLOADS[args.workload]
    if args.nnz:
        w = synth.scaled(w, args.nnz,
                         dims=(1 << args.bits,) * 3 if (args.bits and w.coords == "feistel") else None)
    m = w.nnz
    f32 = torch.float32
    lean = w.coords == "feistel"
    seed = w.seed + rank          # independent replicas: each rank its own seeded batch
    build_ms = None
    if lean:
        idx, t, start_h = make_device_inputs(w, seed, dev)
        idx_h = t_h = None
        # host copies for the end-to-end leg, taken before the build consumes them
        idx_pin = t_pin = None
        if not args.quick and args.solve_probe is None and not args.kernel_probe:
            idx_pin = [torch.empty(m, dtype=torch.int32).pin_memory() for _ in range(3)]
            t_pin = torch.empty(m, dtype=f32).pin_memory()
            for dst, src in zip(idx_pin, idx):
                dst.copy_(src)
            t_pin.copy_(t)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p = tc.build_pattern(idx, w.dims, t, dtype=f32, lean=True, consume_input=True)
        e1.record()
        e1.synchronize()
        build_ms = e0.elapsed_time(e1)
        xbuf = t                  # the consumed values buffer holds TTTP's output
    else:
        seed, idx_h, planted_h, start_h = make_inputs(w, seed_offset=rank)
        idx = [torch.as_tensor(c).to(dev) for c in idx_h]
        planted = [torch.as_tensor(a, dtype=f32).to(dev) for a in planted_h]
        # values: planted model at the observed entries (TTTP on a value-less
        # pattern, mapped back to input order) plus seeded noise
        p0 = tc.build_pattern(idx, w.dims, None, dtype=f32)
        x = tc.tttp(p0, planted)
        perm0 = p0.view(0)[1]
        model = torch.empty(m, dtype=f32, device=dev)
        model[perm0] = x
        t_h = synth.observe(model.double().cpu().numpy(), w.values, seed, w.noise).astype(np.float32)
        del p0, x, perm0, model
        t = torch.as_tensor(t_h).to(dev)
        p = tc.build_pattern(idx, w.dims, t, dtype=f32, refillable=True)
        xbuf = torch.empty(m, dtype=f32, device=dev)
    A0 = [torch.as_tensor(a, dtype=f32).to(dev) for a in start_h]
    A = [a.clone() for a in A0]
    rhs = [torch.empty_like(a) for a in A0]
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    if args.solve_probe is not None:
        # Solve Factor on one mode (right-hand side: the MTTKRP of the values),
        # timed alone in each form of --prec (comma-separated, in that order:
        # one untimed call, then --steps timed calls per form; suffixes force
        # a tuning: "@warp" or "@tc05" the R = 64 Gram engine, "@rpwN" the
        # factorization's rows per warp): the command the Solve Factor
        # profiles use
        d = args.solve_probe
        b = tc.mttkrp(p, A, d)
        out = torch.empty_like(b)
        ms = {}
        engines = {"warp": tc.GRAM_WARP_MMA, "tc05": tc.GRAM_TCGEN05}
        for spec in args.prec.split(","):
            form, *opts = spec.split("@")
            eng = rpw = 0
            for o in opts:
                if o in engines:
                    eng = engines[o]
                elif o.startswith("rpw"):
                    rpw = int(o[3:])
                else:
                    raise SystemExit(f"unknown solve-probe option {o!r}")
            tc.set_solve_tuning(f32, 0, reset=True)
            if eng or rpw:
                tc.set_solve_tuning(f32, w.rank, gram_kernel=eng, chol_rows_per_warp=rpw)
            tc.solve_factor(p, A, d, b, w.lam, out=out, prec=form)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                tc.solve_factor(p, A, d, b, w.lam, out=out, prec=form)
            e1.record()
            e1.synchronize()
            ms[spec] = e0.elapsed_time(e1) / args.steps
        tc.set_solve_tuning(f32, 0, reset=True)
        if tc.last_error(p) != tc.OK:
            raise RuntimeError("device error in the Solve Factor probe")
        if rank == 0:
            print(json.dumps({"solve_probe": {"workload": w.name, "nnz": w.nnz, "mode": d,
                                              "rows": w.dims[d], "ms_per_call": ms}}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    if args.kernel_probe:
        # one kernel alone, --warmup untimed calls then --steps timed (CUDA
        # events): the command the per-kernel ncu captures run
        kind = args.kernel_probe
        xs = [torch.randn_like(a) for a in A]
        ys = [torch.empty_like(a) for a in A]
        if kind == "ggn":
            cgp = tc.CG(p, A, w.loss, w.lam, precondition=False)
            fn = lambda: cgp.matvec(xs, ys)
        elif kind == "mttkrp":
            fn = lambda: tc.mttkrp(p, A, 0, out=rhs[0])
        elif kind == "tttp":
            fn = lambda: tc.tttp(p, A, weights=None, out=xbuf)
        elif kind == "grad":
            fn = lambda: tc.loss_grad(p, A, w.loss, w.lam, grads=ys)
        elif kind == "solve":
            tc.mttkrp(p, A, 0, out=rhs[0])
            fn = lambda: tc.solve_factor(p, A, 0, rhs[0], w.lam, out=ys[0], prec=args.prec)
        else:
            raise SystemExit(f"unknown --kernel-probe {kind}")
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        e1.synchronize()
        if tc.last_error(p) != tc.OK:
            raise RuntimeError("device error in the kernel probe")
        if rank == 0:
            print(json.dumps({"kernel_probe": kind, "workload": w.name, "dims": list(w.dims),
                              "nnz": m, "ms_per_call": e0.elapsed_time(e1) / args.steps}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    state = {"p": p, "cg": tc.CG(p, A, w.loss, w.lam)}

    def step():
        pp, cg = state["p"], state["cg"]
        if not lean:
            tc.refill_pattern(pp, idx, t)
        for a, a0 in zip(A, A0):
            a.copy_(a0)
        tc.tttp(pp, A, weights=None, out=xbuf)
        drivers.als_sweep(pp, A, w.lam, rhs=rhs, prec=args.prec)
        cg.ggn_step(CG_ITERS, loss_out=loss)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if tc.last_error(p) != tc.OK:
        raise RuntimeError("device error during warm-up")

    # ---- timed region: K steps, events on the launching stream
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = tc.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(st)
            step()
            ev[k][1].record(st)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    launches = tc.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = job_time_ms(total_ms, world, dev)
    value = job_value(world, m, args.steps, total_ms)
    if tc.last_error(p) != tc.OK:
        raise RuntimeError("device error in the timed steps")
    if args.quick:      # timed steps only (for profiler runs)
        if rank == 0:
            print(json.dumps({"metric": metric_of(w), "value": value, "unit": "nnz/s",
                              "ms_per_step": total_ms / args.steps, "gpu_launches": int(launches),
                              "build_ms": build_ms,
                              "config": {"workload": w.name, "nnz": w.nnz}}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- per-kernel breakdown (same inputs, events around each call)
    big = m > 500_000_000

    def timed(fn, reps=5):
        if big:
            reps = 1
        else:
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        b.synchronize()
        return a.elapsed_time(b) / reps

    cg = state["cg"]
    for a, a0 in zip(A, A0):
        a.copy_(a0)
    xv = [torch.randn_like(a) for a in A]
    yv = [torch.empty_like(a) for a in A]
    gb = [torch.empty_like(a) for a in A]
    dxv = [torch.empty_like(a) for a in A]
    kern = {}
    if not lean:
        kern["pattern_rebuild"] = timed(lambda: tc.refill_pattern(p, idx, t))
    kern["tttp"] = timed(lambda: tc.tttp(p, A, weights="values", out=xbuf))
    for d in range(3):
        kern[f"mttkrp_mode{d}"] = timed(lambda d=d: tc.mttkrp(p, A, d, out=rhs[d]))
    for d in range(3):
        kern[f"solve_factor_mode{d}"] = timed(
            lambda d=d: tc.solve_factor(p, A, d, rhs[d], w.lam, out=yv[d]))
    for d in range(3):   # the step's ALS: right-hand side formed in the Gram pass
        kern[f"als_update_mode{d}"] = timed(
            lambda d=d: tc.als_update(p, A, d, w.lam, out=yv[d], prec=args.prec))
    kern["loss_grad"] = timed(lambda: tc.loss_grad(p, A, w.loss, w.lam, grads=gb))
    kern["ggn_matvec"] = timed(lambda: tc.ggn_matvec(p, A, xv, w.loss, w.lam, y=yv))
    # the product as the PCG runs it (interleaved factor / direction rows)
    kern["ggn_matvec_pcg"] = timed(lambda: cg.matvec(xv, yv))
    kern["precond_setup"] = timed(lambda: cg.setup())
    kern[f"pcg_{CG_ITERS}_iters_graph"] = timed(lambda: cg.solve(gb, CG_ITERS, dx=dxv))
    B = [a.clone() for a in A0]
    kern["als_sweep"] = timed(lambda: drivers.als_sweep(p, B, w.lam, rhs=rhs, prec=args.prec))
    kern["ggn_step"] = timed(lambda: cg.ggn_step(CG_ITERS, loss_out=loss), reps=3)
    del B
    torch.cuda.synchronize()
    if tc.last_error(p) not in (tc.OK,):
        raise RuntimeError("device error in breakdown")

    # ---- optional: one ALS sweep in each Solve Factor precision form, from the
    # same start, with its time and its objective against the refined FP32 form
    als_forms = None
    if args.als_forms:
        als_forms = {}
        fval = {}
        for form in ("fp32_refine", "fp32", "tf32_refine", "tf32_refine2", "bf16_refine",
                     "fp32_refine_chol32", "tf32_refine_chol32", "bf16_refine_chol32"):
            B = [a.clone() for a in A0]

            def sweep_from_start(form=form, B=B):
                for b, a0 in zip(B, A0):     # (three factor copies, negligible)
                    b.copy_(a0)
                drivers.als_sweep(p, B, w.lam, rhs=rhs, prec=form)

            ms = timed(sweep_from_start, reps=3)
            sweep_from_start()
            f_t, _ = tc.loss_grad(p, B, "ls", w.lam, want_grad=False)
            fval[form] = f_t.item()
            als_forms[form] = {"als_sweep_ms": ms}
        for form in als_forms:
            als_forms[form]["objective_rel_to_fp32_refine"] = abs(fval[form] - fval["fp32_refine"]) / \
                abs(fval["fp32_refine"])
        if tc.last_error(p) not in (tc.OK,):
            raise RuntimeError("device error in the precision forms")

    # ---- roofline of the dominant kernel
    # the step's time by kernel family (the ALS sweep runs fused updates:
    # MTTKRP folded into Solve Factor's Gram pass)
    share = {
        "ggn_matvec": CG_ITERS * kern["ggn_matvec_pcg"],
        "solve_factor": sum(kern[f"als_update_mode{d}"] for d in range(3)) + kern["precond_setup"],
        "tttp": kern["tttp"],
        "loss_grad": kern["loss_grad"],
    }
    if not lean:
        share["pattern_rebuild"] = kern["pattern_rebuild"]
    dominant = max(share, key=share.get)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    def roof(kind, ms):
        b = algorithmic_bytes(kind, w)
        return {"bound": "hbm", "achieved": b / (ms / 1e3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "frac": b / (ms / 1e3) / 1e9 / hbm_peak,
                "algorithmic_bytes": b, "ms": ms}

    roofs = {
        "ggn_matvec": roof("ggn_matvec", kern["ggn_matvec_pcg"]),
        "tttp": roof("tttp", kern["tttp"]),
        "mttkrp": roof("mttkrp", sum(kern[f"mttkrp_mode{d}"] for d in range(3)) / 3),
        "solve_factor": roof("solve_factor", sum(kern[f"solve_factor_mode{d}"] for d in range(3)) / 3),
    }
    main_kind = dominant if dominant in roofs else "ggn_matvec"
    traffic = NCU_TRAFFIC.get((w.name, main_kind))
    roofline = dict(roofs[main_kind])
    roofline["kernel"] = main_kind
    if main_kind == "ggn_matvec":
        roofline["note"] = ("one Gauss-Newton product = 3 launches of the interleaved sweep kernel "
                            "(one per output mode); achieved = one-pass algorithmic bytes / time "
                            "of the product")
    roofline["peak_source"] = peak_src
    roofline["traffic"] = (traffic["bytes"] if traffic and traffic["src"] == src_hash(traffic["file"])
                           else None)

    # ---- the dominant kernel's measured DRAM traffic per launch (ncu) over its
    # time, against the same peak: the algorithmic count above credits each
    # factor row once, while every nonzero's row gathers go to DRAM when the
    # factors are larger than L2
    dram = None
    if roofline["traffic"]:
        rate = roofline["traffic"] / (roofline["ms"] / 1e3) / 1e9
        dram = {"bound": "hbm", "achieved": rate, "peak": hbm_peak, "unit": "GB/s",
                "frac": rate / hbm_peak, "traffic": roofline["traffic"], "kernel": main_kind,
                "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch set "
                        "(scaled from the capture size to this workload) / the event-timed duration"}

    # ---- end to end through the C ABI with host buffers
    if not lean:
        idx_pin = [torch.as_tensor(c).pin_memory() for c in idx_h]
        t_pin = torch.as_tensor(t_h).pin_memory()
    A0_pin = [a.cpu().pin_memory() for a in A0]
    out_pin = [torch.empty_like(a, device="cpu").pin_memory() for a in A0]
    loss_pin = torch.empty(1, dtype=torch.float64).pin_memory()
    h2d = sum(c.numel() * c.element_size() for c in idx_pin) + t_pin.numel() * 4 + \
        sum(a.numel() * 4 for a in A0_pin)
    d2h = sum(a.numel() * 4 for a in out_pin) + 8

    def e2e_step():
        if lean:
            # the lean pattern cannot be refilled: free it (and its solver),
            # copy the input, build again from the consumed input
            state["cg"] = None
            state["p"] = None
        for dst, src in zip(idx, idx_pin):
            dst.copy_(src, non_blocking=True)
        t.copy_(t_pin, non_blocking=True)
        for dst, src in zip(A0, A0_pin):
            dst.copy_(src, non_blocking=True)
        if lean:
            state["p"] = tc.build_pattern(idx, w.dims, t, dtype=f32, lean=True, consume_input=True)
            state["cg"] = tc.CG(state["p"], A, w.loss, w.lam)
        step()
        for dst, src in zip(out_pin, A):
            dst.copy_(src, non_blocking=True)
        loss_pin.copy_(loss, non_blocking=True)

    del cg, p, xv, yv, gb, dxv
    torch.cuda.empty_cache()
    e2e_steps = min(args.steps, 3) if lean else args.steps
    for _ in range(1 if lean else 2):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = job_time_ms((time.perf_counter() - t0) * 1e3, world, dev)
    e2e_val = job_value(world, m, e2e_steps, e2e_ms)
    if tc.last_error(state["p"]) != tc.OK:
        raise RuntimeError("device error in the end-to-end steps")

    result = {
        "metric": metric_of(w),
        "value": value,
        "unit": "nnz/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": ("synthetic (seeded keyed-permutation coordinates, planted CP factors, noise), "
                 "generated on the device" if lean else
                 "synthetic (seeded Philox): coordinates, planted CP factors, noise"),
        "config": {
            "workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "rank": w.rank,
            "lambda": w.lam, "loss": w.loss, "cg_iters": CG_ITERS,
            "pattern": "lean, built once from the consumed input" if lean else
                       "full, rebuilt in every step",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (per-step nonzero streams ~%.0f MB)" % (m * 36 / 1e6),
        },
        "wall_s_timed": wall,
        "kernels_ms": kern,
        "kernels_nnz_per_s": {k: m / (v / 1e3) for k, v in kern.items()},
        "als_sweep_s": kern["als_sweep"] / 1e3,
        "ggn_step_s": kern["ggn_step"] / 1e3,
        "time_share_ms": share,
        "roofline": roofline,
        "dram_roofline": dram,
        "rooflines": roofs,
        "e2e": {"value": e2e_val, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / e2e_steps,
                "steps": e2e_steps,
                "includes": ("host-to-device copy of the coordinates, values and starting "
                             "factors, pattern build, the step, copy of the factors and "
                             "objective back (host clock)" if lean else
                             "host-to-device copy of the coordinates, values and starting "
                             "factors, the step (with its rebuild), copy of the factors and "
                             "objective back (CUDA events)")},
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
    }
    if build_ms is not None:
        result["build_ms"] = build_ms
        result["build_nnz_per_s"] = m / (build_ms / 1e3)
    if args.prec != "fp32":
        result["config"]["solve_factor_form"] = args.prec
    if als_forms is not None:
        result["als_sweep_forms"] = als_forms
    del state
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ oracle arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = synth.WORKLOADS[args.workload]
    cores = oracle.set_parallel(True, os.cpu_count() or 1)
    dims, idx, t, start, desc = cpu_sample(w)
    n = len(idx[0])
    for _ in range(args.warmup):
        oracle_step(dims, idx, t, start, w.lam, w.loss)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(dims, idx, t, start, w.lam, w.loss)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = f"subsample: {desc}; FP64 oracle, OpenMP build on {cores} cores (nproc {os.cpu_count()})"
    print(json.dumps({
        "impl": "reference", "metric": metric_of(w), "value": value, "unit": "nnz/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "rank": w.rank,
                   "lambda": w.lam, "loss": w.loss, "cg_iters": CG_ITERS,
                   "sample_dims": list(dims), "sample_nnz": n},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="setup, warm-up and the timed steps only (for profiler runs)")
    ap.add_argument("--nnz", type=int, default=0,
                    help="use the first NNZ coordinates of the workload (smaller profiling case)")
    ap.add_argument("--bits", type=int, default=0,
                    help="with --nnz, on the generated workload: dims 2^BITS per mode")
    ap.add_argument("--kernel-probe", default=None,
                    choices=["ggn", "mttkrp", "tttp", "grad", "solve"],
                    help="time one kernel alone (--warmup + --steps calls) and exit")
    ap.add_argument("--prec", default="fp32",
                    help="Solve Factor precision form of the ALS sweep (tc.PRECS; default fp32)")
    ap.add_argument("--solve-probe", type=int, default=None, metavar="MODE",
                    help="time Solve Factor on MODE (--steps calls per form of --prec, "
                         "comma-separated) and exit")
    ap.add_argument("--als-forms", action="store_true",
                    help="also time one ALS sweep in every precision form and report the "
                         "objective of each against the refined FP32 form")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
