"""Benchmark of the sparse CP-completion hot path on GB300.

One step = one pass of every hot-path kernel over one batch of synthetic
input, all through the C ABI of libtc:
  1. rebuild the per-mode sorted pattern of the batch (tc_pattern_refill),
  2. TTTP of the current model at the observed entries (tc_tttp),
  3. one ALS sweep: per mode MTTKRP of the tensor, then Solve Factor (Sec. 2.2),
  4. one generalized Gauss-Newton step: objective and gradient, block-diagonal
     preconditioner, 10 PCG iterations replayed from a CUDA graph, update (Sec. 2.5).
The headline value is observed entries per second through that step.

Default workload: order-3 tensor 10^4 x 10^4 x 10^4 with 10^7 distinct uniform
coordinates, values from a planted rank-16 CP model plus N(0, 0.1^2) noise,
FP32 factors, int32 indices, R = 16, lambda = 1e-2, least squares.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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

WORKLOAD = "cp3_10k_m10M_r16"
CG_ITERS = 10
METRIC = ("observed entries/s through one full step (pattern rebuild + TTTP + ALS sweep + "
          "Gauss-Newton step with 10 graph-captured PCG iterations)")

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel from one ncu capture, keyed by the hash of the source file it was
# measured on; a stale hash reports null.  The Gauss-Newton sweep was captured
# at 4e6 nonzeros (36.64 MB read, ~0 written per launch; the capture size rule
# keeps multi-pass ncu runs off the full workload) and scaled by the nonzeros
# to 1e7: three launches per product.
NCU_TRAFFIC = {
    "ggn_matvec": {"bytes": 3 * 36.65e6 * 2.5, "file": "paper_1910_02371_gb300/csrc/sweep.cu",
                   "src": "1d03ab541fb6d2df"},
}


def src_hash(path):
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


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
    """Coordinates, planted and starting factors (host); values are made on the
    device by the caller from the planted model."""
    seed = w.seed + seed_offset
    idx = synth.distinct_coords(w.dims, w.nnz, w.coord_dist, seed, w.zipf_s)
    planted = synth.factor_matrices(w.dims, w.rank, w.factor_dist, seed, dtype=np.float64)
    start = synth.perturb(planted, seed)
    return seed, idx, planted, start


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
        w = synth.scaled(w, args.nnz)
    # independent replicas: each rank its own seeded batch of the same shape
    seed, idx_h, planted_h, start_h = make_inputs(w, seed_offset=rank)
    m = w.nnz
    f32 = torch.float32
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
    A0 = [torch.as_tensor(a, dtype=f32).to(dev) for a in start_h]
    A = [a.clone() for a in A0]
    rhs = [torch.empty_like(a) for a in A0]
    xbuf = torch.empty(m, dtype=f32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    if args.solve_probe is not None:
        # Solve Factor on one mode (right-hand side: the MTTKRP of the values),
        # timed alone in each form of --prec (comma-separated, in that order:
        # one untimed call, then --steps timed calls per form): the command the
        # Solve Factor profiles use
        d = args.solve_probe
        b = tc.mttkrp(p, A, d)
        out = torch.empty_like(b)
        ms = {}
        for form in args.prec.split(","):
            tc.solve_factor(p, A, d, b, w.lam, out=out, prec=form)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                tc.solve_factor(p, A, d, b, w.lam, out=out, prec=form)
            e1.record()
            e1.synchronize()
            ms[form] = e0.elapsed_time(e1) / args.steps
        if tc.last_error(p) != tc.OK:
            raise RuntimeError("device error in the Solve Factor probe")
        if rank == 0:
            print(json.dumps({"solve_probe": {"workload": w.name, "nnz": w.nnz, "mode": d,
                                              "rows": w.dims[d], "ms_per_call": ms}}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    cg = tc.CG(p, A, w.loss, w.lam)

    def step():
        tc.refill_pattern(p, idx, t)
        for a, a0 in zip(A, A0):
            a.copy_(a0)
        tc.tttp(p, A, weights=None, out=xbuf)
        drivers.als_sweep(p, A, w.lam, rhs=rhs, prec=args.prec)
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
    if args.quick:      # timed steps only (for profiler runs)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "nnz/s",
                              "ms_per_step": total_ms / args.steps, "gpu_launches": int(launches),
                              "config": {"workload": w.name, "nnz": w.nnz}}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- per-kernel breakdown (same inputs, events around each call)
    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        b.synchronize()
        return a.elapsed_time(b) / reps

    for a, a0 in zip(A, A0):
        a.copy_(a0)
    xv = [torch.randn_like(a) for a in A]
    yv = [torch.empty_like(a) for a in A]
    gb = [torch.empty_like(a) for a in A]
    dxv = [torch.empty_like(a) for a in A]
    kern = {
        "pattern_rebuild": timed(lambda: tc.refill_pattern(p, idx, t)),
        "tttp": timed(lambda: tc.tttp(p, A, weights="values", out=xbuf)),
    }
    for d in range(3):
        kern[f"mttkrp_mode{d}"] = timed(lambda d=d: tc.mttkrp(p, A, d, out=rhs[d]))
    for d in range(3):
        kern[f"solve_factor_mode{d}"] = timed(
            lambda d=d: tc.solve_factor(p, A, d, rhs[d], w.lam, out=yv[d]))
    kern["loss_grad"] = timed(lambda: tc.loss_grad(p, A, w.loss, w.lam, grads=gb))
    kern["ggn_matvec"] = timed(lambda: tc.ggn_matvec(p, A, xv, w.loss, w.lam, y=yv))
    # the product as the PCG runs it (interleaved factor / direction rows)
    kern["ggn_matvec_pcg"] = timed(lambda: cg.matvec(xv, yv))
    kern["precond_setup"] = timed(lambda: cg.setup())
    kern[f"pcg_{CG_ITERS}_iters_graph"] = timed(lambda: cg.solve(gb, CG_ITERS, dx=dxv))
    B = [a.clone() for a in A0]
    kern["als_sweep"] = timed(lambda: drivers.als_sweep(p, B, w.lam, rhs=rhs, prec=args.prec))
    kern["ggn_step"] = timed(lambda: cg.ggn_step(CG_ITERS, loss_out=loss), reps=3)
    torch.cuda.synchronize()
    if tc.last_error(p) not in (tc.OK,):
        raise RuntimeError("device error in breakdown")

    # ---- optional: one ALS sweep in each Solve Factor precision form, from the
    # same start, with its time and its objective against the refined FP32 form
    als_forms = None
    if args.als_forms:
        als_forms = {}
        fval = {}
        for form in ("fp32_refine", "fp32", "tf32_refine", "bf16_refine", "fp32_refine_chol32",
                     "tf32_refine_chol32", "bf16_refine_chol32"):
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

    # ---- roofline of the dominant kernel (Gauss-Newton matvec: 11 per step)
    share = {
        "ggn_matvec": CG_ITERS * kern["ggn_matvec_pcg"],
        "solve_factor": sum(kern[f"solve_factor_mode{d}"] for d in range(3)) + kern["precond_setup"],
        "mttkrp": sum(kern[f"mttkrp_mode{d}"] for d in range(3)),
        "tttp": kern["tttp"],
        "pattern_rebuild": kern["pattern_rebuild"],
        "loss_grad": kern["loss_grad"],
    }
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
        "mttkrp": roof("mttkrp", share["mttkrp"] / 3),
        "solve_factor": roof("solve_factor", sum(kern[f"solve_factor_mode{d}"] for d in range(3)) / 3),
    }
    main_kind = dominant if dominant in roofs else "ggn_matvec"
    traffic = NCU_TRAFFIC.get(main_kind)
    roofline = dict(roofs[main_kind])
    roofline["kernel"] = main_kind
    if main_kind == "ggn_matvec":
        roofline["note"] = ("one Gauss-Newton product = 3 launches of the interleaved sweep kernel "
                            "(one per output mode); achieved = one-pass algorithmic bytes / time "
                            "of the product")
    roofline["peak_source"] = peak_src
    roofline["traffic"] = (traffic["bytes"] if traffic and traffic["src"] == src_hash(traffic["file"])
                           else None)

    # ---- end to end through the C ABI with host buffers
    idx_pin = [torch.as_tensor(c).pin_memory() for c in idx_h]
    t_pin = torch.as_tensor(t_h).pin_memory()
    A0_pin = [a.cpu().pin_memory() for a in A0]
    out_pin = [torch.empty_like(a, device="cpu").pin_memory() for a in A0]
    loss_pin = torch.empty(1, dtype=torch.float64).pin_memory()
    h2d = sum(c.numel() * c.element_size() for c in idx_pin) + t_pin.numel() * 4 + \
        sum(a.numel() * 4 for a in A0_pin)
    d2h = sum(a.numel() * 4 for a in out_pin) + 8

    def e2e_step():
        for dst, src in zip(idx, idx_pin):
            dst.copy_(src, non_blocking=True)
        t.copy_(t_pin, non_blocking=True)
        for dst, src in zip(A0, A0_pin):
            dst.copy_(src, non_blocking=True)
        step()
        for dst, src in zip(out_pin, A):
            dst.copy_(src, non_blocking=True)
        loss_pin.copy_(loss, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        e2e_step()
    e1.record(st)
    e1.synchronize()
    e2e_ms = job_time_ms(e0.elapsed_time(e1), world, dev)
    e2e_val = job_value(world, m, args.steps, e2e_ms)

    result = {
        "metric": METRIC,
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
        "data": "synthetic (seeded Philox): coordinates, planted CP factors, noise",
        "config": {
            "workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "rank": w.rank,
            "lambda": w.lam, "loss": w.loss, "cg_iters": CG_ITERS,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (per-step nonzero streams ~%.0f MB)" % (m * 32 / 1e6),
        },
        "wall_s_timed": wall,
        "kernels_ms": kern,
        "kernels_nnz_per_s": {k: m / (v / 1e3) for k, v in kern.items()},
        "als_sweep_s": kern["als_sweep"] / 1e3,
        "ggn_step_s": kern["ggn_step"] / 1e3,
        "time_share_ms": share,
        "roofline": roofline,
        "rooflines": roofs,
        "e2e": {"value": e2e_val, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
    }
    if args.prec != "fp32":
        result["config"]["solve_factor_form"] = args.prec
    if als_forms is not None:
        result["als_sweep_forms"] = als_forms
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, idx_h, t_h.astype(np.float64), start_h,
                                              target_s=args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ oracle arm
def oracle_step(dims, idx, t, A, lam, loss):
    """The same step on the FP64 oracle: patterns, TTTP, ALS sweep, GGN step."""
    import oracle
    for d in range(3):
        oracle.counting_sort(idx[d], dims[d])
    oracle.tttp(dims, idx, None, A)
    B = oracle.als_sweep(dims, idx, t, A, lam)
    return oracle.ggn_step(dims, idx, t, B, loss, lam, CG_ITERS)


def sample_sizes(w, target_s, steps=1):
    """Prefix sample size whose oracle step takes about target_s seconds: the
    step time is fitted as a + b n from two small samples (the per-row solves
    give a fixed part)."""
    import oracle  # noqa: F401
    A = synth.init_factors(w.dims, w.rank, w.seed)
    rng = np.random.default_rng(0)
    sizes = (20_000, 80_000)
    idx = synth.distinct_coords(w.dims, sizes[-1], w.coord_dist, w.seed)
    times = []
    for n in sizes:
        t0 = time.perf_counter()
        oracle_step(w.dims, [c[:n] for c in idx], rng.standard_normal(n), A, w.lam, w.loss)
        times.append(time.perf_counter() - t0)
    b = max((times[1] - times[0]) / (sizes[1] - sizes[0]), 1e-9)
    a = max(times[0] - b * sizes[0], 0.0)
    n = int((target_s / steps - a) / b)
    return max(sizes[0], min(w.nnz, n))


def cpu_baseline(w, idx, t, A, target_s=15.0):
    import oracle
    oracle.build()
    n = sample_sizes(w, target_s)
    sub = [c[:n] for c in idx]
    t0 = time.perf_counter()
    oracle_step(w.dims, sub, t[:n], A, w.lam, w.loss)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "nnz/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {w.nnz} coordinates (draw order), full dims and rank, "
                      f"one oracle step (3 counting sorts, TTTP, ALS sweep, GGN step with "
                      f"{CG_ITERS} PCG iterations) in {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = synth.WORKLOADS[args.workload]
    budget = 150.0
    n = sample_sizes(w, budget / max(1, args.steps + args.warmup))
    seed, idx, planted, start = make_inputs(synth.scaled(w, n))
    t = synth.observe(oracle.model_entries(w.dims, idx, planted), w.values, seed, w.noise)
    for _ in range(args.warmup):
        oracle_step(w.dims, idx, t, start, w.lam, w.loss)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(w.dims, idx, t, start, w.lam, w.loss)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = (f"{n} coordinates of workload {w.name} (full dims and rank) per step; FP64 "
              f"oracle, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Philox)",
        "config": {"workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "rank": w.rank,
                   "lambda": w.lam, "loss": w.loss, "cg_iters": CG_ITERS},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="setup, warm-up and the timed steps only (for profiler runs)")
    ap.add_argument("--nnz", type=int, default=0,
                    help="use the first NNZ coordinates of the workload (smaller profiling case)")
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
