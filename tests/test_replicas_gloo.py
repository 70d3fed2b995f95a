"""The benchmark's multi-rank path on CPU: two gloo ranks, as torchrun would
start them (RANK / WORLD_SIZE / MASTER_* in the environment).  Each rank draws
its own seeded batch of the same shape, the job's time is the maximum over
ranks, the whole-job value counts every rank's nonzeros, and the reference
arm runs on rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.scaled(synth.WORKLOADS["cp3_10k_m10M_r16"], 5000)
    seed, idx, planted, start = bench.make_inputs(w, seed_offset=rank)
    digest = [int(seed), [int(c.sum()) for c in idx], float(planted[0].sum())]
    # the ranks' timed regions differ; the job takes the slowest
    local_ms = 10.0 + 5.0 * rank
    job_ms = bench.job_time_ms(local_ms, world)
    value = bench.job_value(world, w.nnz, 4, job_ms)
    dist.barrier()
    # the reference arm: rank 0 runs and prints, the others return at once
    buf = io.StringIO()
    args = type("A", (), dict(workload="cp3_200_m40k_r5", steps=1, warmup=0))()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(args)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(digest=digest, job_ms=job_ms, value=value, ref_out=buf.getvalue()), f)


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    # independent replicas: different seeds and draws, same shape
    assert r[0]["digest"][0] != r[1]["digest"][0]
    assert r[0]["digest"][1] != r[1]["digest"][1]
    # max over ranks, and the value from it counts both ranks' nonzeros
    assert r[0]["job_ms"] == r[1]["job_ms"] == 15.0
    assert r[0]["value"] == r[1]["value"] == pytest.approx(2 * 5000 * 4 / 15e-3)
    # rank 1 ran no reference work and printed nothing
    assert r[1]["ref_out"] == ""


def test_replica_inputs_are_deterministic():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.scaled(synth.WORKLOADS["cp3_10k_m10M_r16"], 3000)
    a = bench.make_inputs(w, seed_offset=1)
    b = bench.make_inputs(w, seed_offset=1)
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    assert bench.job_time_ms(7.5, 1) == 7.5
