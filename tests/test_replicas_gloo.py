"""The multi-process path of bench.py on the CPU (gloo, world size 2).

The source problems and the Rayleigh-Ritz step do not shard across GPUs in this
build: `bench.py --gpus N` runs N independent replicas, one per rank, with no
collective on the data path.  What the ranks share is host logic: every rank
works on its own seeded problem, the job's time is the slowest rank's
(max-reduction behind a barrier), the whole-job value counts all ranks' units,
and only rank 0 runs the oracle leg.  These run here as two gloo processes.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    # each replica its own seeded problem
    p = bench.problem(rank)
    # per-rank "timings": the job takes the slowest
    ms = 10.0 + 5.0 * rank
    dist.barrier()
    t_max = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.replica_throughput(1000, ws, t_max)
    # the oracle leg: rank 0 alone (the others return at once)
    ran_reference = False
    if rank != 0:

        class A:
            steps, warmup = 1, 3

        bench.run_reference(A, ws, rank)  # returns without work on rank != 0
    else:
        ran_reference = True
    out[rank] = (float(p.U0[:5, 0].sum()), t_max, value, ran_reference)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_share_only_the_timing():
    ws = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    seeds0, t0, v0, ref0 = out[0]
    seeds1, t1, v1, ref1 = out[1]
    assert seeds0 != seeds1  # independent replicas draw their own initial orbitals
    assert t0 == t1 == 15.0  # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(2 * 1000 / 15e-3)
    assert ref0 and not ref1


def test_single_process_needs_no_collective():
    import bench

    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.replica_throughput(500, 1, 2.0) == pytest.approx(500 / 2e-3)
    a, b = bench.problem(0), bench.problem(1)
    assert a.n == b.n and a.N == b.N and not np.allclose(a.U0, b.U0)
