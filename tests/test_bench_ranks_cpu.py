"""The N > 1 launch of bench.py on CPU (gloo, world size 2): replicas only.

* every rank draws its own replica (seed = rank) of the same workload shape;
* the job's step time is the slowest rank's, and the job's rate counts the
  units of all ranks (whole-job throughput, weak scaling);
* the reference arm runs on rank 0 alone; the other ranks return at once.
"""
import os
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")
dist_mod = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w = bench.dist_setup()
        step_ms = 2.0 + rank            # rank 1 is the slower one
        ms, rate = bench.job_rate(step_ms, 1000.0, ws, dist, "cpu")
        p = bench.workload("c2", rank)
        class A:                        # the reference arm's arguments
            steps, warmup, headline = 1, 0, "c2"
        ref = bench.run_reference(A, ws, rank) if rank != 0 else "skipped on rank 0 here"
        q.put((rank, w, ms, rate, int(p.d[:50].sum()), ref))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_on_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, w0, ms0, rate0, s0, _), (r1, w1, ms1, rate1, s1, ref1) = out
    assert w0 == (2, 0, 0) and w1 == (2, 1, 1)
    # max over ranks, whole-job rate
    assert ms0 == ms1 == 3.0
    assert rate0 == rate1 == pytest.approx(2 * 1000.0 / 3e-3)
    # independent replicas of the same shape
    assert s0 != s1
    # the reference arm does no work off rank 0
    assert ref1 is None
