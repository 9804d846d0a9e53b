"""The N > 1 path of bench.py (independent replicas, no data-path
collective): the whole-job reduction over ranks, run as two gloo ranks on the
CPU.  The slowest rank's time and the sum of all ranks' work make the value."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r: time 100 + 10 r ms, 7 + r iterations, 3 launches
        (ms, e2e), (iters, e2e_iters, launches) = bench.reduce_replicas([100.0 + 10 * rank, 50.0 - rank],
                                                                        [7 + rank, 5, 3])
        out[rank] = (ms, e2e, iters, e2e_iters, launches, bench.replica_throughput(iters, ms))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, e2e, iters, e2e_iters, launches, value = res[r]
        assert ms == 110.0 and e2e == 50.0                  # max over ranks
        assert iters == 15.0 and e2e_iters == 10.0 and launches == 6.0   # sums over ranks
        assert value == pytest.approx(15.0 / 0.110)
