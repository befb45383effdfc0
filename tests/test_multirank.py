"""The N > 1 path of bench.py on CPU: independent replicas (one per rank, no
data exchange), the slowest rank's time, whole-job throughput.  Two gloo ranks
on 127.0.0.1; the timings are planted per rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist, "cpu")
        value = bench.replica_throughput(world, 1000, 10, t)
        dist.barrier()
        out[rank] = (t, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        times = [0.25, 0.5]
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]                       # every rank sees the same numbers
    t, value = res[0]
    assert t == 0.5                               # the slowest rank's time
    assert value == pytest.approx(2 * 1000 * 10 / 0.5)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(0.125, None, "cpu") == 0.125
    assert bench.replica_throughput(1, 1_048_576, 20, 2.0) == pytest.approx(1_048_576 * 10)
