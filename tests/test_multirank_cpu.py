"""The multi-rank host logic of the bench on CPU: two gloo ranks, each with
its own stream, reduce their frame times to the slowest and agree on the
whole-job throughput.  No GPU and no data-path collective: every rank shades
and trains its own view."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed, view = bench.rank_stream(rank)
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, "cpu")
    value = bench.job_throughput(world, 2_073_600, slowest)
    out[rank] = (seed, view, slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_use_distinct_streams():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    (s0, v0, t0, val0), (s1, v1, t1, val1) = res[0], res[1]
    assert s0 != s1 and v0 != v1
    assert t0 == t1 == 15.0
    assert val0 == val1 == pytest.approx(2 * 2_073_600 / 15e-3 / 1e6)
