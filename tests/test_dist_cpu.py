"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed
region is the maximum over ranks and the reported rate counts the units of
all ranks.  Views are independent, so ranks share no data: the only
cross-rank operations are the barrier and this reduction."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    local_ms = 100.0 + 50.0 * rank                 # rank 1 is the slower one
    dist.barrier()
    max_ms = bench.reduce_max(local_ms, dist)
    rate = bench.whole_job_rate(256, ws, max_ms / 10)
    q.put((r, ws, local, max_ms, rate))
    dist.destroy_process_group()


def test_two_rank_timing_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, ws, local, max_ms, rate) in enumerate(out):
        assert (rank, ws, local) == (r, 2, r)
        assert max_ms == 150.0
        assert rate == pytest.approx(2 * 256 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(12.5) == 12.5
    assert bench.whole_job_rate(256, 1, 128.0) == pytest.approx(2000.0)
