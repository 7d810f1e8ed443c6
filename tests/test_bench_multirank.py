"""The multi-rank path of bench.py on CPU: two gloo ranks, max-over-ranks timing and whole-job
throughput (each rank runs an independent replica; no collective on the data path)."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env()[:2] == (world, rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)          # rank 1 is the slow one
    v = bench.job_throughput(1000, world, 4, ms)
    out[rank] = (ms, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 2 * 1000 * 4 / 0.015)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_throughput(10, 1, 2, 1000.0) == 20.0
