"""The multi-rank bench path on the CPU: two gloo ranks, max-over-ranks timing.

bench.py under torchrun runs one independent replica per rank (the path does not
shard one system across GPUs); the job's time is the slowest rank's and the
throughput is world_size * units / max_ms.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.aggregate_ms(dist, 1.0 + rank)  # rank 1 is slower
    ws, r, _ = bench.dist_env()
    q.put((rank, ms, ws, ws * 1000.0 / ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, ws, value in res:
        assert ws == 2 and ms == 2.0 and value == pytest.approx(1000.0)
