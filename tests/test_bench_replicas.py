"""The multi-rank (replica) logic of bench.py on CPU with the gloo backend, world size 2: every
rank gets its own Philox job id, and the reported time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, dist, torch.device("cpu"))
    jobs = [None] * world
    dist.all_gather_object(jobs, bench.replica_job(rank))
    out.put((rank, t, jobs))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_time_is_max_and_jobs_distinct():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, jobs in res:
        assert t == 2.5
        assert len(set(jobs)) == world
    assert bench_none_identity()


def bench_none_identity():
    import bench
    return bench.max_over_ranks(3.25, None, None) == 3.25
