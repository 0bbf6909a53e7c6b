"""The multi-rank part of bench.py on CPU: two gloo ranks (spawned processes)
take the maximum of their timings and meet at a barrier, as the replica
benchmark does with one GPU per rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench._dist()
    assert (w, r, local) == (world, rank, rank)
    vals = bench.max_over_ranks([float(rank), 10.0 - rank, 3.0], dist)
    dist.barrier()
    out.put((rank, vals))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [1.0, 10.0, 3.0]


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
