"""The benchmark's multi-rank path (one independent bed per rank, no collective on
the data path) with world size 2 over gloo on the CPU: the job time is the max
over ranks and the value counts every rank's particles."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 55.0][rank]
    parts = [200_000, 180_000][rank]
    dist.barrier()
    value, total = bench.aggregate(ms, parts, steps=10, world=world, device="cpu")
    q.put((rank, value, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = (200_000 + 180_000) * 20 * 10 / 0.055
    for rank, value, total in out:
        assert total == 55.0
        assert abs(value - expect) < 1e-6 * expect
