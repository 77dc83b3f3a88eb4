"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
path runs independent replicas, so the only cross-rank steps are the
barriers around the timed region and the max over ranks of its time."""
import os
import socket
import tempfile

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.rank_sync(dist)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    bench.rank_sync(dist)
    with open(os.path.join(out, "r%d" % rank), "w") as f:
        f.write(repr(ms))
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    world = 2
    with tempfile.TemporaryDirectory() as out:
        mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
        got = [float(open(os.path.join(out, "r%d" % r)).read()) for r in range(world)]
    assert got == [20.0, 20.0]


def test_single_rank_passes_time_through():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
