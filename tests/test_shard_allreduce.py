"""Host side of velocity-space sharding on CPU (gloo, world size 2 and 3):
the fixed-order all-reduce that a sharded context's exchange performs gives
every rank the same bits, equal to the sum of the ranks' partial buffers
taken in rank order, for the two exchange buffers' shapes (face sums, cell
moment sums); and the row partition covers the velocity grid."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_09984_gb300 import ugks as U  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def partial(rank, n, seed):
    """This rank's partial sums: values of mixed sign and magnitude, so that
    the order of summation shows in the last bits."""
    rng = np.random.default_rng(seed + 101 * rank)
    return rng.normal(size=n) * 10.0 ** rng.integers(-8, 8, size=n)


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for name, n in (("face", 12 * 1000), ("cell", 6 * 700)):
        t = torch.tensor(partial(rank, n, 7 if name == "face" else 9), dtype=torch.float64)
        U.fixed_order_allreduce(t)
        res[name] = t.numpy()
    np.savez(os.path.join(out, "r%d.npz" % rank), **res)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_fixed_order_allreduce_same_bits_on_every_rank(world):
    with tempfile.TemporaryDirectory() as out:
        mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
        got = [np.load(os.path.join(out, "r%d.npz" % r)) for r in range(world)]
        for name, n, seed in (("face", 12 * 1000, 7), ("cell", 6 * 700, 9)):
            want = partial(0, n, seed).copy()
            for r in range(1, world):
                want = want + partial(r, n, seed)
            for g in got:
                assert np.array_equal(g[name].view(np.int64), want.view(np.int64))


def test_shard_rows_partition():
    for nvy in (2, 7, 32, 64):
        for n in range(1, min(nvy, 8) + 1):
            rows = U.shard_rows(nvy, n)
            assert rows[0][0] == 0 and rows[-1][1] == nvy
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [b - a for a, b in rows]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        U.shard_rows(4, 5)
