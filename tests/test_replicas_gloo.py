"""Right-hand-side sharding with two gloo ranks on CPU: shards cover every column once, the step
time reported is the slowest rank's, and the final gather restores the full column order."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2608_26875_b300.replicas import gather_columns, max_over_ranks, rhs_shard


def test_shards_partition_columns():
    for n in (1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            cols = [c for r in range(world) for c in rhs_shard(n, r, world)]
            assert cols == list(range(n))
    with pytest.raises(ValueError):
        rhs_shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cols = rhs_shard(n, rank, world)
        # each rank's "result": column index encoded in a complex block (M=3, 2, nc=5, ncols)
        local = torch.zeros((3, 2, 5, len(cols)), dtype=torch.complex128)
        for k, c in enumerate(cols):
            local[..., k] = complex(c, -c)
        full = gather_columns(local, n)
        t = max_over_ranks(1.0 + rank)
        q.put((rank, full.shape[-1], [full[0, 0, 0, c].real.item() for c in range(n)], t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n", [7, 64])
def test_two_rank_gather_and_max(n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ncols, vals, t in out:
        assert ncols == n
        assert vals == [float(c) for c in range(n)]
        assert t == 2.0
