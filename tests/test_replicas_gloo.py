"""Right-hand-side sharding with two gloo ranks on CPU: shards cover every column once, the step
time reported is the slowest rank's, and the final gather restores the full column order.  Failure
on the host: a rank that fails before the gather (its solve raised, say) and leaves the group makes
the surviving rank's gather end with an error within the process group's timeout, not hang; a shard
of the wrong width is refused."""
import datetime
import os
import socket
import time

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


def _worker_fail(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    local = torch.ones((3, 2, 5, len(rhs_shard(8, rank, world))), dtype=torch.complex128)
    if rank == 1:
        # this rank's work failed between steps: it leaves without joining the gather
        q.put((1, "left", 0.0))
        q.close()
        q.join_thread()                          # flush the message; os._exit skips the feeder thread
        os._exit(3)
    t0 = time.monotonic()
    try:
        gather_columns(local, 8)
        q.put((0, "completed", time.monotonic() - t0))
    except Exception as e:                      # the collective reports the lost peer
        q.put((0, type(e).__name__, time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)


def test_surviving_rank_gets_an_error_when_a_peer_leaves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (what, dt)) for r, what, dt in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    what, dt = out[0]
    assert what != "completed", out
    assert dt < 60.0, out


def _worker_bad_width(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wrong = len(rhs_shard(7, rank, world)) + 1
        try:
            gather_columns(torch.zeros((2, wrong)), 7)
            q.put((rank, "accepted"))
        except ValueError:
            q.put((rank, "refused"))
    finally:
        dist.destroy_process_group()


def test_gather_refuses_a_shard_of_the_wrong_width():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_bad_width, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(out) == [(0, "refused"), (1, "refused")]
