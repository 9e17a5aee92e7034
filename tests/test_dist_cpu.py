"""The multi-rank host path on CPU: two gloo ranks shard independent problems and reduce the
timing (max over ranks) and the work (sum over ranks) the way bench.py does under torchrun."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1702_03818_gb300 import dist as D

        mine = D.shard_indices(11, rank, world)
        units = sum(10 * (i + 1) for i in mine)       # work of this rank's problems
        ms = 100.0 + 50.0 * rank                       # rank 1 is the slow one
        D.barrier()
        q.put((rank, mine, D.max_over_ranks(ms), D.sum_over_ranks(units)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(11))
    assert not set(shards[0]) & set(shards[1])
    assert all(r[2] == 150.0 for r in res)                # max over ranks
    assert all(r[3] == sum(10 * (i + 1) for i in range(11)) for r in res)


def test_shard_indices_single_rank_and_errors():
    from paper_1702_03818_gb300 import dist as D

    assert D.shard_indices(5, 0, 1) == [0, 1, 2, 3, 4]
    assert D.max_over_ranks(3.5) == 3.5  # no process group: the value itself
    with pytest.raises(ValueError):
        D.shard_indices(5, 2, 2)
