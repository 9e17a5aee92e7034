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


# ---------------------------------------------------------------------------------------
# Slab decomposition of one grid (paper_1702_03818_gb300/slab.py): partition, halo exchange
# and the exchange schedule, with the oracle's stages as the stage engine
# ---------------------------------------------------------------------------------------

def _slab_worker(rank, world, port, q, ny, nx, s, nsteps, halo, m):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np

        import frkc2_inputs as I
        from oracle import frkc2_oracle as O
        from paper_1702_03818_gb300 import slab as SL

        u0 = I.smooth_unit((ny, nx), 3.0, 61)
        kap = I.kappa_field((ny, nx), 62, ell=2.0)
        sl = SL.Slab(ny, world, rank, halo)
        # the conductivity: interior rows from this rank, halo rows by one exchange
        k_ext = torch.zeros((sl.rows_ext, nx), dtype=torch.float64)
        k_ext[sl.interior()] = torch.as_tensor(kap[sl.y0:sl.y1])
        SL.exchange_halos(k_ext, sl)
        halo_ok = bool(np.array_equal(k_ext.numpy(), kap[sl.global_rows()]))
        # the state: interleaved (re, im), interior rows only; halos come with the first exchange
        w_ext = torch.zeros((sl.rows_ext, nx, 2), dtype=torch.float64)
        w_ext[sl.interior(), :, 0] = torch.as_tensor(u0[sl.y0:sl.y1])
        a = O.plan(s)["a"]
        pr_glob = dict(ndim=2, dx=1.0, bc="periodic", kappa="field", kappa_c=1.0, kappa_p=2.5, kappa_field=kap)
        dt = 0.9 * O.beta(s) / O.rho_bound(pr_glob)
        pr_ext = dict(pr_glob, kappa_field=k_ext.numpy().copy())
        calls = []

        def stages(l0, l1):
            calls.append((l0, l1))
            W = w_ext[..., 0].numpy() + 1j * w_ext[..., 1].numpy()
            if l0 == 0:
                W = W.real.astype(np.complex128)
            for al in a[l0:l1]:
                W = W + (dt * al) * O.apply_f(W, pr_ext)
            w_ext[..., 0] = torch.as_tensor(W.real)
            w_ext[..., 1] = torch.as_tensor(W.imag)

        nex = SL.slab_steps(None, s, nsteps, w_ext, sl, stages, stages_per_exchange=m)
        q.put((rank, sl.y0, sl.y1, w_ext[sl.interior(), :, 0].numpy().copy(), halo_ok, nex, calls))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ny,halo,m", [(2, 24, 4, 4), (2, 23, 5, 3), (3, 31, 4, 4), (4, 26, 3, 2)])
def test_gloo_ranks_slab_steps_equal_the_whole_grid(world, ny, halo, m):
    """2 to 4 ranks, each holding its slab of a periodic grid's rows (uneven heights where ny
    does not divide) plus `halo` rows each side, run 2 FRKC2 steps of s = 8 stages exchanging
    halos before every group of m stages; the interior rows equal the oracle's step on the
    whole grid bit for bit, the conductivity's halo rows equal the global rows they stand for,
    and the schedule is ceil(s / m) groups per step."""
    import numpy as np

    import frkc2_inputs as I
    from oracle import frkc2_oracle as O

    nx, s, nsteps = 10, 8, 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, q, ny, nx, s, nsteps, halo, m))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u0 = I.smooth_unit((ny, nx), 3.0, 61)
    kap = I.kappa_field((ny, nx), 62, ell=2.0)
    pr = dict(ndim=2, dx=1.0, bc="periodic", kappa="field", kappa_c=1.0, kappa_p=2.5, kappa_field=kap)
    dt = 0.9 * O.beta(s) / O.rho_bound(pr)
    ref = O.frkc2_step(u0, O.plan(s)["a"], dt, pr, nsteps)
    got = np.concatenate([r[3] for r in res])
    assert [(r[1], r[2]) for r in res] == [(q * ny // world, (q + 1) * ny // world) for q in range(world)]
    assert all(r[4] for r in res)
    groups = -(-s // m)
    assert all(r[5] == groups * nsteps for r in res)
    want_calls = [(l0, min(s, l0 + m)) for l0 in range(0, s, m)] * nsteps
    assert all(r[6] == want_calls for r in res)
    assert np.array_equal(got, ref)


def test_slab_partition_and_rejections():
    import numpy as np

    from paper_1702_03818_gb300 import slab as SL

    parts = [SL.Slab(10, 3, r, 2) for r in range(3)]
    assert [(p.y0, p.y1) for p in parts] == [(0, 3), (3, 6), (6, 10)]
    assert list(parts[0].global_rows()) == [8, 9, 0, 1, 2, 3, 4]
    assert (parts[0].lower, parts[0].upper) == (2, 1)
    assert np.array_equal(parts[2].extend(np.arange(10)), [4, 5, 6, 7, 8, 9, 0, 1])
    with pytest.raises(ValueError):
        SL.Slab(10, 3, 0, 4)   # a slab of 3 rows cannot feed a 4-row halo
    with pytest.raises(ValueError):
        SL.Slab(10, 2, 2, 1)
    one = SL.Slab(6, 1, 0, 2)  # a single rank: the halo is the grid's own wrap
    t = torch.arange(10.0)
    SL.exchange_halos(t, one)
    assert t.tolist() == [6.0, 7.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 2.0, 3.0]
    with pytest.raises(ValueError):
        SL.slab_steps(None, 8, 1, t, one, lambda a, b: None, stages_per_exchange=3)
