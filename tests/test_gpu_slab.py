"""The slab decomposition on the GPU: frkc2_stages on extended slabs, halos exchanged between
groups of stages (paper_1702_03818_gb300/slab.py).

Two processes share cuda:0 and exchange their halo rows through host memory over gloo (each
synchronises its stream before sending; no kernel waits on another process).  The interior rows
must equal the single-process frkc2_step of the whole grid bit for bit: every interior cell
runs the same streaming-pass arithmetic on the same values."""
import os
import socket

import numpy as np
import pytest

import frkc2_inputs as I
from oracle import frkc2_oracle as O
from helpers import oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")


def _recipe(ny, nx):
    u0 = I.smooth_unit((ny, nx), ny / 8.0, 3819)
    kap = I.kappa_field((ny, nx), 3818, ell=ny / 16.0)
    return u0, kap


def _whole_grid(ny, nx, s, nsteps, prec):
    u0, kap = _recipe(ny, nx)
    kd = torch.float64 if prec == "fp64" else torch.float32
    sd = torch.float32 if prec == "fp32" else torch.float64
    kt = torch.as_tensor(kap, dtype=kd, device="cuda")
    pr = F.make_problem(2, (nx, ny), 1.0, "periodic", "field", prec, kappa_field=kt)
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho)
    plan = F.frkc2_plan(s)
    dt = 0.9 * plan.info()["beta"] / rho.item()
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    u = torch.as_tensor(u0, dtype=sd, device="cuda")
    F.frkc2_step(plan, pr, dt, nsteps, 0.0, u, ws, F.make_tuning(k=1, kernel=2))
    return u.cpu().numpy(), dt


def _run_slab(rank, world, ny, nx, s, nsteps, halo, m, dt, prec):
    from paper_1702_03818_gb300 import slab as SL

    u0, kap = _recipe(ny, nx)
    sl = SL.Slab(ny, world, rank, halo)
    kd = torch.float64 if prec == "fp64" else torch.float32
    sd = torch.float32 if prec == "fp32" else torch.float64
    k_ext = torch.zeros((sl.rows_ext, nx), dtype=kd, device="cuda")
    k_ext[sl.interior()] = torch.as_tensor(kap[sl.y0:sl.y1], dtype=kd, device="cuda")
    SL.exchange_halos(k_ext, sl)
    w_ext = torch.zeros((sl.rows_ext, nx, 2), dtype=sd, device="cuda")
    w_ext[sl.interior(), :, 0] = torch.as_tensor(u0[sl.y0:sl.y1], dtype=sd, device="cuda")
    pr = F.make_problem(2, (nx, sl.rows_ext), 1.0, "periodic", "field", prec, kappa_field=k_ext)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    plan = F.frkc2_plan(s)
    n = SL.slab_steps(plan, s, nsteps, w_ext, sl, SL.device_stages(F, plan, pr, dt, w_ext, ws),
                      stages_per_exchange=m)
    assert F.frkc2_workspace_status(ws) == F.OK
    return w_ext[sl.interior(), :, 0].cpu().numpy(), n


def _worker(rank, world, port, q, args):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out, n = _run_slab(rank, world, *args)
        q.put((rank, out, n))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_rank_stages_equal_frkc2_step(prec):
    """One rank: frkc2_stages in groups of 5 stages on the extended grid (halo = its own wrap)
    equals frkc2_step with the streaming pass bit for bit, and the oracle to the precision."""
    from paper_1702_03818_gb300 import slab as SL

    ny, nx, s, nsteps = 96, 130, 16, 2
    ref, dt = _whole_grid(ny, nx, s, nsteps, prec)
    got, n = _run_slab(0, 1, ny, nx, s, nsteps, 6, 5, dt, prec)
    assert n == nsteps * 4
    assert np.array_equal(got, ref)
    u0, kap = _recipe(ny, nx)
    kf = kap if prec == "fp64" else kap.astype(np.float32).astype(np.float64)
    uo = u0 if prec == "fp64" else u0.astype(np.float32).astype(np.float64)
    oref = O.frkc2_step(uo, O.plan(s)["a"], dt, oracle_problem(2, "periodic", "field", 1.0, kf), nsteps)
    assert rel_err(got, oref) < (1e-11 if prec == "fp64" else 1e-4)
    assert SL.Slab(ny, 1, 0, 6).n == ny


@pytest.mark.parametrize("halo,m", [(8, 8), (7, 3)])
def test_two_processes_on_one_gpu_reproduce_the_whole_grid(halo, m):
    """Two ranks (processes on cuda:0, gloo, host-staged halos), FP64, 2 steps of s = 32:
    the gathered interiors equal the single-process frkc2_step bit for bit."""
    import torch.multiprocessing as tmp

    world, ny, nx, s, nsteps = 2, 90, 128, 32, 2
    ref, dt = _whole_grid(ny, nx, s, nsteps, "fp64")
    port = _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    args = (ny, nx, s, nsteps, halo, m, dt, "fp64")
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, args)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = np.concatenate([r[1] for r in res])
    assert all(r[2] == nsteps * -(-s // m) for r in res)
    assert np.array_equal(got, ref)


def test_stages_rejects_unsupported_and_bad_ranges():
    plan = F.frkc2_plan(8)
    kt = torch.ones((16, 16), dtype=torch.float64, device="cuda")
    pr = F.make_problem(2, (16, 16), 1.0, "periodic", "field", "fp64", kappa_field=kt)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    w = torch.zeros((16, 16, 2), dtype=torch.float64, device="cuda")
    for l0, l1 in [(3, 3), (-1, 2), (0, 9)]:
        with pytest.raises(F.Frkc2Error) as e:
            F.frkc2_stages(plan, pr, 0.1, l0, l1, w, ws)
        assert e.value.status == F.EINVAL
    p3 = F.make_problem(3, (8, 8, 8), 1.0, "periodic", "const", "fp64", kappa_c=1.0)
    ws3 = torch.empty(F.frkc2_workspace_size(p3), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.Frkc2Error) as e:
        F.frkc2_stages(plan, p3, 0.1, 0, 2, torch.zeros((8, 8, 8, 2), dtype=torch.float64, device="cuda"), ws3)
    assert e.value.status == F.EUNSUPPORTED
