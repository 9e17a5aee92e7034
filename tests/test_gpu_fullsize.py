"""Parity at the benchmark sizes, in the launch configuration the benchmark times.

One FRKC2 step of s stages makes a cell's new value depend only on the cells within s rows /
columns / planes of it (one cell per stage).  So a sampled output cell of a full-size step is
reproduced exactly by the oracle on a window of radius s + 1 around it (the window's own
boundary error travels one cell per stage and has not reached the centre).  The adjoint, whose
dependence is global after several steps, is checked at full size by the dot-product identity
<J v, w> = <v, J^T w> between the GPU forward and the GPU adjoint.
"""
import numpy as np
import pytest

import frkc2_inputs as I
from oracle import frkc2_oracle as O
from helpers import oracle_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")


def window(a, centre, r):
    """The (2r+1)^d block of a periodic array around ``centre`` (numpy order)."""
    idx = np.ix_(*[np.arange(c - r, c + r + 1) % n for c, n in zip(centre, a.shape)])
    return a[idx]


def sampled_cells(shape, count, seed):
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(0, n)) for n in shape) for _ in range(count)]


def seam_cells_2d(n):
    """Corners, edges and the seams of the launch layouts on an n x n grid: 48-cell output
    tiles of the 64 x 64 register-tiled regions (k = 8), 31- and 30-column warp chunks of the
    streaming passes, the wrap of the periodic grid and the middle of the grid."""
    xs = sorted({0, 1, 30, 31, 47, 48, 61, 62, 95, 96, n // 2 - 1, n // 2, n - 49, n - 48, n - 2, n - 1})
    ys = [0, 47, 48, n // 2, n - 48, n - 1]
    cells = [(y, x) for y in ys for x in xs[::2]] + [(y, x) for y in ys[::3] for x in xs[1::2]]
    return sorted(set(cells))


@pytest.fixture(scope="module")
def varkappa2048():
    cfg = I.CONFIGS["varkappa2d"]
    n = cfg["n"]
    u0 = I.smooth_unit((n, n), 64.0, cfg["u0_seed"])
    kap = I.kappa_field((n, n), cfg["kappa_seed"])
    return u0, kap


@pytest.mark.parametrize("prec,order,tol", [("fp64", "greedy", 1e-11), ("fp32", "greedy", 3e-4),
                                            ("fp32", "lebedev", 5e-6), ("dfloat", "greedy", 2e-6),
                                            ("mixed", "greedy", 2e-6)])
def test_varkappa2d_2048_one_step_sampled(varkappa2048, prec, order, tol):
    """The 2D variable-conductivity workload at 2048^2, s = 64, one step of the benchmark's dt
    and default launch configuration (FP32 also with the plan the precision policy chooses for
    the job, the Lebedev-Finogenov order); 80 cells -- corners, edges, tile and warp seams and
    random cells -- against the oracle on 131^2 windows."""
    u0, kap = varkappa2048
    n, s = u0.shape[0], I.CONFIGS["varkappa2d"]["s"]
    kd = torch.float64 if prec == "fp64" else torch.float32
    sd = torch.float32 if prec == "fp32" else torch.float64
    kt = torch.as_tensor(kap, dtype=kd, device="cuda")
    pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
    if order == "lebedev":
        plan, chosen, _ = F.frkc2_plan_auto(s, pr, I.CONFIGS["varkappa2d"]["steps"], 1e-4)
        assert chosen == prec
    else:
        plan = F.frkc2_plan(s)
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho)
    dt = I.CONFIGS["varkappa2d"]["cfl"] * plan.info()["beta"] / rho.item()
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    u = torch.as_tensor(u0, dtype=sd, device="cuda")
    F.frkc2_step(plan, pr, dt, 1, rho.item(), u, ws)
    assert F.frkc2_workspace_status(ws) == F.OK
    got = u.double().cpu().numpy()
    kap_o = kap if prec == "fp64" else kap.astype(np.float32).astype(np.float64)
    u0_o = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    a = O.plan(s)["a"] if order == "greedy" else O.step_sizes(s)[O.order_lebedev(s)]
    r = s + 1
    cells = seam_cells_2d(n)
    cells += sampled_cells(u0.shape, 80 - len(cells), 2048)
    assert len(cells) >= 64
    for c in cells:
        opr = oracle_problem(2, "dirichlet", "field", 1.0, window(kap_o, c, r))
        ref = O.frkc2_step(window(u0_o, c, r), a, dt, opr, 1)[r, r]
        assert abs(got[c] - ref) <= tol, (c, got[c], ref)  # the state lies in [0, 1]


def test_nonlinear3d_256_one_step_sampled():
    """The 3D kappa(u) workload at 256^3 (hot spot plus 1 % noise, Dirichlet), s = 32, one step
    with the 3D z-streaming pass; 3 sampled cells (one at the hot spot) against the oracle on
    67^3 windows that lie inside the grid (a window reaching past the boundary would evolve the
    ghost cells it contains)."""
    cfg = I.CONFIGS["nonlinear3d"]
    n, s = cfg["n"], cfg["s_stable"]
    u0 = I.hotspot3d_u0(n, sigma=20.0, seed=cfg["seed"])
    plan = F.frkc2_plan(s)
    pr = F.make_problem(3, (n, n, n), 1.0, "dirichlet", "power", "fp64", kappa_c=1.0, kappa_p=2.5)
    ud = torch.as_tensor(u0, device="cuda")
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, ud, rho)
    dt = cfg["cfl"] * plan.info()["beta"] / rho.item()
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step(plan, pr, dt, 1, 0.0, ud, ws)
    assert F.frkc2_workspace_status(ws) == F.OK
    got = ud.cpu().numpy()
    a = O.plan(s)["a"]
    r = s + 1
    rng = np.random.default_rng(256)
    inner = [tuple(int(rng.integers(r, n - r)) for _ in range(3)) for _ in range(2)]
    for c in [(n // 2, n // 2, n // 2)] + inner:
        win = u0[c[0] - r:c[0] + r + 1, c[1] - r:c[1] + r + 1, c[2] - r:c[2] + r + 1]
        opr = oracle_problem(3, "dirichlet", "power", 1.0, None)
        ref = O.frkc2_step(win, a, dt, opr, 1)[r, r, r]
        assert abs(got[c] - ref) <= 1e-11 * max(abs(ref), 1e-3), (c, got[c], ref)


def test_adjoint_1024_dot_product():
    """The adjoint workload's grid and plan (1024^2 periodic var-kappa, s = 100), two steps:
    <J v, w> = <v, J^T w> between the GPU forward map and the GPU adjoint at full size."""
    cfg = I.CONFIGS["adjoint2d"]
    n, s = cfg["n"], cfg["s"]
    kap = I.kappa_field((n, n), cfg["kappa_seed"], ell=32.0 * n / 2048)
    rng = np.random.default_rng(11)
    v, w = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    kt = torch.as_tensor(kap, device="cuda")
    pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp64", kappa_field=kt)
    plan = F.frkc2_plan(s)
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho)
    dt = cfg["cfl"] * plan.info()["beta"] / rho.item()
    nsteps = 2
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    jv = torch.as_tensor(v, device="cuda")
    F.frkc2_step(plan, pr, dt, nsteps, 0.0, jv, ws)
    wsa = torch.empty(F.frkc2_adjoint_workspace_size(plan, pr, nsteps, 1), dtype=torch.uint8, device="cuda")
    du = torch.empty((n, n), dtype=torch.float64, device="cuda")
    F.frkc2_adjoint(plan, pr, dt, nsteps, 1, torch.as_tensor(v, device="cuda"), torch.as_tensor(w, device="cuda"),
                    du, None, wsa)
    lhs = float(torch.sum(jv * torch.as_tensor(w, device="cuda")).item())
    rhs = float(torch.sum(torch.as_tensor(v, device="cuda") * du).item())
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)
