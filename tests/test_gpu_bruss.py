"""GPU parity of the Brusselator stage loop (frkc2_bruss_step, Sec. 3.1, Eq. 17) against the
FP64 oracle, the bit-exact Gershgorin bound, and the persistent launch's bounded barrier."""
import numpy as np
import pytest

import frkc2_inputs as I
from oracle import brusselator as BR
from oracle import frkc2_oracle as O
from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

DT = {"fp64": torch.float64, "fp32": torch.float32}
TOL = {"fp64": 1e-11, "fp32": 1e-4}


def state(shape, bc, seed):
    """The paper's initial state on square periodic grids, else a seeded perturbation of the
    equilibrium (v, w) = (1, 3)."""
    ny, nx = shape
    if bc == "periodic" and nx == ny:
        return I.bruss_u0(nx, ny, 1.0 / nx)
    rng = np.random.default_rng(seed)
    return 1.0 + 0.5 * rng.uniform(-1, 1, shape), 3.0 + 0.5 * rng.uniform(-1, 1, shape)


def run_gpu(plan, shape, bc, prec, v0, w0, dt, nsteps, kernel=0, **tk):
    ny, nx = shape
    p = F.make_bruss_problem((nx, ny), bc=bc, precision=prec)
    ws = torch.empty(F.frkc2_bruss_workspace_size(p), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    v = torch.as_tensor(v0, dtype=DT[prec], device="cuda").contiguous()
    w = torch.as_tensor(w0, dtype=DT[prec], device="cuda").contiguous()
    F.frkc2_bruss_step(plan, p, dt, nsteps, 0.0, v, w, ws, F.make_tuning(kernel=kernel, **tk))
    st = F.frkc2_workspace_status(ws)
    return v.double().cpu().numpy(), w.double().cpu().numpy(), st


def rounded(a, prec):
    return a.astype(np.float32).astype(np.float64) if prec == "fp32" else a


CASES = [
    # (ny, nx), bc, s, nsteps
    ((200, 200), "periodic", 16, 3),
    ((29, 37), "neumann", 8, 4),
    ((33, 64), "periodic", 32, 2),
    ((300, 5), "neumann", 16, 2),
    ((1, 257), "periodic", 8, 3),
    ((17, 1), "neumann", 8, 2),
]


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0][0]}x{c[0][1]}-{c[1]}-s{c[2]}")
def test_bruss_matches_oracle(case, prec, kernel):
    shape, bc, s, nsteps = case
    v0, w0 = state(shape, bc, 100 + s)
    v0, w0 = rounded(v0, prec), rounded(w0, prec)
    pr = BR.problem(shape, bc=bc, dx=1.0 / 200)
    plan = F.frkc2_plan(s)
    oplan = O.plan(s)
    dt = 0.8 * oplan["beta"] / BR.rho_bound(v0, w0, pr)
    rv, rw = BR.frkc2_step(v0, w0, oplan["a"], dt, pr, nsteps)
    p = F.make_bruss_problem((shape[1], shape[0]), dx=1.0 / 200, bc=bc, precision=prec)
    ws = torch.empty(F.frkc2_bruss_workspace_size(p), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    v = torch.as_tensor(v0, dtype=DT[prec], device="cuda").contiguous()
    w = torch.as_tensor(w0, dtype=DT[prec], device="cuda").contiguous()
    F.frkc2_bruss_step(plan, p, dt, nsteps, 0.0, v, w, ws, F.make_tuning(kernel=kernel))
    assert F.frkc2_workspace_status(ws) == F.OK
    gv, gw = v.double().cpu().numpy(), w.double().cpu().numpy()
    ev, ew = rel_err(gv, rv), rel_err(gw, rw)
    assert ev < TOL[prec] and ew < TOL[prec], (ev, ew)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_equals_per_stage_launches(prec):
    shape = (96, 130)
    v0, w0 = state(shape, "periodic", 7)
    plan = F.frkc2_plan(16)
    dt = 0.5 * F.frkc2_plan_info(plan)["beta"] / BR.rho_bound(v0, w0, BR.problem(shape))
    a = run_gpu(plan, shape, "periodic", prec, v0, w0, dt, 3, kernel=1)
    b = run_gpu(plan, shape, "periodic", prec, v0, w0, dt, 3, kernel=2)
    assert a[2] == F.OK and b[2] == F.OK
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1024, 2048])
def test_persistent_waits_at_size(n, prec):
    """Large grids, where the persistent launch's CTAs own thousands of cells: at 1024^2 they
    wait on their neighbours' stage flags, at 2048^2 in FP64 at the grid barrier (FP32 keeps the
    flags).  Bit-identical to one launch per stage, and at 1024^2 FP64 equal to the oracle."""
    shape = (n, n)
    v0, w0 = state(shape, "periodic", 11)
    v0, w0 = rounded(v0, prec), rounded(w0, prec)
    plan = F.frkc2_plan(16)
    pr = BR.problem(shape, dx=1.0 / n)
    dt = 0.8 * F.frkc2_plan_info(plan)["beta"] / BR.rho_bound(v0, w0, pr)
    a = run_gpu(plan, shape, "periodic", prec, v0, w0, dt, 1, kernel=1)
    b = run_gpu(plan, shape, "periodic", prec, v0, w0, dt, 1, kernel=2)
    assert a[2] == F.OK and b[2] == F.OK
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    if n == 1024 and prec == "fp64":
        rv, rw = BR.frkc2_step(v0, w0, O.plan(16)["a"], dt, pr, 1)
        assert rel_err(a[0], rv) < 1e-11 and rel_err(a[1], rw) < 1e-11


def test_more_than_1024_stages_chunked_launches():
    """A 2048-stage plan takes two persistent launches per step; same result as per stage and
    as the oracle on the plan's own step sizes."""
    shape = (16, 16)
    s = 2048
    v0, w0 = state(shape, "neumann", 9)
    plan = F.frkc2_plan(s, flags=F.PLAN_LEBEDEV)
    a = F.frkc2_plan_info(plan)["a"]
    pr = BR.problem(shape, bc="neumann")
    dt = 0.05
    rv, rw = BR.frkc2_step(v0, w0, a, dt, pr, 2)
    F.frkc2_launch_count()
    g1 = run_gpu(plan, shape, "neumann", "fp64", v0, w0, dt, 2, kernel=1)
    assert F.frkc2_launch_count() == 4
    g2 = run_gpu(plan, shape, "neumann", "fp64", v0, w0, dt, 2, kernel=2)
    assert g1[2] == F.OK and g2[2] == F.OK
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1])
    assert rel_err(g1[0], rv) < 1e-11 and rel_err(g1[1], rw) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rho_bound_bit_exact(prec):
    for shape, bc in [((200, 200), "periodic"), ((37, 61), "neumann")]:
        v0, w0 = state(shape, bc, 21)
        v0, w0 = rounded(v0, prec), rounded(w0, prec)
        p = F.make_bruss_problem((shape[1], shape[0]), bc=bc, precision=prec)
        ws = torch.empty(F.frkc2_bruss_workspace_size(p), dtype=torch.uint8, device="cuda")
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        v = torch.as_tensor(v0, dtype=DT[prec], device="cuda")
        w = torch.as_tensor(w0, dtype=DT[prec], device="cuda")
        F.frkc2_bruss_rho_bound(p, v, w, rho, ws)
        assert float(rho.item()) == BR.rho_bound(v0, w0, BR.problem(shape, bc=bc))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_equilibrium_exactly_preserved(prec):
    shape = (50, 70)
    plan = F.frkc2_plan(32)
    v0, w0 = np.ones(shape), np.full(shape, 3.0)
    v, w, st = run_gpu(plan, shape, "periodic", prec, v0, w0, 1e-3, 5)
    assert st == F.OK and np.array_equal(v, v0) and np.array_equal(w, w0)


def test_zero_steps_leave_state():
    shape = (20, 30)
    v0, w0 = state(shape, "neumann", 3)
    v, w, st = run_gpu(F.frkc2_plan(8), shape, "neumann", "fp64", v0, w0, 1e-4, 0)
    assert np.array_equal(v, v0) and np.array_equal(w, w0)


@pytest.mark.parametrize("kernel", [1, 2])
def test_nonfinite_latched(kernel):
    shape = (40, 40)
    v0, w0 = state(shape, "periodic", 4)
    v0[10, 11] = np.nan
    _, _, st = run_gpu(F.frkc2_plan(8), shape, "periodic", "fp64", v0, w0, 1e-5, 1, kernel=kernel)
    assert st == F.ENONFINITE


@pytest.mark.parametrize("shape", [(64, 64), (1, 257)], ids=["neighbour-flags", "grid-barrier"])
def test_barrier_wait_runs_out_and_context_survives(shape):
    """fault_inject: the first wait between stages (on the neighbour CTAs' stage flags, or on
    the grid barrier where a CTA's stencil reaches too many CTAs: one row of 257 cells over
    152 CTAs) waits for a count nothing reaches; every CTA gives up after wait_limit polls,
    the launch returns and FRKC2_ETIMEOUT is latched.  The next call on the same device then
    runs normally."""
    v0, w0 = state(shape, "periodic", 5)
    plan = F.frkc2_plan(8)
    dt = 1e-4
    _, _, st = run_gpu(plan, shape, "periodic", "fp64", v0, w0, dt, 2, kernel=1, wait_limit=2000, fault_inject=1)
    assert st == F.ETIMEOUT
    v, w, st = run_gpu(plan, shape, "periodic", "fp64", v0, w0, dt, 2, kernel=1)
    assert st == F.OK
    rv, rw = BR.frkc2_step(v0, w0, O.plan(8)["a"], dt, BR.problem(shape), 2)
    assert rel_err(v, rv) < 1e-11 and rel_err(w, rw) < 1e-11


def test_launch_counts():
    shape = (32, 32)
    v0, w0 = state(shape, "periodic", 6)
    plan = F.frkc2_plan(16)
    F.frkc2_launch_count()
    run_gpu(plan, shape, "periodic", "fp64", v0, w0, 1e-4, 5, kernel=1)
    assert F.frkc2_launch_count() == 1
    run_gpu(plan, shape, "periodic", "fp64", v0, w0, 1e-4, 5, kernel=2)
    assert F.frkc2_launch_count() == 16 * 5
