"""GPU parity of the forward path (frkc2_rho_bound, frkc2_step) against the FP64 oracle.

Every case builds the same seeded inputs for both sides; the CUDA path is called through
the C ABI (the ctypes binding) and compared element by element with the oracle.
Tolerances (relative L2 against the FP64 oracle): FP64 1e-11, FP32 1e-4 at s <= 64.
"""
import numpy as np
import pytest

from oracle import frkc2_oracle as O
import frkc2_inputs as I
from helpers import oracle_problem, rel_err, seeded_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

TOL = {"fp64": 1e-11, "fp32": 1e-4, "mixed": 1e-6, "dfloat": 1e-6}
DT = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float64, "dfloat": torch.float64}
KDT = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float32, "dfloat": torch.float32}


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def lib_problem(shape, bc, kappa, prec, dx=1.0, field_t=None, c=1.0, p=2.5):
    n = tuple(reversed(shape))  # (nx, ny, nz)
    return F.make_problem(len(shape), n, dx, bc, kappa, prec, kappa_c=c, kappa_p=p, kappa_field=field_t)


def run_gpu(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, dx=1.0, c=1.0, tune=None):
    u = dev(u0, DT[prec])
    kt = dev(field, KDT[prec]) if field is not None else None
    pr = lib_problem(shape, bc, kappa, prec, dx, kt, c)
    ws = torch.empty(F.frkc2_workspace_size(pr, tune), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step(plan, pr, dt, nsteps, 0.0, u, ws, tune)
    st = F.frkc2_workspace_status(ws)
    return u.double().cpu().numpy(), st


def rounded_field(field, prec):
    """The conductivity the GPU sees: float32-rounded for every precision but FP64."""
    if field is None or prec == "fp64":
        return field
    return field.astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------------------
# spectral-radius bound
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape,bc", [((64, 80), "periodic"), ((33, 47), "dirichlet"),
                                      ((9, 10, 11), "periodic"), ((7, 6, 5), "dirichlet"),
                                      ((300,), "dirichlet")])
def test_rho_bound_field_bit_exact(shape, bc):
    _, field = seeded_case(shape, bc, "field", 21)
    kt = dev(field, torch.float64)
    pr = lib_problem(shape, bc, "field", "fp64", 0.37, kt)
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho)
    ref = O.rho_bound(oracle_problem(len(shape), bc, "field", 0.37, field))
    assert rho.item() == ref


def test_rho_bound_const_and_power():
    n = 200
    pr = lib_problem((n, n), "periodic", "const", "fp64", 1.0 / n, c=0.02)
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho)
    assert rho.item() == O.rho_bound(oracle_problem(2, "periodic", "const", 1.0 / n, c=0.02), np.zeros((n, n)))
    u0 = I.hotspot3d_u0(24, sigma=4.0)
    ut = dev(u0, torch.float64)
    pr = lib_problem(u0.shape, "dirichlet", "power", "fp64", 1.0)
    F.frkc2_rho_bound(pr, ut, rho)
    ref = O.rho_bound(oracle_problem(3, "dirichlet", "power", 1.0), u0)
    assert abs(rho.item() / ref - 1.0) < 1e-14
    # FP32 field: the bound is formed in FP64 from the float values
    _, field = seeded_case((40, 50), "periodic", "field", 5)
    pr = lib_problem((40, 50), "periodic", "field", "fp32", 1.0, dev(field, torch.float32))
    F.frkc2_rho_bound(pr, None, rho)
    assert rho.item() == O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, rounded_field(field, "fp32")))


# ---------------------------------------------------------------------------------------
# forward step parity
# ---------------------------------------------------------------------------------------

CASES = [
    # shape, bc, kappa, s, nsteps, k, kernel
    ((100, 77), "periodic", "field", 16, 2, 1, 0),
    ((100, 77), "periodic", "field", 16, 2, 1, 1),
    ((100, 77), "periodic", "field", 16, 2, 4, 1),
    ((70, 130), "dirichlet", "field", 32, 2, 1, 0),
    ((70, 130), "dirichlet", "field", 32, 2, 3, 1),
    ((64, 64), "periodic", "const", 64, 1, 8, 1),
    ((5, 7), "periodic", "field", 8, 3, 4, 1),
    ((5, 7), "dirichlet", "field", 8, 3, 1, 0),
    ((1, 9), "periodic", "field", 4, 2, 1, 0),
    ((257,), "dirichlet", "const", 16, 3, 16, 1),
    ((1000,), "periodic", "field", 16, 2, 5, 1),
    ((12, 10, 14), "periodic", "field", 16, 1, 1, 1),
    ((12, 10, 14), "dirichlet", "field", 16, 1, 2, 1),
    ((10, 11, 9), "dirichlet", "power", 16, 1, 1, 1),
    ((34, 20), "periodic", "power", 16, 1, 2, 1),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-s{c[3]}-k{c[5]}-kern{c[6]}")
def test_step_parity(case, prec):
    shape, bc, kappa, s, nsteps, k, kernel = case
    u0, field = seeded_case(shape, bc, kappa, 100 + s)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    assert np.array_equal(plan.info()["order"], oplan["order"])
    fo = rounded_field(field, prec)
    opr = oracle_problem(len(shape), bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    u0g = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0g, oplan["a"], dt, opr, nsteps)
    tune = F.make_tuning(k=k, kernel=kernel)
    got, st = run_gpu(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, tune=tune)
    assert st == F.OK
    err = rel_err(got, ref)
    assert err < TOL[prec], err


def test_heat1d_workload_matches_closed_form_and_oracle():
    cfg = I.CONFIGS["heat1d"]
    u0, amp, dx = I.heat1d_u0(cfg["n"], 8, cfg["seed"])
    L = cfg["s"]
    plan = F.frkc2_plan(L)
    beta = plan.info()["beta"]
    nsteps = int(np.ceil(cfg["t_end"] / (0.9 * beta * dx * dx / 4.0)))
    dt = cfg["t_end"] / nsteps
    opr = oracle_problem(1, "dirichlet", "const", dx)
    ref = O.frkc2_step(u0, O.plan(L)["a"], dt, opr, nsteps)
    got, st = run_gpu(plan, (cfg["n"],), "dirichlet", "const", "fp64", u0, None, dt, nsteps, dx=dx)
    assert st == F.OK and nsteps == 87
    assert rel_err(got, ref) < 1e-12


def test_varkappa2d_reduced_many_steps_fp64_fp32():
    shape = (256, 256)
    u0 = I.smooth_unit(shape, 64 / 8, 3819)
    field = I.kappa_field(shape, 3818, ell=32 / 8)
    s = 64
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-4)):
        fo = rounded_field(field, prec)
        opr = oracle_problem(2, "periodic", "field", 1.0, fo)
        dt = 0.9 * oplan["beta"] / O.rho_bound(opr)
        u0g = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
        ref = O.frkc2_step(u0g, oplan["a"], dt, opr, 4)
        got, st = run_gpu(plan, shape, "periodic", "field", prec, u0, field, dt, 4)
        assert st == F.OK
        assert rel_err(got, ref) < tol, (prec, rel_err(got, ref))


def test_nsteps_zero_and_nonfinite_flag():
    shape = (32, 32)
    u0, field = seeded_case(shape, "periodic", "field", 3)
    plan = F.frkc2_plan(8)
    got, st = run_gpu(plan, shape, "periodic", "field", "fp64", u0, field, 0.1, 0)
    assert np.array_equal(got, u0) and st == F.OK
    bad = u0.copy()
    bad[5, 5] = np.nan
    _, st = run_gpu(plan, shape, "periodic", "field", "fp64", bad, field, 0.1, 1)
    assert st == F.ENONFINITE


def test_launch_count_matches_passes():
    shape = (64, 64)
    u0, field = seeded_case(shape, "periodic", "field", 4)
    plan = F.frkc2_plan(16)
    F.frkc2_launch_count()
    run_gpu(plan, shape, "periodic", "field", "fp32", u0, field, 0.5, 3, tune=F.make_tuning(k=4, kernel=1))
    # one face-preparation launch plus 16/4 passes per step
    assert F.frkc2_launch_count() == 1 + 3 * 4


TB_CASES = [
    # shape, bc, kappa, s, nsteps, k
    ((100, 77), "periodic", "field", 16, 2, 4),
    ((200, 130), "periodic", "field", 8, 3, 8),  # one pass per step over many regions
    ((100, 77), "periodic", "field", 16, 2, 1),
    ((200, 130), "dirichlet", "field", 32, 2, 3),
    ((64, 64), "periodic", "const", 64, 1, 8),
    ((9, 13), "periodic", "field", 8, 3, 2),
    ((9, 13), "dirichlet", "field", 8, 3, 8),
    ((130, 300), "periodic", "field", 16, 1, 16),
    ((57, 200), "dirichlet", "const", 32, 2, 5),
]


@pytest.mark.parametrize("case", TB_CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-k{c[5]}")
def test_step_parity_fp32_temporal_blocking(case):
    """The FP32 register/shared-memory temporally blocked kernel (kernel 3)."""
    shape, bc, kappa, s, nsteps, k = case
    u0, field = seeded_case(shape, bc, kappa, 300 + s)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    fo = rounded_field(field, "fp32")
    opr = oracle_problem(2, bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    ref = O.frkc2_step(u0.astype(np.float32).astype(np.float64), oplan["a"], dt, opr, nsteps)
    got, st = run_gpu(plan, shape, bc, kappa, "fp32", u0, field, dt, nsteps, tune=F.make_tuning(k=k, kernel=3))
    assert st == F.OK
    assert rel_err(got, ref) < TOL["fp32"], rel_err(got, ref)


WF_CASES = [
    # shape (ny, nx), bc, kappa, s, nsteps, k, rows per chunk (0 = library default)
    ((96, 256), "periodic", "field", 16, 2, 8, 0),
    ((77, 260), "dirichlet", "field", 32, 2, 8, 0),
    ((130, 516), "periodic", "const", 24, 1, 6, 0),
    ((64, 300), "dirichlet", "field", 20, 2, 12, 0),
    ((41, 256), "periodic", "field", 8, 3, 8, 0),
    ((50, 264), "dirichlet", "field", 4, 3, 4, 0),
    ((200, 512), "periodic", "field", 64, 1, 8, 7),
    ((33, 260), "periodic", "field", 10, 2, 2, 5),
    ((40, 256), "dirichlet", "field", 6, 1, 1, 0),
    ((9, 1024), "dirichlet", "field", 16, 2, 8, 2),
]


@pytest.mark.parametrize("case", WF_CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-s{c[3]}-k{c[5]}-H{c[6]}")
def test_step_parity_fp32_wavefront(case):
    """The FP32 wavefront pass (kernel 7): strips of 256 columns walked up in chunks of rows,
    k stage levels in flight, rows staged by TMA bulk copies.  Periodic strips that wrap,
    Dirichlet strips that leave the grid, ragged rows and strips, one pass per step (the real
    state alternating between the caller's array and the workspace), a short last pass (s not a
    multiple of k), k from 1 to 12, and chunks of a few rows.  Against the oracle (grid norm and
    every element) and against the register-tiled FP32 pass."""
    shape, bc, kappa, s, nsteps, k, H = case
    u0, field = seeded_case(shape, bc, kappa, 700 + s)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    fo = rounded_field(field, "fp32")
    opr = oracle_problem(2, bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    ref = O.frkc2_step(u0.astype(np.float32).astype(np.float64), oplan["a"], dt, opr, nsteps)
    got, st = run_gpu(plan, shape, bc, kappa, "fp32", u0, field, dt, nsteps,
                      tune=F.make_tuning(k=k, tile=(0, H, 0), kernel=7))
    assert st == F.OK
    assert rel_err(got, ref) < TOL["fp32"], rel_err(got, ref)
    if 2 * k < 64:
        reg, st = run_gpu(plan, shape, bc, kappa, "fp32", u0, field, dt, nsteps, tune=F.make_tuning(k=k, kernel=3))
        assert rel_err(got, reg) < TOL["fp32"], rel_err(got, reg)  # two roundings of the same stages


def test_wavefront_row_wait_runs_out_and_context_survives():
    """fault_inject on kernel 7: the first pass leaves one row's TMA copies unissued, so every
    thread's bounded wait on that row's mbarrier runs out (wait_limit polls); the CTAs wait
    (bounded) for their copies in flight and return, FRKC2_ETIMEOUT is latched, and the next
    call on the same device matches the oracle."""
    shape = (40, 256)
    u0, field = seeded_case(shape, "periodic", "field", 8)
    s = 16
    plan = F.frkc2_plan(s)
    kt = dev(field, torch.float32)
    pr = lib_problem(shape, "periodic", "field", "fp32", 1.0, kt, 1.0)
    fo = field.astype(np.float32).astype(np.float64)
    opr = oracle_problem(2, "periodic", "field", 1.0, fo)
    dt = 0.9 * O.beta(s) / O.rho_bound(opr)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    u = dev(u0, torch.float32)
    F.frkc2_step(plan, pr, dt, 2, 0.0, u, ws, F.make_tuning(k=8, kernel=7, wait_limit=2000, fault_inject=1))
    assert F.frkc2_workspace_status(ws) == F.ETIMEOUT
    F.frkc2_workspace_reset(ws)
    u = dev(u0, torch.float32)
    F.frkc2_step(plan, pr, dt, 2, 0.0, u, ws, F.make_tuning(k=8, kernel=7))
    assert F.frkc2_workspace_status(ws) == F.OK
    ref = O.frkc2_step(u0.astype(np.float32).astype(np.float64), O.plan(s)["a"], dt, opr, 2)
    assert rel_err(u.double().cpu().numpy(), ref) < TOL["fp32"]


def test_wavefront_launches_and_rejects_unsupported():
    """Kernel 7 on an FP32 2D problem with nx a multiple of 4 and at least 256: one face set-up
    kernel for the call, one for the wavefront layout, then one launch per pass; other widths,
    or a state array off a 16-byte boundary, are refused."""
    shape = (48, 256)
    u0, field = seeded_case(shape, "periodic", "field", 5)
    plan = F.frkc2_plan(16)
    u = dev(u0, torch.float32)
    kt = dev(field, torch.float32)
    pr = lib_problem(shape, "periodic", "field", "fp32", 1.0, kt, 1.0)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_launch_count()
    F.frkc2_step(plan, pr, 0.1, 3, 0.0, u, ws, F.make_tuning(kernel=7))
    assert F.frkc2_launch_count() == 1 + 1 + 3 * 2  # faces, wavefront faces, 2 passes of 8 stages x 3 steps
    a = u.double().cpu().numpy()
    u2 = dev(u0, torch.float32)
    F.frkc2_step(plan, pr, 0.1, 3, 0.0, u2, ws, F.make_tuning(kernel=7))
    assert np.array_equal(a, u2.double().cpu().numpy())  # deterministic
    for bad_shape in [(48, 252), (48, 254), (48, 128)]:
        ub = dev(seeded_case(bad_shape, "periodic", "field", 6)[0], torch.float32)
        kb = dev(seeded_case(bad_shape, "periodic", "field", 6)[1], torch.float32)
        pb = lib_problem(bad_shape, "periodic", "field", "fp32", 1.0, kb, 1.0)
        wsb = torch.empty(F.frkc2_workspace_size(pb), dtype=torch.uint8, device="cuda")
        with pytest.raises(F.Frkc2Error) as e:
            F.frkc2_step(plan, pb, 0.1, 1, 0.0, ub, wsb, F.make_tuning(kernel=7))
        assert e.value.status == F.EUNSUPPORTED
        F.frkc2_step(plan, pb, 0.1, 1, 0.0, ub, wsb)  # the default falls back to another pass
    big = torch.zeros(48 * 256 + 2, dtype=torch.float32, device="cuda")
    with pytest.raises(F.Frkc2Error) as e:  # state array 8 bytes off a 16-byte boundary
        F.frkc2_step(plan, pr, 0.1, 1, 0.0, big[2:].view(48, 256), ws, F.make_tuning(kernel=7))
    assert e.value.status == F.EUNSUPPORTED


def test_tb_kernel_rejects_unsupported():
    shape = (32, 32)
    u0, field = seeded_case(shape, "periodic", "field", 5)
    plan = F.frkc2_plan(8)
    with pytest.raises(F.Frkc2Error) as e:
        run_gpu(plan, shape, "periodic", "field", "fp64", u0, field, 0.1, 1, tune=F.make_tuning(k=4, kernel=3))
    assert e.value.status == F.EUNSUPPORTED


PAIRED_CASES = [
    # shape, bc, kappa, s, nsteps
    ((100, 77), "periodic", "field", 16, 3),
    ((70, 130), "dirichlet", "field", 32, 2),
    ((64, 64), "periodic", "const", 8, 2),
    ((5, 7), "periodic", "field", 8, 2),
    ((9, 40), "dirichlet", "field", 4, 3),
    ((257, 33), "periodic", "field", 64, 1),
]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-6), ("fp32", 5e-4)])
@pytest.mark.parametrize("case", PAIRED_CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-s{c[3]}")
def test_step_parity_paired_real_pairs(case, prec, tol):
    """Conjugate pairs in adjacent stages applied to the real state (kernel 4) against the
    oracle's literal complex stages in the same order."""
    shape, bc, kappa, s, nsteps = case
    u0, field = seeded_case(shape, bc, kappa, 600 + s)
    oplan = O.plan(s, method="paired")
    plan = F.frkc2_plan(s, flags=F.PLAN_PAIRED)
    assert np.array_equal(plan.info()["order"], oplan["order"])
    fo = rounded_field(field, prec)
    opr = oracle_problem(2, bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    u0g = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0g, oplan["a"], dt, opr, nsteps)
    got, st = run_gpu(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, tune=F.make_tuning(kernel=4))
    assert st == F.OK
    assert rel_err(got, ref) < tol, rel_err(got, ref)
    # the oracle's own real pair form agrees with its complex stages
    assert rel_err(O.frkc2_step_paired(u0g, oplan["a"], dt, opr, nsteps), ref) < 1e-12


def test_paired_plan_on_3d_runs_as_complex_stages():
    shape = (9, 10, 11)
    u0, field = seeded_case(shape, "periodic", "field", 77)
    oplan = O.plan(8, method="paired")
    plan = F.frkc2_plan(8, flags=F.PLAN_PAIRED)
    opr = oracle_problem(3, "periodic", "field", 1.0, field)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr)
    ref = O.frkc2_step(u0, oplan["a"], dt, opr, 2)
    got, st = run_gpu(plan, shape, "periodic", "field", "fp64", u0, field, dt, 2)
    assert st == F.OK and rel_err(got, ref) < 1e-11


# ---------------------------------------------------------------------------------------
# DFLOAT: float-pair state on the FP32 pipe (2D fixed conductivity, k = 1 streaming pass)
# ---------------------------------------------------------------------------------------

DF_CASES = [
    # shape, bc, kappa, s, nsteps, kernel, k (0: default)
    ((100, 77), "periodic", "field", 16, 2, 0, 0),
    ((70, 130), "dirichlet", "field", 32, 2, 2, 0),
    ((64, 64), "periodic", "const", 64, 1, 0, 0),
    ((5, 7), "dirichlet", "field", 8, 3, 0, 0),
    ((1, 9), "periodic", "field", 4, 2, 0, 0),
    ((33, 1), "dirichlet", "field", 8, 2, 0, 0),
    ((200, 130), "periodic", "field", 32, 2, 3, 8),
    ((130, 300), "dirichlet", "field", 16, 1, 3, 5),
    ((57, 200), "dirichlet", "const", 32, 2, 3, 16),
    ((9, 13), "periodic", "field", 8, 3, 3, 1),
    # one pass per step on a grid of many regions (s <= k): a pass must not write the array
    # it reads, since its regions' halos overlap other CTAs' output tiles
    ((200, 130), "periodic", "field", 8, 3, 0, 0),
    ((150, 170), "dirichlet", "field", 4, 2, 3, 8),
]


@pytest.mark.parametrize("case", DF_CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-s{c[3]}-kern{c[5]}-k{c[6]}")
def test_step_parity_dfloat(case):
    shape, bc, kappa, s, nsteps, kernel, kk = case
    u0, field = seeded_case(shape, bc, kappa, 300 + s)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    fo = rounded_field(field, "dfloat")
    opr = oracle_problem(len(shape), bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    ref = O.frkc2_step(u0, oplan["a"], dt, opr, nsteps)
    got, st = run_gpu(plan, shape, bc, kappa, "dfloat", u0, field, dt, nsteps, tune=F.make_tuning(k=kk, kernel=kernel))
    assert st == F.OK
    err = rel_err(got, ref)
    assert err < TOL["dfloat"], err


def test_dfloat_keeps_state_precision_fp32_loses():
    """Many steps on a 2D field problem: the float-pair state stays within MIXED-class error of
    the FP64 oracle while the float state drifts an order of magnitude further."""
    shape = (96, 96)
    u0, field = seeded_case(shape, "periodic", "field", 77)
    s, nsteps = 64, 12
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    fo = rounded_field(field, "fp32")
    opr = oracle_problem(2, "periodic", "field", 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr)
    ref = O.frkc2_step(u0, oplan["a"], dt, opr, nsteps)
    ref32 = O.frkc2_step(u0.astype(np.float32).astype(np.float64), oplan["a"], dt, opr, nsteps)
    got_df, st = run_gpu(plan, shape, "periodic", "field", "dfloat", u0, field, dt, nsteps)
    assert st == F.OK
    got_32, _ = run_gpu(plan, shape, "periodic", "field", "fp32", u0, field, dt, nsteps,
                        tune=F.make_tuning(k=1, kernel=2))
    e_df, e_32 = rel_err(got_df, ref), rel_err(got_32, ref32)
    assert e_df < 1e-6 and e_df * 10 < e_32, (e_df, e_32)


def test_dfloat_launch_count():
    shape = (40, 50)
    u0, field = seeded_case(shape, "periodic", "field", 12)
    plan = F.frkc2_plan(16)
    kt = dev(field, torch.float32)
    pr = lib_problem(shape, "periodic", "field", "dfloat", 1.0, kt)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    dt = 0.5 * plan.info()["beta"] / O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, rounded_field(field, "fp32")))
    u = dev(u0, torch.float64)
    F.frkc2_launch_count()
    F.frkc2_step(plan, pr, dt, 3, 0.0, u, ws, F.make_tuning(kernel=2))
    assert F.frkc2_launch_count() == 2 + 3 * 16  # faces, face pairs, one pass per stage
    v = dev(u0, torch.float64)
    F.frkc2_step(plan, pr, dt, 3, 0.0, v, ws)
    assert F.frkc2_launch_count() == 1 + 3 * 2  # faces, then passes of 8 and 8 stages
    assert rel_err(v.cpu().numpy(), u.cpu().numpy()) < 1e-6


# ---------------------------------------------------------------------------------------
# 3D pass streaming along z (kernel 5, the 3D default at k = 1)
# ---------------------------------------------------------------------------------------

S3_CASES = [
    # shape (nz, ny, nx), bc, kappa, s, nsteps, kernel
    ((12, 10, 14), "periodic", "field", 16, 1, 0),
    ((40, 33, 70), "dirichlet", "field", 8, 2, 5),
    ((35, 70, 7), "periodic", "power", 8, 1, 5),
    ((10, 11, 9), "dirichlet", "power", 16, 1, 0),
    ((70, 17, 31), "dirichlet", "power", 8, 1, 5),
    ((9, 1, 33), "periodic", "field", 8, 2, 5),
    ((1, 20, 1), "dirichlet", "const", 4, 2, 5),
    ((2, 2, 2), "periodic", "power", 4, 1, 5),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("case", S3_CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-s{c[3]}-kern{c[5]}")
def test_step_parity_stream3d(case, prec):
    shape, bc, kappa, s, nsteps, kernel = case
    u0, field = seeded_case(shape, bc, kappa, 400 + s)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    fo = rounded_field(field, prec)
    opr = oracle_problem(3, bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    u0g = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0g, oplan["a"], dt, opr, nsteps)
    got, st = run_gpu(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, tune=F.make_tuning(k=1, kernel=kernel))
    assert st == F.OK
    err = rel_err(got, ref)
    assert err < TOL[prec], err


def test_stream3d_equals_tile_pass_and_rejects_k():
    shape = (24, 20, 40)
    u0, field = seeded_case(shape, "dirichlet", "power", 9)
    plan = F.frkc2_plan(8)
    opr = oracle_problem(3, "dirichlet", "power", 1.0, None)
    dt = 0.9 * plan.info()["beta"] / O.rho_bound(opr, u0)
    a, st_a = run_gpu(plan, shape, "dirichlet", "power", "fp64", u0, None, dt, 1, tune=F.make_tuning(k=1, kernel=5))
    b, st_b = run_gpu(plan, shape, "dirichlet", "power", "fp64", u0, None, dt, 1, tune=F.make_tuning(k=1, kernel=1))
    assert st_a == F.OK and st_b == F.OK
    assert rel_err(a, b) < 1e-13
    pr = lib_problem(shape, "dirichlet", "power", "fp64")
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.Frkc2Error) as e:
        F.frkc2_step(plan, pr, dt, 1, 0.0, dev(u0, torch.float64), ws, F.make_tuning(k=2, kernel=5))
    assert e.value.status == F.EUNSUPPORTED


# ---------------------------------------------------------------------------------------
# 1D whole-job cluster kernel (kernel 6, the 1D default for N <= 16384 and s <= 1024)
# ---------------------------------------------------------------------------------------

S1_CASES = [
    # shape, bc, kappa, s, nsteps, kernel
    ((256,), "dirichlet", "const", 16, 5, 0),
    ((257,), "periodic", "field", 16, 3, 6),
    ((1000,), "dirichlet", "field", 32, 2, 6),
    ((31,), "periodic", "field", 8, 4, 6),
    ((2,), "dirichlet", "const", 4, 2, 6),
    ((16384,), "periodic", "field", 8, 1, 6),
    ((5003,), "dirichlet", "field", 64, 1, 0),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("case", S1_CASES, ids=lambda c: f"{c[0][0]}-{c[1]}-{c[2]}-s{c[3]}-kern{c[5]}")
def test_step_parity_small1d(case, prec):
    shape, bc, kappa, s, nsteps, kernel = case
    u0, field = seeded_case(shape, bc, kappa, 500 + s)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    fo = rounded_field(field, prec)
    opr = oracle_problem(1, bc, kappa, 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    u0g = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0g, oplan["a"], dt, opr, nsteps)
    F.frkc2_launch_count()
    got, st = run_gpu(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, tune=F.make_tuning(kernel=kernel))
    assert F.frkc2_launch_count() == 2  # face set-up and the whole job
    assert st == F.OK
    err = rel_err(got, ref)
    assert err < TOL[prec], err


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_small1d_single_cell(bc):
    """One cell: Dirichlet f = -2 kappa u (both faces to a zero ghost), periodic f = 0."""
    u0 = np.array([0.7])
    oplan = O.plan(8)
    plan = F.frkc2_plan(8)
    opr = oracle_problem(1, bc, "const", 1.0, None)
    dt = 0.5 * oplan["beta"] / max(O.rho_bound(opr, u0), 1.0)
    ref = O.frkc2_step(u0, oplan["a"], dt, opr, 3)
    got, st = run_gpu(plan, (1,), bc, "const", "fp64", u0, None, dt, 3, tune=F.make_tuning(kernel=6))
    assert st == F.OK
    assert abs(got[0] - ref[0]) <= 1e-13 * max(abs(ref[0]), 1e-300) + 1e-300


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-4)])
@pytest.mark.parametrize("n", [256, 3001])
def test_small1d_cluster_size_choice(n, prec, tol):
    """The 1D whole-job kernel with 1, 2, 4 and 8 CTAs in its cluster (tile_x) and the
    library's choice: each against the oracle, and all bit-identical (every cell takes the
    same operations in the same order whatever thread or CTA holds it, and a halo cell is
    recomputed exactly as its owner computes it)."""
    u0, field = seeded_case((n,), "dirichlet", "field", 60 + n)
    plan = F.frkc2_plan(16)
    oplan = O.plan(16)
    fo = rounded_field(field, prec)
    opr = oracle_problem(1, "dirichlet", "field", 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    u0o = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0o, oplan["a"], dt, opr, 5)
    outs = []
    for cl in (0, 1, 2, 4, 8):
        got, st = run_gpu(plan, (n,), "dirichlet", "field", prec, u0, field, dt, 5,
                          tune=F.make_tuning(kernel=6, tile=(cl, 0, 0)))
        assert st == F.OK
        assert rel_err(got, ref) < tol, (cl, rel_err(got, ref))
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0]), rel_err(o, outs[0])


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("n", [31, 256, 3001])
def test_small1d_halo_exchange(n, prec, bc):
    """Clusters of 2 to 8 CTAs that hold their chunk plus a halo of K cells and exchange the
    halos every K stages (K = 1, 3, 5, 8, 16; clamped to the smallest chunk), with 32 to 96
    threads per CTA (raised to what holds the chunk): each against the oracle over 3 steps of
    s = 16, so that exchanges fall inside steps and across step ends, and bit-identical to the
    one-CTA launch."""
    u0, field = seeded_case((n,), bc, "field", 90 + n)
    plan = F.frkc2_plan(16)
    oplan = O.plan(16)
    fo = rounded_field(field, prec)
    opr = oracle_problem(1, bc, "field", 1.0, fo)
    dt = 0.9 * oplan["beta"] / O.rho_bound(opr, u0)
    u0o = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0o, oplan["a"], dt, opr, 3)
    one, st = run_gpu(plan, (n,), bc, "field", prec, u0, field, dt, 3, tune=F.make_tuning(kernel=6, tile=(1, 0, 0)))
    assert st == F.OK
    for cl, kx, th in [(2, 1, 0), (2, 8, 32), (8, 3, 0), (8, 8, 64), (8, 16, 0), (4, 5, 96)]:
        got, st = run_gpu(plan, (n,), bc, "field", prec, u0, field, dt, 3,
                          tune=F.make_tuning(k=kx, kernel=6, tile=(cl, th, 0)))
        assert st == F.OK
        assert rel_err(got, ref) < TOL[prec], (cl, kx, th, rel_err(got, ref))
        assert np.array_equal(got, one), (cl, kx, th, rel_err(got, one))


def test_small1d_rejects_out_of_range():
    plan = F.frkc2_plan(8)
    for shape, kappa in [((16385,), "const"), ((100,), "power")]:
        pr = lib_problem(shape, "periodic", kappa, "fp64")
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        with pytest.raises(F.Frkc2Error) as e:
            F.frkc2_step(plan, pr, 1e-3, 1, 0.0, torch.zeros(shape, dtype=torch.float64, device="cuda"), ws,
                         F.make_tuning(kernel=6))
        assert e.value.status == F.EUNSUPPORTED
