"""GPU parity of the adjoint (frkc2_adjoint) against the FP64 oracle, the dot-product test,
central finite differences of the GPU forward, and the autograd wrapper."""
import numpy as np
import pytest

from oracle import frkc2_oracle as O
from helpers import oracle_problem, rel_err, seeded_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

DT = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float64}
KDT = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float32}


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_adjoint(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, ckpt, g, dx=1.0, want_dk=True):
    kt = dev(field, KDT[prec]) if field is not None else None
    pr = F.make_problem(len(shape), tuple(reversed(shape)), dx, bc, kappa, prec, kappa_field=kt)
    ws = torch.empty(F.frkc2_adjoint_workspace_size(plan, pr, nsteps, ckpt), dtype=torch.uint8, device="cuda")
    du = torch.empty(shape, dtype=DT[prec], device="cuda")
    dk = torch.empty(shape, dtype=KDT[prec], device="cuda") if (want_dk and kappa == "field") else None
    F.frkc2_adjoint(plan, pr, dt, nsteps, ckpt, dev(u0, DT[prec]), dev(g, DT[prec]), du, dk, ws)
    torch.cuda.synchronize()
    return du.double().cpu().numpy(), (dk.double().cpu().numpy() if dk is not None else None)


def gpu_forward(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, dx=1.0):
    kt = dev(field, KDT[prec]) if field is not None else None
    pr = F.make_problem(len(shape), tuple(reversed(shape)), dx, bc, kappa, prec, kappa_field=kt)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    u = dev(u0, DT[prec])
    F.frkc2_step(plan, pr, dt, nsteps, 0.0, u, ws)
    return u.double().cpu().numpy()


CASES = [
    # shape, bc, kappa, s, nsteps, ckpt
    ((48, 40), "periodic", "field", 16, 5, 2),
    ((37, 29), "dirichlet", "field", 8, 3, 3),
    ((300,), "dirichlet", "const", 16, 4, 1),
    ((9, 8, 7), "periodic", "field", 8, 2, 1),
    ((8, 7, 6), "dirichlet", "power", 8, 2, 2),
    ((30, 26), "periodic", "power", 8, 2, 1),
]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-3), ("mixed", 1e-5)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}")
def test_adjoint_matches_oracle(case, prec, tol):
    shape, bc, kappa, s, nsteps, ckpt = case
    u0, field = seeded_case(shape, bc, kappa, 500 + s)
    fo = field if (field is None or prec == "fp64") else field.astype(np.float32).astype(np.float64)
    u0o = u0 if prec != "fp32" else u0.astype(np.float32).astype(np.float64)
    opr = oracle_problem(len(shape), bc, kappa, 1.0, fo)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    dt = 0.8 * oplan["beta"] / O.rho_bound(opr, u0o)
    rng = np.random.default_rng(7)
    g = rng.standard_normal(shape)
    if prec == "fp32":
        g = g.astype(np.float32).astype(np.float64)
    ref_u, ref_k = O.frkc2_adjoint(u0o, oplan["a"], dt, opr, nsteps, g)
    du, dk = gpu_adjoint(plan, shape, bc, kappa, prec, u0, field, dt, nsteps, ckpt, g)
    assert rel_err(du, ref_u) < tol, rel_err(du, ref_u)
    if kappa == "field":
        assert rel_err(dk, ref_k) < tol, rel_err(dk, ref_k)


def test_dot_product_gpu_forward_vs_gpu_adjoint():
    """<J v, w> = <v, J^T w> with J the GPU forward map (linear in u0) and J^T the GPU adjoint."""
    shape = (64, 64)
    _, field = seeded_case(shape, "periodic", "field", 41)
    rng = np.random.default_rng(42)
    v, w = rng.standard_normal(shape), rng.standard_normal(shape)
    s, nsteps = 32, 6
    plan = F.frkc2_plan(s)
    opr = oracle_problem(2, "periodic", "field", 1.0, field)
    dt = 0.9 * O.beta(s) / O.rho_bound(opr)
    Jv = gpu_forward(plan, shape, "periodic", "field", "fp64", v, field, dt, nsteps)
    JTw, _ = gpu_adjoint(plan, shape, "periodic", "field", "fp64", v, field, dt, nsteps, 4, w, want_dk=False)
    lhs, rhs = float(np.vdot(Jv, w)), float(np.vdot(v, JTw))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)


def test_kappa_gradient_central_differences_64():
    """dJ/dkappa of J = ||u(T) - u_tgt||^2 against central differences of the GPU forward (64^2)."""
    shape = (64, 64)
    u0, field = seeded_case(shape, "periodic", "field", 43)
    tgt, _ = seeded_case(shape, "periodic", "field", 44)
    s, nsteps = 16, 4
    plan = F.frkc2_plan(s)
    dt = 0.8 * O.beta(s) / O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, field))

    def loss(k, u):
        uT = gpu_forward(plan, shape, "periodic", "field", "fp64", u, k, dt, nsteps)
        return float(np.sum((uT - tgt) ** 2))

    uT = gpu_forward(plan, shape, "periodic", "field", "fp64", u0, field, dt, nsteps)
    du, dk = gpu_adjoint(plan, shape, "periodic", "field", "fp64", u0, field, dt, nsteps, 2, 2 * (uT - tgt))
    for idx in [(0, 0), (10, 33), (63, 5), (40, 63)]:
        h = 1e-6 * field[idx]
        kp, km = field.copy(), field.copy()
        kp[idx] += h
        km[idx] -= h
        fd = (loss(kp, u0) - loss(km, u0)) / (2 * h)
        assert abs(fd - dk[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, dk[idx])
        up, um = u0.copy(), u0.copy()
        up[idx] += 1e-6
        um[idx] -= 1e-6
        fdu = (loss(field, up) - loss(field, um)) / 2e-6
        assert abs(fdu - du[idx]) < 1e-6 * max(1.0, abs(fdu)), (idx, fdu, du[idx])


def test_autograd_wrapper():
    from paper_1702_03818_gb300.autograd import frkc2_steps

    shape = (40, 52)
    u0, field = seeded_case(shape, "periodic", "field", 45)
    s, nsteps = 16, 3
    plan = F.frkc2_plan(s)
    dt = 0.8 * O.beta(s) / O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, field))
    u = dev(u0, torch.float64).requires_grad_(True)
    k = dev(field, torch.float64).requires_grad_(True)
    tgt = dev(np.zeros(shape), torch.float64)
    out = frkc2_steps(u, k, plan, dt, nsteps, ckpt_every=2)
    J = ((out - tgt) ** 2).sum()
    J.backward()
    oplan = O.plan(s)
    opr = oracle_problem(2, "periodic", "field", 1.0, field)
    uT = O.frkc2_step(u0, oplan["a"], dt, opr, nsteps)
    ref_u, ref_k = O.frkc2_adjoint(u0, oplan["a"], dt, opr, nsteps, 2 * uT)
    assert rel_err(u.grad.cpu().numpy(), ref_u) < 1e-10
    assert rel_err(k.grad.cpu().numpy(), ref_k) < 1e-10


@pytest.mark.parametrize("shape,bc", [((50, 44), "periodic"), ((33, 41), "dirichlet")])
def test_split_forward_backward_equals_combined(shape, bc):
    u0, field = seeded_case(shape, bc, "field", 61)
    s, nsteps, ck = 16, 5, 2
    plan = F.frkc2_plan(s)
    dt = 0.8 * O.beta(s) / O.rho_bound(oracle_problem(2, bc, "field", 1.0, field))
    kt = dev(field, torch.float64)
    pr = F.make_problem(2, tuple(reversed(shape)), 1.0, bc, "field", "fp64", kappa_field=kt)
    ws = torch.empty(F.frkc2_adjoint_workspace_size(plan, pr, nsteps, ck), dtype=torch.uint8, device="cuda")
    u0d = dev(u0, torch.float64)
    uT = torch.empty_like(u0d)
    F.frkc2_adjoint_forward(plan, pr, dt, nsteps, ck, u0d, uT, ws)
    ref_uT = gpu_forward(plan, shape, bc, "field", "fp64", u0, field, dt, nsteps)
    assert rel_err(uT.cpu().numpy(), ref_uT) < 1e-13
    g = np.random.default_rng(62).standard_normal(shape)
    du = torch.empty_like(u0d)
    dk = torch.empty_like(kt)
    F.frkc2_adjoint_backward(plan, pr, dt, nsteps, ck, dev(g, torch.float64), du, dk, ws)
    du2, dk2 = gpu_adjoint(plan, shape, bc, "field", "fp64", u0, field, dt, nsteps, ck, g)
    assert np.array_equal(du.cpu().numpy(), du2) and np.array_equal(dk.cpu().numpy(), dk2)
    ref_u, ref_k = O.frkc2_adjoint(u0, O.plan(s)["a"], dt, oracle_problem(2, bc, "field", 1.0, field), nsteps, g)
    assert rel_err(du2, ref_u) < 1e-10 and rel_err(dk2, ref_k) < 1e-10


TB_CASES = [
    # shape (ny, nx), bc, s, nsteps, ckpt: FP32 fixed-conductivity 2D problems run the
    # temporally blocked tape and reverse passes (8 stages each): several 64 x 64 regions,
    # a ragged last pass, grids smaller than a region, segments recomputed from checkpoints
    ((70, 100), "periodic", 20, 3, 2),
    ((61, 97), "dirichlet", 12, 2, 1),
    ((3, 5), "periodic", 8, 2, 2),
    ((50, 130), "dirichlet", 64, 1, 1),
    ((49, 49), "periodic", 10, 4, 3),
]


@pytest.mark.parametrize("case", TB_CASES, ids=lambda c: f"{c[0][0]}x{c[0][1]}-{c[1]}-s{c[2]}")
def test_adjoint_fp32_temporal_blocking_matches_oracle(case):
    shape, bc, s, nsteps, ckpt = case
    u0, field = seeded_case(shape, bc, "field", 900 + s)
    fo = field.astype(np.float32).astype(np.float64)
    u0o = u0.astype(np.float32).astype(np.float64)
    opr = oracle_problem(2, bc, "field", 1.0, fo)
    oplan = O.plan(s)
    plan = F.frkc2_plan(s)
    dt = 0.8 * oplan["beta"] / O.rho_bound(opr, u0o)
    g = np.random.default_rng(8).standard_normal(shape).astype(np.float32).astype(np.float64)
    ref_u, ref_k = O.frkc2_adjoint(u0o, oplan["a"], dt, opr, nsteps, g)
    du, dk = gpu_adjoint(plan, shape, bc, "field", "fp32", u0, field, dt, nsteps, ckpt, g)
    assert rel_err(du, ref_u) < 2e-3, rel_err(du, ref_u)
    assert rel_err(dk, ref_k) < 2e-3, rel_err(dk, ref_k)


def test_adjoint_fp32_dot_product_with_fp32_forward():
    """<J v, w> = <v, J^T w> between the FP32 forward (register-tiled passes) and the FP32
    temporally blocked adjoint, to FP32 rounding."""
    shape = (96, 80)
    _, field = seeded_case(shape, "periodic", "field", 47)
    rng = np.random.default_rng(48)
    v = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    w = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    s, nsteps = 24, 3
    plan = F.frkc2_plan(s)
    opr = oracle_problem(2, "periodic", "field", 1.0, field.astype(np.float32).astype(np.float64))
    dt = 0.9 * O.beta(s) / O.rho_bound(opr)
    Jv = gpu_forward(plan, shape, "periodic", "field", "fp32", v, field, dt, nsteps)
    JTw, _ = gpu_adjoint(plan, shape, "periodic", "field", "fp32", v, field, dt, nsteps, 2, w, want_dk=False)
    lhs, rhs = float(np.vdot(Jv, w)), float(np.vdot(v, JTw))
    assert abs(lhs - rhs) < 1e-4 * np.linalg.norm(Jv) * np.linalg.norm(w), (lhs, rhs)
