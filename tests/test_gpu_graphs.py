"""frkc2_step captured in a CUDA graph: every fast path (2D streaming FP64, 2D register-tiled
FP32, DFLOAT, 3D z-streaming, the 1D cluster kernel, the Brusselator's persistent launch)
queues only kernels and memsets on the caller's stream, so a captured step replays with the
same result as the eager call."""
import numpy as np
import pytest

from oracle import frkc2_oracle as O
from helpers import oracle_problem, seeded_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

DT = {"fp64": torch.float64, "fp32": torch.float32, "dfloat": torch.float64}
KDT = {"fp64": torch.float64, "fp32": torch.float32, "dfloat": torch.float32}

CASES = [
    # shape (numpy order), bc, kappa, precision, s, nsteps
    ((96, 130), "periodic", "field", "fp64", 16, 2),
    ((96, 130), "dirichlet", "field", "fp32", 16, 2),
    ((96, 130), "periodic", "field", "dfloat", 16, 2),
    ((20, 24, 40), "dirichlet", "power", "fp64", 8, 1),
    ((300,), "dirichlet", "field", "fp64", 16, 3),
]


def capture_and_compare(run, reset, outs):
    """Eager call, then the same call captured once and replayed twice: identical results."""
    reset()
    run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    reset()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        run(side)
    for _ in range(2):
        reset()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for o, e in zip(outs, eager):
            assert torch.equal(o, e)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{c[1]}-{c[2]}-{c[3]}")
def test_step_graph_replay(case):
    shape, bc, kappa, prec, s, nsteps = case
    u0, field = seeded_case(shape, bc, kappa, 700 + s)
    plan = F.frkc2_plan(s)
    opr = oracle_problem(len(shape), bc, kappa, 1.0, field)
    dt = 0.8 * plan.info()["beta"] / O.rho_bound(opr, u0)
    kt = torch.as_tensor(field, dtype=KDT[prec], device="cuda") if field is not None else None
    pr = F.make_problem(len(shape), tuple(reversed(shape)), 1.0, bc, kappa, prec, kappa_field=kt)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    u0d = torch.as_tensor(u0, dtype=DT[prec], device="cuda")
    u = u0d.clone()
    capture_and_compare(lambda st: F.frkc2_step(plan, pr, dt, nsteps, 0.0, u, ws, stream=st),
                        lambda: u.copy_(u0d), [u])
    assert F.frkc2_workspace_status(ws) == F.OK


def test_bruss_step_graph_replay():
    import frkc2_inputs as I

    n = 200
    v0, w0 = I.bruss_u0(n, n, 1.0 / n)
    plan = F.frkc2_plan(16)
    pr = F.make_bruss_problem(n)
    ws = torch.empty(F.frkc2_bruss_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    v0d, w0d = torch.as_tensor(v0, device="cuda"), torch.as_tensor(w0, device="cuda")
    v, w = v0d.clone(), w0d.clone()
    dt = 0.8 * plan.info()["beta"] / 6417.0

    def reset():
        v.copy_(v0d)
        w.copy_(w0d)

    capture_and_compare(lambda st: F.frkc2_bruss_step(plan, pr, dt, 5, 0.0, v, w, ws, stream=st), reset, [v, w])
    assert F.frkc2_workspace_status(ws) == F.OK
