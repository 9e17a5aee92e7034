"""Degenerate inputs through the CUDA path: zero steps, and grids of one or two cells along
an axis (the periodic wrap onto the cell itself, a Dirichlet cell whose four neighbours are
ghosts), each against the oracle."""
import numpy as np
import pytest

from oracle import frkc2_oracle as O
from helpers import oracle_problem, rel_err, seeded_case
from test_gpu_forward import F, rounded_field, run_gpu, torch, dev, lib_problem

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-5}


def test_zero_steps_leave_the_state_untouched():
    shape = (40, 33)
    u0, field = seeded_case(shape, "periodic", "field", 31)
    u = dev(u0, torch.float64)
    before = u.clone()
    pr = lib_problem(shape, "periodic", "field", "fp64", 1.0, dev(field, torch.float64))
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_launch_count()
    F.frkc2_step(F.frkc2_plan(16), pr, 1.0, 0, 0.0, u, ws)
    torch.cuda.synchronize()
    assert F.frkc2_launch_count() == 0
    assert torch.equal(u, before)
    assert F.frkc2_workspace_status(ws) == F.OK


SHAPES = [(1, 1), (1, 2), (2, 2), (2, 7), (1,), (2,), (1, 1, 1), (2, 1, 3)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tiny_grids_match_oracle(shape, bc, prec):
    rng = np.random.default_rng(len(shape) * 10 + sum(shape))
    u0 = rng.random(shape)
    field = np.exp(0.5 * rng.standard_normal(shape))
    fo = rounded_field(field, prec)
    opr = oracle_problem(len(shape), bc, "field", 1.0, fo)
    s = 8
    dt = 0.9 * O.beta(s) / O.rho_bound(opr)
    u0g = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    ref = O.frkc2_step(u0g, O.plan(s)["a"], dt, opr, 3)
    got, st = run_gpu(F.frkc2_plan(s), shape, bc, "field", prec, u0, field, dt, 3)
    assert st == F.OK
    if bc == "periodic" and all(n == 1 for n in shape):
        assert np.array_equal(got, u0g)  # every neighbour is the cell itself: f = 0 exactly
    assert rel_err(got, ref) < TOL[prec], rel_err(got, ref)
