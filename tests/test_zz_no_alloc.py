"""frkc2_step_noalloc: the forward step for callers that cannot allocate device memory.

Such callers (a plugin whose host application owns every device allocation, code running
while its allocator is locked) cannot hand frkc2_step a workspace; this entry point takes
its scratch from an array built into the library.  The tests check, through the C ABI,
that two calls in a row give the same result as frkc2_step with a caller workspace, and
that problems larger than the array are refused.  This file is collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

import frkc2_inputs as I


def _case(prec, shape=(150, 200)):
    u0 = I.smooth_unit(shape, 12.0, 77)
    kap = I.kappa_field(shape, 78, ell=8.0)
    sd = torch.float32 if prec == "fp32" else torch.float64
    kd = torch.float64 if prec == "fp64" else torch.float32
    kt = torch.as_tensor(kap, dtype=kd, device="cuda")
    pr = F.make_problem(2, (shape[1], shape[0]), 1.0, "periodic", "field", prec, kappa_field=kt)
    return torch.as_tensor(u0, dtype=sd, device="cuda"), pr


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-4)])
def test_noalloc_matches_workspace_step_twice(prec, tol):
    u0, pr = _case(prec)
    plan = F.frkc2_plan(32)
    rho_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho_t)
    rho = rho_t.item()
    dt = 0.9 * plan.info()["beta"] / rho
    ref = u0.clone()
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    got = u0.clone()
    for call in range(2):  # two calls in a row, the second continuing from the first
        F.frkc2_step(plan, pr, dt, 2, rho, ref, ws)
        F.frkc2_step_noalloc(plan, pr, dt, 2, rho, got)
        torch.cuda.synchronize()
        a = got.double().cpu().numpy()
        b = ref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < tol, call


def test_noalloc_rejects_problems_larger_than_its_array():
    big = F.make_problem(2, (2048, 2048), 1.0, "periodic", "const", "fp64", kappa_c=1.0)
    assert F.frkc2_workspace_size(big) > F.NOALLOC_SCRATCH_BYTES

    class Fake:
        def data_ptr(self):
            return 1 << 20

    with pytest.raises(F.Frkc2Error) as e:
        F.frkc2_step_noalloc(F.frkc2_plan(8), big, 0.1, 1, 0.0, Fake(), stream=0)
    assert e.value.status == F.ENOMEM
