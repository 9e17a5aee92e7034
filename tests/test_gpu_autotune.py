"""GPU checks of the autotuner: it picks a candidate that runs, is no slower than the
library default, gives the same result within tolerance, and caches its choice."""
import json
import os

import numpy as np
import pytest

from oracle import frkc2_oracle as O
from helpers import oracle_problem, rel_err, seeded_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")


def test_autotune_step_fp32_and_cache(tmp_path, monkeypatch):
    from paper_1702_03818_gb300 import autotune as AT

    monkeypatch.setenv("FRKC2_TUNE_CACHE", str(tmp_path / "tune.json"))
    shape = (512, 512)
    u0, field = seeded_case(shape, "periodic", "field", 71)
    s = 32
    plan = F.frkc2_plan(s)
    kt = torch.as_tensor(field, dtype=torch.float32, device="cuda")
    pr = F.make_problem(2, (512, 512), 1.0, "periodic", "field", "fp32", kappa_field=kt)
    dt = 0.9 * O.beta(s) / O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, field.astype(np.float32).astype(np.float64)))
    u = torch.as_tensor(u0, dtype=torch.float32, device="cuda")
    u_before = u.clone()
    best, times = AT.autotune_step(plan, pr, u, dt, nsteps=2)
    assert torch.equal(u, u_before)  # the tuner works on a scratch copy
    assert len(times) >= 5
    assert min(times.values()) <= 1.2 * times[json.dumps(dict(k=1, tile=[0, 0, 0], kernel=2))]
    # the wavefront pass is among the candidates of a 512-wide FP32 grid, and runs
    assert any(json.loads(k)["kernel"] == 7 for k in times)
    cached = json.load(open(tmp_path / "tune.json"))
    assert len(cached) == 1
    again, t2 = AT.autotune_step(plan, pr, u, dt, nsteps=2)
    assert t2 == {} and (again.k, again.kernel) == (best.k, best.kernel)
    ws = torch.empty(F.frkc2_workspace_size(pr, best), dtype=torch.uint8, device="cuda")
    a = u.clone()
    F.frkc2_step(plan, pr, dt, 2, 0.0, a, ws, best)
    b = u.clone()
    ws2 = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_step(plan, pr, dt, 2, 0.0, b, ws2)
    assert rel_err(a.double().cpu().numpy(), b.double().cpu().numpy()) < 1e-4


def test_autotune_batch_runs():
    from paper_1702_03818_gb300 import autotune as AT

    specs = [(96, 80, 16), (128, 128, 32), (40, 200, 16)]
    plans, probs, us, dts = [], [], [], []
    for i, (ny, nx, s) in enumerate(specs):
        u0, field = seeded_case((ny, nx), "periodic", "field", 80 + i)
        kt = torch.as_tensor(field, dtype=torch.float32, device="cuda")
        probs.append(F.make_problem(2, (nx, ny), 1.0, "periodic", "field", "fp32", kappa_field=kt))
        plans.append(F.frkc2_plan(s))
        us.append(torch.as_tensor(u0, dtype=torch.float32, device="cuda"))
        dts.append(0.9 * O.beta(s) / O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, field)))
    best, times = AT.autotune_batch(plans, probs, dts, [2] * 3, us)
    # FP32 items run register-tiled 64 x 64 regions: one candidate per stages-per-pass k
    assert best is not None and len(times) >= 4 and best.k in (6, 8, 10) and best.tile_z in (1, 4, 8, 16)
