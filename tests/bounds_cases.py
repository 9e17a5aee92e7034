"""Child process of tests/test_gpu_debug_bounds.py: runs parity cases of the main pass kernels
through the bounds-checking library (FRKC2_DEBUG_BOUNDS=1 is set by the parent before the
binding loads) and prints one JSON line: per case the latched status and the error against
the oracle."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from helpers import oracle_problem, rel_err, seeded_case  # noqa: E402
from oracle import frkc2_oracle as O  # noqa: E402
from paper_1702_03818_gb300 import frkc2 as F  # noqa: E402

assert F.library_path().endswith("libfrkc2_debug.so"), F.library_path()
DT = {"fp64": torch.float64, "fp32": torch.float32}

# shape (numpy order), bc, kappa, precision, s, nsteps, tuning (k, tile, kernel)
CASES = [
    ((77, 100), "periodic", "field", "fp64", 16, 2, dict(kernel=2)),       # 2D streaming
    ((77, 100), "dirichlet", "field", "fp64", 16, 2, dict(kernel=2)),
    ((70, 260), "periodic", "field", "fp32", 16, 2, dict(k=8, kernel=7)),  # wavefront (TMA rows)
    ((70, 260), "dirichlet", "field", "fp32", 16, 2, dict(k=8, kernel=7)),
    ((77, 100), "periodic", "field", "fp32", 16, 2, dict(k=6, kernel=3)),  # register regions
    ((77, 100), "dirichlet", "field", "fp32", 16, 2, dict(k=6, kernel=3)),
    ((77, 100), "dirichlet", "field", "fp64", 8, 2, dict(k=2, tile=(32, 16, 1), kernel=1)),  # tiles
    ((20, 18, 33), "periodic", "field", "fp64", 8, 1, dict(k=2, tile=(16, 8, 4), kernel=1)),
    ((20, 18, 33), "dirichlet", "power", "fp64", 8, 1, dict(k=1, kernel=5)),  # 3D z-streaming
    ((20, 18, 33), "periodic", "field", "fp32", 8, 1, dict(k=1, kernel=5)),
    ((3001,), "dirichlet", "field", "fp64", 16, 3, dict(k=8, tile=(8, 0, 0), kernel=6)),  # 1D cluster
    ((3001,), "periodic", "field", "fp32", 16, 3, dict(k=5, tile=(4, 64, 0), kernel=6)),
]
# grids of one or two cells along an axis, with the library's default kernel for each (the
# 2D streaming pass, the FP32 register regions, the 1D cluster kernel, the 3D z-streaming
# pass) and the shared-memory tiles
CASES += [(shape, bc, "field", prec, 8, 2, dict())
          for shape in [(1, 1), (2, 2), (1, 3), (1,), (2,), (1, 1, 1), (2, 1, 3)]
          for bc in ("periodic", "dirichlet") for prec in ("fp64", "fp32")]
CASES += [((2, 3), bc, "field", "fp64", 8, 2, dict(k=2, kernel=1)) for bc in ("periodic", "dirichlet")]

out = []
for shape, bc, kappa, prec, s, nsteps, tk in CASES:
    u0, field = seeded_case(shape, bc, kappa, 900 + len(out))
    fo = field if (field is None or prec == "fp64") else field.astype(np.float32).astype(np.float64)
    u0o = u0.astype(np.float32).astype(np.float64) if prec == "fp32" else u0
    opr = oracle_problem(len(shape), bc, kappa, 1.0, fo)
    dt = 0.9 * O.beta(s) / O.rho_bound(opr, u0o)
    ref = O.frkc2_step(u0o, O.plan(s)["a"], dt, opr, nsteps)
    tune = F.make_tuning(**tk)
    kt = torch.as_tensor(field, dtype=DT[prec], device="cuda") if field is not None else None
    pr = F.make_problem(len(shape), tuple(reversed(shape)), 1.0, bc, kappa, prec, kappa_field=kt)
    ws = torch.empty(F.frkc2_workspace_size(pr, tune), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    u = torch.as_tensor(u0, dtype=DT[prec], device="cuda")
    F.frkc2_step(F.frkc2_plan(s), pr, dt, nsteps, 0.0, u, ws, tune)
    st = F.frkc2_workspace_status(ws)
    out.append({"case": f"{shape}-{bc}-{kappa}-{prec}-{tk}", "status": int(st),
                "err": rel_err(u.double().cpu().numpy(), ref), "tol": 1e-11 if prec == "fp64" else 1e-4})
print(json.dumps(out))
