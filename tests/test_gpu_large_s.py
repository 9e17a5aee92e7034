"""Parity at large stage counts: one step of the 2D variable-conductivity recipe on a 512^2
periodic grid for s = 128 (the paper's greedy order and the Lebedev-Finogenov order), 512 and
1024 (the Lebedev-Finogenov order, the library's default above s = 256), FP64 and FP32,
against the FP64 oracle on the whole grid with the same stage order.  These are the stage
counts of the s sweep on 4096^2 grids; at 512^2 the oracle still runs the whole grid.

With T = 0.9 beta / rho the step is long (beta grows like s^2) and diffusion carries the field
far towards its mean, which the flux form conserves; the FP64 check also compares the
deviation from that mean, where the arithmetic of the stages shows."""
import numpy as np
import pytest

import frkc2_inputs as I
from oracle import frkc2_oracle as O
from helpers import oracle_map, oracle_problem, rel_err, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

N = 512
CASES = [(128, "greedy"), (128, "lebedev"), (512, "default"), (1024, "default")]


def _inputs():
    u0 = I.smooth_unit((N, N), 64.0 * N / 2048, 3819)
    kap = I.kappa_field((N, N), 3818, ell=32.0 * N / 2048)
    return u0, kap


def _oracle_order(s, order):
    return O.plan(s)["a"] if order == "greedy" else O.step_sizes(s)[O.order_lebedev(s)]


@pytest.fixture(scope="module")
def refs():
    u0, kap = _inputs()
    jobs, keys = [], []
    for prec in ("fp64", "fp32"):
        k = kap if prec == "fp64" else kap.astype(np.float32).astype(np.float64)
        u = u0 if prec == "fp64" else u0.astype(np.float32).astype(np.float64)
        opr = oracle_problem(2, "periodic", "field", 1.0, k)
        rho = O.rho_bound(opr)
        for s, order in CASES:
            dt = 0.9 * O.beta(s) / rho
            jobs.append((u, _oracle_order(s, order), dt, opr, 1))
            keys.append((prec, s, order))
    return dict(zip(keys, oracle_map(jobs)))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s,order", CASES)
def test_large_s_one_step_matches_oracle(refs, prec, s, order):
    u0, kap = _inputs()
    flags = {"greedy": F.PLAN_GREEDY, "lebedev": F.PLAN_LEBEDEV, "default": 0}[order]
    plan = F.frkc2_plan(s, flags=flags)
    a_o = _oracle_order(s, order)
    # the same stage order; the step sizes agree to the conditioning of 1 - zeta_j (about eps L^2)
    assert np.max(np.abs(plan.info()["a"] - a_o) / np.abs(a_o)) < 1e-9
    kd = torch.float64 if prec == "fp64" else torch.float32
    sd = torch.float32 if prec == "fp32" else torch.float64
    kt = torch.as_tensor(kap, dtype=kd, device="cuda")
    pr = F.make_problem(2, (N, N), 1.0, "periodic", "field", prec, kappa_field=kt)
    k_o = kap if prec == "fp64" else kap.astype(np.float32).astype(np.float64)
    dt = 0.9 * O.beta(s) / O.rho_bound(oracle_problem(2, "periodic", "field", 1.0, k_o))
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    u = torch.as_tensor(u0, dtype=sd, device="cuda")
    F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws)
    assert F.frkc2_workspace_status(ws) == F.OK
    got = u.double().cpu().numpy()
    ref = refs[(prec, s, order)]
    if prec == "fp64":
        assert rel_err(got, ref) < 1e-11
        m = ref.mean()
        assert rel_l2(got - m, ref - m) < 1e-9
    else:
        pred = F.frkc2_precision_policy(plan, pr, 1, 1.0)[1]  # the FP32 forecast (FP32 is chosen at tol 1)
        tol = 3e-4 if order == "greedy" else 1e-4  # the paper's order at s = 128 is above 1e-4 in FP32
        err = rel_err(got, ref)
        assert err < tol, (err, pred)
        assert rel_l2(got, ref) < 2.0 * pred, (rel_l2(got, ref), pred)  # the policy's forecast holds


def test_ten_thousand_stages_keep_seven_digits():
    """The paper's 10^4 stages (Sec. 2.2: internal stability with about 7 of 16 digits kept at
    accelerations above 6000): one FP64 step of s = 10000 in the Lebedev-Finogenov order on a
    64^2 periodic var-kappa grid against the oracle's literal complex stages in the same order."""
    n, s = 64, 10000
    u0 = I.smooth_unit((n, n), 8.0, 4041)
    kap = I.kappa_field((n, n), 4042, ell=4.0)
    plan = F.frkc2_plan(s)
    assert np.array_equal(plan.info()["order"], O.order_lebedev(s))
    a_o = O.step_sizes(s)[O.order_lebedev(s)]
    opr = oracle_problem(2, "periodic", "field", 1.0, kap)
    dt = 0.9 * O.beta(s) / O.rho_bound(opr)
    ref = O.frkc2_step(u0, a_o, dt, opr, 1)
    pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp64",
                        kappa_field=torch.as_tensor(kap, device="cuda"))
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    u = torch.as_tensor(u0, device="cuda")
    F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws)
    assert F.frkc2_workspace_status(ws) == F.OK
    got = u.cpu().numpy()
    m = ref.mean()
    print("s = 10000 FP64 against the oracle: rel", rel_err(got, ref), "deviation from the mean",
          rel_l2(got - m, ref - m))
    assert rel_err(got, ref) < 1e-7
    assert rel_l2(got - m, ref - m) < 1e-7
