"""GPU parity of the batched persistent launch (frkc2_step_batched / batch_prepare + batch_launch)
against the FP64 oracle, CUDA-graph replay, and the bounded device wait (fault injected on
the device side with a counter nothing advances -- the wait runs out, nothing hangs)."""
import numpy as np
import pytest

from oracle import frkc2_oracle as O
from helpers import oracle_problem, rel_err, seeded_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")

DT = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float64, "dfloat": torch.float64}
KDT = {"fp64": torch.float64, "fp32": torch.float32, "mixed": torch.float32, "dfloat": torch.float32}
TOL = {"fp64": 1e-11, "fp32": 1e-4, "mixed": 1e-6, "dfloat": 1e-6}


def make_batch(prec, bc, specs, seed0=900):
    """specs: list of (ny, nx, s, nsteps)."""
    items = []
    for i, (ny, nx, s, nsteps) in enumerate(specs):
        u0, field = seeded_case((ny, nx), bc, "field", seed0 + 3 * i)
        fo = field if prec == "fp64" else field.astype(np.float32).astype(np.float64)
        opr = oracle_problem(2, bc, "field", 1.0, fo)
        dt = 0.9 * O.beta(s) / O.rho_bound(opr)
        kt = torch.as_tensor(field, dtype=KDT[prec], device="cuda")
        pr = F.make_problem(2, (nx, ny), 1.0, bc, "field", prec, kappa_field=kt)
        items.append(dict(u0=u0, opr=opr, dt=dt, s=s, nsteps=nsteps, pr=pr,
                          u=torch.as_tensor(u0, dtype=DT[prec], device="cuda")))
    return items


def oracle_results(items, prec):
    out = []
    for it in items:
        u0 = it["u0"] if prec != "fp32" else it["u0"].astype(np.float32).astype(np.float64)
        out.append(O.frkc2_step(u0, O.plan(it["s"])["a"], it["dt"], it["opr"], it["nsteps"]))
    return out


SPECS = [(20, 33, 8, 2), (64, 64, 16, 1), (150, 97, 32, 2), (7, 5, 8, 3), (40, 128, 16, 1),
         (90, 90, 8, 1), (31, 17, 32, 1), (128, 40, 16, 2)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_batched_matches_oracle(prec, bc):
    items = make_batch(prec, bc, SPECS)
    plans = [F.frkc2_plan(it["s"]) for it in items]
    tune = F.make_tuning(k=8 if prec == "fp32" else 4)  # s = 8, nsteps = 1 gives a single pass
    nst = [it["nsteps"] for it in items]
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, [it["pr"] for it in items], nst, tune),
                     dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_launch_count()
    F.frkc2_step_batched(plans, [it["pr"] for it in items], [it["dt"] for it in items], nst,
                         [it["u"] for it in items], ws, tune)
    assert F.frkc2_workspace_status(ws) == F.OK
    refs = oracle_results(items, prec)
    for it, ref in zip(items, refs):
        err = rel_err(it["u"].double().cpu().numpy(), ref)
        assert err < TOL[prec], (it["u"].shape, it["s"], it["nsteps"], err)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "dfloat"])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
@pytest.mark.parametrize("rows", [0, 7])
def test_batched_streaming_items_match_oracle(prec, bc, rows):
    """FP64 / MIXED / DFLOAT batches with one stage per pass (the default) run the streaming
    body on tiles of 31 columns x a row block split among the warps (128 rows by default; 7
    makes blocks smaller than the warp count); DFLOAT holds the stage states as float pairs.
    Every item against the oracle, grid norm and every element, over ragged grids of 5 .. 150
    cells a side and 1 .. 3 steps."""
    items = make_batch(prec, bc, SPECS, seed0=1300)
    plans = [F.frkc2_plan(it["s"]) for it in items]
    tune = F.make_tuning(tile=(0, rows, 0)) if rows else None
    if prec == "dfloat":  # its default is the float-pair regions; one stage a pass streams
        tune = F.make_tuning(k=1, tile=(0, rows, 0))
    nst = [it["nsteps"] for it in items]
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, [it["pr"] for it in items], nst, tune),
                     dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step_batched(plans, [it["pr"] for it in items], [it["dt"] for it in items], nst,
                         [it["u"] for it in items], ws, tune)
    assert F.frkc2_workspace_status(ws) == F.OK
    refs = oracle_results(items, prec)
    for it, ref in zip(items, refs):
        err = rel_err(it["u"].double().cpu().numpy(), ref)
        assert err < TOL[prec], (it["u"].shape, it["s"], it["nsteps"], err)


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
@pytest.mark.parametrize("k,group", [(8, 4), (6, 1), (4, 3)])
def test_batched_dfloat_regions_match_oracle(bc, k, group):
    """DFLOAT batches with k stages per pass (8 by default) run the float-pair register-tiled
    64 x 64 regions of the single-problem DFLOAT pass, `group` consecutive regions per item:
    every item against the oracle over ragged grids and 1 .. 3 steps (s = 8 .. 32: passes of
    fewer than k stages at a step's end, single-pass steps)."""
    items = make_batch("dfloat", bc, SPECS, seed0=1700)
    plans = [F.frkc2_plan(it["s"]) for it in items]
    tune = F.make_tuning(k=k, tile=(0, 0, group))
    nst = [it["nsteps"] for it in items]
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, [it["pr"] for it in items], nst, tune),
                     dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step_batched(plans, [it["pr"] for it in items], [it["dt"] for it in items], nst,
                         [it["u"] for it in items], ws, tune)
    assert F.frkc2_workspace_status(ws) == F.OK
    refs = oracle_results(items, "dfloat")
    for it, ref in zip(items, refs):
        err = rel_err(it["u"].double().cpu().numpy(), ref)
        assert err < TOL["dfloat"], (it["u"].shape, it["s"], it["nsteps"], err)


@pytest.mark.parametrize("group", [1, 3])
def test_batched_fp32_regions_per_item(group):
    """FP32 items covering `group` consecutive 64 x 64 regions of one pass (the default is 4,
    used by the other tests): the same results as the oracle on ragged grids."""
    items = make_batch("fp32", "periodic", SPECS, seed0=1500)
    plans = [F.frkc2_plan(it["s"]) for it in items]
    tune = F.make_tuning(k=6, tile=(0, 0, group))
    nst = [it["nsteps"] for it in items]
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, [it["pr"] for it in items], nst, tune),
                     dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step_batched(plans, [it["pr"] for it in items], [it["dt"] for it in items], nst,
                         [it["u"] for it in items], ws, tune)
    assert F.frkc2_workspace_status(ws) == F.OK
    for it, ref in zip(items, oracle_results(items, "fp32")):
        assert rel_err(it["u"].double().cpu().numpy(), ref) < TOL["fp32"]


def test_batched_cuda_graph_replay():
    prec = "fp32"
    items = make_batch(prec, "periodic", SPECS[:5], seed0=950)
    plans = [F.frkc2_plan(it["s"]) for it in items]
    probs = [it["pr"] for it in items]
    nst = [it["nsteps"] for it in items]
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, probs, nst), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    us = [it["u"] for it in items]
    u0s = [u.clone() for u in us]
    F.frkc2_batch_prepare(plans, probs, [it["dt"] for it in items], nst, us, ws)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        F.frkc2_batch_launch(ws, stream=s)  # eager launch on the capture stream first
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [u.clone() for u in us]
    g = torch.cuda.CUDAGraph()
    for u, u0 in zip(us, u0s):
        u.copy_(u0)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        F.frkc2_batch_launch(ws, stream=torch.cuda.current_stream())
    for _ in range(2):
        for u, u0 in zip(us, u0s):
            u.copy_(u0)
        g.replay()
        torch.cuda.synchronize()
        for u, e in zip(us, eager):
            assert torch.equal(u, e)
    assert F.frkc2_workspace_status(ws) == F.OK
    refs = oracle_results(items, prec)
    for it, ref in zip(items, refs):
        assert rel_err(it["u"].double().cpu().numpy(), ref) < TOL[prec]


def test_batched_bounded_wait_reports_timeout():
    """A dependent work item waits on a counter nothing advances: the wait gives up after its
    poll limit, the launch returns, and the status word reads FRKC2_ETIMEOUT."""
    items = make_batch("fp32", "periodic", [(64, 64, 16, 2), (32, 48, 16, 3)], seed0=970)
    plans = [F.frkc2_plan(it["s"]) for it in items]
    probs = [it["pr"] for it in items]
    nst = [it["nsteps"] for it in items]
    tune = F.make_tuning(k=4, wait_limit=2000, fault_inject=1)
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, probs, nst, tune), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step_batched(plans, probs, [it["dt"] for it in items], nst, [it["u"] for it in items], ws, tune)
    assert F.frkc2_workspace_status(ws) == F.ETIMEOUT
    # the context is still usable: a normal launch on a fresh workspace succeeds
    tune_ok = F.make_tuning(k=4)
    ws2 = torch.empty_like(ws)
    F.frkc2_workspace_reset(ws2)
    for it in items:
        it["u"].copy_(torch.as_tensor(it["u0"], dtype=torch.float32, device="cuda"))
    F.frkc2_step_batched(plans, probs, [it["dt"] for it in items], nst, [it["u"] for it in items], ws2, tune_ok)
    assert F.frkc2_workspace_status(ws2) == F.OK


def test_batched_rejects_mixed_kinds():
    items = make_batch("fp64", "periodic", SPECS[:2])
    plans = [F.frkc2_plan(it["s"]) for it in items]
    p2 = F.make_problem(2, (16, 16), 1.0, "periodic", "const", "fp32", kappa_c=1.0)
    with pytest.raises(F.Frkc2Error):
        F.frkc2_batch_workspace_size(plans, [items[0]["pr"], p2], [1, 1])
    p3 = F.make_problem(3, (8, 8, 8), 1.0, "periodic", "const", "fp64", kappa_c=1.0)
    with pytest.raises(F.Frkc2Error) as e:
        F.frkc2_batch_workspace_size(plans, [items[0]["pr"], p3], [1, 1])
    assert e.value.status == F.EUNSUPPORTED


@pytest.mark.parametrize("prec", ["fp64", "fp32", "dfloat"])
def test_batched_64_problems_large_s_matches_oracle(prec):
    """64 uneven problems with s from {16, 64, 128, 256} (every problem above the FP32 threshold
    of the paper's order in the FP32 batch), one persistent launch.  FP64 and DFLOAT items run
    the paper's plans (DFLOAT: the float-pair state that keeps those plans within reach where
    FP32 does not); FP32 items the plans the precision policy gives linear problems (the
    Lebedev-Finogenov order, FP32 within 1e-4 at these s).  Each item against the oracle with
    its own stage order, grid norm and every element."""
    from helpers import oracle_map

    rng = np.random.default_rng(6464)
    specs = [(int(rng.integers(9, 80)), int(rng.integers(9, 80)), int(rng.choice([16, 64, 128, 256])),
              int(rng.integers(1, 3))) for _ in range(64)]
    bc = "periodic"
    items = make_batch(prec, bc, specs, seed0=4000)
    if prec == "fp32":
        plans = [F.frkc2_plan_auto(it["s"], it["pr"], it["nsteps"], 1e-4)[0] for it in items]
        assert all(F.frkc2_precision_policy(p, it["pr"], it["nsteps"], 1e-4)[0] == "fp32"
                   for p, it in zip(plans, items))
    else:
        plans = [F.frkc2_plan(it["s"]) for it in items]
    probs = [it["pr"] for it in items]
    nst = [it["nsteps"] for it in items]
    tune = F.make_tuning(k=8) if prec == "fp32" else None  # FP64: streaming items, DFLOAT: regions (k = 8)
    ws = torch.empty(F.frkc2_batch_workspace_size(plans, probs, nst, tune), dtype=torch.uint8, device="cuda")
    F.frkc2_workspace_reset(ws)
    F.frkc2_step_batched(plans, probs, [it["dt"] for it in items], nst, [it["u"] for it in items], ws, tune)
    assert F.frkc2_workspace_status(ws) == F.OK
    jobs = []
    orders = {s: (O.step_sizes(s)[O.order_lebedev(s)] if prec == "fp32" else O.plan(s)["a"])
              for s in sorted({it["s"] for it in items})}
    for it in items:
        a = orders[it["s"]]
        u0 = it["u0"].astype(np.float32).astype(np.float64) if prec == "fp32" else it["u0"]
        jobs.append((u0, a, it["dt"], it["opr"], it["nsteps"]))
    refs = oracle_map(jobs)
    errs = []
    for it, p, ref in zip(items, plans, refs):
        err = rel_err(it["u"].double().cpu().numpy(), ref)
        errs.append(err)
        tol = TOL[prec]
        if prec == "dfloat":
            # float flux arithmetic under the paper's order: the library's precision model
            # forecasts the DFLOAT error from the order's rounding gain (8e-6 at s = 128 and
            # 4e-5 at s = 256 over 2 steps); below s = 128 it stays under the 1e-6 class
            name, forecast = F.frkc2_precision_policy(p, it["pr"], it["nsteps"], 1e-4)
            if name == "dfloat":
                tol = max(tol, forecast)
        assert err < tol, (it["u"].shape, it["s"], it["nsteps"], err, tol)
    print(prec, "largest error", max(errs))
