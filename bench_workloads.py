"""Benchmarks of the other FRKC2 workloads (``python bench.py --workload NAME``).

Each function times one workload on cuda:0 and returns a JSON-ready dict in the bench line
format.  Timing: CUDA events on the launching stream, warm-up runs first, L2 flushed (a
256 MiB write) before every timed run, outside the events.  Errors of FP32 / MIXED runs are
stated against the FP64 GPU result of the same job; parity of every path with the FP64 oracle
is established by the GPU tests (tests/test_gpu_*.py) on reduced instances of these recipes.

Workloads (sizes and seeds from frkc2_inputs.CONFIGS):
  heat1d       1D heat, N = 256 Dirichlet, s = 16, 87 steps to T = 0.05, FP64 (one cluster launch).
  nonlinear3d  3D kappa(u) = 1 + u^2.5, 256^3 Dirichlet hot spot with 1 % noise; one bench
               step = one FRKC2 step at FP64, FP32 and MIXED.  s = 32: with s = 128 the complex
               stages amplify the noise modes until kappa(W) leaves the stability bound and the
               run (and the FP64 oracle on reduced grids) produces non-finite values.
  adjoint2d    2D var-kappa 1024^2, s = 100, 40 steps, checkpoint every 8: forward vs adjoint.
  batched2d    512 2D var-kappa problems (n ~ U{64..1024}, s ~ {16..256}, 10 steps), one
               persistent launch replayed from a CUDA graph, FP32 and FP64; k (and the FP64
               tile) chosen by the autotuner on a 48-problem slice.
  ssweep       4096^2 var-kappa, s in {32, 128, 512, 1024}, 4 steps, FP32 vs FP64 error growth
               with s (internal amplification).
  bruss2d      the paper's Brusselator (Sec. 3.1): 200^2 periodic, s = 16, dt = 0.9 beta/rho, to
               t = 1, FP64 and FP32, persistent launch vs one launch per stage; plus 2048^2,
               s = 64, 10 steps for throughput against the FP64-pipe and HBM rooflines.
"""
from __future__ import annotations

import numpy as np

import frkc2_inputs as I

UNIT = "cell-stage/s"


def _torch():
    import torch
    return torch


def _timed(fn, warmup=2, reps=3, flush=None):
    torch = _torch()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms)), ms


def _dt(torch):
    return {"fp64": (torch.float64, torch.float64), "fp32": (torch.float32, torch.float32),
            "mixed": (torch.float64, torch.float32), "dfloat": (torch.float64, torch.float32)}


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def heat1d(F, sweep: bool = True):
    """The 1D heat workload (N = 256 Dirichlet, s = 16, 87 steps) with the library's default
    whole-job kernel in FP64 and FP32, and (sweep) the kernel's cluster size, stages per halo
    exchange and threads per CTA; each against the FP64 default run."""
    torch = _torch()
    cfg = I.CONFIGS["heat1d"]
    u0, _, dx = I.heat1d_u0(cfg["n"], 8, cfg["seed"])
    s = cfg["s"]
    plan = F.frkc2_plan(s)
    beta = plan.info()["beta"]
    nsteps = int(np.ceil(cfg["t_end"] / (0.9 * beta * dx * dx / 4.0)))
    dt = cfg["t_end"] / nsteps
    cs = cfg["n"] * s * nsteps

    def run(prec, tune=None):
        pr = F.make_problem(1, (cfg["n"],), dx, "dirichlet", "const", prec, kappa_c=1.0)
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        u0d = torch.as_tensor(u0, dtype=_dt(torch)[prec][0], device="cuda")
        u = u0d.clone()

        def job():
            u.copy_(u0d)
            F.frkc2_step(plan, pr, dt, nsteps, 0.0, u, ws, tune)

        med, _ = _timed(job, 3, 5)
        return med, u.double().cpu().numpy()

    ms64, ref = run("fp64")
    ms32, u32 = run("fp32")
    out = {"workload": "heat1d: 1D heat N=256 Dirichlet, s=16, 87 steps, FP64", "metric": "cell-stage/s",
           "value": cs / (ms64 / 1e3), "unit": UNIT, "ms_per_job": ms64, "nsteps": nsteps,
           "fp32": {"ms_per_job": ms32, "value": cs / (ms32 / 1e3), "rel_l2_vs_fp64": _rel(u32, ref)},
           "kernel": "1D whole-job cluster kernel (one launch for all 87 x 16 stages)"}
    if sweep:
        rows = {}
        for prec in ("fp64", "fp32"):
            for cl in (1, 2, 4, 8):
                for kx in ((0,) if cl == 1 else (1, 4, 8, 16)):
                    for th in (32, 64, 128, 256):
                        tune = F.make_tuning(k=kx, kernel=6, tile=(cl, th, 0))
                        try:
                            ms, u = run(prec, tune)
                        except F.Frkc2Error:
                            continue
                        rows[f"{prec}_cl{cl}_k{kx}_t{th}"] = {"ms_per_job": ms, "rel_l2_vs_fp64": _rel(u, ref)}
        out["sweep"] = rows
    return out


def nonlinear3d(F, n=None):
    torch = _torch()
    cfg = I.CONFIGS["nonlinear3d"]
    n = n or cfg["n"]
    s = cfg["s_stable"]
    u0 = I.hotspot3d_u0(n, sigma=20.0 * n / cfg["n"], seed=cfg["seed"])
    plan = F.frkc2_plan(s)
    beta = plan.info()["beta"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out, results = {}, {}
    rho_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    pr64 = F.make_problem(3, (n, n, n), 1.0, "dirichlet", "power", "fp64", kappa_c=1.0, kappa_p=2.5)
    F.frkc2_rho_bound(pr64, torch.as_tensor(u0, device="cuda"), rho_t)
    dt = cfg["cfl"] * beta / rho_t.item()
    for prec in ("fp64", "fp32", "mixed"):
        sd, _ = _dt(torch)[prec]
        pr = F.make_problem(3, (n, n, n), 1.0, "dirichlet", "power", prec, kappa_c=1.0, kappa_p=2.5)
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        u0d = torch.as_tensor(u0, dtype=sd, device="cuda")
        u = u0d.clone()

        def job():
            u.copy_(u0d)
            F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws)

        med, _ = _timed(job, 1, 3, flush)
        results[prec] = u.double().cpu().numpy()
        out[prec] = {"value": n ** 3 * s / (med / 1e3), "ms_per_step": med,
                     "status": F.frkc2_workspace_status(ws)}
        del ws, u, u0d
    for prec in ("fp32", "mixed"):
        out[prec]["rel_l2_vs_fp64_gpu"] = _rel(results[prec], results["fp64"])
    return {"workload": f"nonlinear3d: 3D kappa(u)=1+u^2.5 {n}^3 Dirichlet, s={s}, one FRKC2 step per bench step",
            "metric": "cell-stage/s", "value": out["fp64"]["value"], "unit": UNIT, "dtype": "f64",
            "precisions": out,
            "kernel": "3D pass streaming along z (k = 1)"}


def adjoint2d(F):
    torch = _torch()
    cfg = I.CONFIGS["adjoint2d"]
    n, s, nsteps, ck = cfg["n"], cfg["s"], cfg["steps"], cfg["ckpt"]
    u0 = I.smooth_unit((n, n), 64.0 * n / 2048, cfg["u0_seed"])
    kap = I.kappa_field((n, n), cfg["kappa_seed"], ell=32.0 * n / 2048)
    tgt = I.smooth_unit((n, n), 64.0 * n / 2048, cfg["target_seed"])
    plan = F.frkc2_plan(s)
    beta = plan.info()["beta"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    for prec in ("fp64", "fp32"):
        sd, kd = _dt(torch)[prec]
        kt = torch.as_tensor(kap, dtype=kd, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
        rho_t = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho_t)
        dt = cfg["cfl"] * beta / rho_t.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        u0d = torch.as_tensor(u0, dtype=sd, device="cuda")
        u = u0d.clone()

        def fwd():
            u.copy_(u0d)
            F.frkc2_step(plan, pr, dt, nsteps, 0.0, u, ws)

        tf, _ = _timed(fwd, 1, 3, flush)
        g = 2.0 * (u - torch.as_tensor(tgt, dtype=sd, device="cuda"))
        wsa = torch.empty(F.frkc2_adjoint_workspace_size(plan, pr, nsteps, ck), dtype=torch.uint8, device="cuda")
        du = torch.empty_like(u0d)
        dk = torch.empty_like(kt)

        def adj():
            F.frkc2_adjoint(plan, pr, dt, nsteps, ck, u0d, g, du, dk, wsa)

        ta, _ = _timed(adj, 1, 3, flush)
        uT = torch.empty_like(u0d)

        def adj_fwd():
            F.frkc2_adjoint_forward(plan, pr, dt, nsteps, ck, u0d, uT, wsa)

        def adj_bwd():
            F.frkc2_adjoint_backward(plan, pr, dt, nsteps, ck, g, du, dk, wsa)

        # the backward needs the forward's checkpoints: time the pair, then the forward alone
        tfa, _ = _timed(adj_fwd, 1, 3, flush)
        ms_b = []
        for _ in range(3):
            adj_fwd()
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            adj_bwd()
            e1.record()
            e1.synchronize()
            ms_b.append(e0.elapsed_time(e1))
        tb = float(np.median(ms_b))
        res[prec] = {"forward_ms": tf, "adjoint_ms": ta, "adjoint_over_forward": ta / tf,
                     "adjoint_forward_ms": tfa, "adjoint_backward_ms": tb,
                     "backward_over_forward": tb / tf,
                     "forward_value": n * n * s * nsteps / (tf / 1e3),
                     "workspace_gb": wsa.numel() / 1e9,
                     "grad_norms": [float(du.double().norm()), float(dk.double().norm())]}
        del wsa, ws
    return {"workload": f"adjoint2d: 2D var-kappa {n}^2 periodic, s={s}, {nsteps} steps, checkpoint every {ck}",
            "metric": "adjoint backward time / forward time", "value": res["fp64"]["backward_over_forward"],
            "unit": "ratio", "higher_is_better": False, "precisions": res,
            "note": ("frkc2_adjoint = frkc2_adjoint_forward (the integration keeping checkpoints) + "
                     "frkc2_adjoint_backward (segment recompute + reverse stages); forward = frkc2_step")}


def batched2d(F):
    torch = _torch()
    cfg = I.CONFIGS["batched2d"]
    specs = I.batched_problems(cfg["count"], cfg["seed"])
    nsteps = cfg["steps"]
    plans = {s: F.frkc2_plan(s) for s in sorted({p["s"] for p in specs})}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fields = []
    for p in specs:
        n = p["n"]
        u = I.grf_torch(n, 64.0 * n / 2048, p["u0_seed"])
        u = (u - u.min()) / (u.max() - u.min())
        k = torch.exp(0.5 * I.grf_torch(n, 32.0 * n / 2048, p["kappa_seed"]))
        fields.append((u, k))
    # FP32 items take the plans the precision policy gives these problems at 1e-4 over the job
    # (the Lebedev-Finogenov order; with the paper's order the s = 128 / 256 items would exceed
    # 1e-4 in FP32); the policy must choose FP32 for every item
    probe = F.make_problem(2, (64, 64), 1.0, "periodic", "field", "fp32")
    auto = {sv: F.frkc2_plan_auto(sv, probe, nsteps, 1e-4) for sv in plans}
    assert all(a[1] == "fp32" for a in auto.values()), {sv: a[1] for sv, a in auto.items()}
    res = {}
    finals = {}
    for prec in ("fp32", "fp64", "dfloat"):
        sd, kd = _dt(torch)[prec]
        probs, us, u0s, dts, pl = [], [], [], [], []
        for p, (u, k) in zip(specs, fields):
            kt = k.to(kd).contiguous()
            pr = F.make_problem(2, (p["n"], p["n"]), 1.0, "periodic", "field", prec, kappa_field=kt)
            rho_t = torch.zeros(1, dtype=torch.float64, device="cuda")
            F.frkc2_rho_bound(pr, None, rho_t)
            dts.append(0.9 * plans[p["s"]].info()["beta"] / rho_t.item())
            probs.append(pr)
            u0s.append(u.to(sd).contiguous())
            us.append(u0s[-1].clone())
            pl.append(auto[p["s"]][0] if prec == "fp32" else plans[p["s"]])
        nst = [nsteps] * len(specs)
        # stages per pass and tile from the autotuner, timed on a 48-problem slice of the batch
        from paper_1702_03818_gb300.autotune import autotune_batch
        m = 48
        tune, tt = autotune_batch(pl[:m], probs[:m], dts[:m], nst[:m], us[:m], reps=1)
        for u, u0 in zip(us, u0s):
            u.copy_(u0)
        ws = torch.empty(F.frkc2_batch_workspace_size(pl, probs, nst, tune), dtype=torch.uint8, device="cuda")
        F.frkc2_workspace_reset(ws)
        F.frkc2_batch_prepare(pl, probs, dts, nst, us, ws, tune)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            F.frkc2_batch_launch(ws, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            F.frkc2_batch_launch(ws, stream=torch.cuda.current_stream())

        def reset():
            for u, u0 in zip(us, u0s):
                u.copy_(u0)

        ms = []
        for it in range(4):
            reset()
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            if it >= 1:
                ms.append(e0.elapsed_time(e1))
        assert F.frkc2_workspace_status(ws) == F.OK
        finals[prec] = [u.double() for u in us]
        cs = sum(p["n"] ** 2 * p["s"] * nsteps for p in specs)
        # consistency: three problems against the single-problem path
        errs = []
        for i in (0, len(specs) // 2, len(specs) - 1):
            wsi = torch.empty(F.frkc2_workspace_size(probs[i]), dtype=torch.uint8, device="cuda")
            v = u0s[i].clone()
            F.frkc2_step(pl[i], probs[i], dts[i], nsteps, 0.0, v, wsi)
            errs.append(_rel(us[i].double().cpu().numpy(), v.double().cpu().numpy()))
        # the same 512 problems one frkc2_step call after another on one stream (the library's
        # default kernel for each, one workspace reused), timed the same way
        wsmax = max(F.frkc2_workspace_size(pr) for pr in probs)
        wss = torch.empty(wsmax, dtype=torch.uint8, device="cuda")
        vs = [u0.clone() for u0 in u0s]

        def sequential():
            for i in range(len(specs)):
                F.frkc2_step(pl[i], probs[i], dts[i], nsteps, 0.0, vs[i], wss)

        sequential()  # warm-up: first-call launch configuration queries
        torch.cuda.synchronize()
        sms = []
        for it in range(2):
            for v, u0 in zip(vs, u0s):
                v.copy_(u0)
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sequential()
            e1.record()
            e1.synchronize()
            sms.append(e0.elapsed_time(e1))
        seq_ms = float(min(sms))
        del wss, vs
        res[prec] = {"value": cs / (np.median(ms) / 1e3), "ms_per_launch": float(np.median(ms)),
                     "sequential_single_problem": {"ms": seq_ms, "value": cs / (seq_ms / 1e3),
                                                   "batched_speedup": seq_ms / float(np.median(ms))},
                     "cell_stages": cs, "max_rel_l2_vs_single_problem_path": max(errs),
                     "plans": ("precision policy (Lebedev-Finogenov order), largest predicted FP32 error "
                               f"{max(a[2] for a in auto.values()):.2e}" if prec == "fp32" else "the paper's order"),
                     "workspace_gb": ws.numel() / 1e9,
                     "tuning": {"k": tune.k, "tile": [tune.tile_x, tune.tile_y, tune.tile_z]}, "autotune_ms": tt}
        del ws, g
    # every item of the FP32 and DFLOAT launches against the FP64 launch's result
    for prec in ("fp32", "dfloat"):
        res[prec]["max_rel_l2_vs_fp64_batch"] = max(
            float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(finals[prec], finals["fp64"]))
    del finals
    return {"workload": "batched2d: 512 var-kappa 2D problems, n~U{64..1024}, s~{16..256}, 10 steps, one persistent launch (CUDA graph)",
            "metric": "cell-stage/s", "value": res["fp32"]["value"], "unit": UNIT, "precisions": res}


def ssweep(F):
    torch = _torch()
    n = 4096
    u0 = I.smooth_unit((n, n), 64.0 * 2, 3819)
    kap = I.kappa_field((n, n), 3818, ell=64.0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for s in (32, 128, 512, 1024):
        plan = F.frkc2_plan(s)
        info = plan.info()
        row = {"Q_over_L2": info["Q"] / s ** 2}
        res = {}
        for prec in ("fp64", "fp32"):
            sd, kd = _dt(torch)[prec]
            kt = torch.as_tensor(kap, dtype=kd, device="cuda")
            pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
            rho_t = torch.zeros(1, dtype=torch.float64, device="cuda")
            F.frkc2_rho_bound(pr, None, rho_t)
            dt = 0.9 * info["beta"] / rho_t.item()
            ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
            u0d = torch.as_tensor(u0, dtype=sd, device="cuda")
            u = u0d.clone()

            def job():
                u.copy_(u0d)
                F.frkc2_step(plan, pr, dt, 4, 0.0, u, ws)

            med, _ = _timed(job, 1, 2, flush)
            res[prec] = u.double().cpu().numpy()
            row[prec] = {"value": n * n * s * 4 / (med / 1e3), "ms": med}
            del ws
        row["fp32_rel_l2_vs_fp64_gpu"] = _rel(res["fp32"], res["fp64"])
        out[str(s)] = row
    return {"workload": "ssweep: 4096^2 var-kappa periodic, s in {32,128,512,1024}, 4 steps, FP32 vs FP64",
            "metric": "fp32 error vs fp64 by s", "value": out["1024"]["fp32_rel_l2_vs_fp64_gpu"], "unit": "rel L2",
            "by_s": out}


def precision(F):
    """Error of each reduced precision against the FP64 GPU run of the same 2048^2 var-kappa
    job (the bench recipe) by stage count and ordering, after 1, 10 and 100 steps (the job's
    length): the stage count up to which FP32 state and arithmetic stay within 1e-4 relative
    L2, what the float-pair state (DFLOAT) and MIXED give beyond it, and beside each the
    precision policy's predicted FP32 error and its choice (frkc2_precision_policy)."""
    torch = _torch()
    cfg = I.CONFIGS["varkappa2d"]
    n = cfg["n"]
    u0 = I.smooth_unit((n, n), 64.0, cfg["u0_seed"])
    kap = I.kappa_field((n, n), cfg["kappa_seed"])
    precs = ("fp64", "fp32", "dfloat", "mixed")
    probs, wss = {}, {}
    for prec in precs:
        kd = torch.float64 if prec == "fp64" else torch.float32
        kt = torch.as_tensor(kap, dtype=kd, device="cuda")
        probs[prec] = (F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt), kt)
        wss[prec] = torch.empty(F.frkc2_workspace_size(probs[prec][0]), dtype=torch.uint8, device="cuda")
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(probs["fp64"][0], None, rho)
    rows = {}
    threshold = {}
    for order, flag in (("greedy", F.PLAN_GREEDY), ("lebedev", F.PLAN_LEBEDEV)):
        best = 0
        for s in (16, 32, 48, 64, 96, 128, 192, 256):
            plan = F.frkc2_plan(s, flags=flag)
            info = plan.info()
            dt = cfg["cfl"] * info["beta"] / rho.item()
            row = {"Q_over_L2": info["Q"] / s ** 2, "rounding_gain": F.frkc2_plan_rounding_gain(plan)}
            for nsteps in (1, 10, 100):
                outs = {}
                for prec in precs:
                    sd = torch.float32 if prec == "fp32" else torch.float64
                    u = torch.as_tensor(u0, dtype=sd, device="cuda")
                    F.frkc2_workspace_reset(wss[prec])
                    F.frkc2_step(plan, probs[prec][0], dt, nsteps, 0.0, u, wss[prec])
                    outs[prec] = u.double().cpu().numpy()
                row[f"steps{nsteps}"] = {p: _rel(outs[p], outs["fp64"]) for p in precs if p != "fp64"}
                choice, pred = F.frkc2_precision_policy(plan, probs["fp64"][0], nsteps, 1e-4)
                row[f"steps{nsteps}"]["fp32_predicted"] = pred if choice == "fp32" else pred / 5e-2 if choice in (
                    "dfloat", "mixed") else pred * 2.0 ** 29
                row[f"steps{nsteps}"]["policy_at_1e-4"] = choice
            rows[f"{order}_s{s}"] = row
            if all(row[f"steps{m}"]["fp32"] <= 1e-4 for m in (1, 10, 100)) and s > best:
                best = s
        threshold[order] = best
    return {"workload": "precision: 2048^2 var-kappa periodic (bench recipe), error vs the FP64 GPU run by s and "
                        "ordering, 1, 10 and 100 steps",
            "metric": "largest s with FP32 rel L2 <= 1e-4 after 1, 10 and 100 steps", "value": threshold,
            "unit": "stages", "by_s": rows}


def peaks(F):
    """FMA throughput of the FP64 and FP32 pipes (frkc2_fma_probe: 8 independent FMA chains per
    thread, 152 x 8 CTAs of 256 threads; FP32 also as packed two-lane FMAs), against the
    unit-count figures the rooflines use: 152 SMs x 2 FP64 FMA per clock and x 128 FP32 FMA per
    clock at 2.07 GHz."""
    torch = _torch()
    blocks = 152 * 8
    out = {}
    for prec, iters, units in (("fp64", 4096, 2), ("fp32", 65536, 128), ("fp32x2", 65536, 128)):
        buf = torch.empty(blocks * 256, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")

        def job():
            F.frkc2_fma_probe(prec, blocks, iters, buf)

        med, ms = _timed(job, 2, 5)
        fmas = blocks * 256 * iters * 8
        nominal = 152 * units * 2.07e9
        out[prec] = {"tfma_per_s": fmas / (med / 1e3) / 1e12, "ms": med,
                     "nominal_tfma_per_s": nominal / 1e12, "frac_of_nominal": fmas / (med / 1e3) / nominal}
    return {"workload": "peaks: FP64 / FP32 FMA throughput probe", "metric": "TFMA/s", "unit": "TFMA/s",
            "value": out["fp64"]["tfma_per_s"], "pipes": out}


def fp32passes(F):
    """The FP32 k-stage passes on the 2D var-kappa recipe (2048^2 and 4096^2, s = 64, 10 steps,
    the policy's Lebedev-Finogenov plan): the wavefront pass (kernel 7) by k and rows per chunk
    against the register-tiled 64 x 64 regions (kernel 3), cell-stage/s of the whole frkc2_step
    call and the error of each against the FP64 GPU run of the same plan."""
    torch = _torch()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for n in (2048, 4096):
        u0 = I.smooth_unit((n, n), 64.0 * n / 2048, 3819)
        kap = I.kappa_field((n, n), 3818, ell=32.0 * n / 2048)
        s, nsteps = 64, 10
        plan = F.frkc2_plan(s, flags=F.PLAN_LEBEDEV)
        k64 = torch.as_tensor(kap, dtype=torch.float64, device="cuda")
        p64 = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp64", kappa_field=k64)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(p64, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws64 = torch.empty(F.frkc2_workspace_size(p64), dtype=torch.uint8, device="cuda")
        ref = torch.as_tensor(u0, dtype=torch.float64, device="cuda")
        F.frkc2_step(plan, p64, dt, nsteps, 0.0, ref, ws64)
        ref = ref.cpu().numpy()
        del ws64
        k32 = torch.as_tensor(kap, dtype=torch.float32, device="cuda")
        p32 = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp32", kappa_field=k32)
        ws = torch.empty(F.frkc2_workspace_size(p32), dtype=torch.uint8, device="cuda")
        u0d = torch.as_tensor(u0, dtype=torch.float32, device="cuda")
        u = u0d.clone()
        rows = {}
        cases = [("regions_k8", F.make_tuning(k=8, kernel=3))]
        for k in (4, 6, 8, 10, 12):
            cases.append((f"wavefront_k{k}", F.make_tuning(k=k, kernel=7)))
        for H in (24, 32, 48, 64, 96):
            cases.append((f"wavefront_k8_H{H}", F.make_tuning(k=8, tile=(0, H, 0), kernel=7)))
        for name, tune in cases:
            def job():
                u.copy_(u0d)
                F.frkc2_step(plan, p32, dt, nsteps, 0.0, u, ws, tune)

            med, _ = _timed(job, 2, 3, flush)
            rows[name] = {"value": n * n * s * nsteps / (med / 1e3), "ms": med,
                          "rel_l2_vs_fp64_gpu": _rel(u.double().cpu().numpy(), ref)}
        out[str(n)] = rows
        del ws
    best = max(out["2048"].items(), key=lambda kv: kv[1]["value"])
    return {"workload": "fp32passes: 2D var-kappa periodic, 2048^2 and 4096^2, s = 64 (Lebedev order), 10 steps, "
                        "FP32 wavefront pass by k and chunk rows vs register-tiled regions",
            "metric": "cell-stage/s", "value": best[1]["value"], "best": best[0], "unit": UNIT, "cases": out}


BRUSS_INST_PER_CELL_STAGE = 41  # 4 Laplacians (4 each), v^2 and v^2 w (8), 4 rhs (9), 4 updates (8)
BRUSS_BYTES_PER_CELL_STAGE = {"fp64": 64, "fp32": 32}  # 4 state values read and written
FP64_PEAK_TINST = 152 * 2 * 2.07e9 / 1e12


def bruss2d(F, hbm_peak_gbs: float = 6787.2):
    torch = _torch()
    cfg = I.CONFIGS["bruss2d"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sd = {"fp64": torch.float64, "fp32": torch.float32}
    out = {}

    def case(n, s, nsteps_or_tend, label):
        dx = 1.0 / n
        v0, w0 = I.bruss_u0(n, n, dx)
        plan = F.frkc2_plan(s)
        beta = plan.info()["beta"]
        res, rows = {}, {}
        for prec in ("fp64", "fp32"):
            pr = F.make_bruss_problem(n, dx=dx, bc=cfg["bc"], precision=prec, D=cfg["D"], A=cfg["A"], B=cfg["B"])
            ws = torch.empty(F.frkc2_bruss_workspace_size(pr), dtype=torch.uint8, device="cuda")
            F.frkc2_workspace_reset(ws)
            v0d = torch.as_tensor(v0, dtype=sd[prec], device="cuda")
            w0d = torch.as_tensor(w0, dtype=sd[prec], device="cuda")
            rho_t = torch.zeros(1, dtype=torch.float64, device="cuda")
            F.frkc2_bruss_rho_bound(pr, v0d, w0d, rho_t, ws)
            rho = rho_t.item()
            if label == "paper":
                nsteps = int(np.ceil(nsteps_or_tend / (cfg["cfl"] * beta / rho)))
                dt = nsteps_or_tend / nsteps
            else:
                nsteps = nsteps_or_tend
                dt = cfg["cfl"] * beta / rho
            v, w = v0d.clone(), w0d.clone()
            row = {"rho_bound": rho, "dt": dt, "nsteps": nsteps}
            for kern, name in ((1, "persistent"), (2, "per_stage")):
                t = F.make_tuning(kernel=kern)

                def job():
                    v.copy_(v0d)
                    w.copy_(w0d)
                    F.frkc2_bruss_step(plan, pr, dt, nsteps, 0.0, v, w, ws, t)

                F.frkc2_launch_count()
                med, _ = _timed(job, 2, 5, flush)
                launches = F.frkc2_launch_count() // 7
                cs = n * n * s * nsteps
                r = {"value": cs / (med / 1e3), "ms_per_job": med, "launches_per_job": launches}
                if prec == "fp64":
                    tinst = cs * BRUSS_INST_PER_CELL_STAGE / (med / 1e3) / 1e12
                    r["roofline"] = {"bound": "alu", "achieved": tinst, "peak": FP64_PEAK_TINST,
                                     "unit": "Tinst/s (FP64 pipe)", "frac": tinst / FP64_PEAK_TINST}
                else:
                    gbs = cs * BRUSS_BYTES_PER_CELL_STAGE[prec] / (med / 1e3) / 1e9
                    r["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak_gbs, "unit": "GB/s",
                                     "frac": gbs / hbm_peak_gbs,
                                     "note": "L2-resident state" if n * n * 32 * 2 < 100e6 else "state larger than L2"}
                row[name] = r
            row["status"] = F.frkc2_workspace_status(ws)
            res[prec] = (v.double().cpu().numpy(), w.double().cpu().numpy())
            rows[prec] = row
            del ws
        rows["fp32_rel_l2_vs_fp64_gpu"] = max(_rel(res["fp32"][0], res["fp64"][0]), _rel(res["fp32"][1], res["fp64"][1]))
        return rows

    out["paper_200"] = case(cfg["n"], cfg["s"], cfg["t_end"], "paper")
    out["large_2048"] = case(cfg["n_large"], cfg["s_large"], cfg["steps_large"], "large")
    big = out["large_2048"]["fp64"]["persistent"]
    return {"workload": f"bruss2d: Brusselator D=0.02, A=1, B=3 periodic; 200^2 s={cfg['s']} to t={cfg['t_end']}, "
                        f"and 2048^2 s={cfg['s_large']} {cfg['steps_large']} steps",
            "metric": "cell-stage/s", "value": big["value"], "unit": UNIT, "dtype": "f64", "cases": out,
            "kernel": "k_bruss2d: persistent cooperative launch, grid barrier between stages"}


def order4(F):
    """Work against accuracy for the rank-2 and rank-4 polynomials (Eq. 7, N = 2 and 4) on one
    smooth Fourier mode of a 2048^2 periodic constant-kappa grid, whose exact solution is
    e^{lambda t} u0: s = 64 plans of both ranks at 1, 2, 4 and 8 times their fewest stable steps
    (dt = 0.9 beta / rho) to t with lambda t = -2, each run timed (CUDA events) and compared with
    the closed form.  Reported: time, cell-stage/s and relative L2 error per run, the observed
    order, and the time each rank needs for a relative error of 1e-8 (interpolated in log-log)."""
    torch = _torch()
    n, s, kx, ky = 2048, 64, 3, 5
    dx = 1.0 / n
    x = np.arange(n) / n
    u0 = np.outer(np.sin(2 * np.pi * ky * x), np.sin(2 * np.pi * kx * x))
    lam = -(4.0 / dx ** 2) * (np.sin(np.pi * kx / n) ** 2 + np.sin(np.pi * ky / n) ** 2)
    t_end = 2.0 / -lam
    exact = np.exp(lam * t_end) * u0
    pr = F.make_problem(2, (n, n), dx, "periodic", "const", "fp64", kappa_c=1.0)
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.frkc2_rho_bound(pr, None, rho)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
    out = {}
    for name, flags in (("rank2", 0), ("rank4", F.PLAN_ORDER4)):
        plan = F.frkc2_plan(s, flags=flags)
        beta = plan.info()["beta"]
        m0 = int(np.ceil(t_end * rho.item() / (0.9 * beta)))
        runs = []
        for f in (1, 2, 4, 8):
            m = m0 * f
            u = torch.as_tensor(u0, dtype=torch.float64, device="cuda")
            u_init = u.clone()
            F.frkc2_workspace_reset(ws)

            def run():
                u.copy_(u_init)
                F.frkc2_step(plan, pr, t_end / m, m, rho.item(), u, ws)

            ms, _ = _timed(run, warmup=1, reps=3)
            err = _rel(u.cpu().numpy(), exact)
            assert F.frkc2_workspace_status(ws) == F.OK
            runs.append({"nsteps": m, "ms": ms, "cell_stage_per_s": n * n * s * m / (ms * 1e-3), "rel_err": err})
        e = np.array([r["rel_err"] for r in runs])
        t = np.array([r["ms"] for r in runs])
        slope = np.log2(e[:-1] / e[1:]).tolist()
        how = "interpolated"
        if e.min() <= 1e-8 <= e.max():
            i = int(np.argmax(e <= 1e-8))
            w = (np.log(1e-8) - np.log(e[i - 1])) / (np.log(e[i]) - np.log(e[i - 1]))
            ms_at = float(np.exp(np.log(t[i - 1]) + w * (np.log(t[i]) - np.log(t[i - 1]))))
        elif e.max() < 1e-8:  # already below at the fewest stable steps
            ms_at, how = float(t[0]), "fewest stable steps"
        else:  # time grows as the steps, error falls as steps^-order: extend the last interval
            ms_at = float(t[-1] * (e[-1] / 1e-8) ** (1.0 / slope[-1]))
            how = "extrapolated with the last observed order"
        out[name] = {"beta": beta, "fewest_stable_steps": m0, "runs": runs, "observed_order": slope,
                     "ms_for_rel_err_1e-8": ms_at, "ms_for_rel_err_1e-8_from": how}
    return {"workload": f"order4: 2048^2 periodic const-kappa Fourier mode ({kx},{ky}), s = {s}, lambda t = -2, "
                        "FP64, exact solution e^(lambda t) u0",
            "metric": "ms for relative L2 error 1e-8", "unit": "ms",
            "value": {k: v["ms_for_rel_err_1e-8"] for k, v in out.items()}, "cases": out}


WORKLOADS = {"peaks": peaks, "fp32passes": fp32passes, "heat1d": heat1d, "nonlinear3d": nonlinear3d, "adjoint2d": adjoint2d,
             "batched2d": batched2d, "ssweep": ssweep, "bruss2d": bruss2d, "precision": precision,
             "order4": order4}


def profile_case(F, name: str):
    """One small instance per kernel family for ncu captures (inputs above the 129 MB L2,
    a few GB on the device at most): runs each case twice so a capture can skip the first."""
    torch = _torch()
    if name == "wf2d":  # FP32 wavefront pass, 4096^2, k = 8, the policy's plan
        n, s = 4096, 16
        u0 = I.smooth_unit((n, n), 128.0, 3819)
        k = I.kappa_field((n, n), 3818, ell=64.0)
        plan = F.frkc2_plan(s, flags=F.PLAN_LEBEDEV)
        kt = torch.as_tensor(k, dtype=torch.float32, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp32", kappa_field=kt)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            u = torch.as_tensor(u0, dtype=torch.float32, device="cuda")
            F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws, F.make_tuning(kernel=7))
    elif name in ("small1d", "small1d_fp32"):  # the 1D heat job (N = 256), the default whole-job kernel
        cfg = I.CONFIGS["heat1d"]
        u0, _, dx = I.heat1d_u0(cfg["n"], 8, cfg["seed"])
        plan = F.frkc2_plan(cfg["s"])
        nsteps = int(np.ceil(cfg["t_end"] / (0.9 * plan.info()["beta"] * dx * dx / 4.0)))
        prec = "fp32" if name.endswith("fp32") else "fp64"
        pr = F.make_problem(1, (cfg["n"],), dx, "dirichlet", "const", prec, kappa_c=1.0)
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            u = torch.as_tensor(u0, dtype=torch.float32 if prec == "fp32" else torch.float64, device="cuda")
            F.frkc2_step(plan, pr, cfg["t_end"] / nsteps, nsteps, 0.0, u, ws)
    elif name == "tb2d":  # FP32 temporally blocked pass, 4096^2, k = 8
        n, s = 4096, 16
        u0 = I.smooth_unit((n, n), 128.0, 3819)
        k = I.kappa_field((n, n), 3818, ell=64.0)
        plan = F.frkc2_plan(s)
        kt = torch.as_tensor(k, dtype=torch.float32, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp32", kappa_field=kt)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            u = torch.as_tensor(u0, dtype=torch.float32, device="cuda")
            F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws)
    elif name in ("adj_stream2d", "adj_stream2d_fp32"):  # streaming adjoint, 2048^2, s = 8, 2 steps
        n, s, nsteps = 2048, 8, 2
        prec = "fp32" if name.endswith("fp32") else "fp64"
        sd = torch.float32 if prec == "fp32" else torch.float64
        u0 = I.smooth_unit((n, n), 64.0, 3819)
        k = I.kappa_field((n, n), 3818)
        plan = F.frkc2_plan(s)
        kt = torch.as_tensor(k, dtype=sd, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_adjoint_workspace_size(plan, pr, nsteps, 1), dtype=torch.uint8, device="cuda")
        u = torch.as_tensor(u0, dtype=sd, device="cuda")
        g = torch.ones_like(u)
        du, dk = torch.empty_like(u), torch.empty_like(kt)
        for _ in range(2):
            F.frkc2_adjoint(plan, pr, dt, nsteps, 1, u, g, du, dk, ws)
    elif name == "batched":  # 8 FP32 problems of 1024^2, s = 16, 1 step
        plan = F.frkc2_plan(16)
        probs, us, dts = [], [], []
        for i in range(8):
            u0 = I.grf_torch(1024, 32.0, 20000 + i)
            kt = torch.exp(0.5 * I.grf_torch(1024, 16.0, 30000 + i)).float().contiguous()
            pr = F.make_problem(2, (1024, 1024), 1.0, "periodic", "field", "fp32", kappa_field=kt)
            rho = torch.zeros(1, dtype=torch.float64, device="cuda")
            F.frkc2_rho_bound(pr, None, rho)
            probs.append(pr)
            us.append(u0.float().contiguous())
            dts.append(0.9 * plan.info()["beta"] / rho.item())
        plans = [plan] * 8
        ws = torch.empty(F.frkc2_batch_workspace_size(plans, probs, [1] * 8), dtype=torch.uint8, device="cuda")
        F.frkc2_workspace_reset(ws)
        for _ in range(2):
            F.frkc2_step_batched(plans, probs, dts, [1] * 8, us, ws)
    elif name in ("generic3d", "stream3d", "stream3d_fp32"):  # kappa(u) pass, 192^3, s = 8 (tile / z-streaming)
        n, s = 192, 8
        u0 = I.hotspot3d_u0(n, sigma=15.0, seed=2017)
        plan = F.frkc2_plan(s)
        prec = "fp32" if name.endswith("fp32") else "fp64"
        pr = F.make_problem(3, (n, n, n), 1.0, "dirichlet", "power", prec, kappa_c=1.0, kappa_p=2.5)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        u = torch.as_tensor(u0, dtype=torch.float32 if prec == "fp32" else torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, u, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        t = F.make_tuning(k=1, tile=(32, 4, 4), kernel=1) if name == "generic3d" else F.make_tuning(k=1, kernel=5)
        for _ in range(2):
            v = u.clone()
            F.frkc2_step(plan, pr, dt, 1, 0.0, v, ws, t)
    elif name in ("stream2d_mixed", "stream2d_fp32"):  # k = 1 streaming pass, 2048^2, s = 16, 1 step
        n, s = 2048, 16
        prec = name.split("_")[1]
        sd = torch.float32 if prec == "fp32" else torch.float64
        u0 = I.smooth_unit((n, n), 64.0, 3819)
        k = I.kappa_field((n, n), 3818)
        plan = F.frkc2_plan(s)
        kt = torch.as_tensor(k, dtype=torch.float32, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            u = torch.as_tensor(u0, dtype=sd, device="cuda")
            F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws, F.make_tuning(k=1, kernel=2))
    elif name in ("stream2d_df", "tb2d_df"):  # DFLOAT pass, 2048^2 var-kappa, s = 16, 1 step
        n, s = 2048, 16
        t = F.make_tuning(k=1, kernel=2) if name == "stream2d_df" else F.make_tuning(k=8, kernel=3)
        u0 = I.smooth_unit((n, n), 64.0, 3819)
        k = I.kappa_field((n, n), 3818)
        plan = F.frkc2_plan(s)
        kt = torch.as_tensor(k, dtype=torch.float32, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", "dfloat", kappa_field=kt)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            u = torch.as_tensor(u0, device="cuda")
            F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws, t)
    elif name == "paired":  # FP64 real pair stages (PAIRED plan), 2048^2 var-kappa, s = 16, 1 step
        n, s = 2048, 16
        u0 = I.smooth_unit((n, n), 64.0, 3819)
        k = I.kappa_field((n, n), 3818)
        plan = F.frkc2_plan(s, flags=F.PLAN_PAIRED)
        kt = torch.as_tensor(k, dtype=torch.float64, device="cuda")
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp64", kappa_field=kt)
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_rho_bound(pr, None, rho)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            u = torch.as_tensor(u0, device="cuda")
            F.frkc2_step(plan, pr, dt, 1, 0.0, u, ws, F.make_tuning(kernel=4))
    elif name == "bruss":  # FP64 Brusselator persistent launch, 2048^2, s = 16, 1 step
        n, s = 2048, 16
        v0, w0 = I.bruss_u0(n, n, 1.0 / n)
        plan = F.frkc2_plan(s)
        pr = F.make_bruss_problem(n, precision="fp64")
        ws = torch.empty(F.frkc2_bruss_workspace_size(pr), dtype=torch.uint8, device="cuda")
        F.frkc2_workspace_reset(ws)
        v, w = torch.as_tensor(v0, device="cuda"), torch.as_tensor(w0, device="cuda")
        rho = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.frkc2_bruss_rho_bound(pr, v, w, rho, ws)
        dt = 0.9 * plan.info()["beta"] / rho.item()
        for _ in range(2):
            F.frkc2_bruss_step(plan, pr, dt, 1, 0.0, v, w, ws)
    else:
        raise ValueError(name)
    torch.cuda.synchronize()
    return {"workload": f"profile:{name}", "ok": True}
