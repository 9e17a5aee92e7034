#!/usr/bin/env python
"""FRKC2 benchmark: cell-stage updates/s of the 2D variable-conductivity workload.

Workload (one bench step = the whole job): 2048^2 periodic grid, kappa = exp(0.5 g) with g a
unit Gaussian random field of correlation length 32 cells (seed 3818), u0 a smooth random
field in [0, 1] (correlation length 64, seed 3819), FRKC2 with s = 64 stages, 100 steps of
dt = 0.9 beta / rho.  A step runs every part of the path: the spectral-radius bound (kernel),
dt from it, and frkc2_step over 100 x 64 stages.  The primary line is FP64 with the paper's
stage order; FP32 (with the plan and precision frkc2_plan_auto chooses for this job at a 1e-4
tolerance: the Lebedev-Finogenov order), MIXED and DFLOAT (float-pair state on the FP32 pipe)
runs of the same job, and FP64 with a PAIRED plan, are reported under "variants", each with its
error against the FP64 GPU run and against the FP64 oracle over the whole job length.

Timing: W untimed warm-up steps, then K timed steps, each bracketed by CUDA events on the
launching stream; L2 is flushed (a 256 MiB write) between timed steps, outside the events.
Under torchrun the one job is split into row slabs (paper_1702_03818_gb300/slab.py: halo rows
exchanged between groups of stages), so scaling is strong and value = the job's cell-stages /
the slowest rank's time.

``--impl reference`` times the FP64 oracle (the CPU statement of the method) on the host on a
bounded sample of the same workload, rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import frkc2_inputs as I  # noqa: E402

CFG = I.CONFIGS["varkappa2d"]
METRIC = "FRKC2 cell-stage updates/s (2D var-kappa 2048^2, s=64, 100 steps)"
UNIT = "cell-stage/s"
# spec tolerance of the FP32 state (relative L2 against the FP64 result, s <= 64)
POLICY_TOL = 1e-4
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe: 152 SMs x 2 FP64 instructions per clock x 2.07 GHz (1.259 TFLOP/s with FMA = 2)
FP64_PEAK_TINST = 152 * 2 * 2.07e9 / 1e12
FP64_INST_PER_CELL_STAGE = 16  # 2 x (2 differences + 1 product + 3 multiply-adds) + 4 FMA updates
# FP32 pipe: 152 SMs x 128 lanes per clock x 2.07 GHz, in FP32 operations (a packed two-lane
# instruction counts two)
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
# FP32 operations per cell-stage, each shared difference counted once: FP32 2 x (1 x and 1 y
# difference, 2 x-term and 2 y-term products / multiply-adds) + 4 update FMAs; DFLOAT the same
# with 3-operation pair differences, a float increment (product + FMA) and a 10-operation
# TwoSum update per component
FP32_OPS_PER_CELL_STAGE = {"fp32": 16, "dfloat": 44}
# MIXED: 4 differences in double, their 4 conversions to float, 2 conversions of f back and
# 4 FMA updates in double, all on the FP64 pipe (ncu: 14.5 per cell-stage with the halo lane)
MIXED_FP64_INST_PER_CELL_STAGE = 14
# dram bytes per launch from one ncu capture of each pass kernel, keyed by the source hash of
# the kernel file at capture time (the value is reported only while the source is unchanged)
NCU_TRAFFIC = {
    # profiles/stream2d_fp64_varkappa2d_2048.md: two intermediate passes, mean of
    # (170.4 + 42.7) MB and (170.0 + 40.1) MB
    ("pass_stream2d.cu", "4e3d07b4b9363912"): 211.6e6,
}


def wf2d_recompute(nx, ny, k=8, sms=152, ctas_per_sm=3):
    """Computed / output cell-stages of the FP32 wavefront pass at its default launch: strips of
    256 columns with 2h = 16 halo columns (h = k rounded up to 4), one wave of 3 CTAs per SM
    (ncu occupancy), chunks of H rows in which every level runs H + 2k rows."""
    h = (k + 3) // 4 * 4
    strips = -(-nx // (256 - 2 * h))
    chunks = max(1, min(ny, sms * ctas_per_sm // strips))
    H = -(-ny // chunks)
    return strips * 256 / nx * (H + 2 * k) / H


def kernel_source_hash(name: str) -> str:
    path = os.path.join(ROOT, "paper_1702_03818_gb300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def hbm_peak():
    try:
        return float(json.load(open(MEASURED_PEAKS))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def inputs(n=None):
    n = n or CFG["n"]
    ell_u, ell_k = 64.0 * n / CFG["n"], 32.0 * n / CFG["n"]
    u0 = I.smooth_unit((n, n), ell_u, CFG["u0_seed"])
    kappa = I.kappa_field((n, n), CFG["kappa_seed"], ell=ell_k)
    return u0, kappa


def _oracle_worker(stages, iters, barrier, out):
    """One host core: the first ``stages`` stages of one step of the 2048^2 FP64 job with the
    oracle, ``iters`` times, each start aligned with the other workers by ``barrier``."""
    from oracle import frkc2_oracle as O

    u0, k = inputs()
    pr = dict(ndim=2, dx=1.0, bc="periodic", kappa="field", kappa_c=1.0, kappa_p=2.5, kappa_field=k)
    a = O.plan(CFG["s"])["a"][:stages]
    dt = CFG["cfl"] * O.beta(CFG["s"]) / O.rho_bound(pr)
    times = []
    for _ in range(iters):
        barrier.wait()
        t = time.perf_counter()
        O.frkc2_step(u0, a, dt, pr, 1)
        times.append(time.perf_counter() - t)
    out.put(times)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_on_host_cores(stages, iters):
    """The oracle as it stands, one process per host core (spawned, so no process inherits a
    CUDA context), all cores on the same bounded sample at once.  Returns the per-iteration
    wall times (the slowest core of each iteration) and the number of cores."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    cores = host_cores()
    barrier = ctx.Barrier(cores)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(stages, iters, barrier, out)) for _ in range(cores)]
    for p in procs:
        p.start()
    results = [out.get() for _ in procs]
    for p in procs:
        p.join()
    return [max(r[i] for r in results) for i in range(iters)], cores


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"frkc2_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1702_03818_gb300 import frkc2 as F

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    s, nsteps, n = CFG["s"], CFG["steps"], CFG["n"]
    u0_np, k_np = inputs()
    plan = F.frkc2_plan(s)
    beta = plan.info()["beta"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    cells = n * n
    cell_stages = cells * s * nsteps

    def setup(prec):
        sd = torch.float32 if prec == "fp32" else torch.float64
        kd = torch.float64 if prec == "fp64" else torch.float32
        u0 = torch.as_tensor(u0_np, dtype=sd, device=dev)
        kt = torch.as_tensor(k_np, dtype=kd, device=dev)
        pr = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
        ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device=dev)
        F.frkc2_workspace_reset(ws)
        return dict(u0=u0, u=u0.clone(), k=kt, pr=pr, ws=ws, rho=torch.zeros(1, dtype=torch.float64, device=dev))

    def job(c, pl=None):
        F.frkc2_rho_bound(c["pr"], None, c["rho"])
        rho = c["rho"].item()
        dt = CFG["cfl"] * beta / rho
        F.frkc2_step(pl or plan, c["pr"], dt, nsteps, rho, c["u"], c["ws"])
        return dt

    def timed(prec, K, W, clocks=None, pl=None):
        c = setup(prec)
        for _ in range(W):
            c["u"].copy_(c["u0"])
            job(c, pl)
        torch.cuda.synchronize()
        from paper_1702_03818_gb300 import dist as D
        D.barrier(dev)
        ms = []
        launches = 0
        if clocks:
            clocks.start()
        for _ in range(K):
            c["u"].copy_(c["u0"])
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            F.frkc2_launch_count()
            e0.record(stream)
            job(c, pl)
            e1.record(stream)
            launches += F.frkc2_launch_count()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        D.barrier(dev)
        clk = clocks.stop() if clocks else None
        assert F.frkc2_workspace_status(c["ws"]) == F.OK
        return c, ms, launches, clk

    def step_only_ms(c, reps=2, pl=None):
        """Event time of frkc2_step alone (the pass kernels and the face set-up kernels)."""
        F.frkc2_rho_bound(c["pr"], None, c["rho"])
        rho = c["rho"].item()
        dt = CFG["cfl"] * beta / rho
        out = []
        for _ in range(reps):
            c["u"].copy_(c["u0"])
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F.frkc2_step(pl or plan, c["pr"], dt, nsteps, rho, c["u"], c["ws"])
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.mean(out))

    clocks = Clocks(local_rank)
    c64, ms, launches, clk = timed("fp64", args.steps, args.warmup, clocks)
    total_ms = float(np.sum(ms))
    # max over ranks of the timed region
    from paper_1702_03818_gb300 import dist as D
    total_ms = D.max_over_ranks(total_ms, dev)
    value = world * cell_stages * args.steps / (total_ms / 1e3)
    u64 = c64["u"].double().cpu().numpy()

    npass = nsteps * s  # k = 1 passes per step
    step_ms = step_only_ms(c64)
    launch_s = step_ms / 1e3 / npass
    achieved_tinst = FP64_INST_PER_CELL_STAGE * cells / launch_s / 1e12
    peak_hbm, peak_kind = hbm_peak()
    # algorithmic bytes of the FP64 passes: read U, V, kappa and write U, V (8 B each);
    # the first pass of a step reads no V, the last writes no V
    bytes_step = cells * 8 * (s * 5 - 2)
    hbm_gbs = bytes_step * nsteps / (step_ms / 1e3) / 1e9
    roofline = {
        "bound": "alu", "achieved": achieved_tinst, "peak": FP64_PEAK_TINST,
        "unit": "Tinst/s (FP64 pipe)", "frac": achieved_tinst / FP64_PEAK_TINST,
        "traffic": NCU_TRAFFIC.get(("pass_stream2d.cu", kernel_source_hash("pass_stream2d.cu"))),
        "algorithmic_bytes_per_launch": 40 * cells,
        "kernel": "k_stream2d<double,double,periodic>",
        "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": peak_hbm, "hbm_peak_kind": peak_kind,
        "hbm_frac": hbm_gbs / peak_hbm, "avg_launch_us": launch_s * 1e6,
    }

    # precision policy for this job at the FP32 tolerance: plan (stage order) and precision
    # together; FP32 runs with the plan it returns
    pol_probe = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp64")
    pol_plan, pol_prec, pol_pred = F.frkc2_plan_auto(s, pol_probe, nsteps, POLICY_TOL)
    policy = {"tol": POLICY_TOL, "precision": pol_prec, "predicted_rel_l2": pol_pred,
              "order": "Lebedev-Finogenov (FRKC2_PLAN_LEBEDEV)", "rounding_gain": F.frkc2_plan_rounding_gain(pol_plan),
              "paper_order": {"rounding_gain": F.frkc2_plan_rounding_gain(plan),
                              "precision": F.frkc2_precision_policy(plan, pol_probe, nsteps, POLICY_TOL)[0]}}
    variant_plan = {"fp32": pol_plan if pol_prec == "fp32" else plan}

    variants = {}
    if not args.no_variants:
        for prec in ("fp32", "mixed", "dfloat"):
            c, vms, _, _ = timed(prec, args.steps, max(3, args.warmup // 2), pl=variant_plan.get(prec))
            v = cell_stages * args.steps / (np.sum(vms) / 1e3)
            got = c["u"].double().cpu().numpy()
            err = float(np.linalg.norm(got - u64) / np.linalg.norm(u64))
            smsec = step_only_ms(c, pl=variant_plan.get(prec))
            sbytes = 4 if prec == "fp32" else 8
            kbytes = 8 if prec == "fp64" else 4
            # default passes: k stages each; bytes per cell and pass as for FP64 with the
            # state / kappa sizes of this precision
            k = 8 if prec in ("fp32", "dfloat") else 1
            npv = (s + k - 1) // k
            pass_bytes = cells * (npv * (4 * sbytes + kbytes) - 2 * sbytes)
            g = pass_bytes * nsteps / (smsec / 1e3) / 1e9
            if prec in FP32_OPS_PER_CELL_STAGE:
                # k = 8 passes: compute bound (the FP32 pipe and issue).  FP32 runs the wavefront
                # pass (strips of 256 columns, 16 halo columns; chunks of H rows, every level
                # running H + 16 rows); DFLOAT the 64 x 64 register-tiled regions ((64/48)^2)
                ops = FP32_OPS_PER_CELL_STAGE[prec]
                ach = ops * cells * s * nsteps / (smsec / 1e3) / 1e12
                roof = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TOPS, "unit": "Tops/s (FP32 pipe)",
                        "frac": ach / FP32_PEAK_TOPS, "ops_per_cell_stage": ops,
                        "halo_recompute": wf2d_recompute(n, n) if prec == "fp32" else (64 / 48) ** 2,
                        "kernel": "k_wf2d<8> (wavefront, TMA row ring)" if prec == "fp32" else "k_tb2d_df (regions)",
                        "hbm_achieved_gbs": g, "hbm_frac": g / peak_hbm, "traffic": None}
            else:  # MIXED, k = 1 streaming: bound by the FP64 pipe
                ach = MIXED_FP64_INST_PER_CELL_STAGE * cells * s * nsteps / (smsec / 1e3) / 1e12
                roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TINST, "unit": "Tinst/s (FP64 pipe)",
                        "frac": ach / FP64_PEAK_TINST, "inst_per_cell_stage": MIXED_FP64_INST_PER_CELL_STAGE,
                        "hbm_achieved_gbs": g, "hbm_frac": g / peak_hbm, "traffic": None}
            variants[prec] = {
                "value": v, "ms_per_step": float(np.mean(vms)), "k": k,
                "plan": ("Lebedev-Finogenov order (frkc2_plan_auto, tol 1e-4)" if variant_plan.get(prec) is pol_plan
                         else "the paper's greedy order"),
                "speedup_vs_fp64": v / (cell_stages * args.steps / (float(np.sum(ms)) / 1e3)),
                "rel_l2_vs_fp64_gpu_after_100_steps": err,
                "roofline": roof,
            }
            del c
        # FP64 with conjugate pairs in adjacent stages, each pair applied to the real state
        plan_p = F.frkc2_plan(s, flags=F.PLAN_PAIRED)
        c, vms, _, _ = timed("fp64", args.steps, max(3, args.warmup // 2), pl=plan_p)
        v = cell_stages * args.steps / (np.sum(vms) / 1e3)
        got = c["u"].double().cpu().numpy()
        smsec = step_only_ms(c, pl=plan_p)
        ach = 7.5 * cells * s * nsteps / (smsec / 1e3) / 1e12
        variants["fp64_paired"] = {
            "value": v, "ms_per_step": float(np.mean(vms)), "plan": "FRKC2_PLAN_PAIRED (Lebedev pairs, Q ~ 0.12 L^4)",
            "speedup_vs_fp64": v / (cell_stages * args.steps / (float(np.sum(ms)) / 1e3)),
            "rel_l2_vs_fp64_gpu_after_100_steps": float(np.linalg.norm(got - u64) / np.linalg.norm(u64)),
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TINST,
                         "unit": "Tinst/s (FP64 pipe)", "frac": ach / FP64_PEAK_TINST,
                         "inst_per_cell_stage": 7.5, "traffic": None},
        }
        del c

    # e2e: host buffers, copies inside the timed region (primary precision)
    e2e = None
    if not args.no_e2e:
        c = setup("fp64")
        hu = torch.as_tensor(u0_np).pin_memory()
        hk = torch.as_tensor(k_np).pin_memory()
        hout = torch.empty_like(hu).pin_memory()
        tms = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c["u"].copy_(hu, non_blocking=True)
            c["k"].copy_(hk, non_blocking=True)
            job(c)
            hout.copy_(c["u"], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if it >= args.warmup:
                tms.append(e0.elapsed_time(e1))
        e2e = {"value": cell_stages * len(tms) / (np.sum(tms) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": hu.numel() * 8 + hk.numel() * 8,
               "d2h_bytes_per_step": hout.numel() * 8,
               "rel_l2_vs_device_run": float(np.linalg.norm(hout.numpy() - u64) / np.linalg.norm(u64))}
        del c

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "precision_policy": policy,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded GRF conductivity and initial state)",
        "config": {"workload": "varkappa2d: 2D var-kappa diffusion 2048^2 periodic, FRKC2 s=64, 100 steps, FP64",
                   "grid": [n, n], "s": s, "nsteps": nsteps, "cell_stages_per_step": cell_stages,
                   "kernel": "k = 1 streaming pass (FP64)", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "variants": variants,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"], out["error_vs_oracle"] = cpu_baseline(torch, F, dev, pol_plan)
    return out


def _oracle_job(order, kappa_f32, u0_f32, n, nsteps):
    """The FP64 oracle over the whole job (nsteps steps of s stages) on an n^2 instance of the
    recipe, with the stage order of the variant it checks; inputs rounded to float where the
    variant stores them in float."""
    from oracle import frkc2_oracle as O

    u0, k = inputs(n)
    if kappa_f32:
        k = k.astype(np.float32).astype(np.float64)
    if u0_f32:
        u0 = u0.astype(np.float32).astype(np.float64)
    s = CFG["s"]
    a = {"greedy": lambda: O.plan(s)["a"], "lebedev": lambda: O.step_sizes(s)[O.order_lebedev(s)],
         "paired": lambda: O.plan(s, method="paired")["a"]}[order]()
    pr = dict(ndim=2, dx=1.0, bc="periodic", kappa="field", kappa_c=1.0, kappa_p=2.5, kappa_field=k)
    dt = CFG["cfl"] * O.beta(s) / O.rho_bound(pr)
    return O.frkc2_step(u0, a, dt, pr, nsteps), dt


SLAB_HALO = 16  # halo rows of each slab, and stages per exchange, under torchrun


def run_slabs(args, rank, world, local_rank):
    """N > 1: the one 2048^2 job split into row slabs (paper_1702_03818_gb300/slab.py), each rank
    running frkc2_stages on its slab extended by 16 halo rows each side and exchanging the halo
    rows (NCCL point-to-point, into the receiver's memory) before every 16 stages: strong
    scaling, value = the whole job's cell-stages / the slowest rank's time."""
    import torch
    from paper_1702_03818_gb300 import dist as D
    from paper_1702_03818_gb300 import frkc2 as F
    from paper_1702_03818_gb300 import slab as SL

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    s, nsteps, n = CFG["s"], CFG["steps"], CFG["n"]
    u0_np, k_np = inputs()
    plan = F.frkc2_plan(s)
    # dt from the whole grid's Gershgorin bound (every rank holds the seeded inputs)
    kg = torch.as_tensor(k_np, device=dev)
    pg = F.make_problem(2, (n, n), 1.0, "periodic", "field", "fp64", kappa_field=kg)
    rho_t = torch.zeros(1, dtype=torch.float64, device=dev)
    F.frkc2_rho_bound(pg, None, rho_t)
    dt = CFG["cfl"] * plan.info()["beta"] / rho_t.item()
    del kg
    sl = SL.Slab(n, world, rank, SLAB_HALO)
    k_ext = torch.zeros((sl.rows_ext, n), dtype=torch.float64, device=dev)
    k_ext[sl.interior()] = torch.as_tensor(k_np[sl.y0:sl.y1], device=dev)
    SL.exchange_halos(k_ext, sl)  # the conductivity's halo rows, once
    pr = F.make_problem(2, (n, sl.rows_ext), 1.0, "periodic", "field", "fp64", kappa_field=k_ext)
    ws = torch.empty(F.frkc2_workspace_size(pr), dtype=torch.uint8, device=dev)
    F.frkc2_workspace_reset(ws)
    w_ext = torch.zeros((sl.rows_ext, n, 2), dtype=torch.float64, device=dev)
    u_slab = torch.as_tensor(u0_np[sl.y0:sl.y1], device=dev)
    stages = SL.device_stages(F, plan, pr, dt, w_ext, ws)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def job():
        w_ext[sl.interior(), :, 0] = u_slab
        return SL.slab_steps(plan, s, nsteps, w_ext, sl, stages)

    for _ in range(args.warmup):
        job()
    torch.cuda.synchronize()
    D.barrier(dev)
    clocks = Clocks(local_rank)
    clocks.start()
    ms, launches, exchanges = [], 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        F.frkc2_launch_count()
        e0.record(stream)
        exchanges += job()
        e1.record(stream)
        launches += F.frkc2_launch_count()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    D.barrier(dev)
    clk = clocks.stop()
    assert F.frkc2_workspace_status(ws) == F.OK
    total_ms = D.max_over_ranks(float(np.sum(ms)), dev)
    # e2e: this rank's slab of the inputs from pinned host memory, the conductivity's halo
    # exchange, the job, and the slab's result back to the host, all inside the events
    hu = torch.as_tensor(u0_np[sl.y0:sl.y1]).pin_memory()
    hk = torch.as_tensor(k_np[sl.y0:sl.y1]).pin_memory()
    hout = torch.empty_like(hu).pin_memory()
    tms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        D.barrier(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u_slab.copy_(hu, non_blocking=True)
        k_ext[sl.interior()].copy_(hk, non_blocking=True)
        SL.exchange_halos(k_ext, sl)
        job()
        hout.copy_(w_ext[sl.interior(), :, 0], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            tms.append(e0.elapsed_time(e1))
    e2e_ms = D.max_over_ranks(float(np.sum(tms)), dev)
    e2e = {"value": n * n * s * nsteps * len(tms) / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": D.sum_over_ranks(hu.numel() * 8 + hk.numel() * 8, dev),
           "d2h_bytes_per_step": D.sum_over_ranks(hout.numel() * 8, dev)}
    cell_stages = n * n * s * nsteps
    value = cell_stages * args.steps / (total_ms / 1e3)
    # per-rank FP64-pipe rate on the cells each rank computes (its slab and halo rows)
    mine = sl.rows_ext * n * s * nsteps * args.steps / (float(np.sum(ms)) / 1e3)
    ach = FP64_INST_PER_CELL_STAGE * mine / 1e12
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded GRF conductivity and initial state)",
        "config": {"workload": "varkappa2d: 2D var-kappa diffusion 2048^2 periodic, FRKC2 s=64, 100 steps, FP64",
                   "grid": [n, n], "s": s, "nsteps": nsteps, "cell_stages_per_step": cell_stages,
                   "kernel": "k = 1 streaming pass on row slabs (frkc2_stages)",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"row slabs x{world}, {SLAB_HALO} halo rows exchanged before every "
                                  f"{SLAB_HALO} stages ({args.dist_backend} point-to-point)",
                   "exchanges_per_job": exchanges // max(1, args.steps)},
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TINST, "unit": "Tinst/s (FP64 pipe), rank 0",
                     "frac": ach / FP64_PEAK_TINST, "traffic": None,
                     "computed_over_owned_cells": sl.rows_ext / sl.n},
        "clocks": clk, "gpu_launches": launches, "e2e": e2e,
    }


def cpu_baseline(torch, F, dev, pol_plan, n=128, stages=16):
    """The CPU baseline leg: the FP64 oracle timed on every host core at once (one process per
    core, each on the first ``stages`` stages of one step of the 2048^2 job), and each
    variant's error against the oracle over the whole job length (100 steps of 64 stages) on an
    n^2 instance of the recipe, the oracle taking the variant's stage order."""
    import multiprocessing as mp

    nsteps = CFG["steps"]
    s = CFG["s"]
    u0, k = inputs(n)
    plan = F.frkc2_plan(s)
    pplan = F.frkc2_plan(s, flags=F.PLAN_PAIRED)
    # variant: (precision, library plan, oracle order, kappa in float, u0 in float)
    cases = {"fp64": ("fp64", plan, "greedy", False, False),
             "fp32": ("fp32", pol_plan, "lebedev", True, True),
             "mixed": ("mixed", plan, "greedy", True, False),
             "dfloat": ("dfloat", plan, "greedy", True, False),
             "fp64_paired": ("fp64", pplan, "paired", False, False)}
    jobs = sorted({(c[2], c[3], c[4]) for c in cases.values()})
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        refs = dict(zip(jobs, pool.starmap(_oracle_job, [(o, kf, uf, n, nsteps) for o, kf, uf in jobs])))
    errs = {}
    for name, (prec, pl, order, kf, uf) in cases.items():
        ref, dt = refs[(order, kf, uf)]
        sd = torch.float32 if prec == "fp32" else torch.float64
        kd = torch.float64 if prec == "fp64" else torch.float32
        u = torch.as_tensor(u0, dtype=sd, device=dev)
        kt = torch.as_tensor(k, dtype=kd, device=dev)
        lp = F.make_problem(2, (n, n), 1.0, "periodic", "field", prec, kappa_field=kt)
        ws = torch.empty(F.frkc2_workspace_size(lp), dtype=torch.uint8, device=dev)
        F.frkc2_workspace_reset(ws)
        F.frkc2_step(pl, lp, dt, nsteps, 0.0, u, ws)
        got = u.double().cpu().numpy()
        errs[name] = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                      "max_abs_over_max_ref": float(np.abs(got - ref).max() / np.abs(ref).max())}
    errs["sample"] = (f"the whole job length ({nsteps} steps of {s} stages) on a {n}^2 instance of the recipe "
                      f"(correlation lengths scaled by {n}/2048), the oracle with each variant's stage order")
    times, cores = oracle_on_host_cores(stages, 1)
    N = CFG["n"]
    value = cores * N * N * stages / times[0]
    sample = (f"every host core at once, each on the first {stages} of the 6400 stages of the {N}^2 FP64 "
              f"job (numpy, one process per core), {times[0]:.1f} s")
    return ({"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}, errs)


def run_reference(args, rank, world):
    """The oracle timed on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return None
    stages = args.cpu_stages
    all_times, cores = oracle_on_host_cores(stages, args.warmup + args.steps)
    times = all_times[args.warmup:]
    n = CFG["n"]
    v = cores * n * n * stages * len(times) / sum(times)
    sample = (f"each step: every host core at once, each on the first {stages} of the 6400 stages of the "
              f"2048^2 FP64 job (numpy, one process per core)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded GRF conductivity and initial state)",
            "config": {"workload": "varkappa2d: 2D var-kappa diffusion 2048^2 periodic, FRKC2 s=64, 100 steps, FP64",
                       "grid": [n, n], "s": CFG["s"], "sampled_stages_per_step": stages},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-stages", type=int, default=16)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="torchrun transport of the slab halos (gloo stages them through host memory)")
    ap.add_argument("--workload", default="varkappa2d",
                    help="varkappa2d (the default line) or one of bench_workloads.WORKLOADS")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload != "varkappa2d":
        import bench_workloads as BW
        from paper_1702_03818_gb300 import frkc2 as F
        if rank == 0:
            if args.workload.startswith("profile:"):
                out = BW.profile_case(F, args.workload.split(":", 1)[1])
            else:
                out = BW.WORKLOADS[args.workload](F)
            print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        local_rank %= torch.cuda.device_count()  # ranks sharing a device (gloo, host-staged halos)
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(args.dist_backend)
    out = run_slabs(args, rank, world, local_rank) if world > 1 else run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
