"""Autotuner for the stage-pass kernel choice, stages per pass k and tile shape.

``autotune_step`` times candidate ``frkc2_tuning`` values with ``frkc2_step`` on a scratch copy
of the state (CUDA events on the current stream, one warm-up call each) and returns the
fastest; ``autotune_batch`` does the same for the batched launch.  Results are cached in a
JSON file (``$FRKC2_TUNE_CACHE``, default ``~/.cache/frkc2/tune.json``) keyed by grid size,
stage count, precision, conductivity kind, boundary kind and device name, so a problem
shape is tuned once per machine.  Every candidate runs through the C ABI; nothing here
computes any part of the method.
"""
from __future__ import annotations

import json
import os

import torch

from . import frkc2 as F

PREC_NAMES = {F.FP64: "fp64", F.FP32: "fp32", F.MIXED: "mixed", F.DFLOAT: "dfloat"}


def _cache_path() -> str:
    return os.environ.get("FRKC2_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "frkc2", "tune.json"))


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the cache


def _key(prob, s: int) -> str:
    dev = torch.cuda.get_device_name()
    n = "x".join(str(int(prob.n[d])) for d in range(prob.ndim))
    return f"{dev}|{prob.ndim}d|{n}|s{s}|{PREC_NAMES[prob.precision]}|kappa{prob.kappa_kind}|bc{prob.bc}"


def candidates(prob) -> list:
    """Candidate (kernel, k, tile) tunings for a problem."""
    c = []
    if prob.precision == F.DFLOAT:  # the float-pair state: streaming pass or register-tiled regions
        return [F.make_tuning(k=1, kernel=2)] + [F.make_tuning(k=k, kernel=3) for k in (2, 4, 6, 8, 10)]
    if prob.ndim == 2 and prob.kappa_kind != F.KAPPA_POWER:
        c.append(F.make_tuning(k=1, kernel=2))
        if prob.precision == F.FP32:
            c += [F.make_tuning(k=k, kernel=3) for k in (2, 3, 4, 5, 6, 8, 10, 12)]
            if int(prob.n[0]) % 4 == 0 and int(prob.n[0]) >= 256:  # the wavefront pass
                c += [F.make_tuning(k=k, kernel=7) for k in (4, 6, 8, 10, 12)]
        for k in (1, 2, 4):
            c += [F.make_tuning(k=k, tile=t, kernel=1) for t in ((64, 16, 1), (32, 32, 1), (64, 32, 1))]
    elif prob.ndim == 2:
        for k in (1, 2, 4):
            c += [F.make_tuning(k=k, tile=t, kernel=1) for t in ((64, 16, 1), (32, 32, 1), (32, 16, 1))]
    elif prob.ndim == 3:
        c.append(F.make_tuning(k=1, kernel=5))
        for k in (1, 2):
            c += [F.make_tuning(k=k, tile=t, kernel=1) for t in ((32, 4, 4), (32, 8, 2), (64, 4, 2), (16, 8, 4))]
    else:
        if int(prob.n[0]) <= 16384 and prob.kappa_kind != F.KAPPA_POWER:
            # the 1D whole-job kernel: CTAs in the cluster, stages per halo exchange, threads
            c.append(F.make_tuning(kernel=6))
            c += [F.make_tuning(k=k, tile=(cl, th, 0), kernel=6)
                  for cl in (1, 2, 4, 8) for k in (8, 16) for th in (32, 64, 128) if cl > 1 or k == 16]
        c += [F.make_tuning(k=k, tile=(t, 1, 1), kernel=1) for k in (4, 8, 16) for t in (256, 1024)]
    return c


def _tuning_dict(t) -> dict:
    return dict(k=t.k, tile=[t.tile_x, t.tile_y, t.tile_z], kernel=t.kernel)


def autotune_step(plan, prob, u, dt: float, nsteps: int = 1, reps: int = 3, use_cache: bool = True):
    """Fastest tuning of ``frkc2_step`` for this problem; ``u`` is not modified.

    Returns (frkc2_tuning, {candidate description: milliseconds}).
    """
    s = plan.info()["s"]
    key = _key(prob, s)
    cache = _load() if use_cache else {}
    if key in cache:
        d = cache[key]
        return F.make_tuning(k=d["k"], tile=d["tile"], kernel=d["kernel"]), {}
    scratch = u.clone()
    times = {}
    best, best_ms = None, float("inf")
    stream = torch.cuda.current_stream()
    for t in candidates(prob):
        try:
            ws = torch.empty(F.frkc2_workspace_size(prob, t), dtype=torch.uint8, device=u.device)
            scratch.copy_(u)
            F.frkc2_step(plan, prob, dt, nsteps, 0.0, scratch, ws, t)
        except F.Frkc2Error:
            continue
        ms = []
        for _ in range(reps):
            scratch.copy_(u)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F.frkc2_step(plan, prob, dt, nsteps, 0.0, scratch, ws, t)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = sorted(ms)[len(ms) // 2]
        times[json.dumps(_tuning_dict(t))] = m
        if m < best_ms:
            best, best_ms = t, m
        del ws
    if best is None:
        raise RuntimeError("no candidate tuning ran for this problem")
    if use_cache:
        cache = _load()
        cache[key] = _tuning_dict(best)
        _store(cache)
    return best, times


def autotune_batch(plans, probs, dt, nsteps, u, reps: int = 2):
    """Fastest (k, tile) of the batched launch over a few candidates; ``u`` is not modified.

    Returns (frkc2_tuning, {candidate description: milliseconds}).
    """
    prec = probs[0].precision
    if prec == F.FP32:  # register-tiled 64 x 64 regions: the tile follows from k
        cands = [F.make_tuning(k=k, tile=(0, 0, g)) for k in (6, 8, 10) for g in (1, 4, 8, 16)]
    elif prec == F.DFLOAT:  # float-pair regions, or streaming items of one stage
        cands = [F.make_tuning(k=k, tile=(0, 0, g)) for k in (6, 8, 10) for g in (1, 4, 8)]
        cands += [F.make_tuning(k=1, tile=(0, r, 1)) for r in (128, 256)]
    else:  # streaming items (k = 1) by rows per tile, and the shared-memory tile pass
        cands = [F.make_tuning(k=1, tile=(0, r, 1)) for r in (64, 128, 256)]
        cands += [F.make_tuning(k=k, tile=t, kernel=1) for k in (1, 2) for t in ((64, 16, 1), (32, 32, 1))]
    scratch = [t.clone() for t in u]
    times = {}
    best, best_ms = None, float("inf")
    for t in cands:
        try:
            ws = torch.empty(F.frkc2_batch_workspace_size(plans, probs, nsteps, t), dtype=torch.uint8,
                             device=u[0].device)
            F.frkc2_workspace_reset(ws)
            for a, b in zip(scratch, u):
                a.copy_(b)
            F.frkc2_batch_prepare(plans, probs, dt, nsteps, scratch, ws, t)
        except F.Frkc2Error:
            continue
        ms = []
        for _ in range(reps + 1):
            for a, b in zip(scratch, u):
                a.copy_(b)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            F.frkc2_batch_launch(ws)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = sorted(ms[1:])[len(ms[1:]) // 2]
        times[json.dumps(_tuning_dict(t))] = m
        if m < best_ms:
            best, best_ms = t, m
        del ws
    return best, times
