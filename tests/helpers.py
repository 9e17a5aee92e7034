"""Shared test helpers: build the same seeded problem for the oracle and for the CUDA path."""
from __future__ import annotations

import numpy as np

import frkc2_inputs as I


def oracle_problem(ndim, bc, kappa, dx=1.0, field=None, c=1.0, p=2.5):
    return dict(ndim=ndim, dx=dx, bc=bc, kappa=kappa, kappa_c=c, kappa_p=p, kappa_field=field)


def seeded_case(shape, bc, kappa, seed, dx=1.0, ell=None):
    """Seeded (u0, kappa field) for a grid of numpy shape ``shape`` (last axis x).

    u0 is a smooth field in [0, 1] (GRF), kappa = exp(0.5 GRF); both have correlation length
    ``ell`` cells (default: an eighth of the smallest extent, at least 1).
    """
    ell = ell if ell is not None else max(1.0, min(shape) / 8.0)
    u0 = I.smooth_unit(shape, ell, seed)
    field = np.exp(0.5 * I.grf(shape, ell, seed + 1)) if kappa == "field" else None
    if kappa == "power":
        u0 = 0.5 + u0  # kappa(u) = 1 + u^2.5 on a positive state
    return u0, field


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# per-element bound beside the grid norm: max |a - b| <= ELEM_C * tol * max |b|
ELEM_C = 5.0


def rel_err(a, b):
    """max(relative L2, max|a - b| / (ELEM_C max|b|)): below tol means both the grid norm and
    every single element are within tolerance (one wrong cell or boundary row cannot hide in
    the norm of a large grid)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    elem = float(np.max(np.abs(a - b))) / (ELEM_C * max(float(np.max(np.abs(b))), 1e-300)) if a.size else 0.0
    return max(rel_l2(a, b), elem)


def oracle_steps(args):
    """Worker for a spawned process pool: (u0, a, T, prob, nsteps) -> the oracle's step."""
    from oracle import frkc2_oracle as O

    u0, a, T, prob, nsteps = args
    return O.frkc2_step(u0, a, T, prob, nsteps)


def oracle_map(jobs, procs=8):
    """The oracle on several inputs at once in spawned processes (a spawned process does not
    inherit the parent's CUDA context)."""
    import multiprocessing as mp

    if len(jobs) <= 1:
        return [oracle_steps(j) for j in jobs]
    with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
        return pool.map(oracle_steps, jobs)
