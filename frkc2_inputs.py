"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This module holds input generation only: random fields, initial states and the workload
presets (grid sizes, stage counts, step counts, seeds).  It contains none of the FRKC2
arithmetic (no step sizes, no operator, no stability bound), so the two implementations
it feeds stay independent.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``), so every
array is reproducible from its seed on any machine.

Recipes (the paper gives no data; these stand in for its diffusion workloads):

* ``grf(shape, ell, seed)`` -- Gaussian random field.  White noise N(0, 1) on the grid is
  filtered in Fourier space by exp(-2 pi^2 ell^2 |f|^2), f in cycles per cell (a Gaussian
  smoothing kernel of standard deviation ``ell`` cells), then shifted and scaled to mean 0
  and standard deviation 1.  ``ell`` is the "correlation length" of the workload recipes.
* ``smooth_unit(shape, ell, seed)`` -- a GRF min-max rescaled to [0, 1].
* ``kappa_field(shape, seed)`` -- exp(0.5 * grf(ell=32)), a positive log-normal conductivity.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grf", "grf_torch", "smooth_unit", "kappa_field", "heat1d_u0", "hotspot3d_u0", "batched_problems",
    "CONFIGS",
    "bruss_u0",
]


def grf(shape, ell: float, seed: int) -> np.ndarray:
    """Gaussian random field of mean 0 and standard deviation 1 (float64, C order)."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(shape)
    spec = np.fft.fftn(xi)
    k2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        f = np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[ax] = n
        k2 = k2 + (f ** 2).reshape(sh)
    g = np.real(np.fft.ifftn(spec * np.exp(-2.0 * np.pi ** 2 * ell ** 2 * k2)))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def bruss_u0(nx: int, ny: int, dx: float):
    """The Brusselator initial state of Sec. 3.1 (Eq. 17): v = 1 + sin(2 pi x),
    w = 3 + cos(2 pi y) at grid points x = i dx, y = j dx; arrays of shape (ny, nx)."""
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    v = np.broadcast_to(1.0 + np.sin(2.0 * np.pi * x)[None, :], (ny, nx)).copy()
    w = np.broadcast_to(3.0 + np.cos(2.0 * np.pi * y)[:, None], (ny, nx)).copy()
    return v, w


def grf_torch(n: int, ell: float, seed: int, device="cuda"):
    """``grf((n, n), ell, seed)`` with the Fourier filter applied by torch on ``device``.

    The white noise is the same seeded numpy draw; only the FFTs run on the device (used to
    build large batches of inputs quickly; values agree with ``grf`` to rounding).
    """
    import torch

    xi = torch.as_tensor(np.random.default_rng(seed).standard_normal((n, n)), device=device)
    f = torch.fft.fftfreq(n, device=device, dtype=torch.float64)
    k2 = f[:, None] ** 2 + f[None, :] ** 2
    g = torch.fft.ifft2(torch.fft.fft2(xi) * torch.exp(-2.0 * np.pi ** 2 * ell ** 2 * k2)).real
    g = g - g.mean()
    return g / g.std(unbiased=False)


def smooth_unit(shape, ell: float, seed: int) -> np.ndarray:
    """Smooth random field rescaled to the interval [0, 1] (a constant field, e.g. one cell,
    becomes 1/2 everywhere)."""
    g = grf(shape, ell, seed)
    lo, hi = g.min(), g.max()
    if not hi > lo:
        return np.full(np.shape(g), 0.5)
    return (g - lo) / (hi - lo)


def kappa_field(shape, seed: int, ell: float = 32.0) -> np.ndarray:
    """Log-normal conductivity exp(0.5 g), g a unit GRF with correlation length ``ell``."""
    return np.exp(0.5 * grf(shape, ell, seed))


def heat1d_u0(n: int = 256, modes: int = 8, seed: int = 1702):
    """1D heat initial state: sum of sin(k pi x) for k = 1..modes with N(0,1) amplitudes.

    Vertex-centred interior points x_i = i dx, i = 1..n, dx = 1/(n+1) on [0, 1] with u = 0
    at both ends.  Returns (u0, amplitudes, dx).
    """
    rng = np.random.default_rng(seed)
    amp = rng.standard_normal(modes)
    dx = 1.0 / (n + 1)
    x = dx * np.arange(1, n + 1)
    u0 = np.zeros(n)
    for k in range(1, modes + 1):
        u0 += amp[k - 1] * np.sin(k * np.pi * x)
    return u0, amp, dx


def hotspot3d_u0(n: int = 256, sigma: float = 20.0, peak: float = 2.0, noise: float = 0.02,
                 seed: int = 2017) -> np.ndarray:
    """3D Gaussian hot spot (peak 2, std 20 cells) centred on the grid plus uniform noise.

    The noise is ``noise`` * U[0, 1) (1 % of the peak by default), so the field stays >= 0.
    Array layout is [z][y][x] (x fastest).
    """
    rng = np.random.default_rng(seed)
    c = (n - 1) / 2.0
    i = np.arange(n) - c
    r2 = i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2
    return peak * np.exp(-r2 / (2.0 * sigma ** 2)) + noise * rng.random((n, n, n))


def batched_problems(count: int = 512, seed: int = 512, nmin: int = 64, nmax: int = 1024,
                     stage_choices=(16, 32, 64, 128, 256)):
    """Side lengths and stage counts of the uneven batch: n ~ U{nmin..nmax}, s from a set.

    Per-problem field seeds are 10000 + 2 i (conductivity) and 10001 + 2 i (initial state).
    """
    rng = np.random.default_rng(seed)
    n = rng.integers(nmin, nmax + 1, size=count)
    s = rng.choice(np.asarray(stage_choices), size=count)
    return [dict(n=int(n[i]), s=int(s[i]), kappa_seed=10000 + 2 * i, u0_seed=10001 + 2 * i)
            for i in range(count)]


# Workload presets: sizes, stage counts, step counts and seeds of the five diffusion workloads.
CONFIGS = {
    "heat1d": dict(ndim=1, n=256, bc="dirichlet", kappa="const", s=16, t_end=0.05, seed=1702),
    "varkappa2d": dict(ndim=2, n=2048, bc="periodic", kappa="field", s=64, steps=100,
                       kappa_seed=3818, u0_seed=3819, cfl=0.9),
    "nonlinear3d": dict(ndim=3, n=256, bc="dirichlet", kappa="power", s=128, steps=50,
                        seed=2017, cfl=0.9, s_stable=32),
    "adjoint2d": dict(ndim=2, n=1024, bc="periodic", kappa="field", s=100, steps=40, ckpt=8,
                      kappa_seed=3818, u0_seed=3819, target_seed=4040, cfl=0.9),
    "batched2d": dict(count=512, seed=512, steps=10),
    # the paper's Brusselator demonstration: D = 0.02, A = 1, B = 3 on the unit square, 200^2;
    # end time and boundaries unstated (read: t = 1, periodic); plus a 2048^2 throughput case
    "bruss2d": dict(n=200, bc="periodic", D=0.02, A=1.0, B=3.0, s=16, t_end=1.0, cfl=0.9,
                    n_large=2048, s_large=64, steps_large=10),
}
