"""Brusselator reaction-diffusion oracle: a plain, slow, FP64 CPU statement.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/`` and by the CPU-baseline leg of
``bench.py``; nothing in the product package imports, links or runs it, and it imports
nothing from the product.

The problem is the paper's demonstration system (Sec. 3.1, Eq. 17), a two-species
Brusselator on the unit square,

    v_t = D (v_xx + v_yy) + A - (B + 1) v + v^2 w,
    w_t = D (w_xx + w_yy) + B v - v^2 w,

with the paper's values D = 0.02, A = 1, B = 3 (equilibrium v = A, w = B / A); the paper's
initial state v = 1 + sin(2 pi x), w = 3 + cos(2 pi y) is an input (``frkc2_inputs.bruss_u0``).
Space is discretised with the 5-point Laplacian on an nx-by-ny grid of spacing dx.  The FRKC2 step applies the ordered
complex forward-Euler stages of Eq. 13 to the pair (v, w) in complex arithmetic; the
reaction terms are polynomials, so their complex evaluation is unambiguous.

Readings (the paper states neither boundary conditions nor grid placement):
* boundaries are periodic (the initial state is periodic on the unit square); zero-flux
  (Neumann) boundaries, a ghost cell equal to its boundary cell, are offered as well;
* grid point (i, j) sits at x = i dx, y = j dx with dx = 1 / n;
* the state after a step is the real part of W^L, as for the diffusion problems.

State arrays use numpy order (rows = y, last axis = x).

Parity status: pinned by ``tests/test_oracle_bruss.py`` (the equilibrium is a fixed point,
the reaction Jacobian's trace and determinant at equilibrium, the exact discrete eigenvalues
of Fourier and cosine modes, the paper's spectral radius of about 6400 on 200 x 200, Laplacian
conservation, second-order convergence against a fine RK4 solution).
"""
from __future__ import annotations

import numpy as np

PAPER_D, PAPER_A, PAPER_B = 0.02, 1.0, 3.0


def problem(n: int | tuple, bc: str = "periodic", D: float = PAPER_D, A: float = PAPER_A,
            B: float = PAPER_B, dx: float | None = None) -> dict:
    """Problem dict for an (ny, nx) grid; dx defaults to 1 / nx (unit square)."""
    ny, nx = (n, n) if np.isscalar(n) else n
    return {"ny": int(ny), "nx": int(nx), "bc": bc, "D": float(D), "A": float(A), "B": float(B),
            "dx": float(dx) if dx is not None else 1.0 / nx}


def laplacian(u, prob):
    """5-point Laplacian (u_E + u_W + u_N + u_S - 4 u) / dx^2 with periodic wrap or
    zero-flux ghosts (ghost = boundary cell)."""
    if prob["bc"] == "periodic":
        nb = (np.roll(u, 1, axis=1) + np.roll(u, -1, axis=1)
              + np.roll(u, 1, axis=0) + np.roll(u, -1, axis=0))
    elif prob["bc"] == "neumann":
        g = np.pad(u, 1, mode="edge")
        nb = g[1:-1, :-2] + g[1:-1, 2:] + g[:-2, 1:-1] + g[2:, 1:-1]
    else:
        raise ValueError(prob["bc"])
    return (nb - 4.0 * u) / prob["dx"] ** 2


def bruss_f(v, w, prob):
    """Right-hand side of the semi-discrete Brusselator (Eq. 17) at (v, w), real or complex."""
    D, A, B = prob["D"], prob["A"], prob["B"]
    vvw = v * v * w
    fv = D * laplacian(v, prob) + A - (B + 1.0) * v + vvw
    fw = D * laplacian(w, prob) + B * v - vvw
    return fv, fw


def frkc2_step(v0, w0, a, T, prob, nsteps: int = 1):
    """``nsteps`` FRKC2 steps of size T: per step, W^0 = (v, w) and
    W^{l+1} = W^l + T a_l f(W^l) in complex arithmetic for the ordered step sizes ``a``
    (Sec. 3, Eq. 13); the new state is Re W^L."""
    v = np.array(v0, dtype=np.float64)
    w = np.array(w0, dtype=np.float64)
    for _ in range(nsteps):
        V = v.astype(np.complex128)
        W = w.astype(np.complex128)
        for al in a:
            fv, fw = bruss_f(V, W, prob)
            V = V + (T * al) * fv
            W = W + (T * al) * fw
        v, w = V.real.copy(), W.real.copy()
    return v, w


def rho_bound(v, w, prob) -> float:
    """Gershgorin bound on the spectral radius of the Jacobian of f at the real state (v, w).

    A row of the Jacobian has the Laplacian's 4D/dx^2 on the diagonal and four neighbour
    entries D/dx^2 (absolute row sum 8D/dx^2; a zero-flux boundary row has less, so 8D/dx^2
    bounds it too), plus the reaction block: the v row adds |2vw - (B+1)| + v^2, the w row
    |B - 2vw| + v^2.  The bound is 8D/dx^2 + max over cells of the larger reaction sum, formed
    in this order: p = v w, q = v v, rv = |2p - (B+1)| + q, rw = |B - 2p| + q.
    """
    D, A, B = prob["D"], prob["A"], prob["B"]
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    p = v * w
    q = v * v
    rv = np.abs(2.0 * p - (B + 1.0)) + q
    rw = np.abs(B - 2.0 * p) + q
    diff = 8.0 * D / (prob["dx"] * prob["dx"])
    return float(diff + np.max(np.maximum(rv, rw)))


def rk4(v0, w0, h, prob, nsteps: int):
    """Classical fourth-order Runge-Kutta on the real semi-discrete system, step h."""
    v = np.array(v0, dtype=np.float64)
    w = np.array(w0, dtype=np.float64)
    for _ in range(nsteps):
        k1 = bruss_f(v, w, prob)
        k2 = bruss_f(v + 0.5 * h * k1[0], w + 0.5 * h * k1[1], prob)
        k3 = bruss_f(v + 0.5 * h * k2[0], w + 0.5 * h * k2[1], prob)
        k4 = bruss_f(v + h * k3[0], w + h * k3[1], prob)
        v = v + (h / 6.0) * (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0])
        w = w + (h / 6.0) * (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1])
    return v, w
