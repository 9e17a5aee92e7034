"""Pins of the Brusselator oracle (Sec. 3.1, Eq. 17) against facts the paper and the
mathematics fix: the equilibrium, the reaction Jacobian's invariants, exact discrete
eigenvalues of the 5-point Laplacian, the paper's spectral radius, conservation, the
Gershgorin bound and second-order convergence of the FRKC2 step."""
import json
import os

import numpy as np
import pytest

import frkc2_inputs as I
from oracle import brusselator as BR
from oracle import frkc2_oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("A,B", [(1.0, 3.0), (2.0, 5.0), (0.5, 1.7)])
@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_equilibrium_is_fixed_point(A, B, bc):
    """v = A, w = B/A zeroes both reaction terms and the Laplacian of a constant."""
    pr = BR.problem((7, 9), bc=bc, A=A, B=B)
    v = np.full((7, 9), A)
    w = np.full((7, 9), B / A)
    fv, fw = BR.bruss_f(v, w, pr)
    assert np.max(np.abs(fv)) < 1e-13 and np.max(np.abs(fw)) < 1e-13
    a = O.plan(8)["a"]
    v1, w1 = BR.frkc2_step(v, w, a, 0.01, pr, nsteps=2)
    assert np.max(np.abs(v1 - A)) < 1e-12 and np.max(np.abs(w1 - B / A)) < 1e-12


def _jacobian_uniform(pr, v0, w0, eps=1e-5):
    """2x2 Jacobian of the reaction at a uniform state, by central differences of the
    oracle's f on a uniform grid (the Laplacian of a constant vanishes)."""
    sh = (pr["ny"], pr["nx"])
    J = np.zeros((2, 2))
    for col, (dv, dw) in enumerate([(eps, 0.0), (0.0, eps)]):
        fp = BR.bruss_f(np.full(sh, v0 + dv), np.full(sh, w0 + dw), pr)
        fm = BR.bruss_f(np.full(sh, v0 - dv), np.full(sh, w0 - dw), pr)
        J[0, col] = (fp[0][0, 0] - fm[0][0, 0]) / (2 * eps)
        J[1, col] = (fp[1][0, 0] - fm[1][0, 0]) / (2 * eps)
    return J


@pytest.mark.parametrize("A,B", [(1.0, 3.0), (2.0, 5.0), (1.0, 1.5)])
def test_reaction_jacobian_trace_det(A, B):
    """Textbook Brusselator linearisation at equilibrium: trace B - 1 - A^2, determinant A^2
    (Hopf bifurcation at B = 1 + A^2; the paper's A = 1, B = 3 has eigenvalues (1 +- i sqrt 3)/2)."""
    J = _jacobian_uniform(BR.problem(4, A=A, B=B), A, B / A)
    assert abs(np.trace(J) - (B - 1 - A * A)) < 1e-8
    assert abs(np.linalg.det(J) - A * A) < 1e-8
    if (A, B) == (1.0, 3.0):
        ev = np.sort_complex(np.linalg.eigvals(J))
        assert np.allclose(ev, [0.5 - 0.5j * np.sqrt(3), 0.5 + 0.5j * np.sqrt(3)], atol=1e-8)


@pytest.mark.parametrize("k,axis", [(1, 1), (3, 0), (5, 1)])
def test_periodic_fourier_mode_eigenvalue(k, axis):
    """cos(2 pi k i / n) is an eigenvector of the periodic 5-point Laplacian with eigenvalue
    -(4/dx^2) sin^2(pi k / n)."""
    n = 24
    pr = BR.problem(n)
    i = np.arange(n)
    mode = np.cos(2 * np.pi * k * i / n)
    u = np.broadcast_to(mode[None, :] if axis == 1 else mode[:, None], (n, n)).copy()
    lam = -(4.0 / pr["dx"] ** 2) * np.sin(np.pi * k / n) ** 2
    assert np.max(np.abs(BR.laplacian(u, pr) - lam * u)) < 1e-9 * abs(lam)


@pytest.mark.parametrize("k", [1, 2, 7])
def test_neumann_cosine_mode_eigenvalue(k):
    """cos(pi k (j + 1/2) / n) is an eigenvector of the zero-flux 5-point Laplacian (ghost =
    boundary cell) with eigenvalue -(4/dx^2) sin^2(pi k / (2 n))."""
    ny, nx = 10, 13
    pr = BR.problem((ny, nx), bc="neumann")
    j = np.arange(ny)
    u = np.broadcast_to(np.cos(np.pi * k * (j + 0.5) / ny)[:, None], (ny, nx)).copy()
    lam = -(4.0 / pr["dx"] ** 2) * np.sin(np.pi * k / (2 * ny)) ** 2
    assert np.max(np.abs(BR.laplacian(u, pr) - lam * u)) < 1e-9 * abs(4.0 / pr["dx"] ** 2)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_laplacian_conserves_sum(bc):
    rng = np.random.default_rng(3)
    pr = BR.problem((11, 16), bc=bc)
    u = rng.standard_normal((11, 16))
    assert abs(np.sum(BR.laplacian(u, pr))) < 1e-9 * np.sum(np.abs(BR.laplacian(u, pr)))


def test_spectral_radius_paper_value():
    """Linearisation of the oracle's f at equilibrium on the paper's 200 x 200 grid of the unit
    square: the checkerboard mode of each species spans an invariant pair; the largest
    eigenvalue magnitude is about 6400 (Sec. 3.1)."""
    n = 200
    pr = BR.problem(n)
    A, B = pr["A"], pr["B"]
    cb = np.fromfunction(lambda j, i: (-1.0) ** (i + j), (n, n))
    eps = 1e-6
    v0, w0 = np.full((n, n), A), np.full((n, n), B / A)
    M = np.zeros((2, 2))
    for col, (dv, dw) in enumerate([(eps, 0.0), (0.0, eps)]):
        fp = BR.bruss_f(v0 + dv * cb, w0 + dw * cb, pr)
        fm = BR.bruss_f(v0 - dv * cb, w0 - dw * cb, pr)
        # both results are multiples of the checkerboard mode
        for row in range(2):
            d = (fp[row] - fm[row]) / (2 * eps)
            coef = d[0, 0] * cb[0, 0]
            assert np.max(np.abs(d - coef * cb)) < 1e-6 * max(1.0, abs(coef))
            M[row, col] = coef
    rho = np.max(np.abs(np.linalg.eigvals(M)))
    assert abs(rho / GOLD["brusselator_rho_200"]["value"] - 1.0) < 0.01
    bound = BR.rho_bound(v0, w0, pr)
    assert rho <= bound < rho * 1.002


def test_rho_bound_covers_dense_spectrum():
    """The Gershgorin bound is at least the spectral radius of the dense Jacobian (built
    column by column from central differences of f) at a random state."""
    rng = np.random.default_rng(11)
    for bc in ("periodic", "neumann"):
        ny, nx = 5, 6
        pr = BR.problem((ny, nx), bc=bc, D=0.3)
        v = 1.0 + 0.5 * rng.standard_normal((ny, nx))
        w = 3.0 + 0.5 * rng.standard_normal((ny, nx))
        N = ny * nx
        J = np.zeros((2 * N, 2 * N))
        eps = 1e-6
        for c in range(2 * N):
            dv = np.zeros(N)
            dw = np.zeros(N)
            (dv if c < N else dw)[c % N] = eps
            fp = BR.bruss_f(v + dv.reshape(ny, nx), w + dw.reshape(ny, nx), pr)
            fm = BR.bruss_f(v - dv.reshape(ny, nx), w - dw.reshape(ny, nx), pr)
            J[:, c] = np.concatenate([(fp[0] - fm[0]).ravel(), (fp[1] - fm[1]).ravel()]) / (2 * eps)
        rho = np.max(np.abs(np.linalg.eigvals(J)))
        bound = BR.rho_bound(v, w, pr)
        assert rho <= bound * (1 + 1e-9)
        # and it is within the diagonal-splitting slack of the largest absolute row sum
        rowsum = np.max(np.sum(np.abs(J), axis=1))
        assert rowsum * (1 - 1e-9) <= bound < 1.1 * rowsum


def test_paper_initial_state():
    v, w = I.bruss_u0(8, 8, 1.0 / 8)
    assert np.allclose(v[3], 1.0 + np.sin(2 * np.pi * np.arange(8) / 8))
    assert np.allclose(w[:, 5], 3.0 + np.cos(2 * np.pi * np.arange(8) / 8))


def test_second_order_convergence():
    """FRKC2 steps of the full nonlinear system converge at second order in T to a fine RK4
    solution (paper's initial state, 12 x 12 periodic grid, t = 0.4)."""
    pr = BR.problem(12)
    v0, w0 = I.bruss_u0(12, 12, pr["dx"])
    t_end = 0.4
    vr, wr = BR.rk4(v0, w0, t_end / 800, pr, 800)
    a = O.plan(6)["a"]
    errs = []
    for nsteps in (8, 16, 32):
        v, w = BR.frkc2_step(v0, w0, a, t_end / nsteps, pr, nsteps)
        errs.append(np.sqrt(np.sum((v - vr) ** 2 + (w - wr) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.6 < r2 < 4.4, errs


def test_complex_stages_return_real_state_for_conjugate_pairs():
    """With conjugate-pair step sizes the imaginary part left after a step is a rounding-level
    remainder for a linear problem (here the pure-diffusion limit A = B = 0 about v = w = 0)."""
    pr = BR.problem(16, A=0.0, B=0.0)
    rng = np.random.default_rng(5)
    v0 = rng.standard_normal((16, 16)) * 1e-3
    a = O.plan(8)["a"]
    V, W = v0.astype(complex), np.zeros((16, 16), complex)
    for al in a:
        fv, fw = BR.bruss_f(V, W, pr)
        V, W = V + 0.002 * al * fv, W + 0.002 * al * fw
    assert np.linalg.norm(V.imag) < 1e-12 * np.linalg.norm(V.real)
