"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks an oracle function against something that does not come from the oracle
itself: values printed in the paper (tests/golden/paper_values.json), closed forms,
textbook or library routines (numpy's Chebyshev basis, numpy.linalg.eigh,
scipy.linalg.expm), invariants, manufactured solutions and brute force.
"""
import json
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

from oracle import frkc2_oracle as O
import frkc2_inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
LS = [16, 32, 64, 128]


def R_closed(z, L):
    """1 - alpha/4 + (alpha/4) T_L(1 + 4 z / (L^2 alpha)), T_L from numpy's Chebyshev basis."""
    al = 4.0 * (1.0 - 1.0 / L ** 2) / 3.0  # the value fixed by R''(0) = 1, retyped as a number check below
    TL = C.Chebyshev.basis(L)
    return 1.0 - al / 4.0 + (al / 4.0) * TL(1.0 + 4.0 * np.asarray(z) / (L * L * al))


def R_product(z, a):
    z = np.asarray(z, dtype=np.complex128)
    out = np.ones_like(z)
    for al in a:
        out = out * (1.0 + al * z)
    return out


# --------------------------------------------------------------------------------------
# Stability polynomial (Sec. 2, Eqs. 5-8)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("L", LS + [256, 1024])
def test_order_conditions_taylor(L):
    """R(z) = 1 + z + z^2/2 + O(z^3): the first three Taylor coefficients of prod(1 + a z)."""
    a = O.step_sizes(L)
    coef = np.array([1.0 + 0j])
    for al in a:
        coef = np.convolve(coef, np.array([1.0, al]))  # ascending powers of z
    assert abs(coef[1] - 1.0) < 1e-10
    assert abs(coef[2] - 0.5) < 1e-10
    # the third coefficient is not 1/6: the scheme is second order, not third
    assert abs(coef[3] - 1.0 / 6.0) > 1e-3


@pytest.mark.parametrize("L", LS + [256])
def test_product_equals_chebyshev_closed_form(L):
    a = O.step_sizes(L)
    z = np.linspace(-O.beta(L), 0.0, 4001)
    rp = R_product(z, a)
    assert np.max(np.abs(rp.imag)) < 1e-9
    assert np.max(np.abs(rp.real - R_closed(z, L))) < 1e-9


@pytest.mark.parametrize("L", LS + [256])
def test_conjugate_pairs_and_positive_real_part(L):
    a = O.step_sizes(L)
    assert np.all(a.real > 0)
    assert np.array_equal(a[::-1], np.conj(a))
    assert np.all(np.abs(a.imag) > 0)


@pytest.mark.parametrize("L", LS + [256])
def test_stability_extent(L):
    """|R| <= 1 on [-beta, 0], |R| > 1 just beyond, beta/(L^2 beta_RK2) near the paper's 0.330."""
    a = O.step_sizes(L)
    b = O.beta(L)
    z = np.linspace(-b, 0.0, 20 * L + 1)
    assert np.max(np.abs(R_product(z, a))) <= 1.0 + 1e-9
    assert abs(R_product(-b * (1 + 1e-3), a)) > 1.0
    # bisection on the boundary of |R| <= 1 beyond the last extremum recovers beta
    lo, hi = b * 0.999, b * 1.01
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if abs(R_product(-mid, a)) <= 1.0:
            lo = mid
        else:
            hi = mid
    assert abs(lo / b - 1.0) < 1e-9
    ratio = b / (L * L * GOLD["beta_RK2"]["value"])
    assert GOLD["beta_over_L2_betaRK2_frkc2"]["value"] - 0.003 <= ratio <= 1.0 / 3.0


def test_marginal_interior_points():
    """The undamped polynomial touches |R| = 1 inside the interval (the points Sec. 2.1 damps)."""
    L = 32
    a = O.step_sizes(L)
    al = O.alpha(L)
    # T_L(x) = 1 at x = cos(2 pi m / L); z = (x - 1) L^2 alpha / 4
    for m in range(1, L // 2):
        z = (np.cos(2 * np.pi * m / L) - 1.0) * L * L * al / 4.0
        assert abs(abs(R_product(z, a)) - 1.0) < 1e-10


def test_acceleration_claim():
    """beta grows like (2/3) L^2: at L = 10^4 stages the gain over RK2 per f-evaluation exceeds 6000."""
    L = GOLD["viable_stages"]["value"]
    per_eval = O.beta(L) / L  # real extent per f-evaluation
    assert per_eval / (GOLD["beta_RK2"]["value"] / 2.0) > GOLD["acceleration_factor_min"]["value"]


# --------------------------------------------------------------------------------------
# Internal stability and ordering (Sec. 2.2)
# --------------------------------------------------------------------------------------

def test_realised_Q_brute_force_tiny():
    """realised_Q equals an explicit triple loop over (j, k, x) on a tiny case."""
    a = O.step_sizes(8)[[3, 0, 6, 1, 5, 2, 7, 4]]
    b = O.beta(8)
    pts = 64
    best = 0.0
    for i in range(pts + 1):
        x = -b * i / pts
        for j in range(8):
            p = 1.0
            for k in range(j, 8):
                p *= abs(1 + a[k] * x)
                best = max(best, p)
    assert abs(O.realised_Q(a, b, pts) / best - 1.0) < 1e-12


@pytest.mark.parametrize("L", [6, 8])
def test_greedy_order_attains_brute_force_minimum_Q(L):
    """Sec. 2.2 orders the steps to approximately minimise Q (Eqs. 10-11).  For L = 6 and 8
    every one of the L! orderings is tried by brute force (Q of Eq. 10 on one shared grid of
    x in [-beta, 0], each Q_{j,k} from prefix sums of log|1 + a x|): the plan's greedy order
    attains the smallest Q of them all.  A wrong cost in the greedy step (a dropped factor,
    the rest taken without the candidate, a flipped max) would leave it above the minimum.
    At L = 4, where every order is far inside the paper's bound 10 L^2, the greedy order is
    not the minimum; that case is covered by the bound test below."""
    import itertools

    p = O.plan(L)
    a = O.step_sizes(L)
    x = np.linspace(-O.beta(L), 0.0, 129)
    perms = np.asarray(list(itertools.permutations(range(L))))
    lg = np.log(np.abs(1.0 + a[perms][:, :, None] * x[None, None, :]))
    pre = np.concatenate([np.zeros((len(perms), 1, x.size)), np.cumsum(lg, axis=1)], axis=1)
    best = np.full((len(perms), x.size), -np.inf)
    low = pre[:, 0, :]
    for k in range(1, L + 1):  # max over j <= k of the product of factors j..k
        best = np.maximum(best, pre[:, k, :] - low)
        low = np.minimum(low, pre[:, k, :])
    Q = np.exp(best.max(axis=1))
    g = np.flatnonzero((perms == p["order"][None, :]).all(axis=1))
    assert g.size == 1
    assert Q[g[0]] <= Q.min() * (1.0 + 1e-12)
    assert np.median(Q) > 3.0 * Q.min()  # the minimum is not what a typical order gives


@pytest.mark.parametrize("L", LS)
def test_plan_Q_within_paper_bounds(L):
    p = O.plan(L)
    assert sorted(p["order"].tolist()) == list(range(L))
    assert np.array_equal(p["a"], O.step_sizes(L)[p["order"]])
    lo = GOLD["Q_optimal_factor"]["value"] * L * L / 10.0
    hi = GOLD["Q_bound_factor"]["value"] * L * L
    assert lo <= p["Q"] <= hi
    # the ordering matters: root order amplifies far more (Sec. 2.2 motivation)
    qnat = O.realised_Q(O.step_sizes(L), O.beta(L), 16 * L)
    assert qnat > p["Q"]
    # order does not change the stability polynomial
    z = np.linspace(-O.beta(L), 0.0, 501)
    assert np.max(np.abs(R_product(z, p["a"]) - R_product(z, O.step_sizes(L)))) < 1e-9


def test_plan_n_loop_runs():
    """A tight bound forces the n-loop (Sec. 2.2): n grows and the best ordering is kept."""
    L = 32
    p = O.plan(L, bound=1e-6, n_max=3)
    assert 1 <= p["n"] <= 3
    q1 = O.realised_Q(O.step_sizes(L)[O.order_greedy(O.step_sizes(L), O.beta(L), 1, 16 * L)],
                      O.beta(L), 16 * L)
    assert p["Q"] <= q1


# --------------------------------------------------------------------------------------
# Operator (flux form)
# --------------------------------------------------------------------------------------

def _prob(ndim, bc, kappa, dx=1.0, field=None, c=1.0, p=2.5):
    return dict(ndim=ndim, dx=dx, bc=bc, kappa=kappa, kappa_c=c, kappa_p=p, kappa_field=field)


def dense(prob, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        A[:, i] = O.apply_f(e.reshape(shape), prob).ravel()
    return A


def test_operator_manufactured_2d_field_second_order():
    """f(u_h) -> div(kappa grad u) with error O(dx^2) on a smooth periodic solution."""
    errs = []
    for n in (32, 64, 128):
        dx = 1.0 / n
        x = dx * np.arange(n)
        X, Y = np.meshgrid(x, x, indexing="xy")  # arrays [y][x]
        tp = 2 * np.pi
        u = np.sin(tp * X) * np.sin(2 * tp * Y)
        k = 2.0 + np.sin(tp * X) * np.cos(tp * Y)
        ux = tp * np.cos(tp * X) * np.sin(2 * tp * Y)
        uy = 2 * tp * np.sin(tp * X) * np.cos(2 * tp * Y)
        uxx = -tp ** 2 * u
        uyy = -(2 * tp) ** 2 * u
        kx = tp * np.cos(tp * X) * np.cos(tp * Y)
        ky = -tp * np.sin(tp * X) * np.sin(tp * Y)
        exact = kx * ux + k * uxx + ky * uy + k * uyy
        f = O.apply_f(u, _prob(2, "periodic", "field", dx, k))
        errs.append(np.max(np.abs(f - exact)))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


def test_operator_manufactured_3d_power_second_order():
    """kappa(u) = 1 + u^2.5: f -> kappa'(u)|grad u|^2 + kappa(u) lap u, error O(dx^2)."""
    errs = []
    for n in (16, 32, 64):
        dx = 1.0 / n
        x = dx * np.arange(n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        tp = 2 * np.pi
        s = np.sin(tp * X) * np.sin(tp * Y) * np.sin(tp * Z)
        u = 1.5 + 0.5 * s
        gx = 0.5 * tp * np.cos(tp * X) * np.sin(tp * Y) * np.sin(tp * Z)
        gy = 0.5 * tp * np.sin(tp * X) * np.cos(tp * Y) * np.sin(tp * Z)
        gz = 0.5 * tp * np.sin(tp * X) * np.sin(tp * Y) * np.cos(tp * Z)
        lap = -3 * tp ** 2 * 0.5 * s
        exact = 2.5 * u ** 1.5 * (gx ** 2 + gy ** 2 + gz ** 2) + (1 + u ** 2.5) * lap
        f = O.apply_f(u, _prob(3, "periodic", "power", dx))
        errs.append(np.max(np.abs(f - exact)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_operator_dirichlet_1d_closed_form():
    """1D Dirichlet, kappa = 1: sine modes are exact eigenvectors, lambda_k = -(4/dx^2) sin^2(k pi dx/2)."""
    n = 63
    dx = 1.0 / (n + 1)
    x = dx * np.arange(1, n + 1)
    pr = _prob(1, "dirichlet", "const", dx)
    for k in (1, 5, 40, 63):
        v = np.sin(k * np.pi * x)
        lam = -(4.0 / dx ** 2) * np.sin(k * np.pi * dx / 2) ** 2
        assert np.max(np.abs(O.apply_f(v, pr) - lam * v)) < 1e-9 * abs(lam)


def test_operator_symmetric_conservative():
    rng = np.random.default_rng(0)
    shape = (5, 7)
    k = np.exp(rng.standard_normal(shape))
    for bc in ("periodic", "dirichlet"):
        A = dense(_prob(2, bc, "field", 1.0, k), shape)
        assert np.max(np.abs(A - A.T)) < 1e-14
        assert np.all(np.linalg.eigvalsh(A) < 1e-12)  # negative semi-definite diffusion
    A = dense(_prob(2, "periodic", "field", 1.0, k), shape)
    assert np.max(np.abs(A.sum(axis=0))) < 1e-13  # periodic flux form conserves the total
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-13  # constants are steady
    shape3 = (3, 4, 5)
    k3 = np.exp(rng.standard_normal(shape3))
    A3 = dense(_prob(3, "dirichlet", "field", 0.5, k3), shape3)
    assert np.max(np.abs(A3 - A3.T)) < 1e-13


def test_dirichlet_field_boundary_face_reading():
    """A Dirichlet boundary face carries the boundary cell's own kappa (stated reading)."""
    k = np.array([2.0, 3.0, 5.0])
    A = dense(_prob(1, "dirichlet", "field", 1.0, k), (3,))
    assert A[0, 0] == -(2.0 + 2.5) and A[0, 1] == 2.5
    assert A[2, 2] == -(4.0 + 5.0) and A[2, 1] == 4.0


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_rho_bound_is_gershgorin(bc):
    rng = np.random.default_rng(1)
    shape = (6, 5)
    k = np.exp(rng.standard_normal(shape))
    pr = _prob(2, bc, "field", 0.7, k)
    A = dense(pr, shape)
    gersh = np.max(np.sum(np.abs(A), axis=1))
    assert abs(O.rho_bound(pr) / gersh - 1.0) < 1e-14
    assert O.rho_bound(pr) >= np.max(np.abs(np.linalg.eigvalsh(A)))


def test_rho_bound_brusselator_paper_value():
    """Diffusion 0.02 on a 200 x 200 mesh of the unit square: spectral radius about 6400 (Sec. 3.1)."""
    n = 200
    pr = _prob(2, "periodic", "const", 1.0 / n, c=GOLD["brusselator_diffusion"]["value"])
    rho = O.rho_bound(pr, np.zeros((n, n)))
    assert abs(rho / GOLD["brusselator_rho_200"]["value"] - 1.0) < 0.01
    # the Gershgorin bound is attained by the checkerboard mode for a constant coefficient
    chk = (-1.0) ** np.add.outer(np.arange(n), np.arange(n))
    lam = O.apply_f(chk, pr)[0, 0] / chk[0, 0]
    assert abs(-lam / rho - 1.0) < 1e-12


def test_rho_bound_1d_heat_closed_form():
    n = 256
    dx = 1.0 / (n + 1)
    pr = _prob(1, "dirichlet", "const", dx)
    assert abs(O.rho_bound(pr, np.zeros(n)) / (4.0 / dx ** 2) - 1.0) < 1e-14


# --------------------------------------------------------------------------------------
# Stepping (Sec. 3, Eq. 13)
# --------------------------------------------------------------------------------------

def test_heat1d_closed_form_modes():
    """1D heat workload: every sine mode is amplified by R(T lambda_k) per step (R from T_L)."""
    cfg = I.CONFIGS["heat1d"]
    u0, amp, dx = I.heat1d_u0(cfg["n"], 8, cfg["seed"])
    L = cfg["s"]
    p = O.plan(L)
    dtmax = 0.9 * O.beta(L) * dx * dx / 4.0
    nsteps = int(np.ceil(cfg["t_end"] / dtmax))
    T = cfg["t_end"] / nsteps
    pr = _prob(1, "dirichlet", "const", dx)
    u = O.frkc2_step(u0, p["a"], T, pr, nsteps)
    x = dx * np.arange(1, cfg["n"] + 1)
    exact = np.zeros_like(x)
    for k in range(1, 9):
        lam = -(4.0 / dx ** 2) * np.sin(k * np.pi * dx / 2) ** 2
        exact += amp[k - 1] * R_closed(T * lam, L) ** nsteps * np.sin(k * np.pi * x)
    rel = np.linalg.norm(u - exact) / np.linalg.norm(exact)
    assert rel < 1e-12, rel


def test_periodic_fourier_mode_amplification():
    L = 16
    p = O.plan(L)
    n0, n1 = 12, 10
    pr = _prob(2, "periodic", "const", 1.0, c=1.3)
    y, x = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    for k0, k1 in ((1, 2), (5, 3), (6, 5)):
        v = np.cos(2 * np.pi * (k0 * y / n0 + k1 * x / n1))
        lam = -(4 * 1.3) * (np.sin(np.pi * k0 / n0) ** 2 + np.sin(np.pi * k1 / n1) ** 2)
        T = 0.9 * O.beta(L) / O.rho_bound(pr, v)
        out = O.frkc2_step(v, p["a"], T, pr, 2)
        assert np.max(np.abs(out - R_closed(T * lam, L) ** 2 * v)) < 1e-12


def test_varkappa_eigh_library_pin():
    """Linear var-kappa: u^n = V R(T Lambda)^n V^T u0, eigen-decomposition by numpy.linalg.eigh."""
    rng = np.random.default_rng(7)
    shape = (9, 7)
    k = np.exp(0.5 * rng.standard_normal(shape))
    for bc in ("periodic", "dirichlet"):
        pr = _prob(2, bc, "field", 1.0, k)
        A = dense(pr, shape)
        w, V = np.linalg.eigh(A)
        L = 32
        p = O.plan(L)
        T = 0.9 * O.beta(L) / O.rho_bound(pr)
        u0 = rng.random(shape)
        u = O.frkc2_step(u0, p["a"], T, pr, 3)
        ref = V @ (R_closed(T * w, L) ** 3 * (V.T @ u0.ravel()))
        assert np.linalg.norm(u.ravel() - ref) / np.linalg.norm(ref) < 1e-12


def test_second_order_against_expm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    shape = (8, 8)
    k = np.exp(0.5 * rng.standard_normal(shape))
    pr = _prob(2, "periodic", "field", 1.0, k)
    A = dense(pr, shape)
    u0 = rng.random(shape)
    t_end = 2.0
    ref = scipy_linalg.expm(t_end * A) @ u0.ravel()
    L = 8
    a = O.plan(L)["a"]
    errs = []
    for nsteps in (32, 64, 128):
        u = O.frkc2_step(u0, a, t_end / nsteps, pr, nsteps)
        errs.append(np.linalg.norm(u.ravel() - ref))
    slope = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert all(1.9 < s < 2.1 for s in slope), slope


def test_real_projection_drops_only_rounding():
    """Linear f with conjugate-paired step sizes: Im W^L is rounding noise (reading of w^{n+1} = W^L)."""
    rng = np.random.default_rng(5)
    shape = (16, 16)
    k = np.exp(0.5 * rng.standard_normal(shape))
    pr = _prob(2, "periodic", "field", 1.0, k)
    L = 64
    a = O.plan(L)["a"]
    T = 0.9 * O.beta(L) / O.rho_bound(pr)
    _, worst = O.frkc2_step(rng.random(shape), a, T, pr, 2, return_imag=True)
    assert worst < 1e-12


def test_rk4_fourth_order_against_expm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(4)
    shape = (6, 6)
    pr = _prob(2, "periodic", "field", 1.0, np.exp(0.3 * rng.standard_normal(shape)))
    A = dense(pr, shape)
    u0 = rng.random(shape)
    ref = scipy_linalg.expm(0.5 * A) @ u0.ravel()
    e = [np.linalg.norm(O.rk4(u0, 0.5 / m, pr, m).ravel() - ref) for m in (16, 32)]
    assert 3.7 < np.log2(e[0] / e[1]) < 4.3


def test_nonlinear_second_order_against_rk4():
    """kappa(u) = 1 + u^2.5, Dirichlet 3D: FRKC2 converges at order 2 to a fine RK4 solution."""
    n = 6
    u0 = I.hotspot3d_u0(n, sigma=1.5, seed=11)
    pr = _prob(3, "dirichlet", "power", 1.0)
    t_end = 0.6
    ref = O.rk4(u0, t_end / 400, pr, 400)
    L = 8
    a = O.plan(L)["a"]
    errs = [np.linalg.norm(O.frkc2_step(u0, a, t_end / m, pr, m) - ref) for m in (8, 16, 32)]
    slopes = [np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])]
    assert all(1.85 < s < 2.25 for s in slopes), slopes


def test_internal_stability_fp64_many_stages():
    """Ordered stages keep FP64 accuracy at s = 128 on all modes (Sec. 2.2), root order does not."""
    n = 127
    dx = 1.0 / (n + 1)
    x = dx * np.arange(1, n + 1)
    rng = np.random.default_rng(9)
    amp = rng.standard_normal(n)
    u0 = sum(amp[k - 1] * np.sin(k * np.pi * x) for k in range(1, n + 1))
    pr = _prob(1, "dirichlet", "const", dx)
    L = 128
    p = O.plan(L)
    T = 0.9 * O.beta(L) * dx * dx / 4
    u = O.frkc2_step(u0, p["a"], T, pr, 1)
    exact = sum(amp[k - 1] * R_closed(T * (-(4 / dx ** 2) * np.sin(k * np.pi * dx / 2) ** 2), L)
                * np.sin(k * np.pi * x) for k in range(1, n + 1))
    err = np.linalg.norm(u - exact) / np.linalg.norm(exact)
    assert err < 1e-11, err
    u_nat = O.frkc2_step(u0, O.step_sizes(L), T, pr, 1)
    assert not np.linalg.norm(u_nat - exact) / np.linalg.norm(exact) < 1e-6


# --------------------------------------------------------------------------------------
# Adjoint
# --------------------------------------------------------------------------------------

def test_adjoint_dot_product_linear():
    rng = np.random.default_rng(11)
    shape = (10, 12)
    for bc in ("periodic", "dirichlet"):
        pr = _prob(2, bc, "field", 1.0, np.exp(0.5 * rng.standard_normal(shape)))
        L = 16
        a = O.plan(L)["a"]
        T = 0.9 * O.beta(L) / O.rho_bound(pr)
        v = rng.standard_normal(shape)
        w = rng.standard_normal(shape)
        Jv = O.frkc2_step(v, a, T, pr, 3)
        JTw, _ = O.frkc2_adjoint(v, a, T, pr, 3, w)
        assert abs(np.vdot(Jv, w) - np.vdot(v, JTw)) < 1e-12 * abs(np.vdot(Jv, w)) + 1e-13


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_adjoint_kappa_gradient_central_fd(bc):
    rng = np.random.default_rng(12)
    shape = (7, 6)
    k0 = np.exp(0.5 * rng.standard_normal(shape))
    u0 = rng.random(shape)
    tgt = rng.random(shape)
    L = 8
    a = O.plan(L)["a"]
    T = 0.8 * O.beta(L) / O.rho_bound(_prob(2, bc, "field", 1.0, k0))

    def loss(k, u):
        uT = O.frkc2_step(u, a, T, _prob(2, bc, "field", 1.0, k), 2)
        return np.sum((uT - tgt) ** 2)

    uT = O.frkc2_step(u0, a, T, _prob(2, bc, "field", 1.0, k0), 2)
    gu, gk = O.frkc2_adjoint(u0, a, T, _prob(2, bc, "field", 1.0, k0), 2, 2.0 * (uT - tgt))
    for idx in [(0, 0), (3, 2), (6, 5), (0, 5)]:
        h = 1e-6 * k0[idx]
        kp, km = k0.copy(), k0.copy()
        kp[idx] += h
        km[idx] -= h
        fd = (loss(kp, u0) - loss(km, u0)) / (2 * h)
        assert abs(fd - gk[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, gk[idx])
        up, um = u0.copy(), u0.copy()
        up[idx] += 1e-6
        um[idx] -= 1e-6
        fdu = (loss(k0, up) - loss(k0, um)) / 2e-6
        assert abs(fdu - gu[idx]) < 1e-6 * max(1.0, abs(fdu))


def test_adjoint_nonlinear_central_fd():
    rng = np.random.default_rng(13)
    n = 5
    u0 = 0.5 + rng.random((n, n, n))
    tgt = rng.random((n, n, n))
    pr = _prob(3, "dirichlet", "power", 1.0)
    L = 8
    a = O.plan(L)["a"]
    T = 0.5 * O.beta(L) / O.rho_bound(pr, u0 + 0.5)

    def loss(u):
        return np.sum((O.frkc2_step(u, a, T, pr, 2) - tgt) ** 2)

    uT = O.frkc2_step(u0, a, T, pr, 2)
    gu, gk = O.frkc2_adjoint(u0, a, T, pr, 2, 2 * (uT - tgt))
    assert gk is None
    for idx in [(0, 0, 0), (2, 2, 2), (4, 1, 3)]:
        up, um = u0.copy(), u0.copy()
        up[idx] += 1e-6
        um[idx] -= 1e-6
        fd = (loss(up) - loss(um)) / 2e-6
        assert abs(fd - gu[idx]) < 1e-6 * max(1.0, abs(fd)), (idx, fd, gu[idx])


# --------------------------------------------------------------------------------------
# Input generators (no method arithmetic, but the recipes are checked)
# --------------------------------------------------------------------------------------

def test_inputs_recipes():
    g = I.grf((64, 64), 8.0, 1)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    assert np.array_equal(g, I.grf((64, 64), 8.0, 1))
    s = I.smooth_unit((32, 32), 4.0, 2)
    assert s.min() == 0.0 and s.max() == 1.0
    h = I.hotspot3d_u0(16, sigma=3.0)
    assert h.min() >= 0.0 and 1.5 <= h.max() <= 2.02 + 1e-12
    b = I.batched_problems(16)
    assert all(64 <= p["n"] <= 1024 and p["s"] in (16, 32, 64, 128, 256) for p in b)


@pytest.mark.parametrize("L", [8, 16, 64, 128, 256])
def test_lebedev_order_reaches_single_factor_lower_bound(L):
    """Any order's Q is at least the largest single factor max_l max_x |1 + a_l x|; the
    Lebedev-Finogenov half-then-conjugates order attains it for L a power of two."""
    a = O.step_sizes(L)
    b = O.beta(L)
    pts = 8 * L
    perm = O.order_lebedev(L)
    assert sorted(perm.tolist()) == list(range(L))
    x = -b * np.arange(pts + 1) / pts
    single = float(np.max(np.abs(1.0 + np.outer(a, x))))
    q = O.realised_Q(a[perm], b, pts)
    assert abs(q / single - 1.0) < 1e-12
    assert q < GOLD["Q_optimal_factor"]["value"] * L * L


@pytest.mark.parametrize("L", [6, 10, 12, 24, 48, 96, 100, 192, 320, 600])
def test_lebedev_order_within_paper_bound_for_every_even_L(L):
    """For L not a power of two the Lebedev-Finogenov order no longer attains the single-factor
    bound, but its realised Q stays inside the paper's 10 L^2 (Sec. 2.2, Fig. 3) -- the
    library takes this order for every L above 256 (e.g. 320, 384, 1000)."""
    a = O.step_sizes(L)[O.order_lebedev(L)]
    b = O.beta(L)
    x = -b * np.linspace(0.0, 1.0, 8 * L + 1)
    single = float(np.max(np.abs(1.0 + np.outer(a, x))))
    q = O.realised_Q(a, b, 8 * L)
    assert single * (1 - 1e-12) <= q <= 10.0 * L * L


def test_lebedev_permutation_recursion():
    assert O.lebedev_permutation(1) == [0]
    assert O.lebedev_permutation(2) == [0, 1]
    assert O.lebedev_permutation(4) == [0, 3, 1, 2]
    assert O.lebedev_permutation(8) == [0, 7, 3, 4, 1, 6, 2, 5]
    assert O.lebedev_permutation(3) == [0, 2, 1]
    assert O.lebedev_permutation(5) == [0, 4, 1, 3, 2]
    assert O.lebedev_permutation(6) == [0, 5, 2, 3, 1, 4]
    for m in range(1, 40):
        p = O.lebedev_permutation(m)
        assert sorted(p) == list(range(m))
        # every entry but an odd size's middle one sits next to its mirror m - 1 - v
        for i in range(0, m - (m % 2), 2):
            assert p[i] + p[i + 1] == m - 1
        if m % 2:
            assert p[-1] == m // 2


def test_plan_auto_uses_lebedev_above_256():
    p = O.plan(512, q_points=1024)
    assert p["n"] == 0 and np.array_equal(p["order"], O.order_lebedev(512))
    assert p["Q"] <= 10 * 512 ** 2


@pytest.mark.parametrize("L", [16, 64, 100])
@pytest.mark.parametrize("nu0", [0.05, 0.2])
def test_damping_order_conditions_extent_and_maxima(L, nu0):
    """Sec. 2.1: damped step sizes keep the order conditions, shrink beta by about (1 - nu),
    nu = nu0/2, and lift the marginal interior points off |R| = 1."""
    a, mu = O.damped_step_sizes(L, nu0)
    coef = np.array([1.0 + 0j])
    for al in a:
        coef = np.convolve(coef, np.array([1.0, al]))
    assert abs(coef[1] - 1.0) < 1e-12 and abs(coef[2] - 0.5) < 1e-12
    assert np.array_equal(a[::-1], np.conj(a))
    b = O.stability_extent(a, O.beta(L))
    assert abs(b / O.beta(L) - (1.0 - nu0 / 2.0)) < 0.005
    z = np.linspace(-0.95 * b, -0.05 * b, 4001)
    assert np.max(np.abs(R_product(z, a))) < 1.0 - nu0 / 4.0
    assert np.max(np.abs(R_product(np.linspace(-b, 0.0, 4001), a))) <= 1.0 + 1e-9
    assert abs(R_product(-1.001 * b, a)) > 1.0


def test_damping_zero_is_undamped():
    a, mu = O.damped_step_sizes(32, 0.0)
    assert mu == 0
    assert np.max(np.abs(a - O.step_sizes(32))) < 1e-15


@pytest.mark.parametrize("L", [8, 32, 64])
def test_paired_order_quadratic_factor_bound(L):
    """With conjugates adjacent every pair is a real quadratic factor; Q is at least the largest
    of them (about 0.12 L^4) and the paired order attains it for L a power of two."""
    a = O.step_sizes(L)
    perm = O.order_paired(L)
    ap = a[perm]
    assert np.array_equal(ap[1::2], np.conj(ap[0::2]))
    b = O.beta(L)
    pts = 8 * L
    x = -b * np.arange(pts + 1) / pts
    quad = float(np.max(np.abs((1 + np.outer(ap[0::2], x)) * (1 + np.outer(ap[1::2], x)))))
    q = O.realised_Q(ap, b, pts)
    assert abs(q / quad - 1.0) < 1e-12
    assert 0.1 < q / L ** 4 < 0.13


def test_embedded_solution_first_order():
    """Eq. 14: the embedded solution is first order -- its one-step error against expm falls
    like T^2 while the FRKC2 step's falls like T^3."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(21)
    shape = (8, 8)
    pr = _prob(2, "periodic", "field", 1.0, np.exp(0.5 * rng.standard_normal(shape)))
    A = dense(pr, shape)
    u0 = rng.random(shape)
    a = O.plan(8)["a"]
    e_w, e_h = [], []
    for T in (0.0125, 0.00625, 0.003125):
        ref = scipy_linalg.expm(T * A) @ u0.ravel()
        w, h = O.frkc2_step_embedded(u0, a, T, pr)
        e_w.append(np.linalg.norm(w.ravel() - ref))
        e_h.append(np.linalg.norm(h.ravel() - ref))
    sw = np.log2(e_w[0] / e_w[1]), np.log2(e_w[1] / e_w[2])
    sh = np.log2(e_h[0] / e_h[1]), np.log2(e_h[1] / e_h[2])
    assert all(2.8 < x < 3.2 for x in sw), sw
    assert all(1.8 < x < 2.2 for x in sh), sh  # local error O(T^2): first order
    # the embedded solution uses Re(a) only: sum Re(a) = 1 keeps it consistent
    assert abs(np.sum(a.real) - 1.0) < 1e-13


def test_error_norm_definition():
    w = np.array([1.0, -2.0, 0.0])
    h = np.array([1.5, -2.0, 0.1])
    e = np.array([0.5 / 2.5, 0.0, 0.1 / 1.1]) / 1e-3
    assert abs(O.error_norm(w, h, 1e-3) - np.sqrt(np.mean(e ** 2))) < 1e-12


def test_adaptive_reaches_end_and_tolerance_controls_error():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(22)
    shape = (10, 10)
    pr = _prob(2, "periodic", "field", 1.0, np.exp(0.5 * rng.standard_normal(shape)))
    A = dense(pr, shape)
    u0 = rng.random(shape)
    L = 16
    a = O.plan(L)["a"]
    rho = O.rho_bound(pr)
    t_end = 3.0
    ref = scipy_linalg.expm(t_end * A) @ u0.ravel()
    errs, steps = [], []
    for tol in (1e-3, 1e-5):
        u, st = O.frkc2_adaptive(u0, a, O.beta(L), pr, t_end, tol, dt0=0.01, rho=rho)
        assert abs(st["t"] - t_end) < 1e-12
        errs.append(np.linalg.norm(u.ravel() - ref) / np.linalg.norm(ref))
        steps.append(st["accepted"])
        assert max(st["dts"]) <= O.beta(L) / rho * (1 + 1e-12)
    assert errs[1] < errs[0] and steps[1] > steps[0]


# ---------------------------------------------------------------------------------------
# Convex monotone property (Sec. 2.3, Fig. 4): two materials in contact
# ---------------------------------------------------------------------------------------

def _two_material(ratio, n=200):
    """1D periodic bar: kappa = 1 and hot (u = 1) on the left half, kappa = 1/ratio and cold
    (u = 0) on the right half (the paper's problem, parameters not stated: this reading)."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    kap = np.where(x < 0.5, 1.0, 1.0 / ratio)
    u0 = np.where(x < 0.5, 1.0, 0.0)
    return u0, _prob(1, "periodic", "field", dx, field=kap)


def _sign_changes(u, tiny=1e-12):
    """Sign changes of the periodic differences above ``tiny``: 2 for one maximum region and
    one minimum region, more when spurious extrema ("noise") appear."""
    d = np.diff(np.concatenate([u, u[:1]]))
    d = d[np.abs(d) > tiny]
    sg = np.sign(d)
    return int(np.sum(sg != np.roll(sg, 1)))


@pytest.mark.parametrize("ratio", [100.0, 1000.0])
def test_cmp_uniform_stages_noisy_error_control_clean(ratio):
    """Sec. 2.3: with a uniform 8 stages per step the two-material solution shows noise (here
    spurious extrema); with the error control of Sec. 3 and about the same number of
    f-evaluations it does not, and it keeps the maximum principle."""
    u0, pr = _two_material(ratio)
    pl = O.plan(8)
    rho = O.rho_bound(pr)
    t_end = 0.01
    n = int(np.ceil(t_end / (pl["beta"] / rho)))
    fixed = O.frkc2_step(u0, pl["a"], t_end / n, pr, n)
    ctrl, st = O.frkc2_adaptive(u0, pl["a"], pl["beta"], pr, t_end, 1e-3, dt0=1e-6, rho=rho)
    assert _sign_changes(fixed) > 10
    assert _sign_changes(ctrl) == 2
    assert ctrl.max() <= 1.0 and ctrl.min() >= 0.0
    evals_fixed, evals_ctrl = n * 8, (st["accepted"] + st["rejected"]) * 8
    assert evals_ctrl < 1.5 * evals_fixed


# ---------------------------------------------------------------------------------------
# Step-size controller (Sec. 3, Eqs. 14-16) on a problem with closed-form step errors
# ---------------------------------------------------------------------------------------

def _one_cell_polys(a, L):
    """One Dirichlet cell (1D, n = 1, dx = 1, kappa = 1): f(w) = -2 w, so z = -2 T.  The step's
    factor R(z) comes from the Chebyshev closed form and the embedded factor
    Ehat(z) = 1 + z sum_l Re(a_l) Re(P_l(z)), P_l = prod_{j<l} (1 + a_j z), from polynomial
    algebra on the coefficients -- neither from the oracle's grid stepping."""
    Poly = np.polynomial.Polynomial
    Pl, E = Poly([1.0 + 0j]), Poly([1.0])
    for al in a:
        E = E + Poly([0.0, 1.0]) * al.real * Poly(Pl.coef.real)
        Pl = Pl * Poly([1.0, al])
    return (lambda z: R_closed(z, L)), E


def _controller_by_hand(a, L, u0, tol, dt0, attempts, safe=0.8, mutate=None):
    """Eq. 16 written out from the paper for the one-cell problem: rejection scales T by
    SAFE/sqrt(e); after an accepted step T <- T (SAFE/sqrt(e_n)) (T_n/T_{n-1}) sqrt(e_{n-1}/e_n)
    (SAFE/sqrt(e_n) alone after the first).  ``mutate`` plants a plausible mistake."""
    R, E = _one_cell_polys(a, L)
    lam = -2.0
    u, T, Tp, ep, seq = u0, dt0, None, None, []
    for _ in range(attempts):
        w, h = R(T * lam) * u, E(T * lam) * u
        e = abs(w - h) / (tol * (1.0 + max(abs(w), abs(h))))
        if e > 1.0:
            seq.append((T, e, False))
            T *= safe / np.sqrt(e)
            continue
        seq.append((T, e, True))
        u = w
        expo = 1.0 / 3.0 if mutate == "exponent" else 0.5
        fac = safe / e ** expo
        if Tp is not None:
            if mutate != "no_ratio":
                fac *= T / Tp
            if mutate != "no_err_ratio":
                fac *= np.sqrt(ep / e)
        if mutate == "no_leading_T":
            Tp, ep, T = T, e, min(fac, 5.0)
        else:
            Tp, ep, T = T, e, T * min(fac, 5.0)
    return seq


def test_controller_sequence_closed_form_one_cell():
    """The oracle's attempt sequence (T, ||err||, accepted) equals Eq. 16 evaluated on closed-
    form step errors: one rejection, then accepted steps with changing T.  The same scenario
    tells the reading apart from a dropped leading T^n, a dropped T^n/T^{n-1}, a dropped
    sqrt(e_{n-1}/e_n) and a wrong exponent."""
    L = 16
    a = O.plan(L)["a"]
    pr = _prob(1, "dirichlet", "const", 1.0, c=1.0)
    tol, dt0, attempts = 0.01, 0.5, 7
    _, st = O.frkc2_adaptive(np.array([1.0]), a, O.beta(L), pr, t_end=100.0, tol=tol, dt0=dt0,
                             max_steps=attempts)
    got = st["trace"]
    ref = _controller_by_hand(a, L, 1.0, tol, dt0, attempts)
    assert [g[2] for g in got] == [r[2] for r in ref]
    assert not ref[0][2] and sum(r[2] for r in ref) >= 5
    Ts = [r[0] for r in ref if r[2]]
    assert max(Ts) / min(Ts) > 1.5  # the step size really changes
    for g, r in zip(got, ref):
        assert abs(g[0] / r[0] - 1.0) < 1e-10 and abs(g[1] / r[1] - 1.0) < 1e-8
    for m in ("no_leading_T", "no_ratio", "no_err_ratio", "exponent"):
        bad = _controller_by_hand(a, L, 1.0, tol, dt0, attempts, mutate=m)
        assert max(abs(b[0] / r[0] - 1.0) for b, r in zip(bad, ref)) > 1e-3, m


def test_controller_deadbeat_when_error_scales_as_T_squared():
    """Eq. 16 is built for a local error estimate ||err|| = C T^2 (Eq. 14 is first order): then
    one rejection, or one controlled step, sets ||err|| = SAFE^2 and the predictive factor
    keeps it there.  Small z = T lambda on one cell makes ||err|| proportional to T^2 to
    about 0.1 %."""
    L = 16
    a = O.plan(L)["a"]
    pr = _prob(1, "dirichlet", "const", 1.0, c=1.0)
    _, st = O.frkc2_adaptive(np.array([1.0]), a, O.beta(L), pr, t_end=100.0, tol=1e-9, dt0=1e-3,
                             max_steps=8)
    tr = st["trace"]
    assert not tr[0][2]  # e(dt0) > 1: rejected
    for T, e, ok in tr[1:]:
        assert ok and abs(e - 0.64) < 5e-3, (T, e)


def test_real_pair_form_equals_complex_stages():
    """Two adjacent conjugate stages on a real state, w + 2 T Re(a) f(w) + T^2 |a|^2 f(f(w)) in
    the evaluated real form, equal the two literal complex Euler stages for a linear f
    (a pin of the paired variant, Sec. 2.2 order with pairs adjacent)."""
    rng = np.random.default_rng(31)
    shape = (12, 10)
    pr = _prob(2, "periodic", "field", 1.0, np.exp(0.5 * rng.standard_normal(shape)))
    u0 = rng.random(shape)
    for L in (8, 32):
        a = O.plan(L, method="paired")["a"]
        dt = 0.9 * O.beta(L) / O.rho_bound(pr)
        ref = O.frkc2_step(u0, a, dt, pr, 2)
        got = O.frkc2_step_paired(u0, a, dt, pr, 2)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    # a non-adjacent order is not a pair form: the real form then differs
    a = O.plan(8)["a"]
    dt = 0.9 * O.beta(8) / O.rho_bound(pr)
    assert np.linalg.norm(O.frkc2_step_paired(u0, a, dt, pr, 1) - O.frkc2_step(u0, a, dt, pr, 1)) > 1e-3


# ---------------------------------------------------------------------------------------
# The 3D kappa(u) workload at s = 128 (finding: complex stages of a strongly nonlinear f)
# ---------------------------------------------------------------------------------------

def test_nonlinear3d_recipe_overflows_at_s128_not_s32():
    """The 3D recipe (kappa(u) = 1 + u^2.5, hot spot of peak 2 with 1 % noise, Dirichlet,
    T = 0.9 beta / rho) on a 32^3 instance: at s = 128 the complex stage states of one FP64
    oracle step overflow; at s = 32 the step is finite and stays near [0, 2]; with kappa
    frozen at kappa(u0) -- a linear f with the same rho -- the s = 128 step is finite and
    bounded by max u0.  The failure is the nonlinear kappa evaluated on strongly complex stage
    states (Sec. 2.2: partial products amplify stage states by up to Q), not the stage count
    or the step size."""
    u0 = I.hotspot3d_u0(32, sigma=20.0)
    pr = _prob(3, "dirichlet", "power", 1.0, c=1.0, p=2.5)
    rho = O.rho_bound(pr, u0)
    frozen = _prob(3, "dirichlet", "field", 1.0, field=1.0 + u0 ** 2.5)
    assert abs(O.rho_bound(frozen) / rho - 1.0) < 1e-12
    with np.errstate(all="ignore"):
        for s in (32, 128):
            pl = O.plan(s)
            dt = 0.9 * pl["beta"] / rho
            out = O.frkc2_step(u0, pl["a"], dt, pr, 1)
            lin = O.frkc2_step(u0, pl["a"], dt, frozen, 1)
            assert np.all(np.isfinite(lin)) and np.abs(lin).max() <= u0.max()
            if s == 32:
                assert np.all(np.isfinite(out)) and -0.05 < out.min() and out.max() < 2.1
            else:
                assert not np.all(np.isfinite(out))


# ---------------------------------------------------------------------------------------
# Rounding gain of a stage order (Sec. 2.2 applied to rounding errors)
# ---------------------------------------------------------------------------------------

def _lap5(W, k):
    """Periodic 5-point flux-form operator written out here (not the oracle's), any dtype."""
    kx = 0.5 * (k + np.roll(k, 1, 1))
    ky = 0.5 * (k + np.roll(k, 1, 0))
    fx = kx * (W - np.roll(W, 1, 1))
    fy = ky * (W - np.roll(W, 1, 0))
    return (np.roll(fx, -1, 1) - fx) + (np.roll(fy, -1, 0) - fy)


@pytest.mark.parametrize("method", ["greedy", "lebedev"])
def test_rounding_gain_predicts_float32_step_error(method):
    """One FRKC2 step run in numpy complex64 against the same step in complex128: the
    relative error is (unit roundoff 2^-24) x rounding_gain within a factor of three, for the
    paper's greedy order (g from 30 to 1300) and the Lebedev-Finogenov order (g about 2-3),
    a span of three decades of error."""
    n = 96
    u0 = I.smooth_unit((n, n), 12.0, 3819)
    k = I.kappa_field((n, n), 3818, ell=3.0).astype(np.float32)
    kx = 0.5 * (k + np.roll(k, 1, 1))
    ky = 0.5 * (k + np.roll(k, 1, 0))
    rho = float(np.max(2 * (kx + np.roll(kx, -1, 1) + ky + np.roll(ky, -1, 0))))
    k64 = k.astype(np.float64)
    for s in (16, 64, 128):
        a = O.plan(s, method=method)["a"] if method == "greedy" else O.step_sizes(s)[O.order_lebedev(s)]
        dt = 0.9 * O.beta(s) / rho
        W64 = u0.astype(np.complex128)
        W32 = u0.astype(np.complex64)
        for al in a:
            W64 = W64 + (dt * al) * _lap5(W64, k64)
            W32 = W32 + np.complex64(dt * al) * _lap5(W32, k)
        err = np.linalg.norm(W32.real - W64.real) / np.linalg.norm(W64.real)
        g = O.rounding_gain(a, O.beta(s))
        ratio = err / (2.0 ** -24 * g)
        assert 0.33 < ratio < 3.0, (s, g, err, ratio)


def test_rounding_gain_closed_forms():
    """Two stages a, conj(a) (L = 2): g^2 = 1 + mean_x |1 + conj(a) x|^2, the mean of a
    quadratic in x over midpoints, in closed form; and a reversed order changes g."""
    a = O.step_sizes(2)
    b = O.beta(2)
    P = 4096
    x = -b * (np.arange(P) + 0.5) / P
    m1, m2 = x.mean(), (x * x).mean()
    ab = a[1]
    want = 1.0 + (1.0 + 2.0 * ab.real * m1 + abs(ab) ** 2 * m2)
    assert abs(O.rounding_gain(a, b, P) ** 2 / want - 1.0) < 1e-12
    a16 = O.plan(16)["a"]
    assert abs(O.rounding_gain(a16[::-1], O.beta(16)) / O.rounding_gain(a16, O.beta(16)) - 1.0) > 1e-3


# --------------------------------------------------------------------------------------
# Rank-4 polynomial (Sec. 2, Eq. 7 with N = 4; order conditions Eq. 5, bound Eq. 6)
# --------------------------------------------------------------------------------------


def _taylor_coeffs(a):
    c = np.array([1.0 + 0j])
    for al in a:
        c = np.convolve(c, np.array([1.0, al]))
    return c


def test_rank4_at_L4_is_the_rk4_taylor_polynomial():
    """L = N = 4 (M = 1): degree 4 and five order conditions leave only the Taylor polynomial
    1 + z + z^2/2 + z^3/6 + z^4/24, whose real stability boundary is the real root of
    1 + z/2 + z^2/6 + z^3/24 = 0 (numpy.roots; textbook value 2.78529)."""
    c = _taylor_coeffs(O.chebsum_step_sizes(4, 1))
    assert np.allclose(c, [1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0], rtol=0, atol=1e-14)
    r = np.roots([1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0])
    x = -float(r[np.argmin(np.abs(r.imag))].real)
    assert abs(O.chebsum_beta(4, 1) - x) < 1e-12 * x
    assert abs(x - 2.78529) < 1e-5


@pytest.mark.parametrize("M", [1, 2, 4, 8, 32])
def test_rank_n_construction_at_N2_gives_the_frkc2_polynomial(M):
    """The rank-N route (order conditions for d, largest bounded alpha, roots through
    T_M(x) = y) at N = 2 reproduces alpha = 4(1 - 1/L^2)/3, d_1 = 0 and the FRKC2 roots."""
    L = 2 * M
    al = O.chebsum_alpha(2, M)
    assert abs(al - 4.0 * (1.0 - 1.0 / L ** 2) / 3.0) < 1e-14
    d = O.chebsum_coefficients(2, M, al)
    assert abs(d[1]) < 1e-12 and abs(d[0] - (1.0 - al / 4.0)) < 1e-14 and abs(d[2] - al / 8.0) < 1e-14
    assert np.max(np.abs(O.chebsum_roots(2, M) - O.roots(L))) < 1e-13


@pytest.mark.parametrize("L", [8, 16, 64, 256])
def test_rank4_order_conditions_exactly_fourth(L):
    """prod (1 + a_l z) = e^z + O(z^5): e_n n! = 1 for n <= 4 (Eq. 5), but not for n = 5."""
    c = _taylor_coeffs(O.chebsum_step_sizes(4, L // 4))
    fac = np.array([1.0, 1.0, 2.0, 6.0, 24.0, 120.0])
    err = np.abs(c[:6] * fac - 1.0)
    assert np.all(err[:5] < 1e-11), err
    assert err[5] > 0.05


@pytest.mark.parametrize("L", [8, 32, 128])
def test_rank4_product_equals_chebyshev_sum(L):
    """The roots reproduce B = d_0 + 2 sum d_k T_{kM}(1 + z/(M^2 alpha)), the T_j taken from
    numpy's Chebyshev basis, at real and complex z."""
    M = L // 4
    al = O.chebsum_alpha(4, M)
    d = O.chebsum_coefficients(4, M, al)
    a = O.chebsum_step_sizes(4, M)
    rng = np.random.default_rng(L)
    b = O.chebsum_beta(4, M)
    z = -b * rng.random(40) + 1j * 0.05 * b * rng.standard_normal(40)
    x = 1.0 + z / (M * M * al)
    B = d[0] + 2.0 * sum(d[k] * C.Chebyshev.basis(k * M)(x) for k in range(1, 5))
    Rp = R_product(z, a)
    assert np.max(np.abs(Rp - B)) < 1e-9 * max(1.0, np.max(np.abs(B)))


@pytest.mark.parametrize("L", [8, 16, 64])
def test_rank4_bounded_on_extent_and_alpha_maximal(L):
    """|R| <= 1 on [-beta, 0] (dense grid, product form); the order-condition polynomial for an
    alpha 1e-6 larger leaves the bound, 1e-6 smaller stays inside (Eq. 6)."""
    M = L // 4
    a = O.chebsum_step_sizes(4, M)
    b = O.chebsum_beta(4, M)
    x = -b * np.linspace(0.0, 1.0, 40001)
    assert np.max(np.abs(R_product(x, a))) <= 1.0 + 1e-10
    al = O.chebsum_alpha(4, M)
    y = np.cos(np.linspace(0.0, np.pi, 200001))

    def qmax(alpha_):
        d = O.chebsum_coefficients(4, M, alpha_)
        c = 2.0 * d
        c[0] = d[0]
        return np.max(np.abs(C.chebval(y, c)))

    assert qmax(al * (1 + 1e-6)) > 1.0 + 1e-9
    assert qmax(al * (1 - 1e-6)) <= 1.0


@pytest.mark.parametrize("L", [8, 64])
def test_rank4_conjugate_pairs_positive_real_part(L):
    a = O.chebsum_step_sizes(4, L // 4)
    assert np.array_equal(a[::-1], np.conj(a))
    assert np.all(a.real > 0) and np.all(np.abs(a.imag) > 0)
    assert abs(a.sum() - 1.0) < 1e-13


def test_rank4_fourth_order_against_expm():
    """A rank-4 plan converges at order 4 to expm on a variable-kappa periodic problem (the
    rank-2 plan, same problem, at order 2)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    shape = (8, 8)
    pr = _prob(2, "periodic", "field", 1.0, np.exp(0.5 * rng.standard_normal(shape)))
    A = dense(pr, shape)
    u0 = rng.random(shape)
    t_end = 2.0
    ref = scipy_linalg.expm(t_end * A) @ u0.ravel()
    a = O.plan(16, N=4)["a"]
    errs = [np.linalg.norm(O.frkc2_step(u0, a, t_end / m, pr, m).ravel() - ref) for m in (16, 32, 64)]
    slope = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert all(3.8 < s < 4.2 for s in slope), slope


@pytest.mark.parametrize("L", [16, 64, 256])
def test_rank4_plan_Q_near_single_factor_bound(L):
    """The rank-4 plan meets 10 L^2 with a realised Q within 1.3x of the largest single factor
    max |1 + a_l x| (a lower bound for every ordering, Eq. 10)."""
    p = O.plan(L, N=4)
    x = -p["beta"] * np.linspace(0.0, 1.0, 16 * L + 1)
    single = np.max(np.abs(1.0 + np.outer(p["a"], x)))
    assert p["Q"] <= 10.0 * L * L
    assert single <= p["Q"] * (1 + 1e-12) <= 1.3 * single
    assert sorted(p["order"]) == list(range(L))


def test_rank4_s4_step_equals_rk4_step():
    """On a linear problem the 4-stage rank-4 factorised step and the classical RK4 tableau
    (``rk4``) are the same map."""
    rng = np.random.default_rng(11)
    shape = (12, 10)
    pr = _prob(2, "dirichlet", "field", 1.0, np.exp(0.5 * rng.standard_normal(shape)))
    u0 = rng.random(shape)
    T = 0.9 * O.chebsum_beta(4, 1) / O.rho_bound(pr)
    a = O.plan(4, N=4)["a"]
    ref = O.rk4(u0, T, pr, 3)
    assert np.max(np.abs(O.frkc2_step(u0, a, T, pr, 3) - ref)) < 1e-14 * np.max(np.abs(ref))
