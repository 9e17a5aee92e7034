"""FRKC2 oracle: a plain, slow, FP64 CPU statement of the method.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py`` -- nothing in the
product package imports, links or runs it, and it imports nothing from the product.

Every function follows a passage of O'Sullivan, "Factorized Runge-Kutta-Chebyshev
Methods" (arXiv:1702.03818); the passage is cited in each docstring.  Where the paper is
silent or garbled the reading taken is stated in the docstring ("Reading:").

Contents
--------
* stability polynomial and step sizes (Sec. 2, Eqs. 5-8): ``alpha``, ``beta``, ``roots``,
  ``step_sizes``; the damped step sizes of Sec. 2.1 (``damped_step_sizes``); the rank-N
  Chebyshev-sum polynomial of Eq. 7 (``chebsum_coefficients``, ``chebsum_alpha``,
  ``chebsum_beta``, ``chebsum_roots``, ``chebsum_step_sizes``; N = 4 is the fourth-order plan);
* internal stability (Sec. 2.2, Eqs. 10-12): ``realised_Q`` (brute force over all
  sub-sequences), ``rounding_gain`` (the partial products applied to rounding errors),
  ``order_greedy``, ``order_lebedev`` and ``plan`` (the n-loop);
* the diffusion operator f(w) = div(kappa grad w) in flux form (the semi-discrete system of
  Eq. 1): ``cell_kappa``, ``apply_f``, ``rho_bound``;
* the FRKC2 step (Sec. 3, Eq. 13), stages applied literally as complex forward-Euler steps:
  ``frkc2_step``;
* its discrete adjoint (reverse replay of Eq. 13): ``frkc2_adjoint``;
* a classical RK4 integrator used as a fine-step reference for the nonlinear case: ``rk4``.

Problem description
-------------------
A problem is a dict with keys ``ndim`` (1..3), ``dx`` (grid spacing), ``bc``
(``"periodic"`` or ``"dirichlet"``: u = 0 in the ghost cells outside the grid), ``kappa``
(``"const"``, ``"field"`` or ``"power"``), ``kappa_c`` (the constant, or the coefficient c
of kappa(u) = 1 + c u^p), ``kappa_p`` (the exponent p) and ``kappa_field`` (cell-centred
array, same shape as the state).  State arrays use numpy order, last axis = x.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` except the
greedy ordering itself (``order_greedy``): the paper's coefficient table is not available,
so the permutation it produces is checked through invariants (it is a permutation, the
product is unchanged, the realised Q meets the paper's bound) and, for L = 6 and 8, by brute
force (it attains the smallest Q of all L! orderings) -- parity unpinned for the exact greedy
order of larger plans.  ``order_lebedev`` is pinned by the lower bound it attains.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------------------
# Stability polynomial and step sizes (Sec. 2)
# ----------------------------------------------------------------------------------------


def alpha(L: int) -> float:
    """alpha_M of Eq. 8 for the second-order polynomial of degree L = 2M.

    Reading (the paper defers the closed form to its companion paper): with N = 2 the
    polynomial of Eq. 7 is R(z) = 1 - alpha/4 + (alpha/4) T_L(1 + 4 z / (L^2 alpha)).
    R(0) = 1 and R'(0) = 1 hold for any alpha; R''(0) = 1 (Eq. 5, n = 2) gives
    alpha = 4 (1 - 1/L^2) / 3, which is also the largest alpha keeping |R| <= 1 (Eq. 6).
    """
    return 4.0 * (1.0 - 1.0 / (L * L)) / 3.0


def beta(L: int) -> float:
    """Extent of the real stability interval [-beta, 0] (Eq. 6): beta = L^2 alpha / 2."""
    return 0.5 * L * L * alpha(L)


def roots(L: int) -> np.ndarray:
    """Roots zeta_j of T_L(x) = 1 - 4/alpha, the zeros of the polynomial of Eq. 7.

    zeta_j = cos((pi (2j + 1) - i eta) / L), eta = arccosh(4/alpha - 1), j = 0..L-1.
    Reading: the roots come in conjugate pairs j <-> L-1-j; the second member of each pair
    is set to the exact conjugate of the first so that the pair is conjugate bit for bit.
    """
    if L < 2 or L % 2:
        raise ValueError("L must be even and >= 2")
    eta = np.arccosh(4.0 / alpha(L) - 1.0)
    z = np.empty(L, dtype=np.complex128)
    for j in range(L // 2):
        z[j] = np.cos((np.pi * (2 * j + 1) - 1j * eta) / L)
        z[L - 1 - j] = np.conj(z[j])
    return z


def step_sizes(L: int) -> np.ndarray:
    """Complex Euler step sizes a_j = 1 / (M^2 alpha_M (1 - zeta_j)), L = 2M (Eq. 8).

    Returned in root order j = 0..L-1 (before the internal-stability ordering).
    """
    M = L // 2
    return 1.0 / (M * M * alpha(L) * (1.0 - roots(L)))


def _taylor2(a):
    """First and second coefficients of prod_l (1 + a_l z) (e1 = sum a, e2 = sum_{i<j} a_i a_j)."""
    c = np.array([1.0 + 0j])
    for al in a:
        c = np.convolve(c, np.array([1.0, al]))
    return c[1], c[2]


def damped_step_sizes(L: int, nu0: float):
    """Damped step sizes of Sec. 2.1 and the damping parameter mu.

    a_l = (1 - mu_l) / ((1 - nu) M^2 alpha_M (1 - (1 - 2 mu_l) zeta_l)), nu = nu0 / N, N = 2.
    Reading: the N = 2 distinct values of mu_l belong to the two families of roots (T_M(zeta)
    = +i c for even root index j, -i c for odd j); for the step sizes to stay in conjugate
    pairs they are mu and conj(mu).  Newton-Raphson over (Re mu, Im mu) enforces the order
    conditions sum a = 1, sum_{i<j} a_i a_j = 1/2 (Eq. 5), starting from mu = 0 (the undamped
    solution), with a forward-difference Jacobian.
    """
    nu = nu0 / 2.0
    M = L // 2
    al = alpha(L)
    z = roots(L)
    even = (np.arange(L) % 2) == 0

    def steps(mu):
        m = np.where(even, mu, np.conj(mu))
        return (1.0 - m) / ((1.0 - nu) * M * M * al * (1.0 - (1.0 - 2.0 * m) * z))

    def resid(mu):
        e1, e2 = _taylor2(steps(mu))
        return np.array([(e1 - 1.0).real, (e2 - 0.5).real])

    mu = 0.0 + 0.0j
    for _ in range(60):
        r = resid(mu)
        if np.max(np.abs(r)) < 1e-14:
            break
        h = 1e-7
        J = np.column_stack([(resid(mu + h) - r) / h, (resid(mu + 1j * h) - r) / h])
        d = np.linalg.solve(J, -r)
        mu = mu + d[0] + 1j * d[1]
    a = steps(mu)
    for j in range(L // 2):  # conjugate pairs exact to the bit, as for the undamped roots
        a[L - 1 - j] = np.conj(a[j])
    return a, mu


# ----------------------------------------------------------------------------------------
# The rank-N polynomial (Sec. 2, Eq. 7 with N = 4): a sum of Chebyshev polynomials
# ----------------------------------------------------------------------------------------


def _cheb_deriv_at_one(j: int, n: int) -> float:
    """n-th derivative of the Chebyshev polynomial T_j at x = 1: prod_{m<n} (j^2 - m^2)/(2m+1).

    (The classical identity obtained from the Chebyshev differential equation
    (1 - x^2) T'' - x T' + j^2 T = 0 differentiated n times and taken at x = 1.)
    """
    p = 1.0
    for m in range(n):
        p *= (j * j - m * m) / (2.0 * m + 1.0)
    return p


def chebsum_coefficients(N: int, M: int, alpha_: float) -> np.ndarray:
    """Coefficients d_0..d_N of B(z) = d_0 + 2 sum_{k=1}^N d_k T_{kM}(x), x = 1 + z/(M^2 alpha).

    Reading of Eq. 7: the argument of the Chebyshev polynomials is the shifted variable
    x = 1 + z/(M^2 alpha_M), the map under which the step sizes of Eq. 8 are
    a_l = 1/(M^2 alpha_M (1 - zeta_l)) for the roots zeta_l in x.  The d_k solve the N + 1
    linear order conditions of Eq. 5, R(0) = 1 and R^(n)(0) = 1 for n = 1..N, where
    d^n/dz^n T_j(x(z)) at z = 0 is T_j^(n)(1) / (M^2 alpha)^n.
    """
    A = np.zeros((N + 1, N + 1))
    A[0, 0] = 1.0
    A[0, 1:] = 2.0
    for n in range(1, N + 1):
        for k in range(1, N + 1):
            A[n, k] = 2.0 * _cheb_deriv_at_one(k * M, n) / (M * M * alpha_) ** n
    return np.linalg.solve(A, np.ones(N + 1))


def _chebsum_Q(d: np.ndarray) -> np.ndarray:
    """Chebyshev series of Q(y) = d_0 + 2 sum_k d_k T_k(y): since T_{kM} = T_k(T_M), B = Q(T_M(x))."""
    c = 2.0 * np.asarray(d, dtype=np.float64)
    c[0] = d[0]
    return c


def _max_abs_Q(d: np.ndarray) -> float:
    """max |Q(y)| over [-1, 1] from the end point y = -1 and the real critical points inside.

    Q(1) = R(0) = 1 holds by the first order condition and Q'(1) = alpha > 0 there, so the
    end point y = 1 is left out (it would only contribute its rounding error).
    """
    from numpy.polynomial import chebyshev as C

    c = _chebsum_Q(d)
    cand = [-1.0]
    for r in C.chebroots(C.chebder(c)):
        if abs(r.imag) <= 1e-12 * max(1.0, abs(r.real)) and -1.0 < r.real < 1.0:
            cand.append(float(r.real))
    return float(np.max(np.abs(C.chebval(np.array(cand), c))))


def chebsum_alpha(N: int, M: int) -> float:
    """alpha_M of the rank-N polynomial: the largest alpha whose order-condition polynomial is
    bounded, |R(z)| <= 1 on [-2 M^2 alpha, 0] (Eq. 6).

    Reading: T_M maps x in [-1, 1] onto [-1, 1], so the bound on z in [-2 M^2 alpha, 0] is
    |Q(y)| <= 1 on y in [-1, 1]; alpha is found by bisection on that test (the feasible alphas
    form an interval from 0).  For N = 2 this gives the closed form 4 (1 - 1/L^2) / 3 with
    d_1 = 0; for L = N (M = 1) B is the degree-N Taylor polynomial of e^z.
    """
    lo, hi = 0.25, 4.0
    if _max_abs_Q(chebsum_coefficients(N, M, lo)) > 1.0:
        raise ValueError("lower bisection bracket not feasible")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        if _max_abs_Q(chebsum_coefficients(N, M, mid)) <= 1.0:
            lo = mid
        else:
            hi = mid
    return lo


def chebsum_beta(N: int, M: int) -> float:
    """Real stability extent of the rank-N polynomial: beta = 2 M^2 alpha_M (x = -1)."""
    return 2.0 * M * M * chebsum_alpha(N, M)


def chebsum_roots(N: int, M: int) -> np.ndarray:
    """The L = N M roots zeta of B in x, in the root order used for the stage ordering.

    Q(y) has N roots y_i (numpy's companion-matrix root finder); T_M(x) = y_i has the M
    solutions x = cos((arccos y_i + 2 pi k) / M), k = 0..M-1.  Reading of the root order:
    the roots with Im zeta > 0 sorted by decreasing Re zeta are zeta_0..zeta_{L/2-1}, and
    zeta_{L-1-j} = conj(zeta_j) exactly -- for N = 2 this is the order of ``roots``.  Q has
    real coefficients and, for N = 2 and 4, no real roots, so no zeta is real.
    """
    from numpy.polynomial import chebyshev as C

    L = N * M
    al = chebsum_alpha(N, M)
    ys = C.chebroots(_chebsum_Q(chebsum_coefficients(N, M, al)))
    xs = []
    for y in ys.astype(np.complex128):
        th = np.arccos(y)
        for k in range(M):
            xs.append(np.cos((th + 2.0 * np.pi * k) / M))
    xs = np.array(xs)
    upper = xs[xs.imag > 0.0]
    if len(upper) != L // 2:
        raise ValueError("roots not in conjugate pairs off the real axis")
    upper = upper[np.argsort(-upper.real, kind="stable")]
    z = np.empty(L, dtype=np.complex128)
    z[: L // 2] = upper
    z[L // 2:] = np.conj(upper[::-1])
    return z


def chebsum_step_sizes(N: int, M: int) -> np.ndarray:
    """Step sizes a_l = 1/(M^2 alpha_M (1 - zeta_l)) of the rank-N polynomial (Eq. 8), in root
    order; the second member of each conjugate pair is the exact conjugate of the first."""
    L = N * M
    al = chebsum_alpha(N, M)
    a = 1.0 / (M * M * al * (1.0 - chebsum_roots(N, M)))
    for j in range(L // 2):
        a[L - 1 - j] = np.conj(a[j])
    return a


def stability_extent(a, guess: float) -> float:
    """Largest x with |R(-x)| <= 1 near ``guess`` (bisection on the last crossing, Eq. 6)."""
    def absR(x):
        return float(np.abs(np.prod(1.0 + a * (-x))))
    lo, hi = 0.9 * guess, 1.1 * guess
    while absR(lo) > 1.0:
        lo *= 0.99
    while absR(hi) <= 1.0:
        hi *= 1.01
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if absR(mid) <= 1.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-15 * hi:
            break
    return lo


# ----------------------------------------------------------------------------------------
# Internal stability (Sec. 2.2)
# ----------------------------------------------------------------------------------------


def realised_Q(a: np.ndarray, beta_: float, points: int) -> float:
    """Q = max over 1 <= j <= k <= L and x in [-beta, 0] of prod_{l=j}^{k} |1 + a_l x| (Eqs. 10-11).

    Brute force over every contiguous sub-sequence of the ordered ``a`` on the grid
    x_i = -beta i / points, i = 0..points (products formed as sums of logarithms).
    """
    x = -beta_ * np.arange(points + 1) / points
    logv = np.log(np.abs(1.0 + np.outer(a, x)))
    best = -np.inf
    for j in range(len(a)):
        sub = np.cumsum(logv[j:], axis=0)  # row k-j holds log prod_{l=j}^{k}
        best = max(best, float(sub.max()))
    return float(np.exp(best))


def rounding_gain(a: np.ndarray, beta_: float, points: int | None = None) -> float:
    """Rounding gain of a stage order: g = sqrt(sum_l mean_x |prod_{j>l} (1 + a_j x)|^2).

    A rounding error made in stage l (while forming W^{l+1}) reaches the step's output through
    the factors of the later stages l+1..L-1 (the partial products of Sec. 2.2, Eq. 10), so if
    the rounding is spread evenly over the spectrum x = T lambda in [-beta, 0] one step's
    relative error is about (unit roundoff) * g.  The mean is over ``points`` midpoints
    x_i = -beta (i + 1/2) / points (default max(2048, 4 L)).  Plain definition: each suffix
    product is formed afresh.
    """
    a = np.asarray(a)
    L = len(a)
    P = points or max(2048, 4 * L)
    x = -beta_ * (np.arange(P) + 0.5) / P
    total = 0.0
    for l in range(L):
        prod = np.ones(P, dtype=np.complex128)
        for j in range(l + 1, L):
            prod = prod * (1.0 + a[j] * x)
        total += float(np.mean(np.abs(prod) ** 2))
    return float(np.sqrt(total))


def order_greedy(a: np.ndarray, beta_: float, n: int, samples: int, C: float = 1e-4) -> np.ndarray:
    """Stage ordering that keeps the estimated amplification of Eq. 12 small.

    Reading of Eq. 12 (its printed limits are garbled): the items ordered are the L
    individual step sizes.  The samples are x_k = -beta_bar k / S, k = 1..S, on the reduced
    range beta_bar = (1 - n C) beta.  For position l = 1..L the unplaced step size j that
    minimises sum_k max(P_k v_jk, Rest_k / v_jk) is placed, where v_jk = |1 + a_j x_k|, P is
    the product over the stages already placed and Rest the product over every stage not
    yet placed (j included).  Ties go to the lowest original index.  Sums are formed in log
    space (log-sum-exp) so that no product overflows.

    Returns the permutation (indices into ``a``) in stage order.
    """
    L = len(a)
    beta_bar = (1.0 - n * C) * beta_
    x = -beta_bar * np.arange(1, samples + 1) / samples
    logv = np.log(np.abs(1.0 + np.outer(a, x)))
    remaining = list(range(L))
    placed = []
    logP = np.zeros(samples)
    for _ in range(L):
        rem = np.asarray(remaining)
        cand = logv[rem]
        logRest = cand.sum(axis=0)
        e = np.maximum(logP[None, :] + cand, logRest[None, :] - cand)
        m = e.max(axis=1)
        cost = m + np.log(np.exp(e - m[:, None]).sum(axis=1))
        j = remaining.pop(int(np.argmin(cost)))
        placed.append(j)
        logP = logP + logv[j]
    return np.asarray(placed, dtype=np.int64)


def lebedev_permutation(m: int) -> list:
    """Lebedev-Finogenov recursive permutation of 0..m-1 (the ordering idea of Sec. 2.2).

    P(1) = (0); P(m) interleaves each entry v of P(floor(m / 2)) with its mirror m - 1 - v, and
    for odd m ends with the middle index floor(m / 2).  Reading for odd sizes (the recursion is
    classically stated for powers of two): every root stays paired with its mirror about the
    middle; appending the last index instead (P(2q + 1) = P(2q), 2q) leaves the realised Q at
    17 L^2 for L = 1000 and 1600 L^2 for L = 4094, this rule at 0.71 and 2.7 L^2.
    """
    if m == 1:
        return [0]
    out = []
    for v in lebedev_permutation(m // 2):
        out += [v, m - 1 - v]
    if m % 2:
        out.append(m // 2)
    return out


def order_lebedev(L: int) -> np.ndarray:
    """Stage order: the L/2 roots of the upper half (j < L/2) in Lebedev-Finogenov order, then
    their conjugates (j -> L-1-j) in the same order.

    On the real axis |1 + a_j x| = |1 + conj(a_j) x|, so the second half repeats the magnitudes
    of the first; reading for large L (see ``plan``).
    """
    h = np.asarray(lebedev_permutation(L // 2), dtype=np.int64)
    return np.concatenate([h, L - 1 - h])


def order_paired(L: int) -> np.ndarray:
    """Stage order with each conjugate pair adjacent: for the upper-half roots j in
    Lebedev-Finogenov order, the stages j then L-1-j.  Two adjacent conjugate stages act on a
    real state as the real quadratic factor 1 + 2 Re(a) z + |a|^2 z^2 (the pairs "taken in
    conjugate pairs and evaluated in real arithmetic"); any such order has Q >= the largest
    quadratic factor (about 0.12 L^4)."""
    h = np.asarray(lebedev_permutation(L // 2), dtype=np.int64)
    return np.stack([h, L - 1 - h], axis=1).ravel()


def frkc2_step_paired(u0, a, T, prob, nsteps: int = 1):
    """The FRKC2 step with the stages applied pair by pair in real arithmetic.

    For adjacent stages (a, conj(a)) and a linear f, (1 + T a f)(1 + T conj(a) f) w =
    w + 2 T Re(a) f(w) + T^2 |a|^2 f(f(w)); with alpha = Re a, beta = Im a this is evaluated
    as Y = w + T alpha f(w), w' = w + T (alpha - beta^2/alpha) f(w) + T (|a|^2/alpha) f(Y).
    ``a`` must list each pair as two consecutive entries (``order_paired``).
    """
    u = np.array(u0, dtype=np.float64)
    a = np.asarray(a)
    for _ in range(nsteps):
        for p in range(len(a) // 2):
            al, be = a[2 * p].real, a[2 * p].imag
            fw = apply_f(u, prob)
            Y = u + T * al * fw
            u = u + T * (al - be * be / al) * fw + T * ((al * al + be * be) / al) * apply_f(Y, prob)
    return u


def plan(L: int, samples: int | None = None, q_points: int | None = None, n_max: int = 10,
         bound: float = 10.0, method: str = "auto", nu0: float = 0.0, N: int = 2) -> dict:
    """Ordered FRKC2 step sizes for L stages (Sec. 2.2, the n-loop).

    ``greedy``: the ordering of Eq. 12 is repeated with n = 1, 2, ... until the realised Q is
    at most ``bound`` L^2 (the paper's practical bound 10 L^2) or ``n_max`` is reached; the
    ordering with the smallest realised Q is kept.  Reading: S = 16 L ordering samples and
    16 L + 1 points for the realised Q (the paper's L samples leave Q above 10 L^2 from
    L = 128 on).
    ``lebedev``: ``order_lebedev``.
    ``auto`` (reading): the greedy n-loop for L <= 256, where it meets the bound; above that
    the Lebedev-Finogenov order, and the greedy n-loop as well only if that order misses the
    bound (the smaller realised Q is kept).
    ``paired``: ``order_paired`` (conjugates adjacent, for real-arithmetic pair stages).
    ``nu0`` > 0 uses the damped step sizes of Sec. 2.1, with beta found by bisection.
    ``N`` = 4 takes the step sizes and extent of the rank-4 polynomial (``chebsum_step_sizes``,
    ``chebsum_beta``, L = 4M; undamped only).  Reading for ``auto`` there: the Lebedev-Finogenov
    order first at every L (on the rank-4 roots its realised Q is about 0.1 L^2, close to the
    largest single factor, where the greedy reaches a few L^2), the greedy n-loop only if it
    misses the bound.
    """
    if N not in (2, 4) or (N == 4 and (L % 4 or nu0 > 0.0)):
        raise ValueError("N = 2, or N = 4 with L a multiple of 4 and no damping")
    if N == 4:
        a = chebsum_step_sizes(4, L // 4)
        b = chebsum_beta(4, L // 4)
    elif nu0 > 0.0:
        a, _ = damped_step_sizes(L, nu0)
        b = stability_extent(a, (1.0 - nu0 / 2.0) * beta(L))
    else:
        a = step_sizes(L)
        b = beta(L)
    S = samples if samples is not None else 16 * L
    P = q_points if q_points is not None else 16 * L
    best = None

    def consider(perm, n):
        nonlocal best
        Q = realised_Q(a[perm], b, P)
        if best is None or Q < best["Q"]:
            best = dict(L=L, order=np.asarray(perm), a=a[perm], beta=b, Q=Q, n=n)
        return Q

    if method == "paired":
        consider(order_paired(L), 0)
        return best
    run_greedy = method == "greedy" or (method == "auto" and L <= 256 and N == 2)
    if method == "lebedev" or (method == "auto" and (L > 256 or N == 4)):
        q = consider(order_lebedev(L), 0)
        if method == "auto" and q > bound * L * L:
            run_greedy = True
    if run_greedy:
        for n in range(1, n_max + 1):
            if consider(order_greedy(a, b, n, S), n) <= bound * L * L:
                break
    return best


# ----------------------------------------------------------------------------------------
# The diffusion operator f(w) = div(kappa grad w) (the semi-discrete system of Eq. 1)
# ----------------------------------------------------------------------------------------


def cell_kappa(W, prob):
    """Cell-centred conductivity for state W: a constant, a given field, or kappa(W).

    For ``"power"`` kappa(W) = 1 + c W^p on the principal branch (W may be complex in the
    middle of a step).
    """
    kind = prob["kappa"]
    if kind == "const":
        return np.full(W.shape, float(prob["kappa_c"]))
    if kind == "field":
        return np.asarray(prob["kappa_field"], dtype=np.float64)
    if kind == "power":
        return 1.0 + prob["kappa_c"] * np.power(W, prob["kappa_p"])
    raise ValueError(kind)


def _ghost_kappa(prob, kc):
    """kappa in a Dirichlet ghost cell, as a function of the adjacent interior value.

    Reading (the paper states no boundary treatment): for a given field or a constant the
    ghost cell takes the adjacent interior cell's value, so a boundary face carries the
    boundary cell's own kappa; for kappa(u) the ghost takes kappa(0) = 1, its state being 0.
    """
    if prob["kappa"] == "power":
        return np.ones_like(kc)
    return kc


def _neighbours(A, ax, bc, ghost):
    """(A at i+1, A at i-1) along axis ``ax`` with periodic wrap or ghost values."""
    if bc == "periodic":
        return np.roll(A, -1, axis=ax), np.roll(A, 1, axis=ax)
    n = A.shape[ax]
    plus = np.concatenate([np.take(A, range(1, n), axis=ax),
                           np.take(ghost, [n - 1], axis=ax)], axis=ax)
    minus = np.concatenate([np.take(ghost, [0], axis=ax),
                            np.take(A, range(0, n - 1), axis=ax)], axis=ax)
    return plus, minus


def apply_f(W, prob):
    """f(W)_c = (1/dx^2) sum over the 2 ndim faces of c of kappa_f (W_nb - W_c).

    Flux form with the arithmetic-mean face conductivity kappa_f = (kappa_c + kappa_nb)/2
    (reading: the paper specifies no spatial discretisation; this 2nd-order form keeps the
    linear operator symmetric).  Ghost cells of a Dirichlet grid hold W = 0.
    """
    W = np.asarray(W)
    kc = cell_kappa(W, prob)
    zero = np.zeros_like(W)
    gk = _ghost_kappa(prob, kc)
    out = np.zeros(W.shape, dtype=np.result_type(W, kc))
    for ax in range(W.ndim):
        Wp, Wm = _neighbours(W, ax, prob["bc"], zero)
        kp, km = _neighbours(kc, ax, prob["bc"], gk)
        out = out + 0.5 * (kc + kp) * (Wp - W) + 0.5 * (kc + km) * (Wm - W)
    return out / (prob["dx"] * prob["dx"])


def rho_bound(prob, u=None) -> float:
    """Gershgorin bound on the spectral radius: max_c (2/dx^2) sum_faces kappa_f.

    Used for |lambda|_max of Sec. 3 when choosing T so that T |lambda|_max <= beta (Eq. 6).
    For kappa(u) the bound is taken at the real state ``u``.  Faces are summed axis by axis
    from the x axis outwards, the face on the low side before the high side.
    """
    shape = np.shape(u) if u is not None else np.shape(prob["kappa_field"])
    if prob["kappa"] == "const":
        kc = np.full(shape, float(prob["kappa_c"]))
    elif prob["kappa"] == "field":
        kc = np.asarray(prob["kappa_field"], dtype=np.float64)
    else:
        kc = 1.0 + prob["kappa_c"] * np.power(np.asarray(u, dtype=np.float64), prob["kappa_p"])
    gk = _ghost_kappa(prob, kc)
    acc = np.zeros(shape)
    for ax in reversed(range(len(shape))):
        kp, km = _neighbours(kc, ax, prob["bc"], gk)
        acc = acc + 0.5 * (kc + km)
        acc = acc + 0.5 * (kc + kp)
    return float(np.max((2.0 * acc) / (prob["dx"] * prob["dx"])))


# ----------------------------------------------------------------------------------------
# The FRKC2 step (Sec. 3, Eq. 13)
# ----------------------------------------------------------------------------------------


def frkc2_step(u0, a, T, prob, nsteps: int = 1, return_imag: bool = False):
    """Advance the real state u0 by ``nsteps`` FRKC2 steps of size T.

    Each step sets W^0 = w^n and applies W^{l+1} = W^l + T a_l f(W^l) for the step sizes
    ``a`` in the given order (Eq. 13), in complex arithmetic exactly as written.  The new
    state is w^{n+1} = W^L; reading: its real part is kept (for a linear f the imaginary
    part is zero up to rounding, the step sizes coming in conjugate pairs).  With
    ``return_imag`` the largest ||Im W^L|| / ||Re W^L|| over the steps is also returned.
    """
    u = np.array(u0, dtype=np.float64)
    worst = 0.0
    for _ in range(nsteps):
        W = u.astype(np.complex128)
        for al in a:
            W = W + (T * al) * apply_f(W, prob)
        u = W.real.copy()
        nr = np.linalg.norm(u)
        if nr > 0:
            worst = max(worst, float(np.linalg.norm(W.imag) / nr))
    return (u, worst) if return_imag else u


# ----------------------------------------------------------------------------------------
# Discrete adjoint of the FRKC2 step
# ----------------------------------------------------------------------------------------


def _cell_dkappa(W, prob):
    """d kappa / d W at each cell (zero unless kappa = kappa(W))."""
    if prob["kappa"] != "power":
        return np.zeros_like(W)
    p = prob["kappa_p"]
    return prob["kappa_c"] * p * np.power(W, p - 1.0)


def apply_jh(W, lam, prob):
    """(J_f(W)^H lam)_m for the flux-form operator, J_f the complex Jacobian of ``apply_f``.

    Differentiating f_i = (1/dx^2) sum_nb kappa_f (W_nb - W_i), kappa_f = (kappa(W_i) +
    kappa(W_nb))/2, and transposing gives
    (J^H lam)_m = (1/dx^2) sum_{nb i of m} (lam_i - lam_m) conj(kappa_f - kappa'(W_m)(W_i - W_m)/2),
    with lam = 0 in Dirichlet ghost cells.  For a fixed field kappa' = 0 and this is the
    (symmetric) operator itself applied to lam.
    """
    W = np.asarray(W, dtype=np.complex128)
    lam = np.asarray(lam, dtype=np.complex128)
    kc = cell_kappa(W, prob)
    dk = _cell_dkappa(W, prob)
    zero = np.zeros_like(W)
    gk = _ghost_kappa(prob, kc)
    out = np.zeros_like(W)
    for ax in range(W.ndim):
        Wp, Wm = _neighbours(W, ax, prob["bc"], zero)
        lp, lm = _neighbours(lam, ax, prob["bc"], zero)
        kp, km = _neighbours(kc, ax, prob["bc"], gk)
        out = out + (lp - lam) * np.conj(0.5 * (kc + kp) - 0.5 * dk * (Wp - W))
        out = out + (lm - lam) * np.conj(0.5 * (kc + km) - 0.5 * dk * (Wm - W))
    return out / (prob["dx"] * prob["dx"])


def kappa_grad_stage(W, lam, c, prob):
    """Contribution of one stage W -> W + c f(W) to dJ/dkappa (fixed-field kappa).

    For the face f between cells i and j, d(f(W))/d kappa_f is (W_j - W_i)/dx^2 at i and
    (W_i - W_j)/dx^2 at j; with the real inner product <x, y> = Re(x^H y) the face receives
    Re(c [conj(lam_i)(W_j - W_i) + conj(lam_j)(W_i - W_j)]) / dx^2 (lam, W = 0 in ghosts),
    and kappa_f = (kappa_i + kappa_j)/2 passes half of it to each cell; a Dirichlet
    boundary face depends on its interior cell alone (ghost kappa = interior kappa) and
    passes all of it.
    """
    W = np.asarray(W, dtype=np.complex128)
    lam = np.asarray(lam, dtype=np.complex128)
    zero = np.zeros_like(W)
    g = np.zeros(W.shape)
    h2 = prob["dx"] * prob["dx"]
    for ax in range(W.ndim):
        n = W.shape[ax]
        Wp, _ = _neighbours(W, ax, prob["bc"], zero)
        lp, _ = _neighbours(lam, ax, prob["bc"], zero)
        # face between i and i+1 along ax, indexed by i
        face = np.real(c * (np.conj(lam) * (Wp - W) + np.conj(lp) * (W - Wp))) / h2
        if prob["bc"] == "periodic":
            g = g + 0.5 * face + 0.5 * np.roll(face, 1, axis=ax)
        else:
            inner = np.take(face, range(0, n - 1), axis=ax)
            last = np.take(face, [n - 1], axis=ax)  # boundary face on the high side
            lo = np.concatenate([np.zeros_like(last), 0.5 * inner], axis=ax)
            hi = np.concatenate([0.5 * inner, np.zeros_like(last)], axis=ax)
            g = g + lo + hi
            g = g + np.concatenate([np.zeros_like(inner), last], axis=ax)
            # boundary face on the low side: ghost (index -1) and cell 0
            face_lo = np.real(c * (np.conj(np.take(lam, [0], axis=ax))
                                   * (0.0 - np.take(W, [0], axis=ax)))) / h2
            g = g + np.concatenate([face_lo, np.zeros_like(inner)], axis=ax)
    return g


def frkc2_adjoint(u0, a, T, prob, nsteps, dJdu):
    """Gradients of a scalar J(u(T_end)) for ``nsteps`` FRKC2 steps from u0.

    Forward: the stage states of every step are kept (a plain tape).  Backward: with the
    real projection w^{n+1} = Re W^L the step's adjoint starts from lam^L = dJ/dw^{n+1}
    (imaginary part 0); each stage W^{l+1} = W^l + c_l f(W^l), c_l = T a_l, is reversed as
    lam^l = lam^{l+1} + conj(c_l) J_f(W^l)^H lam^{l+1}; dJ/dw^n = Re lam^0 (W^0 = w^n is
    real).  Returns (dJ/du0, dJ/dkappa) -- the second is None unless kappa is a field.
    """
    tape = []
    u = np.array(u0, dtype=np.float64)
    for _ in range(nsteps):
        W = u.astype(np.complex128)
        states = []
        for al in a:
            states.append(W)
            W = W + (T * al) * apply_f(W, prob)
        tape.append(states)
        u = W.real.copy()
    lam_u = np.array(dJdu, dtype=np.float64)
    gk = np.zeros(np.shape(u0)) if prob["kappa"] == "field" else None
    for n in reversed(range(nsteps)):
        lam = lam_u.astype(np.complex128)
        for l in reversed(range(len(a))):
            c = T * a[l]
            Wl = tape[n][l]
            if gk is not None:
                gk = gk + kappa_grad_stage(Wl, lam, c, prob)
            lam = lam + np.conj(c) * apply_jh(Wl, lam, prob)
        lam_u = lam.real.copy()
    return lam_u, gk


# ----------------------------------------------------------------------------------------
# Fine-step reference
# ----------------------------------------------------------------------------------------


def rk4(u0, h, prob, nsteps):
    """Classical fourth-order Runge-Kutta for w' = f(w) with real state, step h."""
    u = np.array(u0, dtype=np.float64)
    for _ in range(nsteps):
        k1 = apply_f(u, prob)
        k2 = apply_f(u + 0.5 * h * k1, prob)
        k3 = apply_f(u + 0.5 * h * k2, prob)
        k4 = apply_f(u + h * k3, prob)
        u = u + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return np.real(u)


# ----------------------------------------------------------------------------------------
# Embedded first-order solution and step-size control (Sec. 3, Eqs. 14-16)
# ----------------------------------------------------------------------------------------


def frkc2_step_embedded(u0, a, T, prob):
    """One FRKC2 step and its embedded first-order solution (Eq. 14).

    W^{l+1} = W^l + T a_l f(W^l) as in ``frkc2_step``; alongside, What^0 = W^0 and
    What^{l+1} = What^l + T Re(a_l) Re(f(W^l)).  Returns (Re W^L, What^L).
    """
    W = np.array(u0, dtype=np.float64).astype(np.complex128)
    H = np.array(u0, dtype=np.float64)
    for al in a:
        fw = apply_f(W, prob)
        H = H + T * al.real * fw.real
        W = W + (T * al) * fw
    return W.real.copy(), H


def error_norm(w, what, tol: float) -> float:
    """Scaled error of Eq. 15, ||e|| with e_i = |w_i - what_i| / (TOL (1 + max(|w_i|, |what_i|))).

    Reading: the norm is the root mean square over the cells (the convention of the error
    controllers the paper refers to), and w is the step's output Re W^L.
    """
    e = np.abs(w - what) / (tol * (1.0 + np.maximum(np.abs(w), np.abs(what))))
    return float(np.sqrt(np.mean(e * e)))


def frkc2_adaptive(u0, a, beta_, prob, t_end: float, tol: float, dt0: float, rho: float = 0.0,
                   safe: float = 0.8, max_steps: int = 100000):
    """Integrate to ``t_end`` with the error control of Sec. 3.

    A step with ||err|| > 1 is rejected and retried with T scaled by SAFE / sqrt(||err||).
    After an accepted step the next T comes from the predictive controller (Eq. 16), read as
    T^{n+1} = T^n (SAFE / sqrt(e_n)) (T^n / T^{n-1}) sqrt(e_{n-1} / e_n) (the printed formula
    lacks the leading T^n), and from T^n SAFE / sqrt(e_n) for the first step.  Readings: T is
    also capped by the stability limit beta/rho (when rho > 0), by the time left, and may grow
    by at most 5x per step; e is floored at 1e-10.
    Returns (u, dict(accepted, rejected, t, dts, trace)); ``trace`` lists every attempt as
    (T, ||err||, accepted).
    """
    u = np.array(u0, dtype=np.float64)
    t, T = 0.0, float(dt0)
    T_prev, e_prev = None, None
    acc = rej = 0
    dts = []
    trace = []
    while t < t_end * (1.0 - 1e-14) and acc + rej < max_steps:
        T = min(T, t_end - t)
        if rho > 0:
            T = min(T, beta_ / rho)
        w, h = frkc2_step_embedded(u, a, T, prob)
        e = error_norm(w, h, tol)
        if not np.isfinite(e) or e > 1.0:
            rej += 1
            trace.append((T, e, False))
            T = T * safe / np.sqrt(e if np.isfinite(e) else 1e10)
            continue
        acc += 1
        trace.append((T, e, True))
        u = w
        t += T
        dts.append(T)
        e = max(e, 1e-10)
        fac = safe / np.sqrt(e)
        if T_prev is not None:
            fac *= (T / T_prev) * np.sqrt(e_prev / e)
        T_prev, e_prev = T, e
        T = T * min(fac, 5.0)
    return u, dict(accepted=acc, rejected=rej, t=t, dts=dts, trace=trace)
