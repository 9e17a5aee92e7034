// Host-side FRKC2 plan: step sizes from the stability polynomial (Sec. 2, Eqs. 7-8) and
// the internal-stability ordering with its realised amplification (Sec. 2.2, Eqs. 10-12).
// Everything here is FP64 and runs once per stage count; the kernels only see the ordered
// step sizes.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <limits>
#include <new>
#include <thread>
#include <vector>

#include "frkc2.h"
#include "frkc2_internal.h"

using cplx = std::complex<double>;

namespace {

// alpha_M for degree L = 2M: R''(0) = 1 with R(z) = 1 - a/4 + (a/4) T_L(1 + 4z/(L^2 a)).
double poly_alpha(int L) { return 4.0 * (1.0 - 1.0 / (double(L) * double(L))) / 3.0; }
double poly_beta(int L) { return 0.5 * double(L) * double(L) * poly_alpha(L); }

// a_j = 1/(M^2 alpha (1 - zeta_j)), zeta_j = cos((pi(2j+1) - i eta)/L), T_L(zeta_j) = 1 - 4/alpha.
// The second member of each conjugate pair is the exact conjugate of the first.
std::vector<cplx> root_order_steps(int L) {
  const double al = poly_alpha(L);
  const double eta = std::acosh(4.0 / al - 1.0);
  const double M = 0.5 * L;
  std::vector<cplx> a(L);
  for (int j = 0; j < L / 2; ++j) {
    const double th = M_PI * double(2 * j + 1) / double(L);
    const double y = eta / double(L);
    // cos(th - i y) = cos th cosh y + i sin th sinh y
    const cplx zeta(std::cos(th) * std::cosh(y), std::sin(th) * std::sinh(y));
    a[j] = 1.0 / (M * M * al * (1.0 - zeta));
    a[L - 1 - j] = std::conj(a[j]);
  }
  return a;
}

// Damped step sizes of Sec. 2.1: a_l = (1 - mu_l) / ((1 - nu) M^2 alpha (1 - (1 - 2 mu_l) zeta_l)),
// nu = nu0 / 2.  mu_l = mu for even root index j (T_M(zeta_j) = +i c), conj(mu) for odd j, so the
// step sizes stay in conjugate pairs; Newton-Raphson over (Re mu, Im mu) from mu = 0 enforces
// e1 = sum a = 1 and e2 = sum_{i<j} a_i a_j = (e1^2 - sum a^2) / 2 = 1/2.
std::vector<cplx> damped_steps(int L, double nu0) {
  const double nu = 0.5 * nu0, al = poly_alpha(L), eta = std::acosh(4.0 / al - 1.0), M = 0.5 * L;
  std::vector<cplx> z(L);
  for (int j = 0; j < L / 2; ++j) {
    const double th = M_PI * double(2 * j + 1) / double(L), y = eta / double(L);
    z[j] = cplx(std::cos(th) * std::cosh(y), std::sin(th) * std::sinh(y));
    z[L - 1 - j] = std::conj(z[j]);
  }
  auto steps = [&](cplx mu) {
    std::vector<cplx> a(L);
    for (int j = 0; j < L; ++j) {
      const cplx m = (j % 2 == 0) ? mu : std::conj(mu);
      a[j] = (1.0 - m) / ((1.0 - nu) * M * M * al * (1.0 - (1.0 - 2.0 * m) * z[j]));
    }
    return a;
  };
  auto resid = [&](cplx mu, double r[2]) {
    const std::vector<cplx> a = steps(mu);
    cplx e1 = 0.0, p2 = 0.0;
    for (const cplx& v : a) {
      e1 += v;
      p2 += v * v;
    }
    const cplx e2 = 0.5 * (e1 * e1 - p2);
    r[0] = (e1 - 1.0).real();
    r[1] = (e2 - 0.5).real();
  };
  cplx mu = 0.0;
  for (int it = 0; it < 60; ++it) {
    double r[2], rx[2], ry[2];
    resid(mu, r);
    if (std::max(std::abs(r[0]), std::abs(r[1])) < 1e-14) break;
    const double h = 1e-7;
    resid(mu + cplx(h, 0.0), rx);
    resid(mu + cplx(0.0, h), ry);
    const double J00 = (rx[0] - r[0]) / h, J01 = (ry[0] - r[0]) / h;
    const double J10 = (rx[1] - r[1]) / h, J11 = (ry[1] - r[1]) / h;
    const double det = J00 * J11 - J01 * J10;
    if (det == 0.0 || !std::isfinite(det)) break;
    mu += cplx((-r[0] * J11 + r[1] * J01) / det, (-J00 * r[1] + J10 * r[0]) / det);
  }
  std::vector<cplx> a = steps(mu);
  for (int j = 0; j < L / 2; ++j) a[L - 1 - j] = std::conj(a[j]);
  return a;
}

// ---- Rank-N polynomial (Eq. 7 with N = 4): B(z) = d_0 + 2 sum_{k=1}^N d_k T_{kM}(x),
// x = 1 + z/(M^2 alpha), L = N M.  With T_{kM} = T_k(T_M), B(z) = Q(T_M(x)) for the degree-N
// Chebyshev series Q(y) = d_0 + 2 sum d_k T_k(y).

// n-th derivative of T_j at 1: prod_{m<n} (j^2 - m^2)/(2m+1).
double cheb_deriv_at_one(int j, int n) {
  double p = 1.0;
  for (int m = 0; m < n; ++m) p *= (double(j) * j - double(m) * m) / (2.0 * m + 1.0);
  return p;
}

constexpr int RANK_MAX = 4;

// d_0..d_N from the linear order conditions R(0) = 1, R^(n)(0) = 1 (Eq. 5), by Gaussian
// elimination with partial pivoting.  Returns false on a singular system.
bool chebsum_d(int N, int M, double al, double* d) {
  double A[RANK_MAX + 1][RANK_MAX + 2];
  for (int n = 0; n <= N; ++n) {
    for (int k = 0; k <= N; ++k) {
      if (n == 0)
        A[n][k] = k == 0 ? 1.0 : 2.0;
      else
        A[n][k] = k == 0 ? 0.0 : 2.0 * cheb_deriv_at_one(k * M, n) / std::pow(double(M) * M * al, n);
    }
    A[n][N + 1] = 1.0;
  }
  for (int c = 0; c <= N; ++c) {
    int piv = c;
    for (int r = c + 1; r <= N; ++r)
      if (std::abs(A[r][c]) > std::abs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k <= N + 1; ++k) std::swap(A[c][k], A[piv][k]);
    for (int r = 0; r <= N; ++r) {
      if (r == c) continue;
      const double f = A[r][c] / A[c][c];
      for (int k = c; k <= N + 1; ++k) A[r][k] -= f * A[c][k];
    }
  }
  for (int k = 0; k <= N; ++k) d[k] = A[k][N + 1] / A[k][k];
  return true;
}

// Monomial coefficients q[0..N] of Q(y), from T_0 = 1, T_1 = y, T_{k+1} = 2y T_k - T_{k-1}.
void chebsum_monomial(int N, const double* d, double* q) {
  double T[RANK_MAX + 1][RANK_MAX + 1] = {};
  T[0][0] = 1.0;
  if (N >= 1) T[1][1] = 1.0;
  for (int k = 1; k < N; ++k)
    for (int i = 0; i <= N; ++i) T[k + 1][i] = (i > 0 ? 2.0 * T[k][i - 1] : 0.0) - T[k - 1][i];
  for (int i = 0; i <= N; ++i) {
    q[i] = d[0] * T[0][i];
    for (int k = 1; k <= N; ++k) q[i] += 2.0 * d[k] * T[k][i];
  }
}

// All complex roots of sum_{i<=n} c[i] y^i (c[n] != 0, n <= RANK_MAX) by the Aberth-Ehrlich
// simultaneous iteration from points on a circle, then Newton steps on each root.
std::vector<cplx> poly_roots(int n, const double* c) {
  auto P = [&](cplx y, cplx* dp) {
    cplx p = c[n], q = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      q = q * y + p;
      p = p * y + c[i];
    }
    *dp = q;
    return p;
  };
  double rad = 0.0;
  for (int i = 0; i < n; ++i) rad = std::max(rad, std::pow(std::abs(c[i] / c[n]), 1.0 / (n - i)));
  rad = std::max(rad, 1e-3);
  std::vector<cplx> z(n);
  for (int i = 0; i < n; ++i) z[i] = std::polar(rad, 2.0 * M_PI * (i + 0.25) / n);
  for (int it = 0; it < 500; ++it) {
    double moved = 0.0;
    for (int i = 0; i < n; ++i) {
      cplx dp;
      const cplx p = P(z[i], &dp);
      if (p == 0.0) continue;
      const cplx ratio = p / dp;
      cplx s = 0.0;
      for (int j = 0; j < n; ++j)
        if (j != i) s += 1.0 / (z[i] - z[j]);
      const cplx w = ratio / (1.0 - ratio * s);
      z[i] -= w;
      moved = std::max(moved, std::abs(w) / std::max(1.0, std::abs(z[i])));
    }
    if (moved < 1e-15) break;  // converged to rounding; Newton steps polish below
  }
  for (cplx& y : z)
    for (int it = 0; it < 3; ++it) {
      cplx dp;
      const cplx p = P(y, &dp);
      if (dp == 0.0) break;
      y -= p / dp;
    }
  return z;
}

// max |Q(y)| on [-1, 1] from y = -1 and the real critical points inside (Q(1) = R(0) = 1 with
// Q'(1) = alpha > 0, so y = 1 is left out).
double chebsum_max_abs_Q(int N, const double* d) {
  double q[RANK_MAX + 1], dq[RANK_MAX];
  chebsum_monomial(N, d, q);
  for (int i = 1; i <= N; ++i) dq[i - 1] = double(i) * q[i];
  auto Qv = [&](double y) {
    double p = q[N];
    for (int i = N - 1; i >= 0; --i) p = p * y + q[i];
    return p;
  };
  double m = std::abs(Qv(-1.0));
  for (const cplx& r : poly_roots(N - 1, dq))
    if (std::abs(r.imag()) <= 1e-12 * std::max(1.0, std::abs(r.real())) && r.real() > -1.0 &&
        r.real() < 1.0)
      m = std::max(m, std::abs(Qv(r.real())));
  return m;
}

// alpha_M: the largest alpha with |Q| <= 1 on [-1, 1] (Eq. 6), by bisection; the feasible
// alphas form an interval from 0.  N = 2 gives 4(1 - 1/L^2)/3 (d_1 = 0).
double chebsum_alpha(int N, int M) {
  double lo = 0.25, hi = 4.0, d[RANK_MAX + 1];
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (chebsum_d(N, M, mid, d) && chebsum_max_abs_Q(N, d) <= 1.0)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Step sizes a_l = 1/(M^2 alpha (1 - zeta_l)) of the rank-N polynomial in root order: the
// roots of T_M(x) = y_i for the N roots y_i of Q are x = cos((arccos y_i + 2 pi k)/M),
// k = 0..M-1; those with Im x > 0 sorted by decreasing Re x are zeta_0..zeta_{L/2-1} and
// zeta_{L-1-j} = conj(zeta_j).  Returns an empty vector if the roots are not in conjugate
// pairs off the real axis.
std::vector<cplx> chebsum_steps(int N, int M, double* beta_out) {
  const int L = N * M;
  const double al = chebsum_alpha(N, M);
  double d[RANK_MAX + 1], q[RANK_MAX + 1];
  if (!chebsum_d(N, M, al, d)) return {};
  chebsum_monomial(N, d, q);
  std::vector<cplx> upper;
  for (const cplx& y : poly_roots(N, q)) {
    const cplx th = std::acos(y);
    for (int k = 0; k < M; ++k) {
      const cplx x = std::cos((th + 2.0 * M_PI * double(k)) / double(M));
      if (x.imag() > 0.0) upper.push_back(x);
    }
  }
  if (int(upper.size()) != L / 2) return {};
  std::stable_sort(upper.begin(), upper.end(),
                   [](const cplx& u, const cplx& v) { return u.real() > v.real(); });
  std::vector<cplx> a(L);
  for (int j = 0; j < L / 2; ++j) {
    a[j] = 1.0 / (double(M) * M * al * (1.0 - upper[j]));
    a[L - 1 - j] = std::conj(a[j]);
  }
  *beta_out = 2.0 * double(M) * M * al;
  return a;
}

// Largest x with |R(-x)| <= 1 near `guess` (bisection on the last crossing of |R| = 1).
double stability_extent(const std::vector<cplx>& a, double guess) {
  auto absR = [&](double x) {
    cplx p = 1.0;
    for (const cplx& v : a) p *= (1.0 - v * x);
    return std::abs(p);
  };
  double lo = 0.9 * guess, hi = 1.1 * guess;
  while (absR(lo) > 1.0) lo *= 0.99;
  while (absR(hi) <= 1.0) hi *= 1.01;
  for (int i = 0; i < 200 && hi - lo > 1e-15 * hi; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (absR(mid) <= 1.0)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Runs fn(lo, hi) over [0, n) on up to hardware_concurrency threads.
template <class F>
void parallel_ranges(int n, F fn) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = int(std::max(1u, std::min(hw, 16u)));
  nt = std::min(nt, std::max(1, n / 8));
  if (nt <= 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t) {
    int lo = int((long long)n * t / nt), hi = int((long long)n * (t + 1) / nt);
    th.emplace_back([=, &fn] { fn(lo, hi); });
  }
  for (auto& x : th) x.join();
}

// log|1 + a_j x_k| for all j (rows) and k (columns).
std::vector<double> log_factors(const std::vector<cplx>& a, const std::vector<double>& x) {
  const int L = int(a.size()), S = int(x.size());
  std::vector<double> lv(size_t(L) * S);
  parallel_ranges(L, [&](int lo, int hi) {
    for (int j = lo; j < hi; ++j)
      for (int k = 0; k < S; ++k) lv[size_t(j) * S + k] = std::log(std::abs(1.0 + a[j] * x[k]));
  });
  return lv;
}

// Greedy ordering of Eq. 12 (reading: items are the L step sizes; samples
// x_k = -beta_bar k/S; at each position the candidate minimising
// sum_k max(P_k v_jk, Rest_k / v_jk) is placed; log-sum-exp; lowest index on ties).
std::vector<int> order_greedy(const std::vector<cplx>& a, double beta, int n, int S,
                              double C = 1e-4) {
  const int L = int(a.size());
  const double bbar = (1.0 - n * C) * beta;
  std::vector<double> x(S);
  for (int k = 0; k < S; ++k) x[k] = -bbar * double(k + 1) / double(S);
  const std::vector<double> lv = log_factors(a, x);
  std::vector<int> remaining(L);
  for (int j = 0; j < L; ++j) remaining[j] = j;
  std::vector<int> placed;
  placed.reserve(L);
  std::vector<double> logP(S, 0.0), logRest(S), cost(L);
  for (int l = 0; l < L; ++l) {
    const int m = int(remaining.size());
    std::fill(logRest.begin(), logRest.end(), 0.0);
    for (int r = 0; r < m; ++r) {
      const double* row = &lv[size_t(remaining[r]) * S];
      for (int k = 0; k < S; ++k) logRest[k] += row[k];
    }
    parallel_ranges(m, [&](int lo, int hi) {
      std::vector<double> e(S);
      for (int r = lo; r < hi; ++r) {
        const double* row = &lv[size_t(remaining[r]) * S];
        double mx = -std::numeric_limits<double>::infinity();
        for (int k = 0; k < S; ++k) {
          e[k] = std::max(logP[k] + row[k], logRest[k] - row[k]);
          mx = std::max(mx, e[k]);
        }
        double acc = 0.0;
        for (int k = 0; k < S; ++k) acc += std::exp(e[k] - mx);
        cost[r] = mx + std::log(acc);
      }
    });
    int best = 0;
    for (int r = 1; r < m; ++r)
      if (cost[r] < cost[best]) best = r;
    const int j = remaining[best];
    remaining.erase(remaining.begin() + best);
    placed.push_back(j);
    const double* row = &lv[size_t(j) * S];
    for (int k = 0; k < S; ++k) logP[k] += row[k];
  }
  return placed;
}

// Realised Q (Eqs. 10-11): max over x_i = -beta i/P (i = 0..P) and over contiguous runs
// j..k of prod |1 + a_l x|.  For each x the best run ending at k is the prefix sum of logs
// up to k minus the smallest prefix sum before j, so one sweep per x suffices.
double realised_Q(const std::vector<cplx>& a, double beta, int P) {
  const int L = int(a.size());
  std::vector<double> best(P + 1, -std::numeric_limits<double>::infinity());
  parallel_ranges(P + 1, [&](int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      const double x = -beta * double(i) / double(P);
      double s = 0.0, mn = 0.0, b = -std::numeric_limits<double>::infinity();
      for (int l = 0; l < L; ++l) {
        s += std::log(std::abs(1.0 + a[l] * x));
        b = std::max(b, s - mn);
        mn = std::min(mn, s);
      }
      best[i] = b;
    }
  });
  return std::exp(*std::max_element(best.begin(), best.end()));
}

// Rounding gain g = sqrt(sum_l mean_x |prod_{j>l} (1 + a_j x)|^2) over P = max(2048, 4L)
// midpoints x_i = -beta (i + 1/2)/P.  A rounding error of stage l reaches the step's output
// through the factors of the later stages (the partial products of Sec. 2.2), so with the
// rounding spread evenly over the spectrum one step's relative error is about
// (unit roundoff) x g.  Per x the suffix products are built from the last stage backwards.
double rounding_gain(const std::vector<cplx>& a, double beta) {
  const int L = int(a.size()), P = std::max(2048, 4 * L);
  std::vector<double> part(P, 0.0);
  parallel_ranges(P, [&](int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      const double x = -beta * (double(i) + 0.5) / double(P);
      cplx suf = 1.0;
      double acc = 0.0;
      for (int l = L - 1; l >= 0; --l) {
        acc += std::norm(suf);  // |prod_{j>l} (1 + a_j x)|^2
        suf *= 1.0 + a[l] * x;
      }
      part[i] = acc;
    }
  });
  double total = 0.0;
  for (double v : part) total += v;
  return std::sqrt(total / double(P));
}

// Lebedev-Finogenov recursive permutation of 0..m-1: P(1) = (0); P(m) interleaves each v of
// P(m/2) (integer division) with its mirror m-1-v, and for odd m ends with the middle index m/2,
// so every root stays paired with its mirror (for m a power of two the classical recursion).
std::vector<int> lebedev_permutation(int m) {
  if (m == 1) return {0};
  std::vector<int> out;
  for (int v : lebedev_permutation(m / 2)) {
    out.push_back(v);
    out.push_back(m - 1 - v);
  }
  if (m % 2) out.push_back(m / 2);
  return out;
}

// The upper-half roots (j < L/2) in Lebedev-Finogenov order, then their conjugates L-1-j in
// the same order.
std::vector<int> order_lebedev(int L) {
  std::vector<int> h = lebedev_permutation(L / 2), out(h);
  for (int v : h) out.push_back(L - 1 - v);
  return out;
}

// Each conjugate pair adjacent: for j of the upper half in Lebedev-Finogenov order, the
// stages j then L-1-j.
std::vector<int> order_paired(int L) {
  std::vector<int> out;
  for (int v : lebedev_permutation(L / 2)) {
    out.push_back(v);
    out.push_back(L - 1 - v);
  }
  return out;
}

}  // namespace

extern "C" {

// Largest stage count of a plan, and of a plan that may run the greedy ordering (its table of
// log-factors holds 16 s^2 doubles: 2 GB at s = 4096).
constexpr int S_MAX = 16384, S_GREEDY_MAX = 4096;

frkc2_status frkc2_plan(int s, double nu, unsigned flags, frkc2_plan_t* out) {
  if (!out || s < 2 || s > S_MAX || (s & 1)) return FRKC2_EINVAL;
  if (!(nu >= 0.0 && nu < 0.9)) return FRKC2_EINVAL;
  *out = nullptr;
  const int L = s;
  const bool order4 = flags & FRKC2_PLAN_ORDER4;
  if (order4 && (L % 4)) return FRKC2_EINVAL;
  if (order4 && nu > 0.0) return FRKC2_EUNSUPPORTED;
  double beta = 0.0;
  std::vector<cplx> a;
  if (order4) {
    a = chebsum_steps(4, L / 4, &beta);
    if (a.empty()) return FRKC2_EPLAN;
  } else {
    a = nu > 0.0 ? damped_steps(L, nu) : root_order_steps(L);
    beta = nu > 0.0 ? stability_extent(a, (1.0 - 0.5 * nu) * poly_beta(L)) : poly_beta(L);
  }
  const int S = 16 * L, P = 16 * L, n_max = 10;
  const double bound = 10.0 * double(L) * double(L);
  std::vector<int> best_order;
  double best_Q = std::numeric_limits<double>::infinity();
  int best_n = 0;
  auto consider = [&](const std::vector<int>& ord, int n) {
    std::vector<cplx> ao(L);
    for (int l = 0; l < L; ++l) ao[l] = a[ord[l]];
    const double Q = realised_Q(ao, beta, P);
    if (Q < best_Q) {
      best_Q = Q;
      best_order = ord;
      best_n = n;
    }
    return Q;
  };
  const bool force_greedy = flags & FRKC2_PLAN_GREEDY, force_lebedev = flags & FRKC2_PLAN_LEBEDEV;
  const bool paired = flags & FRKC2_PLAN_PAIRED;
  if (int(force_greedy) + int(force_lebedev) + int(paired) > 1) return FRKC2_EINVAL;
  if (force_greedy && L > S_GREEDY_MAX) return FRKC2_EINVAL;
  if (paired) consider(order_paired(L), 0);
  // rank-4 plans take the Lebedev-Finogenov order first at every s: on those roots its
  // realised Q is about 0.1 s^2 where the greedy reaches a few s^2
  bool run_greedy = !paired && (force_greedy || (!force_lebedev && L <= 256 && !order4));
  if (!paired && (force_lebedev || (!force_greedy && (L > 256 || order4)))) {
    const double q = consider(order_lebedev(L), 0);
    if (!force_lebedev && q > bound && L <= S_GREEDY_MAX) run_greedy = true;
  }
  if (run_greedy) {
    for (int n = 1; n <= n_max; ++n)
      if (consider(order_greedy(a, beta, n, S), n) <= bound) break;
  }
  if ((flags & FRKC2_PLAN_STRICT) && best_Q > bound) return FRKC2_EPLAN;
  frkc2_plan_s* p = new (std::nothrow) frkc2_plan_s;
  if (!p) return FRKC2_EINVAL;
  p->s = L;
  p->beta = beta;
  p->Q = best_Q;
  p->n_iter = best_n;
  p->order = best_order;
  p->paired = paired;
  p->a_re.resize(L);
  p->a_im.resize(L);
  std::vector<cplx> ao(L);
  for (int l = 0; l < L; ++l) {
    p->a_re[l] = a[best_order[l]].real();
    p->a_im[l] = a[best_order[l]].imag();
    ao[l] = a[best_order[l]];
  }
  p->gain = rounding_gain(ao, beta);
  *out = p;
  return FRKC2_OK;
}

frkc2_status frkc2_plan_from_steps(int s, const double* a_re, const double* a_im,
                                   frkc2_plan_t* out) {
  if (!out || !a_re || !a_im || s < 2 || s > S_MAX || (s & 1)) return FRKC2_EINVAL;
  *out = nullptr;
  frkc2_plan_s* p = new (std::nothrow) frkc2_plan_s;
  if (!p) return FRKC2_EINVAL;
  p->s = s;
  p->beta = poly_beta(s);
  p->n_iter = 0;
  p->a_re.assign(a_re, a_re + s);
  p->a_im.assign(a_im, a_im + s);
  p->order.assign(s, -1);
  std::vector<cplx> ao(s);
  for (int l = 0; l < s; ++l) ao[l] = cplx(a_re[l], a_im[l]);
  p->Q = realised_Q(ao, p->beta, 16 * s);
  p->gain = rounding_gain(ao, p->beta);
  *out = p;
  return FRKC2_OK;
}

frkc2_status frkc2_plan_info(frkc2_plan_t plan, int* s, double* beta, double* Q, int* n_iter,
                             double* a_re, double* a_im, int* order) {
  if (!plan) return FRKC2_EINVAL;
  if (s) *s = plan->s;
  if (beta) *beta = plan->beta;
  if (Q) *Q = plan->Q;
  if (n_iter) *n_iter = plan->n_iter;
  if (a_re) std::memcpy(a_re, plan->a_re.data(), sizeof(double) * plan->s);
  if (a_im) std::memcpy(a_im, plan->a_im.data(), sizeof(double) * plan->s);
  if (order) std::memcpy(order, plan->order.data(), sizeof(int) * plan->s);
  return FRKC2_OK;
}

frkc2_status frkc2_plan_rounding_gain(frkc2_plan_t plan, double* gain) {
  if (!plan || !gain) return FRKC2_EINVAL;
  *gain = plan->gain;
  return FRKC2_OK;
}

void frkc2_plan_destroy(frkc2_plan_t plan) { delete plan; }

const char* frkc2_status_string(frkc2_status st) {
  switch (st) {
    case FRKC2_OK: return "ok";
    case FRKC2_EINVAL: return "invalid argument";
    case FRKC2_EUNSTABLE: return "dt * rho exceeds the stability extent beta";
    case FRKC2_EPLAN: return "plan: realised internal amplification above 10 L^2";
    case FRKC2_ENOMEM: return "workspace too small";
    case FRKC2_ECUDA: return "CUDA runtime error";
    case FRKC2_ETIMEOUT: return "bounded device wait expired";
    case FRKC2_ENONFINITE: return "non-finite value in a step's output";
    case FRKC2_EUNSUPPORTED: return "not supported by this build";
    case FRKC2_EBOUNDS: return "bounds-checking build: a device index fell outside its array";
  }
  return "unknown status";
}

}  // extern "C"
