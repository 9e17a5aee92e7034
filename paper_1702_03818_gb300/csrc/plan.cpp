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

// Lebedev-Finogenov recursive permutation of 0..m-1: P(1) = (0); P(2q) interleaves each v of
// P(q) with 2q-1-v; P(2q+1) = P(2q) followed by 2q.
std::vector<int> lebedev_permutation(int m) {
  if (m == 1) return {0};
  std::vector<int> out;
  if (m % 2 == 0) {
    for (int v : lebedev_permutation(m / 2)) {
      out.push_back(v);
      out.push_back(m - 1 - v);
    }
    return out;
  }
  out = lebedev_permutation(m - 1);
  out.push_back(m - 1);
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

frkc2_status frkc2_plan(int s, double nu, unsigned flags, frkc2_plan_t* out) {
  if (!out || s < 2 || s > 4096 || (s & 1)) return FRKC2_EINVAL;
  if (!(nu >= 0.0 && nu < 0.9)) return FRKC2_EINVAL;
  *out = nullptr;
  const int L = s;
  const std::vector<cplx> a = nu > 0.0 ? damped_steps(L, nu) : root_order_steps(L);
  const double beta = nu > 0.0 ? stability_extent(a, (1.0 - 0.5 * nu) * poly_beta(L)) : poly_beta(L);
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
  if (paired) consider(order_paired(L), 0);
  bool run_greedy = !paired && (force_greedy || (!force_lebedev && L <= 256));
  if (!paired && (force_lebedev || (!force_greedy && L > 256))) {
    const double q = consider(order_lebedev(L), 0);
    if (!force_lebedev && q > bound) run_greedy = true;
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
  if (!out || !a_re || !a_im || s < 2 || s > 4096 || (s & 1)) return FRKC2_EINVAL;
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
