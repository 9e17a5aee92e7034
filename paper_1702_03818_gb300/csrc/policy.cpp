// Precision policy: the cheapest state precision whose predicted rounding error meets a
// tolerance, from the rounding gain of the plan's stage order (Sec. 2.2: the partial products
// of the later stages amplify what an earlier stage rounds).
//
// Model (relative L2 after n steps of s stages): e(n) = C u (g sqrt(n) + c s n), u the unit
// roundoff, g the plan's rounding gain.  The first term is the rounding each stage makes,
// amplified by the later stages' factors, adding over steps like a random walk (the undamped
// polynomial keeps |R| close to 1 on much of [-beta, 0], so rounding in those modes is not
// damped).  The second is coherent: each stage adds an increment that is small against the
// state of smooth data, and those s n roundings of the state do not cancel.  Calibration on
// GB300 (2048^2 recipe, FP32 against FP64, greedy and Lebedev-Finogenov orders,
// s = 16..256, 1, 10 and 100 steps): with C = 1.5 and c = 4e-3 every measured error is at
// most 0.9 of the model (the Lebedev order at s = 256 over 100 steps is where the coherent
// term matters: 5.7e-6 measured, 1.2e-5 predicted).  DFLOAT and MIXED keep a double-class
// state and round only the flux arithmetic to float, which measured 1.1e-3..2.3e-2 of the
// FP32 error (smooth 2D fields; the 3D hot spot of kappa(u) is the 2.3e-2); the policy takes
// 5e-2 of the FP32 model.
#include <cmath>

#include "frkc2.h"
#include "frkc2_internal.h"

namespace {

constexpr double kC = 1.5;
constexpr double kCoherent = 4e-3;
constexpr double kU32 = 5.9604644775390625e-08;  // 2^-24
constexpr double kU64 = 1.1102230246251565e-16;  // 2^-53
constexpr double kPairFactor = 5e-2;

bool shape_ok(const frkc2_problem* p) {
  return p && p->ndim >= 1 && p->ndim <= 3 && p->kappa_kind >= FRKC2_KAPPA_CONST &&
         p->kappa_kind <= FRKC2_KAPPA_POWER;
}

}  // namespace

extern "C" {

frkc2_status frkc2_precision_policy(frkc2_plan_t plan, const frkc2_problem* prob, int nsteps,
                                    double tol, int* precision, double* predicted) {
  if (!plan || !shape_ok(prob) || nsteps < 1 || !(tol > 0.0) || !precision) return FRKC2_EINVAL;
  const double n = double(nsteps);
  const double amp = plan->gain * std::sqrt(n) + kCoherent * double(plan->s) * n;
  const double e32 = kC * kU32 * amp;
  const double epair = kPairFactor * e32;
  const double e64 = kC * kU64 * amp;
  const bool dfloat_ok = prob->ndim == 2 && prob->kappa_kind != FRKC2_KAPPA_POWER;
  int prec;
  double e;
  if (e32 <= tol) {
    prec = FRKC2_FP32;
    e = e32;
  } else if (epair <= tol) {
    // 2D fixed conductivity: the float-pair state runs on the FP32 pipe; elsewhere MIXED
    prec = dfloat_ok ? FRKC2_DFLOAT : FRKC2_MIXED;
    e = epair;
  } else {
    prec = FRKC2_FP64;
    e = e64;
  }
  *precision = prec;
  if (predicted) *predicted = e;
  return FRKC2_OK;
}

frkc2_status frkc2_plan_auto(int s, const frkc2_problem* prob, int nsteps, double tol,
                             frkc2_plan_t* plan, int* precision, double* predicted) {
  if (!plan || !shape_ok(prob) || nsteps < 1 || !(tol > 0.0) || !precision) return FRKC2_EINVAL;
  *plan = nullptr;
  // a linear f takes the order of least rounding gain; kappa(u) keeps the default order,
  // whose stage states stay closer to the real axis
  const unsigned flags = prob->kappa_kind == FRKC2_KAPPA_POWER ? 0u : unsigned(FRKC2_PLAN_LEBEDEV);
  frkc2_plan_t p = nullptr;
  frkc2_status st = frkc2_plan(s, 0.0, flags, &p);
  if (st != FRKC2_OK) return st;
  st = frkc2_precision_policy(p, prob, nsteps, tol, precision, predicted);
  if (st != FRKC2_OK) {
    frkc2_plan_destroy(p);
    return st;
  }
  *plan = p;
  return FRKC2_OK;
}

}  // extern "C"
