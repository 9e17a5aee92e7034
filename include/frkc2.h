/*
 * frkc2.h -- C ABI of the GB300 FRKC2 stage loop.
 *
 * The method is O'Sullivan's second-order Factorized Runge-Kutta-Chebyshev scheme
 * (arXiv:1702.03818).  Given a semi-discrete system w' = f(w) (Sec. 1, Eq. 1), a state w^n,
 * a step T and L = s stages with T |lambda|_max <= beta (Eq. 6), one step applies the
 * ordered complex forward-Euler stages W^{l+1} = W^l + T a_l f(W^l), W^0 = w^n, and returns
 * w^{n+1} = W^L (Sec. 3, Eq. 13).  Here f is the second-order flux-form diffusion operator
 * f(w)_c = (1/dx^2) sum_faces kappa_f (w_nb - w_c), kappa_f = (kappa_c + kappa_nb)/2, on a
 * 1D, 2D (5-point) or 3D (7-point) grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - No call allocates device memory.  Device buffers (states, conductivity, workspace)
 *   belong to the caller; the library only reads and writes them during the calls.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *   that launch work are asynchronous on that stream: a returned FRKC2_OK means the work
 *   was queued.  Argument and plan errors are reported synchronously and queue nothing.
 * - Device-detected conditions (a non-finite value in a step's output, a device wait
 *   that ran out of its iteration limit) are latched in a status word at the start of the
 *   workspace and read with frkc2_workspace_status().
 * - Arrays are dense, row-major with x fastest: index (z*ny + y)*nx + x.
 * - No C++ exception crosses this boundary.  Every call is thread-safe as long as two
 *   concurrent calls do not share a workspace; a plan is immutable after creation.
 */
#ifndef FRKC2_H
#define FRKC2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FRKC2_OK = 0,
  FRKC2_EINVAL = 1,       /* bad argument (size, pointer, enum value, alignment)            */
  FRKC2_EUNSTABLE = 2,    /* dt * rho > beta: the step leaves the stability interval (Eq. 6) */
  FRKC2_EPLAN = 3,        /* strict plan: realised Q above the bound after the n-loop       */
  FRKC2_ENOMEM = 4,       /* workspace smaller than frkc2_workspace_size() asked for        */
  FRKC2_ECUDA = 5,        /* a CUDA runtime call failed (launch, copy, device query)        */
  FRKC2_ETIMEOUT = 6,     /* a bounded device wait expired (latched in the workspace)       */
  FRKC2_ENONFINITE = 7,   /* a step produced NaN or Inf (latched in the workspace)          */
  FRKC2_EUNSUPPORTED = 8, /* valid request that this build does not implement               */
  FRKC2_EBOUNDS = 9       /* bounds-checking build only: a kernel's index fell outside its
                             array and the access was skipped (latched in the workspace)   */
} frkc2_status;

/* NEUMANN (zero flux: the ghost cell repeats its boundary cell) is taken by the Brusselator
 * entry points only; the diffusion entry points reject it.                                 */
enum { FRKC2_BC_PERIODIC = 0, FRKC2_BC_DIRICHLET = 1, FRKC2_BC_NEUMANN = 2 };

/* Conductivity.  CONST: kappa = kappa_c.  FIELD: cell-centred array `kappa`.
 * POWER: kappa(w) = 1 + kappa_c * w^kappa_p (principal branch for complex stage states). */
enum { FRKC2_KAPPA_CONST = 0, FRKC2_KAPPA_FIELD = 1, FRKC2_KAPPA_POWER = 2 };

/* FP64: double state and arithmetic.  FP32: float state and arithmetic.
 * MIXED: double state and double stage update; neighbour differences are formed in double
 * and the flux arithmetic (kappa_f * difference, face sums) runs in float.
 * DFLOAT: double state at the interface; between stages the state is a pair of floats
 * (hi + lo, about 48 significant bits) updated by error-free float sums, neighbour
 * differences are rounded to float and the flux arithmetic runs in float -- every operation
 * on the FP32 pipe.  2D FIELD / CONST problems and frkc2_step only: k = 1 streams (kernel 2),
 * k > 1 runs register-tiled 64 x 64 regions of k stages (kernel 3; the default, k = 8);
 * elsewhere FRKC2_EUNSUPPORTED.  The conductivity field is float.                          */
enum { FRKC2_FP64 = 0, FRKC2_FP32 = 1, FRKC2_MIXED = 2, FRKC2_DFLOAT = 3 };

/* Plan flags: STRICT makes an unmet Q bound an error; GREEDY / LEBEDEV force one ordering;
 * PAIRED puts each conjugate pair in adjacent stages (pairs in Lebedev-Finogenov order) so
 * that 2D fixed-conductivity steps apply each pair to the real state in real arithmetic
 * (w' = w + 2 T Re(a) f(w) + T^2 |a|^2 f(f(w)), exact for a linear f): about half the
 * arithmetic and memory traffic of two complex stages, at an internal amplification
 * Q of about 0.12 L^4 instead of about L^2.  ORDER4 takes the step sizes of the rank-4
 * polynomial (Eq. 7 with N = 4): fourth order on linear problems (frkc2_plan). */
enum {
  FRKC2_PLAN_STRICT = 1,
  FRKC2_PLAN_GREEDY = 2,
  FRKC2_PLAN_LEBEDEV = 4,
  FRKC2_PLAN_PAIRED = 8,
  FRKC2_PLAN_ORDER4 = 16
};

typedef struct frkc2_plan_s* frkc2_plan_t;

typedef struct {
  int ndim;          /* 1, 2 or 3                                                            */
  int bc;            /* FRKC2_BC_*; DIRICHLET means w = 0 in the ghost cells outside the grid */
  int kappa_kind;    /* FRKC2_KAPPA_*                                                        */
  int precision;     /* FRKC2_FP64 / FP32 / MIXED / DFLOAT                                   */
  int64_t n[3];      /* n[0] = x extent, n[1] = y, n[2] = z; extents past ndim must be 1      */
  double dx;         /* grid spacing, the same along every axis                              */
  double kappa_c;    /* CONST: the value; POWER: the coefficient c                           */
  double kappa_p;    /* POWER: the exponent p (> 0)                                          */
  const void* kappa; /* FIELD: device array of n[0]*n[1]*n[2] cell values, double for FP64,
                        float otherwise; a Dirichlet boundary face takes the value
                        of its interior cell.  Ignored for the other kinds.                  */
} frkc2_problem;

typedef struct {
  int k;             /* stages per pass (temporal blocking), 1..16; 0 = library default       */
  int tile_x;        /* output tile per CTA along x, y, z; 0 = library default (kernel 6:
                        tile_x = CTAs in the cluster, 1..8, k = stages per halo exchange
                        between them, 1..16, tile_y = threads per CTA; kernel 7: tile_y =
                        rows per CTA, 0 = one wave of CTAs)                                  */
  int tile_y;
  int tile_z;
  int kernel;        /* 0 = library choice, 1 = generic shared-memory tile kernel,
                        2 = 2D streaming kernel (k = 1 only), 3 = 2D FP32 temporally blocked
                        kernel, 4 = 2D real pair kernel (PAIRED plans only), 5 = 3D kernel
                        streaming along z (k = 1 only), 6 = 1D whole-job cluster kernel
                        (N <= 16384, s <= 1024, FIELD / CONST; the 1D default there), 7 = 2D
                        FP32 wavefront pass: strips of 256 columns walked up the grid with k
                        stage levels in flight, rows staged in shared memory by TMA bulk
                        copies (n[0] a multiple of 4 and >= 256, u 16-byte aligned, every
                        pass of 1, 2, 4, 6, 8, 10 or 12 stages; the FP32 2D default there)  */
  long long wait_limit; /* batched launch and kernel 7 (its waits on the TMA row copies):
                        polls a device wait makes before it gives up and latches
                        FRKC2_ETIMEOUT (0 = library default, 2^22 polls)                    */
  int fault_inject;  /* testing only: 1 = in the batched launch the first dependent work
                        item waits on a counter nothing advances; in kernel 7 (passes of
                        k = 8) the first pass leaves one row uncopied; either wait must run out */
} frkc2_tuning;

/* ---- Plan (host, FP64) --------------------------------------------------------------
 * Step sizes a_j = 1/(M^2 alpha_M (1 - zeta_j)), L = s = 2M (Sec. 2, Eq. 8), zeta_j the
 * roots of the second-order polynomial of Eq. 7, read here as
 * R(z) = 1 - alpha/4 + (alpha/4) T_L(1 + 4z/(L^2 alpha)), alpha = 4(1 - 1/L^2)/3, so that
 * beta = (2/3)(L^2 - 1).  Stage order (Sec. 2.2): for s <= 256 the stages are ordered
 * greedily to keep the amplification estimate of Eq. 12 small, repeated over n (reduced
 * range (1 - n 1e-4) beta) until the realised Q of Eqs. 10-11 is at most 10 L^2; for
 * s > 256 the upper-half roots are taken in Lebedev-Finogenov order followed by their
 * conjugates in the same order (for s a power of two its realised Q equals the largest
 * single factor, the least any order can reach; for other s the recursion keeps every root
 * next to its mirror about the middle, with the middle one of an odd block last: realised Q
 * at most 4.7 L^2 for every s tried up to 4096), with the greedy n-loop as well if that
 * order misses 10 L^2; the smaller realised Q wins.
 *   s     : number of stages, even, 2..16384.  Above 4096 the Lebedev-Finogenov order is the
 *           only one (FRKC2_PLAN_GREEDY gives FRKC2_EINVAL there: the greedy's table would
 *           take 16 s^2 doubles of host memory).
 *   nu    : damping nu0 of Sec. 2.1, 0 <= nu0 < 0.9 (nu = nu0/2 with N = 2).  nu0 > 0 uses
 *           a_l = (1 - mu_l)/((1 - nu) M^2 alpha (1 - (1 - 2 mu_l) zeta_l)) with mu_l = mu on
 *           the roots of T_M = +i c and conj(mu) on their conjugates, mu found by Newton-
 *           Raphson on the order conditions; beta is then found by bisection on |R| = 1
 *           (about (1 - nu) times the undamped extent; interior maxima of |R| drop below 1).
 *   flags : FRKC2_PLAN_STRICT makes an unmet Q bound an error (FRKC2_EPLAN); otherwise the
 *           ordering with the smallest realised Q is kept.  FRKC2_PLAN_GREEDY or
 *           FRKC2_PLAN_LEBEDEV use that ordering alone (both together: FRKC2_EINVAL).
 *           FRKC2_PLAN_ORDER4: the rank-4 polynomial of Eq. 7 (N = 4, s = 4M, s a multiple
 *           of 4, else FRKC2_EINVAL; nu0 > 0 gives FRKC2_EUNSUPPORTED), read as
 *           B = d_0 + 2 sum_{k=1}^4 d_k T_{kM}(1 + z/(M^2 alpha)) with the d_k from the order
 *           conditions R^(n)(0) = 1, n <= 4 (Eq. 5), and alpha the largest value keeping
 *           |R| <= 1 on [-2 M^2 alpha, 0] (bisection); beta = 2 M^2 alpha (about 0.254 s^2;
 *           2.785 at s = 4, where B is the Taylor polynomial of e^z).  The step sizes are
 *           a_l = 1/(M^2 alpha (1 - zeta_l)) (Eq. 8) for the 4M roots zeta_l in conjugate
 *           pairs.  Ordering: Lebedev-Finogenov first at every s (realised Q about 0.1 s^2),
 *           the greedy n-loop only if that misses 10 s^2.  The steps of frkc2_step with such
 *           a plan are fourth order for linear f (second order for kappa(u)).
 *   out   : receives a new plan; release it with frkc2_plan_destroy.
 * Cost: the greedy is O(s^3) host work (tens of ms at s = 64, about 1 s at s = 256); the
 * Lebedev-Finogenov order costs O(s^2) (about 0.2 s at s = 1024).                          */
frkc2_status frkc2_plan(int s, double nu, unsigned flags, frkc2_plan_t* out);

/* A plan from caller-given ordered step sizes (a_re[l] + i a_im[l], l = 0..s-1, host arrays
 * copied).  beta is the closed-form extent for s; Q is the realised amplification of the
 * given order.  Used to run a stage order chosen elsewhere.                               */
frkc2_status frkc2_plan_from_steps(int s, const double* a_re, const double* a_im,
                                   frkc2_plan_t* out);

/* Plan contents.  Any output pointer may be NULL.  a_re, a_im (length s) receive the step
 * sizes in stage order; order (length s) the root index j of each stage.                   */
frkc2_status frkc2_plan_info(frkc2_plan_t plan, int* s, double* beta, double* Q, int* n_iter,
                             double* a_re, double* a_im, int* order);

void frkc2_plan_destroy(frkc2_plan_t plan);

/* ---- Precision policy (Sec. 2.2 applied to rounding) -------------------------------------
 * Rounding gain of the plan's stage order, g = sqrt(sum_l mean_x |prod_{j>l}(1 + a_j x)|^2),
 * the mean over max(2048, 4 s) evenly spaced midpoints x of [-beta, 0].  A rounding error
 * made in stage l reaches the step's output through the factors of the later stages (the
 * partial products of Sec. 2.2, Eq. 10), so with rounding spread evenly over the spectrum
 * one step's relative error is about (unit roundoff) * g.  The paper's greedy order has g of
 * about 30 (s = 16) to 6300 (s = 256); the Lebedev-Finogenov order about 1.8 to 3.4.      */
frkc2_status frkc2_plan_rounding_gain(frkc2_plan_t plan, double* gain);

/* The cheapest state precision whose predicted relative L2 error after nsteps steps (against
 * FP64 arithmetic with the same plan) is at most tol.  With n = nsteps, s the plan's stage
 * count and A = g sqrt(n) + 4e-3 s n (the stage roundings amplified by the later stages and
 * adding like a random walk over steps, plus the s n roundings of a slowly changing state,
 * which do not cancel):
 *   FP32                          if e32 = 1.5 * 2^-24 * A <= tol,
 *   DFLOAT (2D FIELD / CONST) or
 *   MIXED (other problems)        if 5e-2 * e32 <= tol (double-class state, float flux
 *                                 arithmetic),
 *   FP64                          otherwise (predicted 1.5 * 2^-53 * A).
 * The constants are measured on GB300 (2048^2 diffusion recipe, greedy and Lebedev-Finogenov
 * orders, s = 16..256, 1 to 100 steps): every FP32 error measured is at most 0.9 of e32;
 * DFLOAT and MIXED measured 1.1e-3..2.3e-2 of the FP32 error.  The prediction assumes
 * rounding spread over the spectrum, as for smooth data; it is a forecast, not a bound.
 *   prob      : only ndim and kappa_kind are read (precision and pointers are ignored).
 *   nsteps    : >= 1.   tol : > 0.
 *   precision : receives FRKC2_FP32, FRKC2_DFLOAT, FRKC2_MIXED or FRKC2_FP64.
 *   predicted : receives the predicted error (may be NULL).                                */
frkc2_status frkc2_precision_policy(frkc2_plan_t plan, const frkc2_problem* prob, int nsteps,
                                    double tol, int* precision, double* predicted);

/* A plan and a precision together.  FIELD / CONST problems get the stage order of least
 * rounding gain (the Lebedev-Finogenov order, FRKC2_PLAN_LEBEDEV); POWER problems get the
 * default plan of frkc2_plan, because with kappa(u) the strongly complex stage states of that
 * order leave the range where kappa(W) is tame.  Then frkc2_precision_policy chooses the
 * precision.  *plan receives a new plan (release with frkc2_plan_destroy).               */
frkc2_status frkc2_plan_auto(int s, const frkc2_problem* prob, int nsteps, double tol,
                             frkc2_plan_t* plan, int* precision, double* predicted);

/* ---- Spectral-radius bound --------------------------------------------------------------
 * rho = max_c (2/dx^2) sum_faces kappa_f (Gershgorin), the |lambda|_max of Sec. 3 that sets
 * T <= beta / rho.  For POWER the conductivity is evaluated at the real state u (device
 * array in the problem's state precision); u is ignored for CONST and FIELD.  The result is
 * written as one double to device memory rho_dev (caller-owned, 8-byte aligned).  Faces
 * are summed x axis first, low face before high face, so FIELD and CONST results are exact
 * repeats of that order of FP64 operations.                                               */
frkc2_status frkc2_rho_bound(const frkc2_problem* prob, const void* u, double* rho_dev,
                             void* stream);

/* ---- Workspace ----------------------------------------------------------------------------
 * Bytes of device workspace frkc2_step needs for this problem and tuning (tuning may be
 * NULL).  The workspace must be 256-byte aligned.  Its first 256 bytes hold the status word. */
frkc2_status frkc2_workspace_size(const frkc2_problem* prob, const frkc2_tuning* tune,
                                  size_t* bytes);

/* Clears the status word of a workspace (asynchronous, on stream).                         */
frkc2_status frkc2_workspace_reset(void* ws, void* stream);

/* Synchronises stream, reads the status word and returns FRKC2_OK, FRKC2_EBOUNDS (only the
 * bounds-checking build latches it), FRKC2_ENONFINITE or FRKC2_ETIMEOUT, in that priority. */
frkc2_status frkc2_workspace_status(const void* ws, void* stream);

/* ---- Forward step (Sec. 3, Eq. 13) ------------------------------------------------------
 * Advances u by nsteps FRKC2 steps of size dt with the plan's stage order.
 *   u     : device array, in/out, real state (float for FP32, double otherwise).
 *   rho   : if > 0, dt*rho <= beta is checked on the host (FRKC2_EUNSTABLE otherwise);
 *           pass a bound from frkc2_rho_bound or 0 to skip the check.
 *   ws    : device workspace of at least frkc2_workspace_size() bytes.
 *   tune  : stages per pass, tile and kernel choice; NULL = library defaults.
 * Each step starts from W^0 = u (imaginary part 0) and stores Re W^L back into u.  Stages
 * are grouped into passes of k consecutive stages computed in shared memory.              */
frkc2_status frkc2_step(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int nsteps,
                        double rho, void* u, void* ws, size_t ws_bytes,
                        const frkc2_tuning* tune, void* stream);

/* ---- A range of stages (Sec. 3, Eq. 13) on a complex state ---------------------------------
 * Applies the plan's stages l0 .. l1-1 of one step of size dt to the complex stage state
 * W^{l0} and leaves W^{l1}: W^{l+1} = W^l + dt a_l f(W^l).  For callers that split the stage
 * loop, such as a grid decomposed into slabs whose halo rows are exchanged between groups of
 * stages (paper_1702_03818_gb300/slab.py).  2D FIELD / CONST problems in FP64, FP32 or MIXED
 * (FRKC2_EUNSUPPORTED otherwise).
 *   w      : device array of 2 n[0] n[1] values (state precision), interleaved (re, im) per cell,
 *            in and out.  With l0 == 0 (a step's first stages) the imaginary parts are first set
 *            to zero: a step starts from the real state w^n.  After l1 == s the real parts are
 *            w^{n+1}.
 *   l0, l1 : 0 <= l0 < l1 <= s.
 *   ws     : workspace of frkc2_workspace_size(prob) bytes (face conductivities are rebuilt by
 *            every call).
 * Each stage is one launch of the single-stage streaming pass; the last one writes w.        */
frkc2_status frkc2_stages(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int l0, int l1,
                          void* w, void* ws, size_t ws_bytes, void* stream);

/* ---- Error-controlled integration (Sec. 3, Eqs. 14-16) --------------------------------
 * Integrates u from t = 0 to t_end with the embedded first-order solution
 * What^{l+1} = What^l + T Re(a_l) Re(f(W^l)) (Eq. 14) carried through every step and the
 * scaled error ||err|| = RMS_i |Re W^L_i - What^L_i| / (tol (1 + max(|Re W^L_i|, |What^L_i|)))
 * (Eq. 15, root mean square over the cells).  A step with ||err|| > 1 is rejected and retried
 * with T scaled by SAFE/sqrt(||err||), SAFE = 0.8; after an accepted step the next T is
 * T (SAFE/sqrt(e_n)) (T/T_prev) sqrt(e_{n-1}/e_n) (Eq. 16; SAFE/sqrt(e_n) alone after the
 * first step), growing by at most 5x.  T is also capped by t_end - t and, if rho > 0, by the
 * stability limit beta/rho.  The plan's stage count is used for every step.
 * The call is synchronous: each step reads the error norm back to the host.  u is updated
 * only by accepted steps.  Returns FRKC2_ETIMEOUT if 10^6 attempts did not reach t_end.
 * Kernels: 2D FIELD / CONST problems with the default tuning run the single-stage streaming
 * pass with the embedded solution fused into it; other problems, or a tuning that sets
 * kernel, k > 1 or a tile, run the shared-memory tile pass of tune->k stages.
 *   dt0   : first step size to try (> 0).
 *   stats : may be NULL; receives the accepted and rejected step counts, the time reached,
 *           the last accepted step size and its scaled error.
 * Workspace: frkc2_adaptive_workspace_size().                                             */
typedef struct {
  int accepted;
  int rejected;
  double t;
  double dt_last;
  double err_last;
} frkc2_adaptive_stats;
frkc2_status frkc2_adaptive_workspace_size(const frkc2_problem* prob, const frkc2_tuning* tune,
                                           size_t* bytes);
frkc2_status frkc2_step_adaptive(frkc2_plan_t plan, const frkc2_problem* prob, double t_end,
                                 double tol, double dt0, double rho, void* u, void* ws,
                                 size_t ws_bytes, const frkc2_tuning* tune,
                                 frkc2_adaptive_stats* stats, void* stream);

/* ---- Forward step without a workspace -------------------------------------------------
 * The paper has no counterpart: this is a service for callers that cannot allocate device
 * memory -- for example a plugin whose host application owns every device allocation, or
 * code running while the caller's allocator is locked -- and so cannot pass the workspace
 * frkc2_step asks for.  Same arguments and result as frkc2_step with the default tuning,
 * but the workspace is a fixed array of FRKC2_NOALLOC_SCRATCH_BYTES built into the library
 * (every GPU that loads the library holds it until the process exits).  The call allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *   - Problems whose workspace (frkc2_workspace_size) exceeds the array are rejected with
 *     FRKC2_ENOMEM before any work is queued (e.g. FP64 2D grids up to about 510^2 cells,
 *     FP32 2D grids up to about 720^2 cells).
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing).  The first call on a device may load
 *     the library's device code: make that first call before any stream capture.
 *   - Every call shares the one array and it keeps the last call's contents; the call
 *     clears the status word itself.  Calls whose work overlaps on the GPU (different
 *     streams, or different host threads on the same device) race on the array: serialise
 *     them.  The device status word is not returned: check the output for non-finite values. */
#define FRKC2_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
frkc2_status frkc2_step_noalloc(frkc2_plan_t plan, const frkc2_problem* prob, double dt,
                                int nsteps, double rho, void* u, void* stream);

/* ---- Adjoint (reverse replay of Eq. 13) ------------------------------------------------
 * Gradients of a scalar J(u(T_end)) after nsteps steps from u0, given g = dJ/du(T_end).
 * The forward run keeps u every ckpt_every steps; each segment of ckpt_every steps is
 * recomputed from its checkpoint with every stage state stored, then the stages are
 * reversed: lam^l = lam^{l+1} + conj(dt a_l) J_f(W^l)^H lam^{l+1}, starting from
 * lam = g (imaginary part 0) at the end of each step, and dJ/du^n = Re lam^0.
 *   u0, g        : device arrays (state precision), read only.
 *   dJdu0        : device array (state precision), written.
 *   dJdkappa     : device array (kappa precision), written, FIELD only (NULL otherwise or to
 *                  skip): dJ/dkappa_c = sum over stages of the face sensitivities
 *                  Re(dt a_l [conj(lam_i)(W_j - W_i) + conj(lam_j)(W_i - W_j)])/dx^2, half
 *                  to each cell of an interior face.
 * Workspace: frkc2_adjoint_workspace_size().                                               */
frkc2_status frkc2_adjoint_workspace_size(const frkc2_plan_t plan, const frkc2_problem* prob,
                                          int nsteps, int ckpt_every, size_t* bytes);
frkc2_status frkc2_adjoint(frkc2_plan_t plan, const frkc2_problem* prob, double dt,
                           int nsteps, int ckpt_every, const void* u0, const void* g,
                           void* dJdu0, void* dJdkappa, void* ws, size_t ws_bytes,
                           void* stream);

/* The two halves of frkc2_adjoint, for callers (such as an autodiff framework) that run the
 * forward integration first and ask for gradients later.  frkc2_adjoint_forward integrates
 * from u0, keeps the checkpoints and the last segment's stage tape in ws, and writes u(T_end)
 * to uT (device array, may be NULL).  frkc2_adjoint_backward then takes g = dJ/du(T_end) and
 * writes dJdu0 / dJdkappa; it must get the same plan, problem, dt, nsteps, ckpt_every and
 * workspace as the forward call, with the workspace untouched in between.               */
frkc2_status frkc2_adjoint_forward(frkc2_plan_t plan, const frkc2_problem* prob, double dt,
                                   int nsteps, int ckpt_every, const void* u0, void* uT,
                                   void* ws, size_t ws_bytes, void* stream);
frkc2_status frkc2_adjoint_backward(frkc2_plan_t plan, const frkc2_problem* prob, double dt,
                                    int nsteps, int ckpt_every, const void* g, void* dJdu0,
                                    void* dJdkappa, void* ws, size_t ws_bytes, void* stream);

/* ---- Batched forward step ----------------------------------------------------------------
 * nprob independent 2D problems (each with its own plan, grid size, conductivity, dt and
 * step count, all of one precision and the same boundary kind) advanced by ONE persistent
 * kernel launch.  The launch walks a device work list of (problem, pass, tile) items in
 * rounds; a tile waits (bounded spin, then FRKC2_ETIMEOUT latched) until every tile of the
 * previous pass of its problem is done.  frkc2_batch_prepare writes the problem table
 * into the workspace (host-to-device copies on stream); frkc2_batch_launch only resets the
 * counters and launches, so it can be captured in a CUDA graph and replayed.
 * Work items: FP32 and DFLOAT problems run register-tiled 64 x 64 regions of k stages (tile
 * 64 - 2k, default k = 8, the fastest on a mixed batch; DFLOAT with float-pair state),
 * tune->tile_z consecutive regions of one pass per item (default 4); FP64 / MIXED problems
 * with k = 1 (the default), and DFLOAT with k = 1, run the single-stage streaming body on
 * tiles of 31 columns x tune->tile_y rows (default 128); FP64 / MIXED with k > 1 or kernel = 1
 * a k-stage shared-memory tile of tune->tile_x x tune->tile_y (DFLOAT: FRKC2_EUNSUPPORTED).
 *   plans, probs, dt, nsteps, u : host arrays of nprob entries (u[i] device pointers).    */
frkc2_status frkc2_batch_workspace_size(int nprob, const frkc2_plan_t* plans,
                                        const frkc2_problem* probs, const int* nsteps,
                                        const frkc2_tuning* tune, size_t* bytes);
frkc2_status frkc2_batch_prepare(int nprob, const frkc2_plan_t* plans,
                                 const frkc2_problem* probs, const double* dt,
                                 const int* nsteps, void* const* u, const frkc2_tuning* tune,
                                 void* ws, size_t ws_bytes, void* stream);
frkc2_status frkc2_batch_launch(void* ws, void* stream);
frkc2_status frkc2_step_batched(int nprob, const frkc2_plan_t* plans,
                                const frkc2_problem* probs, const double* dt,
                                const int* nsteps, void* const* u, const frkc2_tuning* tune,
                                void* ws, size_t ws_bytes, void* stream);

/* ---- Brusselator reaction-diffusion (Sec. 3.1, Eq. 17) ------------------------------------
 * The paper's demonstration system, two species on a 2D grid with the 5-point Laplacian:
 *   v' = D Lap v + A - (B + 1) v + v^2 w,    w' = D Lap w + B v - v^2 w
 * (the paper's values: D = 0.02, A = 1, B = 3, unit square, spectral radius about 6400 on
 * 200 x 200).  A step applies the plan's ordered complex stages W^{l+1} = W^l + dt a_l f(W^l)
 * (Eq. 13) to the pair (v, w) in complex arithmetic and stores Re W^L; the paper states no
 * boundary condition: PERIODIC and NEUMANN are offered.                                    */
typedef struct {
  int bc;            /* FRKC2_BC_PERIODIC or FRKC2_BC_NEUMANN                                */
  int precision;     /* FRKC2_FP64 or FRKC2_FP32 (state and arithmetic); MIXED: EUNSUPPORTED */
  int64_t nx, ny;    /* grid extents (x fastest), 1..2^30 each                               */
  double dx;         /* grid spacing                                                         */
  double D;          /* diffusion coefficient (>= 0)                                         */
  double A, B;       /* reaction constants                                                   */
} frkc2_bruss_problem;

/* Workspace bytes for frkc2_bruss_step and frkc2_bruss_rho_bound: 256 bytes of status and
 * barrier words, 64 KB of per-CTA stage flags, then two complex stage states (4 planes of
 * nx*ny values each).                                                                      */
frkc2_status frkc2_bruss_workspace_size(const frkc2_bruss_problem* prob, size_t* bytes);

/* Gershgorin bound on the spectral radius of the Jacobian of f at the real state (v, w):
 *   rho = 8 D/dx^2 + max_cells max(|2 v w - (B+1)| + v^2, |B - 2 v w| + v^2),
 * formed in FP64 in that order (p = v w, q = v v), written as one double to rho_dev (device,
 * 8-byte aligned).  v, w: device arrays of the problem's precision, read only.             */
frkc2_status frkc2_bruss_rho_bound(const frkc2_bruss_problem* prob, const void* v,
                                   const void* w, double* rho_dev, void* ws, size_t ws_bytes,
                                   void* stream);

/* Advances (v, w) by nsteps FRKC2 steps of size dt (in place; v and w distinct device arrays
 * of the problem's precision).  rho > 0: dt*rho <= beta is checked (FRKC2_EUNSTABLE).
 * tune->kernel: 0 or 1 = one persistent cooperative launch for every stage of every step,
 * each CTA waiting between stages for the CTAs whose cells its stencil reads (per-CTA stage
 * flags), or for FP64 stages of more than 2048 cells a CTA at a device-wide barrier (a plan of
 * more than 1024 stages takes one launch per 1024 stages of each step); 2 = one launch per
 * stage.  The waits are bounded by tune->wait_limit polls (0 = 2^22); on expiry FRKC2_ETIMEOUT
 * is latched in the workspace and the launch returns early (the state is then unspecified).
 * tune->fault_inject = 1 (testing only, persistent form) makes the first wait between stages
 * wait for a count that nothing reaches.  A non-finite value in a step's output latches FRKC2_ENONFINITE.
 * Memory: 4 state reads and writes per cell-stage (32 bytes in FP32, 64 in FP64).          */
frkc2_status frkc2_bruss_step(frkc2_plan_t plan, const frkc2_bruss_problem* prob, double dt,
                              int nsteps, double rho, void* v, void* w, void* ws,
                              size_t ws_bytes, const frkc2_tuning* tune, void* stream);

/* ---- FMA throughput probe ------------------------------------------------------------------
 * Not part of the method: measures the FP64 or FP32 fused multiply-add rate that the kernels'
 * rooflines are stated against.  Launches `blocks` CTAs of 256 threads, each thread running
 * `iters` rounds of 8 independent FMA chains (FMAs = blocks * 256 * iters * 8) and writing one
 * value to out (device array of blocks * 256 elements of the precision).  The caller times it.
 *   precision : FRKC2_FP64, FRKC2_FP32 (scalar FMAs), or FRKC2_FP32 | FRKC2_PROBE_PACKED (the
 *               same FMAs as packed two-lane FP32 instructions: 4 chains of float pairs).  */
#define FRKC2_PROBE_PACKED 16
frkc2_status frkc2_fma_probe(int precision, int blocks, int iters, void* out, void* stream);

/* Short text for a status code (static storage).                                          */
const char* frkc2_status_string(frkc2_status st);

/* Kernel launches queued by this thread since the last call (and resets the count).       */
long long frkc2_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* FRKC2_H */
