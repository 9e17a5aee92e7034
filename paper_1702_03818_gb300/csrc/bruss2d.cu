// Brusselator reaction-diffusion (Sec. 3.1, Eq. 17) advanced by FRKC2 stages on the GPU.
//
// Two species (v, w) on an nx-by-ny grid, 5-point Laplacian, periodic or zero-flux
// boundaries:  f_v = D Lap v + A - (B+1) v + v^2 w,   f_w = D Lap w + B v - v^2 w.
// Each stage applies W^{l+1} = W^l + h_l f(W^l), h_l = dt a_l (Sec. 3, Eq. 13), to the complex
// pair (v, w) in real arithmetic: 41 floating-point instructions per cell-stage (four
// Laplacians, the complex products v^2 and v^2 w, the four right-hand sides and the four
// complex updates).  Stage states live in the workspace as four planar arrays (Re v, Im v,
// Re w, Im w), ping-ponged between two copies; the first stage of a step reads the caller's
// real (v, w) and the last stage writes the real parts back there.
//
// Two launch forms:
//  * persistent (default): ONE cooperative launch runs every stage of every step; the CTAs
//    are all co-resident (a multiple of the SM count).  Between stages a CTA waits only for
//    the CTAs whose cells its stencil reads (the owners of the cells within one grid row of
//    its own range, a handful), which are also the CTAs that read its cells: each CTA
//    publishes the count of stages it has finished in a flag of its own, and a CTA starts a
//    stage when every neighbour's flag shows the previous one done.  A neighbour set too
//    large for that (tiny grids) falls back to a grid barrier on a monotone arrival counter.
//    Each wait is bounded (polls counted, then FRKC2_ETIMEOUT is latched, an abort word set
//    and every CTA returns).  Stage inputs are read through L2 (ld.global.cg), never from a
//    possibly stale L1 line.
//  * per stage: one ordinary launch per stage, same cell code, no barrier.
// Work split: CTA b owns the contiguous cells [b N / G, (b+1) N / G) of the row-major grid,
// thread t of the CTA takes cells c0 + t, c0 + t + 256, ... (coalesced rows).
#include <algorithm>
#include <cmath>
#include <memory>
#include <type_traits>

#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int BR_THREADS = 256;
constexpr int BR_MAXS = 1024;  // stage coefficients one persistent launch carries
constexpr long long BR_DEFAULT_WAIT = 1ll << 22;
constexpr int BR_MAXCTA = 8192;  // CTAs with a stage flag in the workspace
constexpr int BR_MAXNB = 32;     // neighbour CTAs a CTA waits for, one lane each (more: the grid barrier)

template <int NS>
struct BrussArgs {
  void* v;                   // caller's real state: read by stage 0, written by stage s-1
  void* w;
  void* P[2][4];             // complex stage states, planar: Re v, Im v, Re w, Im w
  int nx, ny;
  long long ncell;
  double Dd, A, B1, B;       // D / dx^2, A, B + 1, B
  int s, l_begin, l_end;     // stages [l_begin, l_end) of each step of an s-stage plan
  int nsteps;
  int coop;                  // 1: grid barrier between stages
  int check_finite;
  int fault_inject;          // testing only: the first barrier waits for a count nothing reaches
  long long wait_limit;
  unsigned* status;
  unsigned* abort_flag;
  unsigned long long* bar;   // barrier arrival counter (zeroed before the launch)
  unsigned long long* flags; // per CTA: stages finished in this launch (zeroed before it)
  int nbsync;                // 1: neighbour flags between stages, 0: the grid barrier (the
                             // choice is the host's, the same for every CTA)
  double hr[NS];             // dt Re a_l, l = l_begin + index
  double hi[NS];             // dt Im a_l
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool bad_bits(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool bad_bits(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }

// Grid-wide barrier for a cooperative launch; false if the launch is being aborted.
template <int NS>
__device__ bool grid_barrier(const BrussArgs<NS>& a, unsigned long long target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(a.bar, 1ull);
    const unsigned long long want = a.fault_inject ? ~0ull : target;
    long long polls = 0;
    while (ld_acquire_u64(a.bar) < want) {
      if (*((volatile unsigned*)a.abort_flag) || ++polls > a.wait_limit) {
        atomicOr(a.status, ST_TIMEOUT);
        atomicExch(a.abort_flag, 1u);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The CTAs whose cells CTA b's stencil reads: the owners of the cells [c0 - nx, c1 + nx) (with
// the periodic wrap), at most two ranges of CTA indices [lo, hi] (the host enables this only
// where every CTA's set is at most BR_MAXNB CTAs and shorter than the grid).  Cell c belongs to
// CTA ceil((c+1) G / N) - 1.
struct NbSet {
  int lo[2], hi[2], n;
};

__device__ __forceinline__ int br_owner(long long c, long long N, long long G) {
  return int(((c + 1) * G - 1) / N);
}

__device__ NbSet br_neighbours(long long c0, long long c1, long long N, long long G, int nx, bool periodic) {
  NbSet s;
  s.n = 0;
  s.lo[0] = s.lo[1] = 0;
  s.hi[0] = s.hi[1] = -1;
  long long a = c0 - nx, z = c1 - 1 + nx;  // inclusive
  if (z - a + 1 >= N) return s;           // the whole grid: too many
  if (!periodic) {
    a = a < 0 ? 0 : a;
    z = z >= N ? N - 1 : z;
    s.lo[0] = br_owner(a, N, G);
    s.hi[0] = br_owner(z, N, G);
  } else if (a < 0) {
    s.lo[0] = br_owner(a + N, N, G);
    s.hi[0] = int(G) - 1;
    s.lo[1] = 0;
    s.hi[1] = br_owner(z, N, G);
  } else if (z >= N) {
    s.lo[0] = br_owner(a, N, G);
    s.hi[0] = int(G) - 1;
    s.lo[1] = 0;
    s.hi[1] = br_owner(z - N, N, G);
  } else {
    s.lo[0] = br_owner(a, N, G);
    s.hi[0] = br_owner(z, N, G);
  }
  s.n = (s.hi[0] - s.lo[0] + 1) + (s.hi[1] - s.lo[1] + 1);
  return s;
}

// Neighbour wait: publish that this CTA finished `done` stages, then wait until every
// neighbour has; false if the launch is being aborted.  Lane i of warp 0 watches neighbour i,
// so the flags are polled together (one L2 round trip per poll, not one per neighbour).
template <int NS>
__device__ bool nb_wait(const BrussArgs<NS>& a, const NbSet& nb, unsigned long long done) {
  __shared__ int s_ok;
  __syncthreads();  // every thread's stores of the finished stage are issued
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane == 0) {
      __threadfence();
      atomicMax(a.flags + blockIdx.x, done);  // performed at L2, like the grid barrier's arrival
    }
    __syncwarp();
    const int n0 = nb.hi[0] - nb.lo[0] + 1;
    int j = -1;
    if (lane < nb.n) j = lane < n0 ? nb.lo[0] + lane : nb.lo[1] + (lane - n0);
    if (j == int(blockIdx.x) && !a.fault_inject) j = -1;  // its own flag is set
    const unsigned long long want = a.fault_inject ? ~0ull : done;
    int ok = 1;
    long long polls = 0;
    while (true) {
      const bool ready = j < 0 || ld_acquire_u64(a.flags + j) >= want;
      if (__all_sync(0xffffffffu, ready)) break;
      const bool stop = *((volatile unsigned*)a.abort_flag) != 0 || ++polls > a.wait_limit;
      if (__any_sync(0xffffffffu, stop)) {
        if (lane == 0) {
          atomicOr(a.status, ST_TIMEOUT);
          atomicExch(a.abort_flag, 1u);
        }
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    if (lane == 0) {
      __threadfence();
      s_ok = ok;
    }
  }
  __syncthreads();
  return s_ok != 0;
}

template <class S>
__device__ __forceinline__ S ldc(const S* p, long long i) {
  return p ? __ldcg(p + i) : S(0);
}

template <class S, bool PERIODIC, int NS>
__global__ void __launch_bounds__(BR_THREADS) k_bruss2d(const BrussArgs<NS> a) {
  const int nx = a.nx, ny = a.ny;
  const long long G = gridDim.x;
  const long long c0 = (long long)blockIdx.x * a.ncell / G;
  const long long c1 = ((long long)blockIdx.x + 1) * a.ncell / G;
  const long long cfirst = c0 + threadIdx.x;
  const int y_first = int(cfirst / nx);
  const int x_first = int(cfirst - (long long)y_first * nx);
  const S Dd = S(a.Dd), A = S(a.A), B1 = S(a.B1), B = S(a.B);
  const bool use_nb = a.coop && a.nbsync;
  const NbSet nb = use_nb ? br_neighbours(c0, c1, a.ncell, G, nx, PERIODIC) : NbSet{};
  unsigned long long target = 0, done = 0;
  bool bad = false;

  for (int n = 0; n < a.nsteps; ++n) {
    for (int l = a.l_begin; l < a.l_end; ++l) {
      if (a.coop && (n > 0 || l > a.l_begin)) {
        ++done;
        if (use_nb) {
          if (!nb_wait(a, nb, done)) return;
        } else {
          target += (unsigned long long)G;
          if (!grid_barrier(a, target)) return;
        }
      }
      const bool first = l == 0, last = l == a.s - 1;
      const S hr = S(a.hr[l - a.l_begin]), hi = S(a.hi[l - a.l_begin]);
      const S* Ivr;
      const S* Ivi;
      const S* Iwr;
      const S* Iwi;
      if (first) {
        Ivr = static_cast<const S*>(a.v);
        Iwr = static_cast<const S*>(a.w);
        Ivi = Iwi = nullptr;
      } else {
        void* const* Q = a.P[(l - 1) & 1];
        Ivr = static_cast<const S*>(Q[0]);
        Ivi = static_cast<const S*>(Q[1]);
        Iwr = static_cast<const S*>(Q[2]);
        Iwi = static_cast<const S*>(Q[3]);
      }
      S* Ovr;
      S* Ovi;
      S* Owr;
      S* Owi;
      if (last) {
        Ovr = static_cast<S*>(a.v);
        Owr = static_cast<S*>(a.w);
        Ovi = Owi = nullptr;
      } else {
        void* const* Q = a.P[l & 1];
        Ovr = static_cast<S*>(Q[0]);
        Ovi = static_cast<S*>(Q[1]);
        Owr = static_cast<S*>(Q[2]);
        Owi = static_cast<S*>(Q[3]);
      }
      int x = x_first, y = y_first;
      for (long long c = cfirst; c < c1; c += BR_THREADS) {
        int xe, xw, yn, ys;
        if (PERIODIC) {
          xe = x + 1 == nx ? 0 : x + 1;
          xw = x == 0 ? nx - 1 : x - 1;
          yn = y + 1 == ny ? 0 : y + 1;
          ys = y == 0 ? ny - 1 : y - 1;
        } else {  // zero flux: the ghost cell repeats the boundary cell
          xe = min(x + 1, nx - 1);
          xw = max(x - 1, 0);
          yn = min(y + 1, ny - 1);
          ys = max(y - 1, 0);
        }
        const long long row = (long long)y * nx;
        const long long iE = row + xe, iW = row + xw;
        const long long iN = (long long)yn * nx + x, iS = (long long)ys * nx + x;
        const S vr = ldc(Ivr, c), vi = ldc(Ivi, c), wr = ldc(Iwr, c), wi = ldc(Iwi, c);
        const S Lvr = ((ldc(Ivr, iE) + ldc(Ivr, iW)) + (ldc(Ivr, iN) + ldc(Ivr, iS))) - S(4) * vr;
        const S Lvi = ((ldc(Ivi, iE) + ldc(Ivi, iW)) + (ldc(Ivi, iN) + ldc(Ivi, iS))) - S(4) * vi;
        const S Lwr = ((ldc(Iwr, iE) + ldc(Iwr, iW)) + (ldc(Iwr, iN) + ldc(Iwr, iS))) - S(4) * wr;
        const S Lwi = ((ldc(Iwi, iE) + ldc(Iwi, iW)) + (ldc(Iwi, iN) + ldc(Iwi, iS))) - S(4) * wi;
        // v^2 and v^2 w in complex arithmetic
        const S qr = vr * vr - vi * vi;
        const S qi = (vr + vr) * vi;
        const S pr = qr * wr - qi * wi;
        const S pi = qr * wi + qi * wr;
        const S fvr = Dd * Lvr + ((A - B1 * vr) + pr);
        const S fvi = Dd * Lvi + (pi - B1 * vi);
        const S fwr = Dd * Lwr + (B * vr - pr);
        const S fwi = Dd * Lwi + (B * vi - pi);
        const S nvr = vr + hr * fvr - hi * fvi;
        const S nwr = wr + hr * fwr - hi * fwi;
        Ovr[c] = nvr;
        Owr[c] = nwr;
        if (!last) {
          Ovi[c] = vi + hr * fvi + hi * fvr;
          Owi[c] = wi + hr * fwi + hi * fwr;
        } else if (a.check_finite) {
          bad |= bad_bits(nvr) || bad_bits(nwr);
        }
        x += BR_THREADS;
        if (x >= nx) {
          const int q = x / nx;
          x -= q * nx;
          y += q;
        }
      }
    }
  }
  if (bad) atomicOr(a.status, ST_NONFINITE);
}

// Gershgorin bound: max over cells of the larger reaction row sum (the Laplacian part is
// added by the finishing kernel).  FP64 throughout, the operations in a fixed order.
template <class S>
__global__ void k_bruss_rho(const S* __restrict__ v, const S* __restrict__ w, long long n, double B1,
                            double B, unsigned long long* acc) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double vv = double(v[i]), ww = double(w[i]);
    const double p = __dmul_rn(vv, ww);
    const double q = __dmul_rn(vv, vv);
    const double rv = __dadd_rn(fabs(__dsub_rn(__dmul_rn(2.0, p), B1)), q);
    const double rw = __dadd_rn(fabs(__dsub_rn(B, __dmul_rn(2.0, p))), q);
    m = fmax(m, fmax(rv, rw));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(acc, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_bruss_rho_finish(const unsigned long long* acc, double diff, double* rho) {
  *rho = __dadd_rn(diff, __longlong_as_double((long long)*acc));
}

struct BrLayout {
  size_t status, abort_flag, bar, acc, flags, planes[2][4], total;
};

BrLayout br_layout(const frkc2_bruss_problem& p) {
  BrLayout L{};
  L.status = 0;
  L.abort_flag = 4;
  L.bar = 8;
  L.acc = 16;
  L.flags = 256;
  size_t off = 256 + align256(size_t(BR_MAXCTA) * 8);
  const size_t plane = align256(size_t(p.nx) * size_t(p.ny) * state_bytes(p.precision));
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < 4; ++c) {
      L.planes[b][c] = off;
      off += plane;
    }
  L.total = off;
  return L;
}

frkc2_status validate(const frkc2_bruss_problem* p) {
  if (!p) return FRKC2_EINVAL;
  if (p->bc != FRKC2_BC_PERIODIC && p->bc != FRKC2_BC_NEUMANN) return FRKC2_EINVAL;
  if (p->precision != FRKC2_FP64 && p->precision != FRKC2_FP32) {
    return p->precision == FRKC2_MIXED ? FRKC2_EUNSUPPORTED : FRKC2_EINVAL;
  }
  if (p->nx < 1 || p->ny < 1 || p->nx > (1 << 30) || p->ny > (1 << 30)) return FRKC2_EINVAL;
  if ((long long)p->nx * p->ny > (1ll << 34)) return FRKC2_EINVAL;
  if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return FRKC2_EINVAL;
  if (!(p->D >= 0.0) || !std::isfinite(p->D) || !std::isfinite(p->A) || !std::isfinite(p->B)) return FRKC2_EINVAL;
  return FRKC2_OK;
}

template <class S, bool PER, int NS>
cudaError_t launch_one(const BrussArgs<NS>& a, bool coop, int grid, cudaStream_t st) {
  auto kern = k_bruss2d<S, PER, NS>;
  if (coop) {
    void* args[] = {const_cast<BrussArgs<NS>*>(&a)};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(BR_THREADS), args, 0, st);
    count_launch();
    return e;
  }
  kern<<<grid, BR_THREADS, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <class S, bool PER>
cudaError_t run(const frkc2_plan_s& plan, const frkc2_bruss_problem& p, double dt, int nsteps, void* v, void* w,
                char* ws, int kern, long long wait_limit, int fault_inject, cudaStream_t st) {
  const BrLayout L = br_layout(p);
  // device properties, queried once per kernel on the first (eager) call
  static const Residency res = query_residency(k_bruss2d<S, PER, BR_MAXS>, BR_THREADS, 0);
  static const int coop_ok = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
      return 0;
    return v;
  }();
  if (res.err != cudaSuccess) return res.err;
  const int sms = res.sms, occ = res.per_sm;
  const bool coop = kern != 2 && coop_ok && occ >= 1;
  const long long ncell = (long long)p.nx * p.ny;
  // a multiple of the SM count, about one 256-cell sweep per CTA, at most the resident CTAs
  long long per_sm = (ncell + (long long)sms * BR_THREADS - 1) / ((long long)sms * BR_THREADS);
  per_sm = std::max(1ll, std::min(per_sm, (long long)std::max(occ, 1)));
  long long grid = (long long)sms * per_sm;
  grid = std::min(grid, std::max(1ll, ncell));  // every CTA owns at least one cell
  // neighbour flags where every CTA waits for at most BR_MAXNB others: a CTA owns floor(N/G)
  // or ceil(N/G) cells and reads a span of at most ceil(N/G) + 2 nx cells, which meets at most
  // ceil(span / floor(N/G)) + 1 ranges, one more where it wraps.  Used in FP32 and for FP64
  // CTAs of at most 2048 cells: at the paper's 200^2 the stage is short and the neighbour wait
  // shorter than the grid barrier (FP64 3.91 against 4.12 ms a job, FP32 1.88 against 2.08);
  // an FP64 stage of 2048^2 keeps the FP64 pipe busy and runs faster with every SM's CTAs on
  // the same stage (202.7 ms against 242.6 ms for 10 steps of s = 64).
  const long long mlo = ncell / grid, mhi = (ncell + grid - 1) / grid, span = mhi + 2ll * p.nx;
  const bool nbsync = grid <= BR_MAXCTA && span < ncell && (span + mlo - 1) / mlo + 2 <= BR_MAXNB &&
                      (std::is_same<S, float>::value || mhi <= 2048);

  auto fill = [&](auto& a) {
    a.v = v;
    a.w = w;
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 4; ++c) a.P[b][c] = ws + L.planes[b][c];
    a.nx = int(p.nx);
    a.ny = int(p.ny);
    a.ncell = ncell;
    a.Dd = p.D / (p.dx * p.dx);
    a.A = p.A;
    a.B1 = p.B + 1.0;
    a.B = p.B;
    a.s = plan.s;
    a.check_finite = 1;
    a.fault_inject = fault_inject;
    a.wait_limit = wait_limit;
    a.status = reinterpret_cast<unsigned*>(ws + L.status);
    a.abort_flag = reinterpret_cast<unsigned*>(ws + L.abort_flag);
    a.bar = reinterpret_cast<unsigned long long*>(ws + L.bar);
    a.flags = reinterpret_cast<unsigned long long*>(ws + L.flags);
    a.nbsync = nbsync ? 1 : 0;
  };

  if (coop) {
    auto ap = std::make_unique<BrussArgs<BR_MAXS>>();  // 16 KB parameter block
    BrussArgs<BR_MAXS>& a = *ap;
    fill(a);
    a.coop = 1;
    auto launch_range = [&](int lb, int le, int ns) -> cudaError_t {
      a.l_begin = lb;
      a.l_end = le;
      a.nsteps = ns;
      for (int l = lb; l < le; ++l) {
        a.hr[l - lb] = dt * plan.a_re[l];
        a.hi[l - lb] = dt * plan.a_im[l];
      }
      cudaError_t e2 = cudaMemsetAsync(ws + L.abort_flag, 0, 12, st);  // abort word and barrier count
      if (e2 == cudaSuccess) e2 = cudaMemsetAsync(ws + L.flags, 0, size_t(std::min<long long>(grid, BR_MAXCTA)) * 8, st);
      if (e2 != cudaSuccess) return e2;
      return launch_one<S, PER, BR_MAXS>(a, true, int(grid), st);
    };
    if (plan.s <= BR_MAXS) return launch_range(0, plan.s, nsteps);
    for (int n = 0; n < nsteps; ++n)
      for (int lb = 0; lb < plan.s; lb += BR_MAXS) {
        const cudaError_t e2 = launch_range(lb, std::min(plan.s, lb + BR_MAXS), 1);
        if (e2 != cudaSuccess) return e2;
      }
    return cudaSuccess;
  }
  BrussArgs<1> a;
  fill(a);
  a.coop = 0;
  a.nsteps = 1;
  for (int n = 0; n < nsteps; ++n)
    for (int l = 0; l < plan.s; ++l) {
      a.l_begin = l;
      a.l_end = l + 1;
      a.hr[0] = dt * plan.a_re[l];
      a.hi[0] = dt * plan.a_im[l];
      const cudaError_t e2 = launch_one<S, PER, 1>(a, false, int(grid), st);
      if (e2 != cudaSuccess) return e2;
    }
  return cudaSuccess;
}

}  // namespace
}  // namespace frkc2

using namespace frkc2;

extern "C" {

frkc2_status frkc2_bruss_workspace_size(const frkc2_bruss_problem* prob, size_t* bytes) {
  if (!bytes) return FRKC2_EINVAL;
  const frkc2_status v = validate(prob);
  if (v != FRKC2_OK) return v;
  *bytes = br_layout(*prob).total;
  return FRKC2_OK;
}

frkc2_status frkc2_bruss_rho_bound(const frkc2_bruss_problem* prob, const void* v, const void* w, double* rho_dev,
                                   void* ws, size_t ws_bytes, void* stream) {
  const frkc2_status vs = validate(prob);
  if (vs != FRKC2_OK) return vs;
  const size_t sb = state_bytes(prob->precision);
  if (!v || !w || !rho_dev || !ws) return FRKC2_EINVAL;
  if ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(w)) & (sb - 1)) return FRKC2_EINVAL;
  if ((reinterpret_cast<uintptr_t>(rho_dev) & 7) || (reinterpret_cast<uintptr_t>(ws) & 255)) return FRKC2_EINVAL;
  if (ws_bytes < br_layout(*prob).total) return FRKC2_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* acc = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + br_layout(*prob).acc);
  if (cudaMemsetAsync(acc, 0, 8, st) != cudaSuccess) return FRKC2_ECUDA;
  const long long n = prob->nx * prob->ny;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FRKC2_ECUDA;
  const long long blocks = std::max(1ll, std::min((n + 255) / 256, (long long)sms * 8));
  if (prob->precision == FRKC2_FP64)
    k_bruss_rho<double><<<unsigned(blocks), 256, 0, st>>>(static_cast<const double*>(v), static_cast<const double*>(w), n,
                                                          prob->B + 1.0, prob->B, acc);
  else
    k_bruss_rho<float><<<unsigned(blocks), 256, 0, st>>>(static_cast<const float*>(v), static_cast<const float*>(w), n,
                                                         prob->B + 1.0, prob->B, acc);
  const double diff = 8.0 * prob->D / (prob->dx * prob->dx);
  k_bruss_rho_finish<<<1, 1, 0, st>>>(acc, diff, rho_dev);
  count_launch(2);
  return cudaGetLastError() == cudaSuccess ? FRKC2_OK : FRKC2_ECUDA;
}

frkc2_status frkc2_bruss_step(frkc2_plan_t plan, const frkc2_bruss_problem* prob, double dt, int nsteps, double rho,
                              void* v, void* w, void* ws, size_t ws_bytes, const frkc2_tuning* tune, void* stream) {
  const frkc2::NvtxRange call_range("frkc2_bruss_step");
  if (!plan || !v || !w || !ws || nsteps < 0) return FRKC2_EINVAL;
  const frkc2_status vs = validate(prob);
  if (vs != FRKC2_OK) return vs;
  if (!(dt > 0.0) || !std::isfinite(dt)) return FRKC2_EINVAL;
  const size_t sb = state_bytes(prob->precision);
  if ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(w)) & (sb - 1)) return FRKC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return FRKC2_EINVAL;
  if (v == w) return FRKC2_EINVAL;
  if (rho > 0.0 && dt * rho > plan->beta * (1.0 + 1e-12)) return FRKC2_EUNSTABLE;
  if (ws_bytes < br_layout(*prob).total) return FRKC2_ENOMEM;
  const int kern = tune ? tune->kernel : 0;
  if (kern < 0 || kern > 2) return FRKC2_EINVAL;
  const long long wait_limit = (tune && tune->wait_limit > 0) ? tune->wait_limit : BR_DEFAULT_WAIT;
  const int fault = tune ? tune->fault_inject : 0;
  if (fault && kern == 2) return FRKC2_EINVAL;  // only the persistent form has a device wait
  if (nsteps == 0) return FRKC2_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);
  const bool per = prob->bc == FRKC2_BC_PERIODIC;
  cudaError_t e;
  if (prob->precision == FRKC2_FP64)
    e = per ? run<double, true>(*plan, *prob, dt, nsteps, v, w, wsb, kern, wait_limit, fault, st)
            : run<double, false>(*plan, *prob, dt, nsteps, v, w, wsb, kern, wait_limit, fault, st);
  else
    e = per ? run<float, true>(*plan, *prob, dt, nsteps, v, w, wsb, kern, wait_limit, fault, st)
            : run<float, false>(*plan, *prob, dt, nsteps, v, w, wsb, kern, wait_limit, fault, st);
  return e == cudaSuccess ? FRKC2_OK : FRKC2_ECUDA;
}

}  // extern "C"
