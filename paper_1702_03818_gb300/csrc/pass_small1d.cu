// Whole-job kernel for small 1D problems: every stage of every step in one launch on a
// thread-block cluster, the state never leaving the chip.
//
// The N cells are split into CL contiguous chunks, one per CTA of a cluster of CL <= 8 CTAs
// (co-scheduled by the hardware).  A CTA holds its chunk extended by H halo cells on each side
// (H = 0 for a Dirichlet grid in one CTA); thread t holds R consecutive cells of the extended
// chunk in registers (complex state and the R + 1 face conductivities around them) for the
// whole job, R a compile-time 1, 2, 4 or 8, the cells past the extended chunk's end zero and
// never updated (as are Dirichlet cells outside the grid).  Per stage each thread takes the
// neighbour cells beyond its ends from the adjacent lanes by shuffles; only the warps' end
// lanes go through shared memory, at one CTA barrier (none when the CTA is one warp).  The
// halo cells at the ends of the extended chunk go stale one cell per stage; every H stages the
// CTAs refresh them from their neighbours' edge cells (a periodic grid in one CTA from its own)
// through the cluster's distributed shared memory, at one cluster barrier.  The stage shares
// each neighbour difference d_i = W_i - W_{i-1} between the two cells of face i:
// f_i = kappa_{i+1} d_{i+1} - kappa_i d_i, then W_i += dt a_l f_i / dx^2 (Sec. 3, Eq. 13): 10
// floating-point instructions per cell-stage, with no product contracted into an add, so every
// launch shape gives the same bits.  At the end of each step the state is Re W^L.  The stage
// coefficients of the whole plan (up to 1024 stages) are copied once to shared memory.
#include <algorithm>
#include <memory>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace cg = cooperative_groups;

namespace frkc2 {
namespace {

constexpr int S1_MAXS = 1024;
constexpr int S1_RMAX = 8;      // cells per thread
constexpr int S1_TMAX = 512;    // threads per CTA
constexpr int S1_WMAX = S1_TMAX / 32;
constexpr int S1_CMAX = 8;      // CTAs per cluster (portable size)
constexpr int S1_HMAX = KMAX;   // halo cells per side (stages per halo exchange)

template <class T> struct V2o;
template <> struct V2o<double> { using type = double2; };
template <> struct V2o<float> { using type = float2; };

struct Small1dArgs {
  void* u;               // caller's real state, read at the start and written at the end
  const void* fx;        // face conductivities, N + 1 (face i between cells i - 1 and i)
  unsigned* status;
  int n, nsteps, s;
  int H;                 // halo cells per side and stages per halo exchange (0: none)
  double ca[S1_MAXS];    // dt Re a_l / dx^2
  double cb[S1_MAXS];    // dt Im a_l / dx^2
};

// products that are never contracted into a neighbouring add: every cell position of every
// launch shape then rounds the same way, so all shapes give the same bits
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ bool bad1(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool bad1(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }

template <class S, class A, bool PERIODIC, int R>
__global__ void __launch_bounds__(S1_TMAX, 1) k_small1d(const Small1dArgs a) {
  using S2 = typename V2o<S>::type;
  __shared__ S2 wlo[2][S1_WMAX];      // each warp's first cell (lane 0), by stage parity
  __shared__ S2 whi[2][S1_WMAX];      // its last cell (lane 31)
  __shared__ S2 own_lo[2][S1_HMAX];   // the chunk's first H cells, by exchange parity
  __shared__ S2 own_hi[2][S1_HMAX];   // its last H cells
  __shared__ S cs[2][S1_MAXS];        // the stage coefficients (ca, cb)
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = int(cluster.num_blocks());
  const int c = int(cluster.block_rank());
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5, nw = nt >> 5;
  const int n = a.n, H = a.H;
  const int c0 = int((long long)c * n / CL), c1 = int((long long)(c + 1) * n / CL);
  const int cp = (c + CL - 1) % CL, cn = (c + 1) % CL;
  const int E = (c1 - c0) + 2 * H;          // cells of the extended chunk, from global c0 - H
  const int lo = t * R;
  const S* __restrict__ U0 = static_cast<const S*>(a.u);
  const A* __restrict__ FX = static_cast<const A*>(a.fx);
  auto wrapn = [n](int g) { return g < 0 ? g + n : (g >= n ? g - n : g); };  // |g| < 2n here

  S U[R], V[R];
  A kf[R + 1];           // faces west of the held cells, and east of the last
  unsigned live = 0;     // bit i: held cell i is updated (in the extended chunk and the grid)
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = lo + i, g = c0 - H + e;
    const bool in = e < E && (PERIODIC || (g >= 0 && g < n));
    if (in) live |= 1u << i;
    const int gi = PERIODIC ? wrapn(g) : g;
    U[i] = in && in_bounds(gi >= 0 && gi < n, a.status) ? U0[gi] : S(0);
    V[i] = S(0);
  }
#pragma unroll
  for (int i = 0; i <= R; ++i) {
    const int e = lo + i, g = c0 - H + e;  // face g lies between cells g - 1 and g
    A v = A(0);
    if (e <= E) {
      const int fi = PERIODIC ? wrapn(g) : g;
      if ((PERIODIC || (g >= 0 && g <= n)) && in_bounds(fi >= 0 && fi <= n, a.status)) v = FX[fi];
    }
    kf[i] = v;
  }
  for (int l = t; l < a.s; l += nt) {
    cs[0][l] = S(a.ca[l]);
    cs[1][l] = S(a.cb[l]);
  }
  cluster.sync();  // every CTA of the cluster is running before any remote access

  bool bad = false;
  int par = 0, xpar = 0, since = 0;  // stages since the last halo exchange (the halo starts exact)
  for (int step = 0; step < a.nsteps; ++step) {
    for (int l = 0; l < a.s; ++l, par ^= 1) {
      if (H > 0 && since == H) {
        // halo exchange: the chunk's own first and last H cells out, the neighbours' in
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int e = lo + i;
          S2 v;
          v.x = U[i];
          v.y = V[i];
          if (e >= H && e < 2 * H && in_bounds(e - H < S1_HMAX, a.status)) own_lo[xpar][e - H] = v;
          if (e >= E - 2 * H && e < E - H && in_bounds(e - (E - 2 * H) < S1_HMAX, a.status))
            own_hi[xpar][e - (E - 2 * H)] = v;
        }
        cluster.sync();
        const S2* rlo = cluster.map_shared_rank(&own_hi[xpar][0], cp);  // global cells c0 - H .. c0 - 1
        const S2* rhi = cluster.map_shared_rank(&own_lo[xpar][0], cn);  // global cells c1 .. c1 + H - 1
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int e = lo + i;
          if (live & (1u << i)) {
            if (e < H) {
              const S2 v = rlo[e];
              U[i] = v.x;
              V[i] = v.y;
            } else if (e >= E - H) {
              const S2 v = rhi[e - (E - H)];
              U[i] = v.x;
              V[i] = v.y;
            }
          }
        }
        xpar ^= 1;
        since = 0;
      }
      // west neighbour of the first cell, east neighbour of the last: the adjacent lanes; at a
      // warp's ends the adjacent warps' end lanes through shared memory; beyond the extended
      // chunk's ends zero (a stale halo's neighbour, or a Dirichlet ghost)
      S wU = __shfl_up_sync(0xffffffffu, U[R - 1], 1), wV = __shfl_up_sync(0xffffffffu, V[R - 1], 1);
      S eU = __shfl_down_sync(0xffffffffu, U[0], 1), eV = __shfl_down_sync(0xffffffffu, V[0], 1);
      if (nw > 1) {
        if (lane == 0) wlo[par][wid] = S2{U[0], V[0]};
        if (lane == 31) whi[par][wid] = S2{U[R - 1], V[R - 1]};
        __syncthreads();
        if (lane == 0) {
          const S2 v = wid > 0 ? whi[par][wid - 1] : S2{S(0), S(0)};
          wU = v.x;
          wV = v.y;
        }
        if (lane == 31) {
          const S2 v = wid < nw - 1 ? wlo[par][wid + 1] : S2{S(0), S(0)};
          eU = v.x;
          eV = v.y;
        }
      } else {
        if (lane == 0) wU = wV = S(0);
        if (lane == 31) eU = eV = S(0);
      }
      const S ca = cs[0][l], cb = cs[1][l];
      // d across the thread's first face, then cell by cell
      A dU = A(U[0] - wU), dV = A(V[0] - wV);
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const S nU = i + 1 < R ? U[i + 1 < R ? i + 1 : i] : eU;
        const S nV = i + 1 < R ? V[i + 1 < R ? i + 1 : i] : eV;
        const A xU = A(nU - U[i]), xV = A(nV - V[i]);
        const A fU = fma(kf[i + 1], xU, -mul_rn(kf[i], dU));
        const A fV = fma(kf[i + 1], xV, -mul_rn(kf[i], dV));
        if (live & (1u << i)) {
          U[i] = fma(-cb, S(fV), fma(ca, S(fU), U[i]));
          V[i] = fma(cb, S(fU), fma(ca, S(fV), V[i]));
        }
        dU = xU;
        dV = xV;
      }
      if (l == a.s - 1) {  // step output: the real part
#pragma unroll
        for (int i = 0; i < R; ++i) V[i] = S(0);
      }
      ++since;
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = lo + i;
    if (e >= H && e < E - H && in_bounds(c0 - H + e >= 0 && c0 - H + e < n, a.status)) {
      static_cast<S*>(a.u)[c0 - H + e] = U[i];
      bad |= bad1(U[i]);
    }
  }
  if (bad) atomicOr(a.status, ST_NONFINITE);
}

template <class S, class A, bool PERIODIC, int R>
cudaError_t launch_r(const Small1dArgs& a, int CL, int threads, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_small1d<S, A, PERIODIC, R>, a);
  count_launch();
  return e;
}

template <class S, class A, bool PERIODIC>
cudaError_t launch_t(const Small1dArgs& a, int CL, int threads, int R, cudaStream_t st) {
  switch (R) {
    case 1: return launch_r<S, A, PERIODIC, 1>(a, CL, threads, st);
    case 2: return launch_r<S, A, PERIODIC, 2>(a, CL, threads, st);
    case 4: return launch_r<S, A, PERIODIC, 4>(a, CL, threads, st);
    case 8: return launch_r<S, A, PERIODIC, 8>(a, CL, threads, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool small1d_supported(const frkc2_problem& p, int s) {
  return p.ndim == 1 && p.kappa_kind != FRKC2_KAPPA_POWER && s <= S1_MAXS && p.n[0] >= 1 &&
         p.n[0] <= int64_t(S1_CMAX) * S1_TMAX * S1_RMAX / 2 &&
         (p.precision == FRKC2_FP64 || p.precision == FRKC2_FP32 || p.precision == FRKC2_MIXED);
}

cudaError_t launch_small1d(const frkc2_problem& p, const frkc2_plan_s& plan, double dt, int nsteps, void* u,
                           const void* fx, unsigned* status, cudaStream_t st, int cluster, int stages_per_exchange,
                           int threads_per_cta) {
  const int n = int(p.n[0]);
  const bool periodic = p.bc == FRKC2_BC_PERIODIC;
  // cluster size (or the caller's): 32 cells a CTA, up to 8 CTAs (N = 256: FP64 0.89 ms a job
  // against 1.22 in one CTA, FP32 0.16 against 0.20)
  const bool f32 = p.precision == FRKC2_FP32;
  int CL = cluster > 0 ? std::min(S1_CMAX, std::min(cluster, n)) : std::max(1, std::min(S1_CMAX, n / 32));
  CL = std::max(CL, (n + S1_TMAX * S1_RMAX / 2 - 1) / (S1_TMAX * S1_RMAX / 2));  // room for a halo
  if (CL > S1_CMAX) return cudaErrorInvalidValue;
  const int chunk = (n + CL - 1) / CL, min_chunk = n / CL;
  // halo cells = stages per exchange (default 16): at most the smallest chunk (a halo comes
  // from one neighbour); none for a Dirichlet grid in one CTA
  int H = 0;
  if (CL > 1 || periodic) {
    H = stages_per_exchange > 0 ? stages_per_exchange : 16;
    H = std::min(H, std::min(S1_HMAX, min_chunk));
    if (H < 1) return cudaErrorInvalidValue;
  }
  const int ext = chunk + 2 * H;
  // threads per CTA (a multiple of 32, at most 512) and cells per thread (1, 2, 4 or 8): the
  // caller's thread count, raised to what holds the extended chunk; by default in FP32 one
  // warp while it holds the extended chunk (no CTA barrier), in FP64 and MIXED one cell a
  // thread (the FP64 instructions of a stage spread over the SM's schedulers)
  int threads = threads_per_cta > 0 ? ((threads_per_cta + 31) / 32) * 32
                                    : (f32 ? 32 : std::min(S1_TMAX, ((ext + 31) / 32) * 32));
  threads = std::max(threads, ((ext + S1_RMAX * 32 - 1) / (S1_RMAX * 32)) * 32);
  if (threads > S1_TMAX) return cudaErrorInvalidValue;
  int R = 1;
  while (R * threads < ext) R *= 2;
  if (R > S1_RMAX) return cudaErrorInvalidValue;
  auto a = std::make_unique<Small1dArgs>();
  a->u = u;
  a->fx = fx;
  a->status = status;
  a->n = n;
  a->nsteps = nsteps;
  a->s = plan.s;
  a->H = H;
  const double h2 = p.dx * p.dx;
  for (int l = 0; l < plan.s; ++l) {
    a->ca[l] = dt * plan.a_re[l] / h2;
    a->cb[l] = dt * plan.a_im[l] / h2;
  }
  switch (p.precision) {
    case FRKC2_FP64:
      return periodic ? launch_t<double, double, true>(*a, CL, threads, R, st)
                      : launch_t<double, double, false>(*a, CL, threads, R, st);
    case FRKC2_FP32:
      return periodic ? launch_t<float, float, true>(*a, CL, threads, R, st)
                      : launch_t<float, float, false>(*a, CL, threads, R, st);
    default:
      return periodic ? launch_t<double, float, true>(*a, CL, threads, R, st)
                      : launch_t<double, float, false>(*a, CL, threads, R, st);
  }
}

}  // namespace frkc2
