// Whole-job kernel for small 1D problems: every stage of every step in one launch on a
// thread-block cluster, the state never leaving the chip.
//
// The N cells are split into CL contiguous chunks, one per CTA of a cluster of CL <= 8 CTAs
// (co-scheduled by the hardware); thread t of a CTA holds R consecutive cells of its chunk in
// registers (complex state and the R + 1 face conductivities around them) for the whole job.
// Per stage each thread publishes its first and last cell in shared memory (double-buffered
// by stage parity), the cluster meets at one hardware barrier, and each thread reads the
// neighbour cell beyond either end from the adjacent thread -- or, at a chunk end, from the
// adjacent CTA's shared memory through the cluster's distributed shared memory.  The stage
// shares each neighbour difference d_i = W_i - W_{i-1} between the two cells of face i:
// f_i = kappa_{i+1} d_{i+1} - kappa_i d_i, then W_i += dt a_l f_i / dx^2 (Sec. 3, Eq. 13):
// 10 floating-point instructions per cell-stage.  At the end of each step the state is Re W^L.
// The stage coefficients of the whole plan (up to 1024 stages) travel in the parameter block.
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
constexpr int S1_TMAX = 256;    // threads per CTA
constexpr int S1_CMAX = 8;      // CTAs per cluster (portable size)

template <class T> struct V2o;
template <> struct V2o<double> { using type = double2; };
template <> struct V2o<float> { using type = float2; };

struct Small1dArgs {
  void* u;               // caller's real state, read at the start and written at the end
  const void* fx;        // face conductivities, N + 1 (face i between cells i - 1 and i)
  unsigned* status;
  int n, nsteps, s;
  int R;                 // cells per thread
  double ca[S1_MAXS];    // dt Re a_l / dx^2
  double cb[S1_MAXS];    // dt Im a_l / dx^2
};

__device__ __forceinline__ bool bad1(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool bad1(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }

template <class S, class A, bool PERIODIC>
__global__ void __launch_bounds__(S1_TMAX) k_small1d(const Small1dArgs a) {
  using S2 = typename V2o<S>::type;
  __shared__ S2 edge_lo[2][S1_TMAX];  // each thread's first cell, by stage parity
  __shared__ S2 edge_hi[2][S1_TMAX];  // its last cell
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = int(cluster.num_blocks());
  const int c = int(cluster.block_rank());
  const int t = threadIdx.x;
  const int n = a.n, R = a.R;
  // chunk of this CTA and of the previous one (for the index of its last occupied thread)
  const int c0 = int((long long)c * n / CL), c1 = int((long long)(c + 1) * n / CL);
  const int cp = (c + CL - 1) % CL, cn = (c + 1) % CL;
  const int p0 = int((long long)cp * n / CL), p1 = int((long long)(cp + 1) * n / CL);
  const int prev_last = (p1 - p0 - 1) / R;  // occupied thread holding the previous chunk's end
  const int lo = c0 + t * R, hi = min(lo + R, c1);
  const int m = max(0, hi - lo);  // cells held by this thread
  const S* __restrict__ U0 = static_cast<const S*>(a.u);
  const A* __restrict__ FX = static_cast<const A*>(a.fx);

  S U[S1_RMAX], V[S1_RMAX];
  A kf[S1_RMAX + 1];  // faces lo .. lo + m
#pragma unroll
  for (int i = 0; i < S1_RMAX; ++i) {
    U[i] = i < m ? U0[lo + i] : S(0);
    V[i] = S(0);
  }
#pragma unroll
  for (int i = 0; i <= S1_RMAX; ++i) kf[i] = i <= m && m > 0 ? FX[lo + i] : A(0);
  cluster.sync();  // every CTA of the cluster is running before any remote access

  bool bad = false;
  int par = 0;
  for (int step = 0; step < a.nsteps; ++step) {
    for (int l = 0; l < a.s; ++l, par ^= 1) {
      if (m > 0) {
        S2 e;
        e.x = U[0];
        e.y = V[0];
        edge_lo[par][t] = e;
        // the last held cell, selected without a run-time register index (which would move
        // the arrays to local memory)
#pragma unroll
        for (int i = 1; i < S1_RMAX; ++i) {
          e.x = i < m ? U[i] : e.x;
          e.y = i < m ? V[i] : e.y;
        }
        edge_hi[par][t] = e;
      }
      cluster.sync();
      if (m > 0) {
        // west neighbour of the first cell, east neighbour of the last cell
        S2 w, ea;
        w.x = w.y = ea.x = ea.y = S(0);
        if (lo > c0) {
          w = edge_hi[par][t - 1];
        } else if (PERIODIC || c > 0) {
          const S2* rem = cluster.map_shared_rank(&edge_hi[par][0], cp);
          w = rem[prev_last];
        }
        if (hi < c1) {
          ea = edge_lo[par][t + 1];
        } else if (PERIODIC || c < CL - 1) {
          const S2* rem = cluster.map_shared_rank(&edge_lo[par][0], cn);
          ea = rem[0];
        }
        const S ca = S(a.ca[l]), cb = S(a.cb[l]);
        // d across the thread's first face, then cell by cell
        A dU = A(U[0] - w.x), dV = A(V[0] - w.y);
#pragma unroll
        for (int i = 0; i < S1_RMAX; ++i) {
          if (i < m) {
            const int in = i + 1 < S1_RMAX ? i + 1 : i;  // a compile-time index inside the array
            const S nU = i + 1 < m ? U[in] : ea.x;
            const S nV = i + 1 < m ? V[in] : ea.y;
            const A eU = A(nU - U[i]), eV = A(nV - V[i]);
            const A fU = kf[i + 1] * eU - kf[i] * dU;
            const A fV = kf[i + 1] * eV - kf[i] * dV;
            U[i] = U[i] + ca * S(fU) - cb * S(fV);
            V[i] = V[i] + ca * S(fV) + cb * S(fU);
            dU = eU;
            dV = eV;
          }
        }
        if (l == a.s - 1) {  // step output: the real part
#pragma unroll
          for (int i = 0; i < S1_RMAX; ++i) V[i] = S(0);
        }
      }
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
#pragma unroll
  for (int i = 0; i < S1_RMAX; ++i)
    if (i < m) {
      static_cast<S*>(a.u)[lo + i] = U[i];
      bad |= bad1(U[i]);
    }
  if (bad) atomicOr(a.status, ST_NONFINITE);
}

template <class S, class A, bool PERIODIC>
cudaError_t launch_t(const Small1dArgs& a, int CL, int threads, cudaStream_t st) {
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
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_small1d<S, A, PERIODIC>, a);
  count_launch();
  return e;
}

}  // namespace

bool small1d_supported(const frkc2_problem& p, int s) {
  return p.ndim == 1 && p.kappa_kind != FRKC2_KAPPA_POWER && s <= S1_MAXS && p.n[0] >= 1 &&
         p.n[0] <= int64_t(S1_CMAX) * S1_TMAX * S1_RMAX &&
         (p.precision == FRKC2_FP64 || p.precision == FRKC2_FP32 || p.precision == FRKC2_MIXED);
}

cudaError_t launch_small1d(const frkc2_problem& p, const frkc2_plan_s& plan, double dt, int nsteps, void* u,
                           const void* fx, unsigned* status, cudaStream_t st, int cluster) {
  const int n = int(p.n[0]);
  // cluster size (or the caller's): the per-stage cluster barrier grows with the CTAs, the
  // FP64 pipe time per stage shrinks with them -- FP64 state spreads 128 cells a CTA (N = 256:
  // 2 CTAs, 1.44 ms a job against 1.52 with 8), FP32 keeps one CTA while it fits (0.87 ms
  // against 1.00)
  const bool f32 = p.precision == FRKC2_FP32;
  int CL = cluster > 0 ? std::min(S1_CMAX, std::min(cluster, n))
                       : (f32 ? 1 : std::max(1, std::min(S1_CMAX, n / 128)));
  CL = std::max(CL, (n + S1_TMAX * S1_RMAX - 1) / (S1_TMAX * S1_RMAX));  // at most S1_RMAX cells a thread
  const int chunk = (n + CL - 1) / CL;
  // threads per CTA: a multiple of 32, at most 256, holding at most S1_RMAX cells each
  int threads = std::min(S1_TMAX, ((chunk + 31) / 32) * 32);
  int R = (chunk + threads - 1) / threads;
  if (R > S1_RMAX) return cudaErrorInvalidValue;
  auto a = std::make_unique<Small1dArgs>();
  a->u = u;
  a->fx = fx;
  a->status = status;
  a->n = n;
  a->nsteps = nsteps;
  a->s = plan.s;
  a->R = R;
  const double h2 = p.dx * p.dx;
  for (int l = 0; l < plan.s; ++l) {
    a->ca[l] = dt * plan.a_re[l] / h2;
    a->cb[l] = dt * plan.a_im[l] / h2;
  }
  const bool per = p.bc == FRKC2_BC_PERIODIC;
  switch (p.precision) {
    case FRKC2_FP64:
      return per ? launch_t<double, double, true>(*a, CL, threads, st) : launch_t<double, double, false>(*a, CL, threads, st);
    case FRKC2_FP32:
      return per ? launch_t<float, float, true>(*a, CL, threads, st) : launch_t<float, float, false>(*a, CL, threads, st);
    default:
      return per ? launch_t<double, float, true>(*a, CL, threads, st) : launch_t<double, float, false>(*a, CL, threads, st);
  }
}

}  // namespace frkc2
