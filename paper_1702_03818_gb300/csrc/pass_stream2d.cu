// 2D single-stage pass (k = 1) streaming straight from global memory, for the fixed
// conductivity (FIELD / CONST) flux-form operator.
//
// Each warp owns 31 consecutive columns plus one halo lane on the low-x side and walks rows
// upward.  Every face flux kappa_f (W_nb - W_c) is computed once and used by both cells of
// the face: the x flux of a lane's east face reaches the next lane through a warp shuffle
// (the halo lane supplies the chunk's west edge), and the y flux of a cell's north face is
// carried in registers as the next row's south flux.  Per cell and stage this leaves 2
// differences, 2 products and 3 sums for each of U and V plus 4 fused multiply-adds for the
// complex update -- 18 floating-point instructions, which is what bounds the FP64 path on
// GB300 (its FP64 pipe issues 2 lanes per clock per SM, far below its memory system).
//
// Work split: the grid is persistent (every CTA resident) and the (column chunk, row)
// pairs, chunk-major, are cut into one contiguous range per warp, so every SM gets the same
// number of cell updates.  A range that crosses into the next chunk restarts the stream.
#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int ST_THREADS = 256;
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int ST_COLS = 31;  // output columns per warp
constexpr int ST_MIN_BLOCKS = 6;

__device__ __forceinline__ bool nonfinite_bits(double v) {
  return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool nonfinite_bits(float v) {
  return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

template <class S, class A, bool PERIODIC>
__global__ void __launch_bounds__(ST_THREADS, ST_MIN_BLOCKS)
    k_stream2d(const PassArgs p, int ncolw, long long total, long long nwarps_grid) {
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * ST_WARPS + (threadIdx.x >> 5);
  const int nx = p.nx, ny = p.ny;
  long long idx = gw * total / nwarps_grid;
  const long long end = (gw + 1) * total / nwarps_grid;
  const S* __restrict__ U = static_cast<const S*>(p.U_in);
  const S* __restrict__ V = static_cast<const S*>(p.V_in);
  const A* __restrict__ FX = static_cast<const A*>(p.fx);
  const A* __restrict__ FY = static_cast<const A*>(p.fy);
  S* __restrict__ Uo = static_cast<S*>(p.U_out);
  S* __restrict__ Vo = static_cast<S*>(p.V_out);
  const bool hasV = V != nullptr;
  const S ca = S(p.ca[0]), cb = S(p.cb[0]);
  bool bad = false;

  while (idx < end) {  // warp-uniform
    const int wcol = int(idx / ny);
    const int y0 = int(idx - (long long)wcol * ny);
    const int y1 = int(min((long long)ny, (long long)y0 + (end - idx)));
    idx += y1 - y0;
    const int x = wcol * ST_COLS + lane - 1;

    // column read by this lane, and whether it holds a real cell
    int xr;
    bool xin;
    if (PERIODIC) {
      xr = ((x % nx) + nx) % nx;
      xin = true;
    } else {
      xr = x;
      xin = x >= 0 && x < nx;
    }
    // east face of the lane's cell: face index xr + 1 (x faces have nx + 1 entries per row)
    const bool has_east_face = PERIODIC ? true : (x >= -1 && x < nx);
    const int xe_face = PERIODIC ? xr + 1 : x + 1;
    // lane 31 reads its east neighbour itself
    int xeast;
    bool eastin;
    if (PERIODIC) {
      xeast = xr + 1 == nx ? 0 : xr + 1;
      eastin = true;
    } else {
      xeast = x + 1;
      eastin = xeast >= 0 && xeast < nx;
    }
    const bool out_ok = lane >= 1 && x >= 0 && x < nx;

    auto load = [&](const S* __restrict__ P, int yy, int xx, bool inx) -> S {
      if (PERIODIC) {
        const int yw = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        return P[size_t(yw) * nx + xx];
      }
      return (inx && yy >= 0 && yy < ny) ? P[size_t(yy) * nx + xx] : S(0);
    };
    // y face j (between rows j-1 and j) of this lane's column
    auto yface = [&](int j) -> A {
      if (PERIODIC) return FY[size_t(j) * nx + xr];
      return xin ? FY[size_t(j) * nx + xr] : A(0);
    };

    // prime the stream: the cell row y0 and the flux through its south face
    S Uc = load(U, y0, xr, xin);
    S Vc = hasV ? load(V, y0, xr, xin) : S(0);
    A FsU, FsV;
    {
      const S Us = load(U, y0 - 1, xr, xin);
      const S Vs = hasV ? load(V, y0 - 1, xr, xin) : S(0);
      const A ks = yface(y0);
      FsU = ks * A(Us - Uc);
      FsV = ks * A(Vs - Vc);
    }
    for (int y = y0; y < y1; ++y) {
      const S Un = load(U, y + 1, xr, xin);
      const S Vn = hasV ? load(V, y + 1, xr, xin) : S(0);
      const A kn = yface(y + 1);
      const A ke = has_east_face ? FX[size_t(y) * (nx + 1) + xe_face] : A(0);
      S Ue = __shfl_down_sync(0xffffffffu, Uc, 1);
      S Ve = __shfl_down_sync(0xffffffffu, Vc, 1);
      if (lane == 31) {
        Ue = load(U, y, xeast, eastin);
        Ve = hasV ? load(V, y, xeast, eastin) : S(0);
      }
      const A FnU = kn * A(Un - Uc), FnV = kn * A(Vn - Vc);
      const A FeU = ke * A(Ue - Uc), FeV = ke * A(Ve - Vc);
      const A FwU = -__shfl_up_sync(0xffffffffu, FeU, 1);
      const A FwV = -__shfl_up_sync(0xffffffffu, FeV, 1);
      const A fU = (FeU + FwU) + (FnU + FsU);
      const A fV = (FeV + FwV) + (FnV + FsV);
      const S un = Uc + ca * S(fU) - cb * S(fV);
      const S vn = Vc + ca * S(fV) + cb * S(fU);
      if (out_ok) {
        const size_t g = size_t(y) * nx + x;
        Uo[g] = un;
        if (Vo) Vo[g] = vn;
        if (p.check_finite) bad |= nonfinite_bits(un);
      }
      FsU = -FnU;
      FsV = -FnV;
      Uc = Un;
      Vc = Vn;
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

template <class S, class A, bool PERIODIC>
cudaError_t launch_t(const PassArgs& a, cudaStream_t st) {
  static int blocks_per_sm = 0, sms = 0;
  auto kern = k_stream2d<S, A, PERIODIC>;
  if (!blocks_per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, ST_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int ncolw = (a.nx + ST_COLS - 1) / ST_COLS;
  const long long total = (long long)ncolw * a.ny;  // (chunk, row) pairs
  long long grid = (long long)sms * blocks_per_sm;
  const long long max_useful = (total + ST_WARPS - 1) / ST_WARPS;
  if (grid > max_useful) grid = max_useful;
  kern<<<unsigned(grid), ST_THREADS, 0, st>>>(a, ncolw, total, grid * ST_WARPS);
  count_launch();
  return cudaGetLastError();
}

template <class S, class A>
cudaError_t launch_s(const PassArgs& a, cudaStream_t st) {
  return a.bc == FRKC2_BC_PERIODIC ? launch_t<S, A, true>(a, st) : launch_t<S, A, false>(a, st);
}

}  // namespace

cudaError_t launch_pass_stream2d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st) {
  switch (p.precision) {
    case FRKC2_FP64: return launch_s<double, double>(a, st);
    case FRKC2_FP32: return launch_s<float, float>(a, st);
    default: return launch_s<double, float>(a, st);
  }
}

}  // namespace frkc2
