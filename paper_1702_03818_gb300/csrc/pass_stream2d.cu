// 2D single-stage pass (k = 1) streaming straight from global memory, for the fixed
// conductivity (FIELD / CONST) flux-form operator.
//
// Each warp owns 31 consecutive columns plus one halo lane on the low-x side and walks a
// strip of rows upward.  Every face flux kappa_f (W_nb - W_c) is computed once and used by
// both cells of the face: the x flux of a lane's east face reaches the next lane through a
// warp shuffle (the halo lane supplies the strip's west edge), and the y flux of a cell's
// north face is carried in registers as the next row's south flux.  Per cell and stage this
// leaves 2 differences, 2 products and 3 sums for each of U and V plus 4 fused
// multiply-adds for the complex update -- 18 floating-point instructions, which is what
// bounds the FP64 path on GB300 (its FP64 pipe is far narrower than its memory system).
#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int ST_THREADS = 256;
constexpr int ST_COLS = 31;  // output columns per warp

template <class S, class A, bool PERIODIC>
__global__ void __launch_bounds__(ST_THREADS) k_stream2d(const PassArgs p, int rows, int ncolw,
                                                          int nwarps) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (ST_THREADS / 32) + (threadIdx.x >> 5);
  if (gw >= nwarps) return;  // whole warp leaves together
  const int wcol = gw % ncolw, wrow = gw / ncolw;
  const int nx = p.nx, ny = p.ny;
  const int x = wcol * ST_COLS + lane - 1;
  const int y0 = wrow * rows;
  const int y1 = min(y0 + rows, ny);
  const S* __restrict__ U = static_cast<const S*>(p.U_in);
  const S* __restrict__ V = static_cast<const S*>(p.V_in);
  const A* __restrict__ FX = static_cast<const A*>(p.fx);
  const A* __restrict__ FY = static_cast<const A*>(p.fy);
  S* __restrict__ Uo = static_cast<S*>(p.U_out);
  S* __restrict__ Vo = static_cast<S*>(p.V_out);
  const bool hasV = V != nullptr;

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
  const S ca = S(p.ca[0]), cb = S(p.cb[0]);

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

  // prime the strip: south neighbour and the flux through the strip's lowest face
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
      if (p.check_finite && !isfinite(double(un))) atomicOr(p.status, ST_NONFINITE);
    }
    FsU = -FnU;
    FsV = -FnV;
    Uc = Un;
    Vc = Vn;
  }
}

template <class S, class A>
cudaError_t launch_s(const PassArgs& a, cudaStream_t st) {
  const int rows = a.ty > 0 ? a.ty : 64;
  const int ncolw = (a.nx + ST_COLS - 1) / ST_COLS;
  const int nroww = (a.ny + rows - 1) / rows;
  const int nwarps = ncolw * nroww;
  const int wpb = ST_THREADS / 32;
  const int grid = (nwarps + wpb - 1) / wpb;
  if (a.bc == FRKC2_BC_PERIODIC)
    k_stream2d<S, A, true><<<grid, ST_THREADS, 0, st>>>(a, rows, ncolw, nwarps);
  else
    k_stream2d<S, A, false><<<grid, ST_THREADS, 0, st>>>(a, rows, ncolw, nwarps);
  count_launch();
  return cudaGetLastError();
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
