// 3D single-stage pass (k = 1) streaming along z, for every conductivity kind and precision.
//
// A CTA is TY warps; warp w is grid row y = by (TY - 2) + w - 1 and lane l is column
// x = bx 30 + l - 1, so the CTA covers a 32 x TY column block whose outer lanes and rows are
// halo: it outputs the 30 x (TY - 2) interior columns.  The CTA walks up its z chunk; each
// thread keeps its own column's W(z), W(z+1) (and for kappa(u) the conductivities of both)
// and the flux through its down face in registers.  Per plane:
//   - x neighbours come by warp shuffle, y neighbours through a shared plane (W, and kappa
//     for kappa(u)), double-buffered by z parity;
//   - each cell forms the fluxes through its east, north and up faces, F = kappa_f (W_nb - W_c);
//     the west flux is lane - 1's east flux (shuffle), the south flux row - 1's north flux (a
//     second shared plane), the down flux the up flux of the plane below (register):
//     f = (F_e - F_w) + (F_n - F_s) + (F_u - F_d), every face flux formed once;
//   - for kappa(u) = 1 + c u^p every cell's kappa(W) is evaluated once per stage (when its
//     plane is loaded) and a face takes kappa_c + kappa_nb, the factor 1/2 folded into the
//     stage coefficients; for FIELD / CONST the face conductivities are read from the face
//     arrays.
// Work per output cell-stage: the halo lanes and rows add 32 TY / (30 (TY - 2)) (1.22 for
// TY = 16); no other redundant work, against the (T + 2)^3 / T^3 halo of a tile pass.
#include <algorithm>
#include <type_traits>

#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "frkc2_math.cuh"

namespace frkc2 {
namespace {

#ifndef FRKC2_S3_TY
#define FRKC2_S3_TY 16
#endif
constexpr int S3_TY = FRKC2_S3_TY;  // warps (grid rows incl. 2 halo rows) per CTA
constexpr int S3_THREADS = 32 * S3_TY;
constexpr int S3_OX = 30, S3_OY = S3_TY - 2;  // output columns / rows per CTA

template <class T> struct V2s;
template <> struct V2s<double> { using type = double2; };
template <> struct V2s<float> { using type = float2; };

__device__ __forceinline__ bool nonfinite3(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool nonfinite3(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }

__device__ __forceinline__ int wrap3(int g, int n) {
  if (g < 0) g += n;
  while (g >= n) g -= n;
  return g;
}

// P25: kappa(u) with the exponent 2.5, evaluated as w^2 sqrt(w) without the general path
template <class S, class A, bool PERIODIC, bool POWER, bool P25>
__global__ void __launch_bounds__(S3_THREADS) k_stream3d(const PassArgs p, int zchunk) {
  // launched with programmatic stream serialization: the next launch may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  using S2 = typename V2s<S>::type;
  using A2 = typename V2s<A>::type;
  __shared__ S2 shW[2][S3_TY][32];
  __shared__ A2 shK[2][S3_TY][POWER ? 32 : 1];
  __shared__ A2 shF[2][S3_TY][32];
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int gx = blockIdx.x * S3_OX + lane - 1;
  const int gy = blockIdx.y * S3_OY + row - 1;
  const int z0 = blockIdx.z * zchunk, z1 = min(nz, z0 + zchunk);
  const int xr = PERIODIC ? wrap3(gx, nx) : gx;
  const int yr = PERIODIC ? wrap3(gy, ny) : gy;
  const bool colin = PERIODIC || (gx >= 0 && gx < nx && gy >= 0 && gy < ny);
  const bool out_ok = lane >= 1 && lane <= 30 && row >= 1 && row <= S3_TY - 2 && gx < nx && gy < ny && gx >= 0 &&
                      gy >= 0;
  const size_t plane = size_t(nx) * ny;
  const size_t col = size_t(yr) * nx + xr;  // in-plane offset of this thread's column (if colin)
  const int in_mode = p.in_mode, out_mode = p.out_mode;
  const S* __restrict__ Ur = static_cast<const S*>(p.U_in);
  const S* __restrict__ Vr = static_cast<const S*>(p.V_in);
  S* __restrict__ Uo = static_cast<S*>(p.U_out);
  S* __restrict__ Vo = static_cast<S*>(p.V_out);
  const A* __restrict__ FX = static_cast<const A*>(p.fx);
  const A* __restrict__ FY = static_cast<const A*>(p.fy);
  const A* __restrict__ FZ = static_cast<const A*>(p.fz);
  // kappa(u): the face factor 1/2 of (kappa_c + kappa_nb)/2 is folded into the coefficients
  const S ca = S(POWER ? 0.5 * p.ca[0] : p.ca[0]), cb = S(POWER ? 0.5 * p.cb[0] : p.cb[0]);
  const A kc = A(p.kc), kp = A(p.kp);

  auto load = [&](int z) -> S2 {
    S2 w;
    w.x = S(0);
    w.y = S(0);
    int zz = z;
    if (PERIODIC) {
      zz = wrap3(z, nz);
    } else if (!colin || z < 0 || z >= nz) {
      return w;
    }
    const size_t g = size_t(zz) * plane + col;
    if (!in_bounds(g < size_t(nz) * plane, p.status)) return w;
    w.x = __ldg(Ur + g);
    if (in_mode == PASS_IO_PLANAR) w.y = __ldg(Vr + g);
    return w;
  };
  // face array sizes, for the bounds-checking build's index checks
  const size_t nfx = size_t(nz) * ny * (nx + 1), nfy = size_t(nz) * (ny + 1) * nx, nfz = size_t(nz + 1) * ny * nx;
  auto ldf = [&](const A* F, size_t i, size_t n) -> A { return in_bounds(i < n, p.status) ? __ldg(F + i) : A(0); };
  auto kap = [&](S2 w) -> A2 {
    A2 k;
    if constexpr (P25)
      kappa_power25<A>(A(w.x), A(w.y), kc, k.x, k.y);
    else
      kappa_power<A>(A(w.x), A(w.y), kc, kp, k.x, k.y);
    return k;
  };
  // face conductivities (FIELD / CONST): east (x face x+1), north (y face y+1), up (z face z+1)
  auto face_e = [&](int z) -> A {
    if (PERIODIC) return ldf(FX, (size_t(wrap3(z, nz)) * ny + yr) * (nx + 1) + xr + 1, nfx);
    if (z < 0 || z >= nz || gy < 0 || gy >= ny || gx < -1 || gx >= nx) return A(0);
    return ldf(FX, (size_t(z) * ny + gy) * (nx + 1) + gx + 1, nfx);
  };
  auto face_n = [&](int z) -> A {
    if (PERIODIC) return ldf(FY, (size_t(wrap3(z, nz)) * (ny + 1) + yr + 1) * nx + xr, nfy);
    if (z < 0 || z >= nz || gx < 0 || gx >= nx || gy < -1 || gy >= ny) return A(0);
    return ldf(FY, (size_t(z) * (ny + 1) + gy + 1) * nx + gx, nfy);
  };
  auto face_u = [&](int z) -> A {  // z face z+1, above cell z
    if (PERIODIC) return ldf(FZ, (size_t(wrap3(z, nz) + 1) * ny + yr) * nx + xr, nfz);
    if (!colin || z < -1 || z >= nz) return A(0);
    return ldf(FZ, (size_t(z + 1) * ny + gy) * nx + gx, nfz);
  };
  // complex flux kappa_f * d with kappa_f real (FIELD) or complex (kappa(u))
  auto flux = [&](A2 kf, A dr, A di) -> A2 {
    A2 F;
    if (POWER) {
      F.x = kf.x * dr - kf.y * di;
      F.y = kf.x * di + kf.y * dr;
    } else {
      F.x = kf.x * dr;
      F.y = kf.x * di;
    }
    return F;
  };

  // prime: W(z0 - 1), W(z0), W(z0 + 1) and the flux through the down face of z0
  S2 Wc = load(z0), Wp = load(z0 + 1);
  A2 Kc, Kp;
  A2 Fd;
  {
    const S2 Wm = load(z0 - 1);
    A2 kf;
    if (POWER) {
      Kc = kap(Wc);
      Kp = kap(Wp);
      const A2 Km = kap(Wm);
      kf.x = Km.x + Kc.x;
      kf.y = Km.y + Kc.y;
    } else {
      kf.x = face_u(z0 - 1);
      kf.y = A(0);
    }
    Fd = flux(kf, A(Wc.x - Wm.x), A(Wc.y - Wm.y));
  }
  bool bad = false;
  for (int z = z0; z < z1; ++z) {
    const int b = z & 1;
    const S2 Wpp = load(z + 2);  // the plane after next, issued early
    A ke = A(0), kn = A(0), ku = A(0);
    if (!POWER) {
      ke = face_e(z);
      kn = face_n(z);
      ku = face_u(z);
    }
    shW[b][row][lane] = Wc;
    if (POWER) shK[b][row][lane] = Kc;
    __syncthreads();
    // east neighbour by shuffle (lane 31 is a halo lane: its east values are not used)
    S2 We;
    We.x = __shfl_down_sync(0xffffffffu, Wc.x, 1);
    We.y = __shfl_down_sync(0xffffffffu, Wc.y, 1);
    const int rn = row + 1 < S3_TY ? row + 1 : row;  // the top halo row has no north cell here
    const S2 Wn = shW[b][rn][lane];
    A2 kfe, kfn, kfu;
    if (POWER) {
      A2 Ke, Kn;
      Ke.x = __shfl_down_sync(0xffffffffu, Kc.x, 1);
      Ke.y = __shfl_down_sync(0xffffffffu, Kc.y, 1);
      Kn = shK[b][rn][lane];
      kfe.x = Kc.x + Ke.x;
      kfe.y = Kc.y + Ke.y;
      kfn.x = Kc.x + Kn.x;
      kfn.y = Kc.y + Kn.y;
      kfu.x = Kc.x + Kp.x;
      kfu.y = Kc.y + Kp.y;
    } else {
      kfe.x = ke;
      kfn.x = kn;
      kfu.x = ku;
      kfe.y = kfn.y = kfu.y = A(0);
    }
    const A2 Fe = flux(kfe, A(We.x - Wc.x), A(We.y - Wc.y));
    const A2 Fn = flux(kfn, A(Wn.x - Wc.x), A(Wn.y - Wc.y));
    const A2 Fu = flux(kfu, A(Wp.x - Wc.x), A(Wp.y - Wc.y));
    shF[b][row][lane] = Fn;
    __syncthreads();
    const int rs = row > 0 ? row - 1 : row;  // the bottom halo row has no south flux here
    const A2 Fs = shF[b][rs][lane];
    A2 Fw;
    Fw.x = __shfl_up_sync(0xffffffffu, Fe.x, 1);
    Fw.y = __shfl_up_sync(0xffffffffu, Fe.y, 1);
    const A fR = ((Fe.x - Fw.x) + (Fn.x - Fs.x)) + (Fu.x - Fd.x);
    const A fI = ((Fe.y - Fw.y) + (Fn.y - Fs.y)) + (Fu.y - Fd.y);
    if (out_ok && in_bounds(size_t(z) * plane + col < size_t(nz) * plane, p.status)) {
      const size_t g = size_t(z) * plane + col;
      const S un = Wc.x + ca * S(fR) - cb * S(fI);
      Uo[g] = un;
      if (out_mode == PASS_IO_PLANAR) Vo[g] = Wc.y + ca * S(fI) + cb * S(fR);
      if (p.check_finite) bad |= nonfinite3(un);
    }
    Fd = Fu;
    Wc = Wp;
    Wp = Wpp;
    if (POWER) {
      Kc = Kp;
      Kp = kap(Wpp);
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

template <class S, class A, bool PERIODIC, bool POWER>
cudaError_t launch_t(const PassArgs& a, cudaStream_t st) {
  // z chunks of 32 planes: (32 + 2) / 32 planes loaded per plane output
  const int zchunk = 32;
  dim3 grid((a.nx + S3_OX - 1) / S3_OX, (a.ny + S3_OY - 1) / S3_OY, (a.nz + zchunk - 1) / zchunk);
  // (MIXED measured 8 % slower with the specialisation, so it keeps the general evaluation)
  const auto kern = POWER && a.kp == 2.5 && std::is_same<S, A>::value ? k_stream3d<S, A, PERIODIC, POWER, true>
                                                                        : k_stream3d<S, A, PERIODIC, POWER, false>;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(S3_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, a, zchunk);
    if (le != cudaSuccess) return le;
  }
  count_launch();
  return cudaGetLastError();
}

template <class S, class A>
cudaError_t launch_s(const frkc2_problem& p, const PassArgs& a, cudaStream_t st) {
  const bool per = p.bc == FRKC2_BC_PERIODIC, pw = p.kappa_kind == FRKC2_KAPPA_POWER;
  if (per) return pw ? launch_t<S, A, true, true>(a, st) : launch_t<S, A, true, false>(a, st);
  return pw ? launch_t<S, A, false, true>(a, st) : launch_t<S, A, false, false>(a, st);
}

}  // namespace

cudaError_t launch_pass_stream3d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st) {
  switch (p.precision) {
    case FRKC2_FP64: return launch_s<double, double>(p, a, st);
    case FRKC2_FP32: return launch_s<float, float>(p, a, st);
    default: return launch_s<double, float>(p, a, st);
  }
}

}  // namespace frkc2
