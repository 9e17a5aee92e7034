// 2D pass applying one conjugate pair of stages in real arithmetic (fixed conductivity).
//
// Two adjacent stages with step sizes a and conj(a) (Sec. 3, Eq. 13) act on a real state w of a
// linear problem as the real quadratic factor (1 + T a f)(1 + T conj(a) f) w =
// w + 2 T alpha f(w) + T^2 |a|^2 f(f(w)), alpha = Re a, beta = Im a, evaluated here as
//   Y = w + cy f(w),   w' = w + c1 f(w) + c2 f(Y),
//   cy = T alpha / dx^2,  c1 = T (alpha - beta^2/alpha) / dx^2,  c2 = T (|a|^2/alpha) / dx^2
// (f here without the 1/dx^2, which the coefficients carry).  The state stays real: 8 bytes
// per cell in FP64 instead of 16, and 15 floating-point instructions per pair (two stencils
// f = k_e d_e - k_w d_w + k_n d_n - k_s d_s of 2 differences + 4 multiply-adds each, with
// every neighbour difference formed once and shared, plus 1 + 2 fused multiply-adds)
// instead of 2 x 16 for two complex stages.
//
// Streaming layout: a warp owns 32 consecutive columns, outputs 29 of them (lanes 2..30), and
// walks rows upward.  At row y it reads w(y+2), forms f(w) and Y for row y+1 and f(Y) and w'
// for row y; x-neighbours come by shuffle (lane 31 reads its east neighbour itself), the
// north differences of w and Y are carried to the next row as its south ones.  Same persistent, balanced work
// split as the complex streaming pass.
#include <algorithm>

#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_WARPS = PR_THREADS / 32;
constexpr int PR_COLS = 29;  // output columns per warp (lanes 2..30)
#ifndef FRKC2_PAIRED_MIN_BLOCKS
#define FRKC2_PAIRED_MIN_BLOCKS 3
#endif

template <class T> struct P2t;
template <> struct P2t<double> { using type = double2; };
template <> struct P2t<float> { using type = float2; };

__device__ __forceinline__ bool bad_bits(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool bad_bits(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }

template <class S, class A, bool PERIODIC>
__global__ void __launch_bounds__(PR_THREADS, FRKC2_PAIRED_MIN_BLOCKS)
    k_paired2d(const PassArgs p, const void* __restrict__ fen_v, long long total, long long nwarps_grid) {
  // launched with programmatic stream serialization: the next launch may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  using A2 = typename P2t<A>::type;
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * PR_WARPS + (threadIdx.x >> 5);
  const int nx = p.nx, ny = p.ny;
  long long idx = gw * total / nwarps_grid;
  const long long end = (gw + 1) * total / nwarps_grid;
  const A2* __restrict__ FEN = static_cast<const A2*>(fen_v);
  const S* __restrict__ W = static_cast<const S*>(p.U_in);
  S* __restrict__ Wo = static_cast<S*>(p.U_out);
  const S cy = S(p.ca[0]), c1 = S(p.ca[1]), c2 = S(p.cb[0]);
  bool bad = false;

  while (idx < end) {  // warp-uniform
    const int wcol = int(idx / ny);
    const int y0 = int(idx - (long long)wcol * ny);
    const int y1 = int(min((long long)ny, (long long)y0 + (end - idx)));
    idx += y1 - y0;
    const int x = wcol * PR_COLS + lane - 2;
    int xr;
    bool xin;
    if (PERIODIC) {
      xr = ((x % nx) + nx) % nx;
      xin = true;
    } else {
      xr = x;
      xin = x >= 0 && x < nx;
    }
    int xeast;
    bool eastin;
    if (PERIODIC) {
      xeast = xr + 1 == nx ? 0 : xr + 1;
      eastin = true;
    } else {
      xeast = x + 1;
      eastin = xeast >= 0 && xeast < nx;
    }
    const bool has_faces = PERIODIC || (x >= -1 && x < nx);
    const int fcol = (PERIODIC ? xr : x) + 1;
    const bool out_ok = lane >= 2 && lane <= 30 && x >= 0 && x < nx;

    auto wrapy = [&](int yy) { return PERIODIC ? (yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy)) : yy; };
    auto ld = [&](int yy, int xx, bool inx) -> S {
      if (!PERIODIC && !(inx && yy >= 0 && yy < ny)) return S(0);
      return __ldg(W + size_t(wrapy(yy)) * nx + xx);
    };
    auto faces = [&](int yy) -> A2 {
      A2 f;
      f.x = A(0);
      f.y = A(0);
      if (!has_faces) return f;
      return __ldg(FEN + size_t(wrapy(yy) + 1) * (nx + 1) + fcol);
    };
    auto cell_in = [&](int yy) { return PERIODIC || (xin && yy >= 0 && yy < ny); };
    auto east_of = [&](S wc, int yy) -> S {
      S e = __shfl_down_sync(0xffffffffu, wc, 1);
      if (lane == 31) e = ld(yy, xeast, eastin);
      return e;
    };
    // f at one cell from its neighbour differences: the east one formed here, the west one
    // (and the west face) from lane - 1, the north one given, the south one carried
    auto fdiff = [&](S wc, S we, A2 f, A dN, A ks, A dS) -> A {
      const A dE = A(we - wc);
      const A dW = __shfl_up_sync(0xffffffffu, dE, 1);
      const A kw = __shfl_up_sync(0xffffffffu, f.x, 1);
      return f.y * dN - ks * dS - kw * dW + f.x * dE;
    };

    // prologue: rows y0-2 .. y0+1 of w; f(w) and Y of rows y0-1, y0
    const S wm2 = ld(y0 - 2, xr, xin), wm1 = ld(y0 - 1, xr, xin), w0 = ld(y0, xr, xin), w1 = ld(y0 + 1, xr, xin);
    const A2 fm2 = faces(y0 - 2), fm1 = faces(y0 - 1), f0 = faces(y0);
    const A dNm2 = A(wm1 - wm2), dNm1 = A(w0 - wm1), dN0 = A(w1 - w0);
    const A fWm1 = fdiff(wm1, east_of(wm1, y0 - 1), fm1, dNm1, fm2.y, dNm2);
    A fWc = fdiff(w0, east_of(w0, y0), f0, dN0, fm1.y, dNm1);
    const S Ym1 = cell_in(y0 - 1) ? wm1 + cy * S(fWm1) : S(0);
    S Yc = cell_in(y0) ? w0 + cy * S(fWc) : S(0);
    // rolling registers for row y (= current output row)
    A dNYs = A(Yc - Ym1);  // north difference of Y at row y - 1, and that face
    A kYs = fm1.y;
    S wc = w0, wn = w1;
    A dNWc = dN0;  // north difference of w at row y
    A2 fc = f0;    // faces of row y

    for (int y = y0; y < y1; ++y) {
      // row y+1: f(w) and Y
      const S wnn = ld(y + 2, xr, xin);
      const A2 fn = faces(y + 1);
      const A dNWn = A(wnn - wn);
      const A fWn = fdiff(wn, east_of(wn, y + 1), fn, dNWn, fc.y, dNWc);
      const S Yn = cell_in(y + 1) ? wn + cy * S(fWn) : S(0);
      // row y: f(Y) and the new state (lane 31 has no east neighbour for Y; its f(Y) is
      // not an output)
      const A dNYc = A(Yn - Yc);
      const A fY = fdiff(Yc, __shfl_down_sync(0xffffffffu, Yc, 1), fc, dNYc, kYs, dNYs);
      const S wnew = wc + c1 * S(fWc) + c2 * S(fY);
      if (out_ok) {
        Wo[size_t(y) * nx + x] = wnew;
        if (p.check_finite) bad |= bad_bits(wnew);
      }
      // roll
      dNYs = dNYc;
      kYs = fc.y;
      fWc = fWn;
      dNWc = dNWn;
      Yc = Yn;
      wc = wn;
      wn = wnn;
      fc = fn;
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

template <class S, class A, bool PERIODIC>
cudaError_t launch_t(const PassArgs& a, const void* fen, cudaStream_t st) {
  const auto kern = k_paired2d<S, A, PERIODIC>;
  static const Residency res = query_residency(kern, PR_THREADS, 0);
  if (res.err != cudaSuccess) return res.err;
  const int ncolw = (a.nx + PR_COLS - 1) / PR_COLS;
  const long long total = (long long)ncolw * a.ny;
  long long grid = (long long)res.sms * res.per_sm;
  const long long max_useful = (total + PR_WARPS - 1) / PR_WARPS;
  if (grid > max_useful) grid = max_useful;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid), 1, 1);
    cfg.blockDim = dim3(PR_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, a, fen, total, grid * PR_WARPS);
    if (le != cudaSuccess) return le;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass_paired2d(const frkc2_problem& p, const PassArgs& a, const void* fen, cudaStream_t st) {
  const bool per = p.bc == FRKC2_BC_PERIODIC;
  switch (p.precision) {
    case FRKC2_FP64: return per ? launch_t<double, double, true>(a, fen, st) : launch_t<double, double, false>(a, fen, st);
    case FRKC2_FP32: return per ? launch_t<float, float, true>(a, fen, st) : launch_t<float, float, false>(a, fen, st);
    default: return per ? launch_t<double, float, true>(a, fen, st) : launch_t<double, float, false>(a, fen, st);
  }
}

}  // namespace frkc2
