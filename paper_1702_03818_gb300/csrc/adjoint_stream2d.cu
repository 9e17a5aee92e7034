// 2D adjoint stage (fixed conductivity) streamed from global memory, the reverse of the
// streaming forward pass: lam^l = lam^{l+1} + conj(c_l) A lam^{l+1} (A symmetric, so J^H = A)
// and, for a conductivity field, the face sensitivities
//   G_f = Re(c_l conj(lam_m - lam_i)(W_i - W_m)) / dx^2
// of every face, added to dJ/dkappa of its two cells with weight 1/2 (1 for a Dirichlet
// boundary face).  Same layout as the forward streaming pass: a warp owns 31 columns plus a
// west halo lane and walks rows upward; each face's lambda difference, lambda flux, W
// difference and sensitivity are formed once (x faces shared by shuffle, y faces carried
// to the next row).  lam and the stage state W^l are read interleaved (U, V).
#include <algorithm>

#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int AS_THREADS = 256;
constexpr int AS_WARPS = AS_THREADS / 32;
constexpr int AS_COLS = 31;

template <class T> struct V2t;
template <> struct V2t<double> { using type = double2; };
template <> struct V2t<float> { using type = float2; };

template <class S, class A, bool PERIODIC>
__global__ void __launch_bounds__(AS_THREADS, 4)
    k_adj_stream2d(const AdjStreamArgs p, long long total, long long nwarps_grid) {
  using S2 = typename V2t<S>::type;
  using A2 = typename V2t<A>::type;
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * AS_WARPS + (threadIdx.x >> 5);
  const int nx = p.nx, ny = p.ny;
  long long idx = gw * total / nwarps_grid;
  const long long end = (gw + 1) * total / nwarps_grid;
  const A2* __restrict__ FEN = static_cast<const A2*>(p.fen);
  const S2* __restrict__ Wc2 = static_cast<const S2*>(p.W);       // W^l interleaved (or real)
  const S* __restrict__ Wr = static_cast<const S*>(p.W);
  const S2* __restrict__ Lin = static_cast<const S2*>(p.L_in);    // lam^{l+1} interleaved (or real)
  const S* __restrict__ Lr = static_cast<const S*>(p.L_in);
  S2* __restrict__ Lout = static_cast<S2*>(p.L_out);
  double* __restrict__ dk = p.dk;
  const S ca = S(p.ca), cb = S(p.cb);
  const A cad = A(p.ca), cbd = A(p.cb);

  while (idx < end) {
    const int wcol = int(idx / ny);
    const int y0 = int(idx - (long long)wcol * ny);
    const int y1 = int(min((long long)ny, (long long)y0 + (end - idx)));
    idx += y1 - y0;
    const int x = wcol * AS_COLS + lane - 1;
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
    const bool out_ok = lane >= 1 && x >= 0 && x < nx;
    // Dirichlet: a boundary face passes all of its sensitivity to its interior cell
    const A wW = (!PERIODIC && x == 0) ? A(1) : A(0.5);
    const A wE = (!PERIODIC && x == nx - 1) ? A(1) : A(0.5);

    auto wrapy = [&](int yy) { return PERIODIC ? (yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy)) : yy; };
    auto ld = [&](const S2* __restrict__ P2, const S* __restrict__ P1, int cplx, int yy, int xx, bool inx) -> S2 {
      S2 w;
      w.x = S(0);
      w.y = S(0);
      const int yw = wrapy(yy);
      if (!PERIODIC && !(inx && yy >= 0 && yy < ny)) return w;
      const size_t g = size_t(yw) * nx + xx;
      if (cplx == 1) {
        w = __ldg(P2 + g);
      } else if (cplx == 2) {
        w.x = __ldg(P2 + g).x;
      } else {
        w.x = __ldg(P1 + g);
      }
      return w;
    };
    auto faces = [&](int yy) -> A2 {
      A2 f;
      f.x = A(0);
      f.y = A(0);
      yy = wrapy(yy);
      if (!has_faces) return f;
      return __ldg(FEN + size_t(yy + 1) * (nx + 1) + fcol);
    };

    // prime: row y0 and its south face (lambda flux and sensitivity through it)
    S2 Lc = ld(Lin, Lr, p.l_complex, y0, xr, xin);
    S2 Wc = ld(Wc2, Wr, p.w_complex, y0, xr, xin);
    A PnU, PnV;      // lambda flux into row y0-1 through its north face
    A Gs;            // sensitivity of the south face of row y0
    {
      const S2 Ls = ld(Lin, Lr, p.l_complex, y0 - 1, xr, xin);
      const S2 Ws = ld(Wc2, Wr, p.w_complex, y0 - 1, xr, xin);
      const A ks = faces(y0 - 1).y;
      const A dlr = A(Lc.x - Ls.x), dli = A(Lc.y - Ls.y);
      PnU = ks * dlr;
      PnV = ks * dli;
      const A dWr = A(Wc.x - Ws.x), dWi = A(Wc.y - Ws.y);
      const A zr = dlr * dWr + dli * dWi;
      const A zi = dlr * dWi - dli * dWr;
      Gs = cbd * zi - cad * zr;
    }
    for (int y = y0; y < y1; ++y) {
      const S2 Ln = ld(Lin, Lr, p.l_complex, y + 1, xr, xin);
      const S2 Wn = ld(Wc2, Wr, p.w_complex, y + 1, xr, xin);
      const A2 f = faces(y);
      S Le_r = __shfl_down_sync(0xffffffffu, Lc.x, 1);
      S Le_i = __shfl_down_sync(0xffffffffu, Lc.y, 1);
      S We_r = __shfl_down_sync(0xffffffffu, Wc.x, 1);
      S We_i = __shfl_down_sync(0xffffffffu, Wc.y, 1);
      if (lane == 31) {
        const S2 Le = ld(Lin, Lr, p.l_complex, y, xeast, eastin);
        const S2 We = ld(Wc2, Wr, p.w_complex, y, xeast, eastin);
        Le_r = Le.x;
        Le_i = Le.y;
        We_r = We.x;
        We_i = We.y;
      }
      // east face: lambda difference, flux, W difference, sensitivity
      const A dEr = A(Le_r - Lc.x), dEi = A(Le_i - Lc.y);
      const A FeU = f.x * dEr, FeV = f.x * dEi;
      A Ge;
      {
        const A dWr = A(We_r - Wc.x), dWi = A(We_i - Wc.y);
        const A zr = dEr * dWr + dEi * dWi;
        const A zi = dEr * dWi - dEi * dWr;
        Ge = cbd * zi - cad * zr;
      }
      // north face
      const A dNr = A(Ln.x - Lc.x), dNi = A(Ln.y - Lc.y);
      const A FnU = f.y * dNr, FnV = f.y * dNi;
      A Gn;
      {
        const A dWr = A(Wn.x - Wc.x), dWi = A(Wn.y - Wc.y);
        const A zr = dNr * dWr + dNi * dWi;
        const A zi = dNr * dWi - dNi * dWr;
        Gn = cbd * zi - cad * zr;
      }
      const A wU = __shfl_up_sync(0xffffffffu, FeU, 1);
      const A wV = __shfl_up_sync(0xffffffffu, FeV, 1);
      const A Gw = __shfl_up_sync(0xffffffffu, Ge, 1);
      const A fU = (FeU - wU) + (FnU - PnU);
      const A fV = (FeV - wV) + (FnV - PnV);
      if (out_ok) {
        const size_t g = size_t(y) * nx + x;
        S2 o;
        o.x = Lc.x + ca * S(fU) + cb * S(fV);
        o.y = Lc.y + ca * S(fV) - cb * S(fU);
        Lout[g] = o;
        if (dk) {
          const A wS = (!PERIODIC && y == 0) ? A(1) : A(0.5);
          const A wN = (!PERIODIC && y == ny - 1) ? A(1) : A(0.5);
          dk[g] += double((wE * Ge + wW * Gw) + (wN * Gn + wS * Gs));
        }
      }
      PnU = FnU;
      PnV = FnV;
      Gs = Gn;
      Lc = Ln;
      Wc = Wn;
    }
  }
}

template <class S, class A, bool PERIODIC>
cudaError_t launch_t(const AdjStreamArgs& a, cudaStream_t st) {
  static int blocks_per_sm = 0, sms = 0;
  auto kern = k_adj_stream2d<S, A, PERIODIC>;
  if (!blocks_per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, AS_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int ncolw = (a.nx + AS_COLS - 1) / AS_COLS;
  const long long total = (long long)ncolw * a.ny;
  long long grid = (long long)sms * blocks_per_sm;
  const long long max_useful = (total + AS_WARPS - 1) / AS_WARPS;
  if (grid > max_useful) grid = max_useful;
  kern<<<unsigned(grid), AS_THREADS, 0, st>>>(a, total, grid * AS_WARPS);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adj_stream2d(const frkc2_problem& p, const AdjStreamArgs& a, cudaStream_t st) {
  const bool per = p.bc == FRKC2_BC_PERIODIC;
  switch (p.precision) {
    case FRKC2_FP64:
      return per ? launch_t<double, double, true>(a, st) : launch_t<double, double, false>(a, st);
    case FRKC2_FP32:
      return per ? launch_t<float, float, true>(a, st) : launch_t<float, float, false>(a, st);
    default:
      return per ? launch_t<double, float, true>(a, st) : launch_t<double, float, false>(a, st);
  }
}

}  // namespace frkc2
