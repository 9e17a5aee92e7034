// 2D adjoint stage (fixed conductivity) streamed from global memory, the reverse of the
// streaming forward pass: lam^l = lam^{l+1} + conj(c_l) A lam^{l+1} (A symmetric, so J^H = A)
// and, for a conductivity field, the face sensitivities
//   G_f = Re(c_l conj(lam_m - lam_i)(W_i - W_m)) / dx^2
// of every face, added to dJ/dkappa of its two cells with weight 1/2 (1 for a Dirichlet
// boundary face).  A warp owns 30 columns plus a halo lane on each side and walks rows
// upward; each face's lambda difference and sensitivity are formed once (x faces shared by
// shuffle, y faces carried to the next row), and A lam = k_e d_e - k_w d_w + k_n d_n - k_s d_s
// takes one product and three fused multiply-adds per component.  Each cell forms
// Y = -(c/2) W^l once (in the state precision), so a face's sensitivity share is
// Re(conj(lam_m - lam_i)(Y_m - Y_i)): two differences and one multiply-add, the face weight
// 1/2 folded into Y (a Dirichlet boundary face, weight 1, counts twice).  Per cell-stage: 4
// lambda differences, 4 for Y, 2 x (2 differences + 2) for the sensitivities, 8 for A lam,
// 4 for the update and 4 for the dJ/dkappa sum -- 32 floating-point instructions.  lam and
// the stage state W^l are read interleaved (U, V).
#include <algorithm>

#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int AS_THREADS = 256;
constexpr int AS_WARPS = AS_THREADS / 32;
constexpr int AS_COLS = 30;  // output columns per warp: lanes 1..30 (lanes 0 and 31 are halos)
#ifndef FRKC2_ADJ_MIN_BLOCKS
#define FRKC2_ADJ_MIN_BLOCKS 2
#endif
#ifndef FRKC2_ADJ_PREFETCH
#define FRKC2_ADJ_PREFETCH 1
#endif
#ifndef FRKC2_ADJ_UNROLL
#define FRKC2_ADJ_UNROLL 2
#endif
constexpr int AS_UNROLL = FRKC2_ADJ_UNROLL;
#ifndef FRKC2_ADJ_MIN_BLOCKS_F32
#define FRKC2_ADJ_MIN_BLOCKS_F32 4
#endif
template <class S>
constexpr int adj_min_blocks() {
  return sizeof(S) == 4 ? FRKC2_ADJ_MIN_BLOCKS_F32 : FRKC2_ADJ_MIN_BLOCKS;
}

template <class T> struct V2t;
template <> struct V2t<double> { using type = double2; };
template <> struct V2t<float> { using type = float2; };

template <class S, class A, bool PERIODIC>
__global__ void __launch_bounds__(AS_THREADS, adj_min_blocks<S>())
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
  const S hr = S(0.5 * p.ca), hi = S(0.5 * p.cb);  // c/2: each face gives half to each cell

  // launched with programmatic stream serialization: the next launch may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
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
    const bool has_faces = PERIODIC || (x >= -1 && x < nx);
    const int fcol = (PERIODIC ? xr : x) + 1;
    const bool out_ok = lane >= 1 && lane <= 30 && x >= 0 && x < nx;
    // Dirichlet: a boundary face passes all of its sensitivity to its interior cell
    const bool bW = !PERIODIC && x == 0;
    const bool bE = !PERIODIC && x == nx - 1;

    // rows run from y0 - 1 to y1: more than one period past the grid when ny is 1
    auto wrapy = [&](int yy) {
      if (PERIODIC) {
        if (yy < 0) yy += ny;
        while (yy >= ny) yy -= ny;
      }
      return yy;
    };
    auto ld = [&](const S2* __restrict__ P2, const S* __restrict__ P1, int cplx, int yy) -> S2 {
      S2 w;
      w.x = S(0);
      w.y = S(0);
      const int yw = wrapy(yy);
      if (!PERIODIC && !(xin && yy >= 0 && yy < ny)) return w;
      const size_t g = size_t(yw) * nx + xr;
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
      if (!has_faces || (!PERIODIC && yy >= ny)) return f;  // face pairs: rows -1 .. ny-1
      return __ldg(FEN + size_t(yy + 1) * (nx + 1) + fcol);
    };
    // Y = -(c/2) W: a face's sensitivity is then Re(conj(lam_m - lam_i)(Y_m - Y_i))
    auto yof = [&](S2 w) -> S2 {
      S2 y;
      y.x = hi * w.y - hr * w.x;
      y.y = -(hi * w.x) - hr * w.y;
      return y;
    };

    // prime: row y0 and its south face (lambda difference, conductivity and sensitivity)
    S2 Lc = ld(Lin, Lr, p.l_complex, y0);
    S2 Yc = yof(ld(Wc2, Wr, p.w_complex, y0));
    A dSr, dSi, ks;  // lambda difference across the south face of row y0, and that face
    A Gs;            // sensitivity of the south face of row y0
    {
      const S2 Ls = ld(Lin, Lr, p.l_complex, y0 - 1);
      const S2 Ys = yof(ld(Wc2, Wr, p.w_complex, y0 - 1));
      ks = faces(y0 - 1).y;
      dSr = A(Lc.x - Ls.x);
      dSi = A(Lc.y - Ls.y);
      Gs = dSr * A(Yc.x - Ys.x) + dSi * A(Yc.y - Ys.y);
    }
#if FRKC2_ADJ_PREFETCH
    // the next row's lam, tape entry and faces are loaded one iteration ahead of their use
    S2 Ln = ld(Lin, Lr, p.l_complex, y0 + 1);
    S2 Wn = ld(Wc2, Wr, p.w_complex, y0 + 1);
    A2 f = faces(y0);
#endif
#pragma unroll AS_UNROLL
    for (int y = y0; y < y1; ++y) {
#if FRKC2_ADJ_PREFETCH
      const S2 Lnn = ld(Lin, Lr, p.l_complex, y + 2);
      const S2 Wnn = ld(Wc2, Wr, p.w_complex, y + 2);
      const A2 fnext = faces(y + 1);
#else
      const S2 Ln = ld(Lin, Lr, p.l_complex, y + 1);
      const S2 Wn = ld(Wc2, Wr, p.w_complex, y + 1);
      const A2 f = faces(y);
#endif
      const S2 Yn = yof(Wn);
      // east face (lane 31 is a halo: its east values are not used)
      const S Le_r = __shfl_down_sync(0xffffffffu, Lc.x, 1);
      const S Le_i = __shfl_down_sync(0xffffffffu, Lc.y, 1);
      const S Ye_r = __shfl_down_sync(0xffffffffu, Yc.x, 1);
      const S Ye_i = __shfl_down_sync(0xffffffffu, Yc.y, 1);
      const A dEr = A(Le_r - Lc.x), dEi = A(Le_i - Lc.y);
      const A Ge = dEr * A(Ye_r - Yc.x) + dEi * A(Ye_i - Yc.y);
      // north face
      const A dNr = A(Ln.x - Lc.x), dNi = A(Ln.y - Lc.y);
      const A Gn = dNr * A(Yn.x - Yc.x) + dNi * A(Yn.y - Yc.y);
      // west face from lane - 1
      const A dWr = __shfl_up_sync(0xffffffffu, dEr, 1);
      const A dWi = __shfl_up_sync(0xffffffffu, dEi, 1);
      const A kw = __shfl_up_sync(0xffffffffu, f.x, 1);
      const A Gw = __shfl_up_sync(0xffffffffu, Ge, 1);
      const A fU = f.y * dNr - ks * dSr - kw * dWr + f.x * dEr;
      const A fV = f.y * dNi - ks * dSi - kw * dWi + f.x * dEi;
      if (out_ok) {
        const size_t g = size_t(y) * nx + x;
        S2 o;
        o.x = Lc.x + ca * S(fU) + cb * S(fV);
        o.y = Lc.y + ca * S(fV) - cb * S(fU);
        Lout[g] = o;
        if (dk) {
          A ge = Ge, gw = Gw, gn = Gn, gs = Gs;
          if (!PERIODIC) {
            if (bE) ge = Ge + Ge;
            if (bW) gw = Gw + Gw;
            if (y == ny - 1) gn = Gn + Gn;
            if (y == 0) gs = Gs + Gs;
          }
          dk[g] += double((ge + gw) + (gn + gs));
        }
      }
      dSr = dNr;
      dSi = dNi;
      ks = f.y;
      Gs = Gn;
      Lc = Ln;
      Yc = Yn;
#if FRKC2_ADJ_PREFETCH
      Ln = Lnn;
      Wn = Wnn;
      f = fnext;
#endif
    }
  }
}

template <class S, class A, bool PERIODIC>
cudaError_t launch_t(const AdjStreamArgs& a, cudaStream_t st) {
  const auto kern = k_adj_stream2d<S, A, PERIODIC>;
  static const Residency res = query_residency(kern, AS_THREADS, 0);
  if (res.err != cudaSuccess) return res.err;
  const int ncolw = (a.nx + AS_COLS - 1) / AS_COLS;
  const long long total = (long long)ncolw * a.ny;
  long long grid = (long long)res.sms * res.per_sm;
  const long long max_useful = (total + AS_WARPS - 1) / AS_WARPS;
  if (grid > max_useful) grid = max_useful;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid), 1, 1);
    cfg.blockDim = dim3(AS_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, a, total, grid * AS_WARPS);
    if (le != cudaSuccess) return le;
  }
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
