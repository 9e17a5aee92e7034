// 2D single-stage pass (k = 1) for the DFLOAT precision: stage states held as float pairs
// (hi + lo, a "double-float" of about 48 significant bits) and every operation on the FP32
// pipe, which on GB300 issues 64 times as many lanes per clock as the FP64 pipe.
//
// Per cell and stage:
//  * neighbour differences rounded to float from the pairs, (hi_nb - hi_c) + (lo_nb - lo_c)
//    (the hi difference is exact when the two values are within a factor of two): 3 ops
//    for each of the east and north neighbours of U and V, 12 in all;
//  * f = kappa_e d_e - kappa_w d_w + kappa_n d_n - kappa_s d_s in float, each difference
//    shared with the cell across the face (x by shuffle, y carried): 4 ops each for U, V;
//  * the increment dU = ca fU - cb fV, dV = ca fV + cb fU in float (4 ops), added to the
//    pair by an error-free sum (Knuth's TwoSum, then a fast renormalisation): 10 ops each.
// About 44 FP32 instructions per cell-stage and no FP64 instruction in the passes between a
// step's first and last, so the pass is bound by memory: 16 bytes of state in, 16 out and 8
// of face conductivities per cell.  The state sum keeps about 48 bits
// across stages (the FP64 path keeps 53); the flux arithmetic is float, as in MIXED.
//
// A step's first pass reads the caller's double state and splits it (hi = float(u),
// lo = float(u - hi)); its last pass writes hi + lo back as a double.  Between passes the
// state is stored as one float4 (U hi, U lo, V hi, V lo) per cell.  Same warp layout and
// persistent balanced work split as the FP64 streaming pass; since the arithmetic is cheap,
// each warp keeps the loads of the next DF_PF rows in flight while it computes a row.
#include <algorithm>

#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int DF_THREADS = 256;
constexpr int DF_WARPS = DF_THREADS / 32;
constexpr int DF_COLS = 31;  // output columns per warp
#ifndef FRKC2_DF_MIN_BLOCKS
#define FRKC2_DF_MIN_BLOCKS 3
#endif
#ifndef FRKC2_DF_PREFETCH
#define FRKC2_DF_PREFETCH 1
#endif
constexpr int DF_MIN_BLOCKS = FRKC2_DF_MIN_BLOCKS;
constexpr int DF_PF = FRKC2_DF_PREFETCH;  // rows loaded ahead of their use (1 or 2)
static_assert(DF_PF == 1 || DF_PF == 2, "prefetch distance 1 or 2");
constexpr int DF_UNROLL = DF_PF + 1;

__device__ __forceinline__ float4 split_real(double u) {
  float4 w;
  w.x = __double2float_rn(u);
  w.y = __double2float_rn(u - double(w.x));
  w.z = 0.f;
  w.w = 0.f;
  return w;
}

// (h, l) + d as a renormalised pair
__device__ __forceinline__ void df_add(float& h, float& l, float d) {
  const float s = h + d;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (d - bb);
  const float t = l + e;
  const float hi = s + t;
  l = t - (hi - s);
  h = hi;
}

__device__ __forceinline__ bool nonfinite_d(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }

// IN_REAL / OUT_REAL: the step's first / last pass (double state in / out).  They are template
// arguments so that the passes in between hold no double arithmetic at all: a runtime test,
// even a uniform one, lets the compiler predicate the conversions into every pass, where they
// would occupy GB300's narrow FP64 pipe.
template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
__global__ void __launch_bounds__(DF_THREADS, DF_MIN_BLOCKS)
    k_stream2d_df(const PassArgs p, const float2* __restrict__ FEN, long long total, long long nwarps_grid) {
  // launched with programmatic stream serialization: the next launch may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * DF_WARPS + (threadIdx.x >> 5);
  const int nx = p.nx, ny = p.ny;
  long long idx = gw * total / nwarps_grid;
  const long long end = (gw + 1) * total / nwarps_grid;
  const double* __restrict__ Ur = static_cast<const double*>(p.U_in);
  const float4* __restrict__ Wi = static_cast<const float4*>(p.U_in);
  double* __restrict__ Uo = static_cast<double*>(p.U_out);
  float4* __restrict__ Wo = static_cast<float4*>(p.U_out);
  const float ca = p.caf[0], cb = p.cbf[0];
  bool bad = false;

  while (idx < end) {  // warp-uniform
    const int wcol = int(idx / ny);
    const int y0 = int(idx - (long long)wcol * ny);
    const int y1 = int(min((long long)ny, (long long)y0 + (end - idx)));
    idx += y1 - y0;
    const int x = wcol * DF_COLS + lane - 1;
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

    // rows run from y0 - 1 to y1 + DF_PF: a periodic row index may lie up to DF_PF + 1 rows
    // past the grid, more than one period when ny <= DF_PF
    auto wrap = [&](int yy) {
      if (yy < 0) yy += ny;
      while (yy >= ny) yy -= ny;
      return yy;
    };
    auto load = [&](int yy, int xx, bool inx) -> float4 {
      int yw = yy;
      if (PERIODIC) {
        yw = wrap(yy);
      } else if (!(inx && yy >= 0 && yy < ny)) {
        return make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const size_t g = size_t(yw) * nx + xx;
      if (IN_REAL) return split_real(__ldg(Ur + g));
      return __ldg(Wi + g);
    };
    // face pairs exist for rows -1 .. ny-1; prefetched rows past the grid are never used
    auto faces = [&](int yy) -> float2 {
      if (PERIODIC) {
        yy = wrap(yy);
      } else if (yy >= ny) {
        return make_float2(0.f, 0.f);
      }
      if (!has_faces) return make_float2(0.f, 0.f);
      return __ldg(FEN + size_t(yy + 1) * (nx + 1) + fcol);
    };
    auto diff = [](float ah, float al, float bh, float bl) -> float { return (ah - bh) + (al - bl); };

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto east = [&](int yy) -> float4 { return lane == 31 ? load(yy, xeast, eastin) : zero4; };
    float4 Wc = load(y0, xr, xin);
    float dSU, dSV, ks;
    {
      const float4 Ws = load(y0 - 1, xr, xin);
      ks = faces(y0 - 1).y;
      dSU = diff(Wc.x, Wc.y, Ws.x, Ws.y);
      dSV = diff(Wc.z, Wc.w, Ws.z, Ws.w);
    }
    // rows y+1 .. y+DF_PF of W, faces and the east column of lane 31 for rows y .. y+DF_PF-1
    float4 W1 = load(y0 + 1, xr, xin);
    float4 W2 = DF_PF == 2 ? load(y0 + 2, xr, xin) : zero4;
    float2 F0 = faces(y0);
    float2 F1 = DF_PF == 2 ? faces(y0 + 1) : make_float2(0.f, 0.f);
    float4 E0 = east(y0);
    float4 E1 = DF_PF == 2 ? east(y0 + 1) : zero4;
    // unrolled DF_PF + 1 times, so the row registers rotate by renaming: a move at the end of
    // each row would wait for the load it copies and defeat the prefetch
#pragma unroll DF_UNROLL
    for (int y = y0; y < y1; ++y) {
      // loads for the row DF_PF ahead, issued before this row's arithmetic
      const float4 Wf = load(y + 1 + DF_PF, xr, xin);
      const float2 Ff = faces(y + DF_PF);
      const float4 Ef = east(y + DF_PF);
      const float4 Wn = W1;
      const float2 f = F0;
      float4 We;
      We.x = __shfl_down_sync(0xffffffffu, Wc.x, 1);
      We.y = __shfl_down_sync(0xffffffffu, Wc.y, 1);
      We.z = __shfl_down_sync(0xffffffffu, Wc.z, 1);
      We.w = __shfl_down_sync(0xffffffffu, Wc.w, 1);
      if (lane == 31) We = E0;
      const float dEU = diff(We.x, We.y, Wc.x, Wc.y), dEV = diff(We.z, We.w, Wc.z, Wc.w);
      const float dNU = diff(Wn.x, Wn.y, Wc.x, Wc.y), dNV = diff(Wn.z, Wn.w, Wc.z, Wc.w);
      const float dWU = __shfl_up_sync(0xffffffffu, dEU, 1);
      const float dWV = __shfl_up_sync(0xffffffffu, dEV, 1);
      const float kw = __shfl_up_sync(0xffffffffu, f.x, 1);
      const float fU = f.y * dNU - ks * dSU - kw * dWU + f.x * dEU;
      const float fV = f.y * dNV - ks * dSV - kw * dWV + f.x * dEV;
      float uh = Wc.x, ul = Wc.y, vh = Wc.z, vl = Wc.w;
      df_add(uh, ul, ca * fU - cb * fV);
      df_add(vh, vl, ca * fV + cb * fU);
      if (out_ok) {
        const size_t g = size_t(y) * nx + x;
        if (OUT_REAL) {
          const double un = double(uh) + double(ul);
          Uo[g] = un;
          if (p.check_finite) bad |= nonfinite_d(un);
        } else {
          Wo[g] = make_float4(uh, ul, vh, vl);
        }
      }
      dSU = dNU;
      dSV = dNV;
      ks = f.y;
      Wc = Wn;
      if (DF_PF == 2) {
        W1 = W2;
        W2 = Wf;
        F0 = F1;
        F1 = Ff;
        E0 = E1;
        E1 = Ef;
      } else {
        W1 = Wf;
        F0 = Ff;
        E0 = Ef;
      }
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
cudaError_t launch_t(const PassArgs& a, const void* fen, cudaStream_t st) {
  const auto kern = k_stream2d_df<PERIODIC, IN_REAL, OUT_REAL>;
  static const Residency res = query_residency(kern, DF_THREADS, 0);
  if (res.err != cudaSuccess) return res.err;
  const int ncolw = (a.nx + DF_COLS - 1) / DF_COLS;
  const long long total = (long long)ncolw * a.ny;
  long long grid = (long long)res.sms * res.per_sm;
  const long long max_useful = (total + DF_WARPS - 1) / DF_WARPS;
  if (grid > max_useful) grid = max_useful;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid), 1, 1);
    cfg.blockDim = dim3(DF_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, a, static_cast<const float2*>(fen), total, grid * DF_WARPS);
    if (le != cudaSuccess) return le;
  }
  count_launch();
  return cudaGetLastError();
}

template <bool PERIODIC>
cudaError_t launch_bc(const PassArgs& a, const void* fen, cudaStream_t st) {
  const bool in_real = a.in_mode == PASS_IO_REAL, out_real = a.out_mode == PASS_IO_REAL;
  if (in_real) return out_real ? launch_t<PERIODIC, true, true>(a, fen, st) : launch_t<PERIODIC, true, false>(a, fen, st);
  return out_real ? launch_t<PERIODIC, false, true>(a, fen, st) : launch_t<PERIODIC, false, false>(a, fen, st);
}

}  // namespace

cudaError_t launch_pass_stream2d_df(const frkc2_problem& p, const PassArgs& a, const void* fen, cudaStream_t st) {
  return p.bc == FRKC2_BC_PERIODIC ? launch_bc<true>(a, fen, st) : launch_bc<false>(a, fen, st);
}

}  // namespace frkc2
