// 2D single-stage pass (k = 1) streaming straight from global memory, for the fixed
// conductivity (FIELD / CONST) flux-form operator.
//
// Each warp owns 31 consecutive columns plus one halo lane on the low-x side and walks rows
// upward.  Every neighbour difference W_nb - W_c is formed once and used by both cells of
// the face: a lane's east difference (and east face conductivity) reaches the next lane
// through a warp shuffle as its west difference (the halo lane supplies the chunk's west
// edge), and a cell's north difference and north face conductivity are carried in registers
// to the next row as its south ones.  Each cell then forms
//   f = kappa_e d_e - kappa_w d_w + kappa_n d_n - kappa_s d_s
// with one product and three fused multiply-adds per component: per cell and stage 2
// differences and 4 multiply-adds for each of U and V plus 4 fused multiply-adds for the
// complex update -- 16 floating-point instructions, which is what bounds the FP64 path on
// GB300 (its FP64 pipe issues 2 lanes per clock per SM, far below its memory system).
// Every term is a conductivity times a neighbour difference, as in the flux form; the face
// sum is rounded per cell, so the two cells of a face see its flux to within rounding.
//
// Memory: the stage state between passes is stored interleaved (U, V) so one 16-byte (FP64)
// load brings a cell's complex value, and each cell's east and north face conductivities
// are read as one pair from a face-pair array; a step's first pass reads the real state and
// its last pass writes it.  Planar (U, V) input and output are also accepted (the adjoint's
// stage tape uses them).
//
// Work split: the grid is persistent (every CTA resident) and the (column chunk, row)
// pairs, chunk-major, are cut into one contiguous range per warp, so every SM gets the same
// number of cell updates.  A range that crosses into the next chunk restarts the stream.
#include <algorithm>

#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int ST_THREADS = 256;
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int ST_COLS = 31;  // output columns per warp
#ifndef FRKC2_STREAM_MIN_BLOCKS
#define FRKC2_STREAM_MIN_BLOCKS 3
#endif
#ifndef FRKC2_STREAM_PREFETCH
#define FRKC2_STREAM_PREFETCH 1  // loads for row y + 1 issued one row ahead
#endif
constexpr int ST_MIN_BLOCKS = FRKC2_STREAM_MIN_BLOCKS;  // CTAs per SM the register budget allows

template <class T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

__device__ __forceinline__ bool nonfinite_bits(double v) {
  return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool nonfinite_bits(float v) {
  return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

// HAT: the pass also advances the embedded first-order solution of Eq. 14 (real, one value a
// cell): What <- What + ca f_R, read from H_in and written to H_out (the adaptive step).
template <class S, class A, bool PERIODIC, bool HAT>
__global__ void __launch_bounds__(ST_THREADS, ST_MIN_BLOCKS)
    k_stream2d(const PassArgs p, const void* __restrict__ fen_v, int ncolw, long long total,
               long long nwarps_grid) {
  using S2 = typename Vec2<S>::type;
  using A2 = typename Vec2<A>::type;
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * ST_WARPS + (threadIdx.x >> 5);
  const int nx = p.nx, ny = p.ny;
  long long idx = gw * total / nwarps_grid;
  const long long end = (gw + 1) * total / nwarps_grid;
  const A2* __restrict__ FEN = static_cast<const A2*>(fen_v);  // [(ny+1)][(nx+1)], index (y+1, x+1)
  const int in_mode = p.in_mode, out_mode = p.out_mode;
  const S* __restrict__ Ur = static_cast<const S*>(p.U_in);
  const S* __restrict__ Vr = static_cast<const S*>(p.V_in);
  const S2* __restrict__ Wi = static_cast<const S2*>(p.U_in);
  S* __restrict__ Uo = static_cast<S*>(p.U_out);
  S* __restrict__ Vo = static_cast<S*>(p.V_out);
  S2* __restrict__ Wo = static_cast<S2*>(p.U_out);
  const S ca = S(p.ca[0]), cb = S(p.cb[0]);
  bool bad = false;
  // launched with programmatic stream serialization: the next pass may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  while (idx < end) {  // warp-uniform
    const int wcol = int(idx / ny);
    const int y0 = int(idx - (long long)wcol * ny);
    const int y1 = int(min((long long)ny, (long long)y0 + (end - idx)));
    idx += y1 - y0;
    const int x = wcol * ST_COLS + lane - 1;

    // column read by this lane (wrapped when periodic) and whether it holds a real cell
    int xr;
    bool xin;
    if (PERIODIC) {
      xr = ((x % nx) + nx) % nx;
      xin = true;
    } else {
      xr = x;
      xin = x >= 0 && x < nx;
    }
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
    // the lane's face-pair column (x = -1 is the Dirichlet west boundary, column 0)
    const bool has_faces = PERIODIC || (x >= -1 && x < nx);
    const int fcol = (PERIODIC ? xr : x) + 1;
    const bool out_ok = lane >= 1 && x >= 0 && x < nx;

    auto load = [&](int yy, int xx, bool inx) -> S2 {
      S2 w;
      w.x = S(0);
      w.y = S(0);
      int yw = yy;
      if (PERIODIC) {
        // rows run from y0 - 1 to y1 (y1 + 1 with the prefetch variant): more than one
        // period past the grid when ny is 1 or 2
        if (yw < 0) yw += ny;
        while (yw >= ny) yw -= ny;
      } else if (!(inx && yy >= 0 && yy < ny)) {
        return w;
      }
      const size_t g = size_t(yw) * nx + xx;
      if (!in_bounds(g < size_t(nx) * ny, p.status)) return w;
      if (in_mode == PASS_IO_COMPLEX) {
        w = __ldg(Wi + g);
      } else {
        w.x = __ldg(Ur + g);
        if (in_mode == PASS_IO_PLANAR) w.y = __ldg(Vr + g);
      }
      return w;
    };
    // face pair (east face, north face) of the cell in row yy of this lane's column
    auto faces = [&](int yy) -> A2 {
      A2 f;
      f.x = A(0);
      f.y = A(0);
      if (PERIODIC) {
        if (yy < 0) yy += ny;
        while (yy >= ny) yy -= ny;
      } else if (yy >= ny) {
        return f;  // face pairs exist for rows -1 .. ny-1
      }
      if (!has_faces) return f;
      const size_t fi = size_t(yy + 1) * (nx + 1) + fcol;
      if (!in_bounds(fi < size_t(ny + 1) * (nx + 1), p.status)) return f;
      return __ldg(FEN + fi);
    };

    // prime the stream: row y0, and the difference across the south face of row y0 (the
    // north difference of row y0 - 1) with that face's conductivity
    S2 Wc = load(y0, xr, xin);
    A dSU, dSV, ks;
    {
      const S2 Ws = load(y0 - 1, xr, xin);
      ks = faces(y0 - 1).y;
      dSU = A(Wc.x - Ws.x);
      dSV = A(Wc.y - Ws.y);
    }
#if FRKC2_STREAM_PREFETCH
    // loads for row y+1 are issued one iteration ahead of their use
    S2 Wn = load(y0 + 1, xr, xin);
    A2 f = faces(y0);
    S2 Wen = lane == 31 ? load(y0, xeast, eastin) : Wc;
#endif
#pragma unroll 2
    for (int y = y0; y < y1; ++y) {
#if FRKC2_STREAM_PREFETCH
      const S2 Wnn = load(y + 2, xr, xin);
      const A2 fnext = faces(y + 1);
      const S2 Wenn = lane == 31 ? load(y + 1, xeast, eastin) : Wn;
      S Ue = __shfl_down_sync(0xffffffffu, Wc.x, 1);
      S Ve = __shfl_down_sync(0xffffffffu, Wc.y, 1);
      if (lane == 31) {
        Ue = Wen.x;
        Ve = Wen.y;
      }
#else
      const S2 Wn = load(y + 1, xr, xin);
      const A2 f = faces(y);
      S Ue = __shfl_down_sync(0xffffffffu, Wc.x, 1);
      S Ve = __shfl_down_sync(0xffffffffu, Wc.y, 1);
      if (lane == 31) {
        const S2 We = load(y, xeast, eastin);
        Ue = We.x;
        Ve = We.y;
      }
#endif
      // differences toward the east and north neighbours
      const A dEU = A(Ue - Wc.x), dEV = A(Ve - Wc.y);
      const A dNU = A(Wn.x - Wc.x), dNV = A(Wn.y - Wc.y);
      // west face: the west neighbour's east difference and conductivity; south face: the
      // north difference and conductivity of the row below
      const A dWU = __shfl_up_sync(0xffffffffu, dEU, 1);
      const A dWV = __shfl_up_sync(0xffffffffu, dEV, 1);
      const A kw = __shfl_up_sync(0xffffffffu, f.x, 1);
      const A fU = f.y * dNU - ks * dSU - kw * dWU + f.x * dEU;
      const A fV = f.y * dNV - ks * dSV - kw * dWV + f.x * dEV;
      const S un = Wc.x + ca * S(fU) - cb * S(fV);
      const S vn = Wc.y + ca * S(fV) + cb * S(fU);
      if (out_ok && in_bounds(size_t(y) * nx + x < size_t(nx) * ny, p.status)) {
        const size_t g = size_t(y) * nx + x;
        if (out_mode == PASS_IO_COMPLEX) {
          S2 w;
          w.x = un;
          w.y = vn;
          Wo[g] = w;
        } else {
          Uo[g] = un;
          if (out_mode == PASS_IO_PLANAR) Vo[g] = vn;
        }
        if (p.check_finite) bad |= nonfinite_bits(un);
        if (HAT) static_cast<S*>(p.H_out)[g] = __ldg(static_cast<const S*>(p.H_in) + g) + ca * S(fU);
      }
      dSU = dNU;
      dSV = dNV;
      ks = f.y;
      Wc = Wn;
#if FRKC2_STREAM_PREFETCH
      Wn = Wnn;
      f = fnext;
      Wen = Wenn;
#endif
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

// Face pairs for the streaming pass: FEN(y, x) = (x face x+1 of row y, y face y+1 of column x)
// for y, x in [-1, n), stored at ((y+1)(nx+1) + x+1); entries with no such face are 0.
template <class A>
__global__ void k_face_pairs(const A* __restrict__ fx, const A* __restrict__ fy, void* out, int nx, int ny) {
  using A2 = typename Vec2<A>::type;
  A2* F = static_cast<A2*>(out);
  const size_t total = size_t(ny + 1) * (nx + 1);
  for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
    const int y = int(t / (nx + 1)) - 1, x = int(t % (nx + 1)) - 1;
    A2 v;
    v.x = y >= 0 ? fx[size_t(y) * (nx + 1) + (x + 1)] : A(0);
    v.y = x >= 0 ? fy[size_t(y + 1) * nx + x] : A(0);
    F[t] = v;
  }
}

template <class S, class A, bool PERIODIC, bool HAT>
cudaError_t launch_t(const PassArgs& a, const void* fen, cudaStream_t st) {
  const auto kern = k_stream2d<S, A, PERIODIC, HAT>;
  static const Residency res = query_residency(kern, ST_THREADS, 0);
  if (res.err != cudaSuccess) return res.err;
  const int ncolw = (a.nx + ST_COLS - 1) / ST_COLS;
  const long long total = (long long)ncolw * a.ny;  // (chunk, row) pairs
  long long grid = (long long)res.sms * res.per_sm;
  const long long max_useful = (total + ST_WARPS - 1) / ST_WARPS;
  if (grid > max_useful) grid = max_useful;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid), 1, 1);
  cfg.blockDim = dim3(ST_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, fen, ncolw, total, grid * ST_WARPS);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <class S, class A>
cudaError_t launch_s(const PassArgs& a, const void* fen, cudaStream_t st) {
  if (a.H_out) return a.bc == FRKC2_BC_PERIODIC ? launch_t<S, A, true, true>(a, fen, st) : launch_t<S, A, false, true>(a, fen, st);
  return a.bc == FRKC2_BC_PERIODIC ? launch_t<S, A, true, false>(a, fen, st) : launch_t<S, A, false, false>(a, fen, st);
}

}  // namespace

size_t face_pair_bytes(const frkc2_problem& p) {
  // the streaming passes' [ny + 1][nx + 1] pairs, or the FP32 wavefront pass's padded
  // [ny + 1][nx + 4] pairs (wf2d_face_pitch), whichever the call builds
  return size_t(p.n[1] + 1) * size_t(p.n[0] + 4) * 2 * arith_bytes(p.precision);
}

cudaError_t launch_face_pairs(const frkc2_problem& p, const void* fx, const void* fy, void* out, cudaStream_t st) {
  const int nx = int(p.n[0]), ny = int(p.n[1]);
  const size_t total = size_t(ny + 1) * (nx + 1);
  const int threads = 256;
  const int blocks = int(std::min<size_t>((total + threads - 1) / threads, 152 * 16));
  if (p.precision == FRKC2_FP64)
    k_face_pairs<double><<<blocks, threads, 0, st>>>(static_cast<const double*>(fx), static_cast<const double*>(fy), out, nx, ny);
  else
    k_face_pairs<float><<<blocks, threads, 0, st>>>(static_cast<const float*>(fx), static_cast<const float*>(fy), out, nx, ny);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pass_stream2d(const frkc2_problem& p, const PassArgs& a, const void* fen, cudaStream_t st) {
  switch (p.precision) {
    case FRKC2_FP64: return launch_s<double, double>(a, fen, st);
    case FRKC2_FP32: return launch_s<float, float>(a, fen, st);
    default: return launch_s<double, float>(a, fen, st);
  }
}

}  // namespace frkc2
