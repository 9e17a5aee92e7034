// 2D adjoint for FP32 with a fixed conductivity, temporally blocked: both halves of the
// backward sweep run k stages per HBM round trip on the register-tiled 64 x 64 regions of
// the FP32 forward pass (16 x 16 threads, 4 x 4 cells each, k-cell recomputed halo, rows
// exchanged through shared memory, columns by 16-lane shuffles, cells held as horizontal
// pairs for the packed f32x2 instructions).
//
// Tape pass (k_tape_tb2d): the forward stages of Sec. 3, Eq. 13 from the tape entry W^{l0},
// writing every stage state W^{l0+1} .. W^{l0+k} of the output tile to the tape (the last as
// the real step output when the pass ends the step) -- 8 bytes written per cell-stage.
//
// Reverse pass (k_adjrev_tb2d): k adjoint stages, last stage first.  The operator is
// symmetric (J^H = A for a fixed conductivity), so stage l maps
//   lam <- lam + conj(c_l) A lam,                        c_l = dt a_l / dx^2,
// and contributes to dJ/dkappa through every face f between cells m and i
//   G_f = Re(conj(lam_m - lam_i)(Y_m - Y_i)),            Y = -(c_l / 2) W^l,
// half of the face's sensitivity to each of its cells (the 1/2 folded into Y; a Dirichlet
// boundary face gives all of it to its interior cell), both with lam^{l+1}, before the update.
// lam stays in registers for the k stages and each cell sums its dJ/dkappa over them in a
// register (its east and north faces' sensitivities formed by itself, the west one by shuffle,
// the south one from the row below -- for a thread's bottom row from the thread below, one
// stage later), added to the FP64 accumulator once per pass.  The tape entries arrive by
// cp.async in a per-thread ring in shared memory (the thread's four rows and the row above),
// each row's entry for the next stage issued as soon as the current one is read, so the loads
// run a whole stage ahead of their use without holding registers.  Per cell-stage the pass
// reads the tape entry W^l (8 bytes; the halo recomputes (64/48)^2 of it at k = 8) and, once
// per pass, lam in and out, the faces and the accumulator.
#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "tb2d_region.cuh"

namespace frkc2 {
namespace {

constexpr int AT_KMAX = 16;

struct AdjTbArgs {
  int nx, ny;
  int k;    // halo width of the launch (the output tile is 64 - 2k)
  int nst;  // stages in this pass, 1 .. k
  const float* fx;  // x faces [ny][nx + 1], y faces [ny + 1][nx] (face i between cells i-1, i)
  const float* fy;
  // tape pass
  const void* in;           // W^{l0}: interleaved (U, V) or real
  int in_complex;
  void* out[AT_KMAX];       // W^{l0+1+j}, interleaved; the last real when last_real
  int last_real;
  // reverse pass, stage j = the j-th stage from the end of the pass
  const void* W[AT_KMAX];   // W^l: interleaved, or real (imaginary part 0) when !w_complex[j]
  int w_complex[AT_KMAX];
  const void* L_in;         // lam^{l_hi}
  int l_mode;               // 0: real array, 1: interleaved, 2: real part of an interleaved array
  float2* L_out;            // lam^{l_hi - nst}, interleaved
  double* dk;               // dJ/dkappa per cell (FP64 accumulator) or nullptr
  float ca[AT_KMAX];        // dt Re(a_l) / dx^2 of stage j, rounded to float once on the host
  float cb[AT_KMAX];
  unsigned* status;
  int check_finite;
};

struct RevShared {
  float4 bot[2][2][16][16];  // [parity][lam x, lam y][ty][tx]: the thread's row 0
  float4 top[2][3][16][16];  // [parity][lam x, lam y, north-face sensitivity][ty][tx]: its row 3
  float4 fx4[4][RT_THREADS];  // x faces 0..3 of row r (face 4 is the east thread's face 0)
  float4 fy4[4][RT_THREADS];  // y faces of row r (row 4 is the north thread's row 0)
  float4 ring[5][2][RT_THREADS];  // tape entries of the thread's rows 0..3 and the row above,
                                  // two cells per float4, filled by cp.async a stage ahead
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(unsigned(__cvta_generic_to_shared(smem))), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(unsigned(__cvta_generic_to_shared(smem))), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(unsigned(__cvta_generic_to_shared(smem))), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// at most 4 groups still in flight: with one group committed per ring row and stage, the
// group of the row about to be read (issued a stage earlier) has landed
__device__ __forceinline__ void cp_wait4() { asm volatile("cp.async.wait_group 4;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Grid rows / columns of a thread's cells (fifth entry: the next row / column), their
// in-grid flags, the Dirichlet inside mask and the output-tile mask (bit 4r + c).
struct RegionIdx {
  int gyr[5], gxc[5];
  bool yin[5], xin[5];
  unsigned inside, outm;
};

template <bool PERIODIC>
__device__ __forceinline__ RegionIdx region_idx(int nx, int ny, int k, int x0, int y0, int tx, int ty) {
  RegionIdx R;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int gx = x0 + 4 * tx + i, gy = y0 + 4 * ty + i;
    R.gxc[i] = PERIODIC ? wrap_r(gx, nx) : gx;
    R.gyr[i] = PERIODIC ? wrap_r(gy, ny) : gy;
    R.xin[i] = gx >= 0 && gx < nx;
    R.yin[i] = gy >= 0 && gy < ny;
  }
  R.inside = 0;
  R.outm = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int ry = 4 * ty + r, rx = 4 * tx + c;
      if (R.xin[c] && R.yin[r]) {
        R.inside |= 1u << (4 * r + c);
        if (ry >= k && ry < RT_R - k && rx >= k && rx < RT_R - k) R.outm |= 1u << (4 * r + c);
      }
    }
  return R;
}

// x face c of row r and y face r of column c, 0 outside a Dirichlet grid
template <bool PERIODIC>
__device__ __forceinline__ float face_x(const RegionIdx& R, const float* __restrict__ FX, int nx, int r, int c) {
  if (PERIODIC || (R.yin[r] && R.gxc[c] >= 0 && R.gxc[c] <= nx)) return FX[size_t(R.gyr[r]) * (nx + 1) + R.gxc[c]];
  return 0.f;
}
template <bool PERIODIC>
__device__ __forceinline__ float face_y(const RegionIdx& R, const float* __restrict__ FY, int nx, int ny, int r, int c) {
  if (PERIODIC || (R.xin[c] && R.gyr[r] >= 0 && R.gyr[r] <= ny)) return FY[size_t(R.gyr[r]) * nx + R.gxc[c]];
  return 0.f;
}

__device__ __forceinline__ float2 pairh(float4 a, int h) { return h ? make_float2(a.z, a.w) : make_float2(a.x, a.y); }
__device__ __forceinline__ float halfv(float2 a, int i) { return i ? a.y : a.x; }
__device__ __forceinline__ void set_half(float2& a, int i, float v) {
  if (i)
    a.y = v;
  else
    a.x = v;
}

// ------------------------------------------------------------------------------------------
// Tape pass: forward stages, every stage state of the output tile written.

template <bool PERIODIC>
__global__ void __launch_bounds__(RT_THREADS, 2) k_tape_tb2d(const AdjTbArgs a) {
  __shared__ float4 sh_bot[2][2][16][16];  // [parity][U, V][ty][tx]: the thread's row 0
  __shared__ float4 sh_top[2][2][16][16];  // its row 3
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k = a.k, T = RT_R - 2 * k;
  const int x0 = blockIdx.x * T - k, y0 = blockIdx.y * T - k;
  const int nx = a.nx, ny = a.ny;
  // launched with programmatic stream serialization: the next launch may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const RegionIdx R = region_idx<PERIODIC>(nx, ny, k, x0, y0, tx, ty);
  // x faces 0..3 of each row; face 4 (the east face of cell 3) is the east thread's face 0, taken
  // by shuffle where it is used (the region's east column of threads gets its own face 0 there,
  // which only reaches halo cells: a wrong edge face spreads one cell per stage, nst <= k)
  float fx[4][4];
  float2 FY2[5][2];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    if (r < 4)
#pragma unroll
      for (int c = 0; c < 4; ++c) fx[r][c] = face_x<PERIODIC>(R, a.fx, nx, r, c);
#pragma unroll
    for (int h = 0; h < 2; ++h)
      FY2[r][h] = make_float2(face_y<PERIODIC>(R, a.fy, nx, ny, r, 2 * h), face_y<PERIODIC>(R, a.fy, nx, ny, r, 2 * h + 1));
  }
  float2 U2[4][2], V2[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float uu = 0.f, vv = 0.f;
      if (PERIODIC || (R.inside & (1u << (4 * r + c)))) {
        const size_t g = size_t(R.gyr[r]) * nx + R.gxc[c];
        if (a.in_complex) {
          const float2 w = static_cast<const float2*>(a.in)[g];
          uu = w.x;
          vv = w.y;
        } else {
          uu = static_cast<const float*>(a.in)[g];
        }
      }
      set_half(U2[r][c >> 1], c & 1, uu);
      set_half(V2[r][c >> 1], c & 1, vv);
    }

  bool bad = false;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = 0; j < a.nst; ++j) {
    const int b = j & 1;
    sh_bot[b][0][ty][tx] = make_float4(U2[0][0].x, U2[0][0].y, U2[0][1].x, U2[0][1].y);
    sh_bot[b][1][ty][tx] = make_float4(V2[0][0].x, V2[0][0].y, V2[0][1].x, V2[0][1].y);
    sh_top[b][0][ty][tx] = make_float4(U2[3][0].x, U2[3][0].y, U2[3][1].x, U2[3][1].y);
    sh_top[b][1][ty][tx] = make_float4(V2[3][0].x, V2[3][0].y, V2[3][1].x, V2[3][1].y);
    __syncthreads();
    const float4 su4 = ty > 0 ? sh_top[b][0][ty - 1][tx] : z4, sv4 = ty > 0 ? sh_top[b][1][ty - 1][tx] : z4;
    const float4 nu4 = ty < 15 ? sh_bot[b][0][ty + 1][tx] : z4, nv4 = ty < 15 ? sh_bot[b][1][ty + 1][tx] : z4;
    const float ca = a.ca[j], cb = a.cb[j];
    const float2 ca2 = make_float2(ca, ca), cb2 = make_float2(cb, cb), ncb2 = make_float2(-cb, -cb);
    float2 dsU[2], dsV[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      dsU[h] = sub2(U2[0][h], pairh(su4, h));
      dsV[h] = sub2(V2[0][h], pairh(sv4, h));
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float wU = __shfl_up_sync(0xffffffffu, U2[r][1].y, 1, 16);
      const float wV = __shfl_up_sync(0xffffffffu, V2[r][1].y, 1, 16);
      const float eU = __shfl_down_sync(0xffffffffu, U2[r][0].x, 1, 16);
      const float eV = __shfl_down_sync(0xffffffffu, V2[r][0].x, 1, 16);
      const float u[6] = {wU, U2[r][0].x, U2[r][0].y, U2[r][1].x, U2[r][1].y, eU};
      const float v[6] = {wV, V2[r][0].x, V2[r][0].y, V2[r][1].x, V2[r][1].y, eV};
      float dxU[5], dxV[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        dxU[c] = u[c + 1] - u[c];
        dxV[c] = v[c + 1] - v[c];
      }
      const float kx[5] = {fx[r][0], fx[r][1], fx[r][2], fx[r][3], __shfl_down_sync(0xffffffffu, fx[r][0], 1, 16)};
      float2 fU[2], fV[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 2 * h;
        fU[h].x = kx[c + 1] * dxU[c + 1] - kx[c] * dxU[c];
        fU[h].y = kx[c + 2] * dxU[c + 2] - kx[c + 1] * dxU[c + 1];
        fV[h].x = kx[c + 1] * dxV[c + 1] - kx[c] * dxV[c];
        fV[h].y = kx[c + 2] * dxV[c + 2] - kx[c + 1] * dxV[c + 1];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 nU = r < 3 ? U2[r + 1][h] : pairh(nu4, h);
        const float2 nV = r < 3 ? V2[r + 1][h] : pairh(nv4, h);
        const float2 dnU = sub2(nU, U2[r][h]), dnV = sub2(nV, V2[r][h]);
        const float2 nks = make_float2(-FY2[r][h].x, -FY2[r][h].y);
        fU[h] = __ffma2_rn(nks, dsU[h], __ffma2_rn(FY2[r + 1][h], dnU, fU[h]));
        fV[h] = __ffma2_rn(nks, dsV[h], __ffma2_rn(FY2[r + 1][h], dnV, fV[h]));
        float2 un = __ffma2_rn(ncb2, fV[h], __ffma2_rn(ca2, fU[h], U2[r][h]));
        float2 vn = __ffma2_rn(cb2, fU[h], __ffma2_rn(ca2, fV[h], V2[r][h]));
        if (!PERIODIC) {
          if (!(R.inside & (1u << (4 * r + 2 * h)))) un.x = vn.x = 0.f;
          if (!(R.inside & (1u << (4 * r + 2 * h + 1)))) un.y = vn.y = 0.f;
        }
        U2[r][h] = un;
        V2[r][h] = vn;
        dsU[h] = dnU;
        dsV[h] = dnV;
      }
    }
    // this stage's state of the output tile to the tape
    const bool real_out = a.last_real && j == a.nst - 1;
    void* out = a.out[j];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (!(R.outm & (1u << (4 * r + c)))) continue;
        const size_t g = size_t(y0 + 4 * ty + r) * nx + (x0 + 4 * tx + c);
        const float uu = halfv(U2[r][c >> 1], c & 1);
        if (real_out) {
          static_cast<float*>(out)[g] = uu;
          if (a.check_finite) bad |= (__float_as_uint(uu) & 0x7f800000u) == 0x7f800000u;
        } else {
          static_cast<float2*>(out)[g] = make_float2(uu, halfv(V2[r][c >> 1], c & 1));
        }
      }
  }
  if (bad) atomicOr(a.status, ST_NONFINITE);
}

// ------------------------------------------------------------------------------------------
// Reverse pass.

template <bool PERIODIC>
__global__ void __launch_bounds__(RT_THREADS, 2) k_adjrev_tb2d(const AdjTbArgs a) {
  extern __shared__ __align__(16) unsigned char at_smem[];
  RevShared& sh = *reinterpret_cast<RevShared*>(at_smem);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int k = a.k, T = RT_R - 2 * k;
  const int x0 = blockIdx.x * T - k, y0 = blockIdx.y * T - k;
  const int nx = a.nx, ny = a.ny;
  // launched with programmatic stream serialization: the next launch may start its CTAs as this
  // one's exit, and every global load below comes after the previous launch has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const RegionIdx R = region_idx<PERIODIC>(nx, ny, k, x0, y0, tx, ty);

  // tape entries of stage jj for ring row i (i = 4: the grid row above the thread's rows):
  // complex entries as (x, y) per cell, two cells per float4; real entries as the four values
  // of ring[i][0].  Four consecutive aligned cells go as 16-byte copies.
  auto issue = [&](int jj, int i) {
    if (jj < a.nst) {
      const bool wc = a.w_complex[jj] != 0;
      const char* Wp = static_cast<const char*>(a.W[jj]);
      const int g0 = R.gyr[i] * nx + R.gxc[0];  // cells < 2^31 (checked on the host)
      const bool run = PERIODIC ? R.gxc[3] == R.gxc[0] + 3 : (R.yin[i] && R.xin[0] && R.xin[3]);
      if (run && (g0 & (wc ? 1 : 3)) == 0) {
        if (wc) {
          cp_async16(&sh.ring[i][0][tid], Wp + size_t(g0) * 8);
          cp_async16(&sh.ring[i][1][tid], Wp + size_t(g0) * 8 + 16);
        } else {
          cp_async16(&sh.ring[i][0][tid], Wp + size_t(g0) * 4);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (!(PERIODIC || (R.yin[i] && R.xin[c]))) continue;
          const int g = R.gyr[i] * nx + R.gxc[c];
          if (wc)
            cp_async8(reinterpret_cast<float*>(&sh.ring[i][c >> 1][tid]) + 2 * (c & 1), Wp + size_t(g) * 8);
          else
            cp_async4(reinterpret_cast<float*>(&sh.ring[i][0][tid]) + c, Wp + size_t(g) * 4);
        }
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int i = 0; i < 5; ++i) issue(0, i);

#pragma unroll
  for (int r = 0; r < 4; ++r) {
    sh.fx4[r][tid] = make_float4(face_x<PERIODIC>(R, a.fx, nx, r, 0), face_x<PERIODIC>(R, a.fx, nx, r, 1),
                                 face_x<PERIODIC>(R, a.fx, nx, r, 2), face_x<PERIODIC>(R, a.fx, nx, r, 3));
    sh.fy4[r][tid] = make_float4(face_y<PERIODIC>(R, a.fy, nx, ny, r, 0), face_y<PERIODIC>(R, a.fy, nx, ny, r, 1),
                                 face_y<PERIODIC>(R, a.fy, nx, ny, r, 2), face_y<PERIODIC>(R, a.fy, nx, ny, r, 3));
  }
  // the faces beyond the thread's own cells (x face 4 of each row, the y faces of row 4) are
  // the east thread's x face 0 and the north thread's row-0 y faces, read from shared memory;
  // the region's east column and north row of threads take 0 there, which only reaches halo
  // cells (a wrong face at the region's edge spreads one cell per stage, at most nst <= k)
  // Dirichlet: a boundary face gives all of its sensitivity to its interior cell
  unsigned bE = 0, bW = 0, bN = 0, bS = 0;
  if (!PERIODIC) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gx = x0 + 4 * tx + c, gy = y0 + 4 * ty + r, bit = 1 << (4 * r + c);
        if (gx == nx - 1) bE |= bit;
        if (gx == 0) bW |= bit;
        if (gy == ny - 1) bN |= bit;
        if (gy == 0) bS |= bit;
      }
  }
  auto wgt = [&](unsigned m, int bit, float g) { return (!PERIODIC && (m & (1u << bit))) ? g + g : g; };

  // lam as horizontal cell pairs: LX[r][h] = (Re lam of cell (r, 2h), of cell (r, 2h + 1))
  float2 LX[4][2], LY[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float lx = 0.f, ly = 0.f;
      if (PERIODIC || (R.inside & (1u << (4 * r + c)))) {
        const size_t g = size_t(R.gyr[r]) * nx + R.gxc[c];
        if (a.l_mode == 1) {
          const float2 w = static_cast<const float2*>(a.L_in)[g];
          lx = w.x;
          ly = w.y;
        } else if (a.l_mode == 2) {
          lx = static_cast<const float2*>(a.L_in)[g].x;
        } else {
          lx = static_cast<const float*>(a.L_in)[g];
        }
      }
      set_half(LX[r][c >> 1], c & 1, lx);
      set_half(LY[r][c >> 1], c & 1, ly);
    }
  float dk[4][4];  // dJ/dkappa of each cell over the pass's stages
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) dk[r][c] = 0.f;
  float gn3[4] = {0.f, 0.f, 0.f, 0.f};  // north-face sensitivities of row 3, passed up a stage later
  __syncthreads();  // faces in shared memory

  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = 0; j < a.nst; ++j) {
    const int b = j & 1;
    const float ca = a.ca[j], cb = a.cb[j];
    const float hr = 0.5f * ca, hi = 0.5f * cb;
    const bool wc = a.w_complex[j] != 0;
    // Y = -(c/2) W^l of ring row i (0 outside a Dirichlet grid); ring rows hold stage j now
    auto yrow = [&](int i, float2 (&yx2)[2], float2 (&yy2)[2]) {
      const float4 p0 = sh.ring[i][0][tid], p1 = sh.ring[i][1][tid];
      const float w[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
      const float wr[4] = {p0.x, p0.y, p0.z, p0.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const bool in = PERIODIC || (R.yin[i] && R.xin[c]);
        const float wx = in ? (wc ? w[2 * c] : wr[c]) : 0.f;
        const float wy = in && wc ? w[2 * c + 1] : 0.f;
        set_half(yx2[c >> 1], c & 1, hi * wy - hr * wx);
        set_half(yy2[c >> 1], c & 1, -(hi * wx) - hr * wy);
      }
    };
    cp_wait4();
    float2 YXc[2], YYc[2];
    yrow(0, YXc, YYc);
    issue(j + 1, 0);
    sh.bot[b][0][ty][tx] = make_float4(LX[0][0].x, LX[0][0].y, LX[0][1].x, LX[0][1].y);
    sh.bot[b][1][ty][tx] = make_float4(LY[0][0].x, LY[0][0].y, LY[0][1].x, LY[0][1].y);
    sh.top[b][0][ty][tx] = make_float4(LX[3][0].x, LX[3][0].y, LX[3][1].x, LX[3][1].y);
    sh.top[b][1][ty][tx] = make_float4(LY[3][0].x, LY[3][0].y, LY[3][1].x, LY[3][1].y);
    sh.top[b][2][ty][tx] = make_float4(gn3[0], gn3[1], gn3[2], gn3[3]);  // previous stage's
    __syncthreads();
    // the region's outermost thread rows have no neighbour row here: their edge goes stale
    const float4 slx = ty > 0 ? sh.top[b][0][ty - 1][tx] : z4, sly = ty > 0 ? sh.top[b][1][ty - 1][tx] : z4;
    const float4 nlx = ty < 15 ? sh.bot[b][0][ty + 1][tx] : z4, nly = ty < 15 ? sh.bot[b][1][ty + 1][tx] : z4;
    {  // the south faces of row 0, from the thread below, one stage late
      const float4 gs = ty > 0 ? sh.top[b][2][ty - 1][tx] : z4;
      dk[0][0] += wgt(bS, 0, gs.x);
      dk[0][1] += wgt(bS, 1, gs.y);
      dk[0][2] += wgt(bS, 2, gs.z);
      dk[0][3] += wgt(bS, 3, gs.w);
    }
    const float2 ca2 = make_float2(ca, ca), cb2 = make_float2(cb, cb), ncb2 = make_float2(-cb, -cb);
    float2 dsX[2], dsY[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      dsX[h] = sub2(LX[0][h], pairh(slx, h));
      dsY[h] = sub2(LY[0][h], pairh(sly, h));
    }
    float gs[4] = {0.f, 0.f, 0.f, 0.f};  // north-face sensitivities of the row below (this stage)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // Y of the row above (ring row r + 1; row 4 is the grid row above the thread's)
      cp_wait4();
      float2 YXn[2], YYn[2];
      yrow(r + 1, YXn, YYn);
      issue(j + 1, r + 1);
      const float wX = __shfl_up_sync(0xffffffffu, LX[r][1].y, 1, 16);
      const float wY = __shfl_up_sync(0xffffffffu, LY[r][1].y, 1, 16);
      const float eX = __shfl_down_sync(0xffffffffu, LX[r][0].x, 1, 16);
      const float eY = __shfl_down_sync(0xffffffffu, LY[r][0].x, 1, 16);
      const float yeX = __shfl_down_sync(0xffffffffu, YXc[0].x, 1, 16);
      const float yeY = __shfl_down_sync(0xffffffffu, YYc[0].x, 1, 16);
      const float lx[6] = {wX, LX[r][0].x, LX[r][0].y, LX[r][1].x, LX[r][1].y, eX};
      const float ly[6] = {wY, LY[r][0].x, LY[r][0].y, LY[r][1].x, LY[r][1].y, eY};
      const float yx[5] = {YXc[0].x, YXc[0].y, YXc[1].x, YXc[1].y, yeX};
      const float yy[5] = {YYc[0].x, YYc[0].y, YYc[1].x, YYc[1].y, yeY};
      // lam differences across x faces 0..4 (face c between cells c - 1 and c)
      float dX[5], dY[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        dX[c] = lx[c + 1] - lx[c];
        dY[c] = ly[c + 1] - ly[c];
      }
      const float4 k4 = sh.fx4[r][tid];
      const float kx[5] = {k4.x, k4.y, k4.z, k4.w, tx < 15 ? sh.fx4[r][tid + 1].x : 0.f};
      float2 fX[2], fY[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 2 * h;
        fX[h].x = kx[c + 1] * dX[c + 1] - kx[c] * dX[c];
        fX[h].y = kx[c + 2] * dX[c + 2] - kx[c + 1] * dX[c + 1];
        fY[h].x = kx[c + 1] * dY[c + 1] - kx[c] * dY[c];
        fY[h].y = kx[c + 2] * dY[c + 2] - kx[c + 1] * dY[c + 1];
      }
      // east-face sensitivities; the west face of cell 0 is the west thread's cell 3 east face
      float ge[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) ge[c] = dX[c + 1] * (yx[c + 1] - yx[c]) + dY[c + 1] * (yy[c + 1] - yy[c]);
      const float gw0 = __shfl_up_sync(0xffffffffu, ge[3], 1, 16);
      const float4 ks4 = sh.fy4[r][tid];
      const float4 kn4 = r < 3 ? sh.fy4[r + 1 < 4 ? r + 1 : 3][tid] : (ty < 15 ? sh.fy4[0][tid + 16] : z4);
      float2 gn2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 nX = r < 3 ? LX[r + 1 < 4 ? r + 1 : 3][h] : pairh(nlx, h);
        const float2 nY = r < 3 ? LY[r + 1 < 4 ? r + 1 : 3][h] : pairh(nly, h);
        const float2 dnX = sub2(nX, LX[r][h]), dnY = sub2(nY, LY[r][h]);
        // north-face sensitivities, two cells per instruction
        gn2[h] = __ffma2_rn(dnY, sub2(YYn[h], YYc[h]), __fmul2_rn(dnX, sub2(YXn[h], YXc[h])));
        const float2 ks = pairh(ks4, h), kn = pairh(kn4, h);
        const float2 nks = make_float2(-ks.x, -ks.y);
        fX[h] = __ffma2_rn(nks, dsX[h], __ffma2_rn(kn, dnX, fX[h]));
        fY[h] = __ffma2_rn(nks, dsY[h], __ffma2_rn(kn, dnY, fY[h]));
        // lam += conj(c) A lam
        float2 ox = __ffma2_rn(cb2, fY[h], __ffma2_rn(ca2, fX[h], LX[r][h]));
        float2 oy = __ffma2_rn(ncb2, fX[h], __ffma2_rn(ca2, fY[h], LY[r][h]));
        if (!PERIODIC) {
          if (!(R.inside & (1u << (4 * r + 2 * h)))) ox.x = oy.x = 0.f;
          if (!(R.inside & (1u << (4 * r + 2 * h + 1)))) ox.y = oy.y = 0.f;
        }
        LX[r][h] = ox;
        LY[r][h] = oy;
        dsX[h] = dnX;
        dsY[h] = dnY;
      }
      const float gn[4] = {gn2[0].x, gn2[0].y, gn2[1].x, gn2[1].y};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int bit = 4 * r + c;
        const float gwc = c == 0 ? gw0 : ge[c > 0 ? c - 1 : 0];
        float acc = wgt(bE, bit, ge[c]) + wgt(bW, bit, gwc) + wgt(bN, bit, gn[c]);
        if (r > 0) acc += wgt(bS, bit, gs[c]);  // row 0's comes from the thread below, later
        dk[r][c] += acc;
        gs[c] = gn[c];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        YXc[h] = YXn[h];
        YYc[h] = YYn[h];
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) gn3[c] = gs[c];
  }
  cp_wait0();

  // the last stage's south faces of row 0, through the parity buffer the last stage did not
  // read (its last readers finished before that stage's barrier)
  const int b = a.nst & 1;
  sh.top[b][2][ty][tx] = make_float4(gn3[0], gn3[1], gn3[2], gn3[3]);
  __syncthreads();
  {
    const float4 gs = ty > 0 ? sh.top[b][2][ty - 1][tx] : z4;
    dk[0][0] += wgt(bS, 0, gs.x);
    dk[0][1] += wgt(bS, 1, gs.y);
    dk[0][2] += wgt(bS, 2, gs.z);
    dk[0][3] += wgt(bS, 3, gs.w);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(R.outm & (1u << (4 * r + c)))) continue;
      const size_t g = size_t(y0 + 4 * ty + r) * nx + (x0 + 4 * tx + c);
      a.L_out[g] = make_float2(halfv(LX[r][c >> 1], c & 1), halfv(LY[r][c >> 1], c & 1));
      if (a.dk) a.dk[g] += double(dk[r][c]);
    }
}

template <bool PERIODIC>
cudaError_t launch_rev(const AdjTbArgs& a, dim3 grid, cudaStream_t st) {
  const auto kern = k_adjrev_tb2d<PERIODIC>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(RevShared)));
  if (attr != cudaSuccess) return attr;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(RT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = sizeof(RevShared);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, a);
    if (le != cudaSuccess) return le;
  }
  count_launch();
  return cudaGetLastError();
}

AdjTbArgs base_args(const frkc2_problem& p, int k, int nst, const void* fx, const void* fy, unsigned* status) {
  AdjTbArgs a{};
  a.nx = int(p.n[0]);
  a.ny = int(p.n[1]);
  a.k = k;
  a.nst = nst;
  a.fx = static_cast<const float*>(fx);
  a.fy = static_cast<const float*>(fy);
  a.status = status;
  return a;
}

dim3 region_grid(const frkc2_problem& p, int k) {
  const int T = RT_R - 2 * k;
  return dim3(unsigned((p.n[0] + T - 1) / T), unsigned((p.n[1] + T - 1) / T), 1);
}

}  // namespace

bool adj_tb2d_supported(const frkc2_problem& p, int k) {
  return p.ndim == 2 && p.precision == FRKC2_FP32 && p.kappa_kind != FRKC2_KAPPA_POWER && k >= 1 &&
         k <= AT_KMAX && 2 * k < RT_R && p.n[0] * p.n[1] < (int64_t(1) << 31);
}

cudaError_t launch_tape_tb2d(const frkc2_problem& p, int k, const AdjTbPass& t, const void* fx, const void* fy,
                             unsigned* status, cudaStream_t st) {
  AdjTbArgs a = base_args(p, k, t.nst, fx, fy, status);
  a.in = t.in;
  a.in_complex = t.in_complex;
  a.last_real = t.last_real;
  a.check_finite = t.last_real;
  for (int j = 0; j < t.nst; ++j) {
    a.out[j] = t.out[j];
    a.ca[j] = float(t.ca[j]);
    a.cb[j] = float(t.cb[j]);
  }
  const dim3 grid = region_grid(p, k);
  const auto tk = p.bc == FRKC2_BC_PERIODIC ? k_tape_tb2d<true> : k_tape_tb2d<false>;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(RT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, tk, a);
    if (le != cudaSuccess) return le;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_adjrev_tb2d(const frkc2_problem& p, int k, const AdjTbPass& t, const void* fx, const void* fy,
                               unsigned* status, cudaStream_t st) {
  AdjTbArgs a = base_args(p, k, t.nst, fx, fy, status);
  a.L_in = t.L_in;
  a.l_mode = t.l_mode;
  a.L_out = static_cast<float2*>(t.L_out);
  a.dk = t.dk;
  a.check_finite = 0;
  for (int j = 0; j < t.nst; ++j) {
    a.W[j] = t.W[j];
    a.w_complex[j] = t.w_complex[j];
    a.ca[j] = float(t.ca[j]);
    a.cb[j] = float(t.cb[j]);
  }
  const dim3 grid = region_grid(p, k);
  return p.bc == FRKC2_BC_PERIODIC ? launch_rev<true>(a, grid, st) : launch_rev<false>(a, grid, st);
}

}  // namespace frkc2
