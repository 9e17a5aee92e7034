// 2D temporally blocked pass for FP32 (fixed conductivity) with the state in registers:
// k stages of Sec. 3, Eq. 13 per HBM round trip.
//
// A CTA of 16 x 16 threads owns a 64 x 64 region: its output tile (64 - 2k)^2 plus a k-cell
// halo recomputed redundantly (region-edge values go stale one cell per stage, which never
// reaches the output tile).  Thread (tx, ty) owns the 4 x 4 cells at columns 4tx..4tx+3,
// rows 4ty..4ty+3 and keeps, for all k stages, their complex state (32 floats) and their 40
// face conductivities in registers.  Per stage:
//   - the thread's bottom and top rows go to shared memory (double-buffered by stage parity,
//     one barrier per stage); its south and north neighbour rows come back from the threads
//     below and above;
//   - the columns beyond its own come from the adjacent threads by 16-lane shuffles, one row
//     at a time, before that row is updated;
//   - every neighbour difference inside the block is formed once and used by both cells of
//     the face: f = k_n d_n - k_s d_s + k_e d_e - k_w d_w, then the complex update;
//   - the cells are held as horizontal pairs (float2), so the y differences, the y terms of f
//     and the complex update run as packed two-lane FP32 instructions (add / fma .f32x2, new
//     with the sm_100 family), two cells per instruction; the x differences and x terms, whose
//     pairs would straddle the register pairs, stay scalar: 11.5 FP32 instructions per
//     cell-stage for 16.5 floating-point operations.
// Shared memory traffic: 8 bytes per cell-stage (the two exchanged rows), against the full
// state of a shared-memory ping-pong.
// The batched launch runs the same region computation from tb2d_region.cuh; this kernel keeps
// its own copy because, written as that shared device function, it compiled to an 11 % slower
// pass (4.15e11 against 4.61e11 cell-stage/s at 2048^2, k = 8) with the same registers.
#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int RT_R = 64;          // region edge (cells)
constexpr int RT_THREADS = 256;   // 16 x 16 threads of 4 x 4 cells
#ifndef FRKC2_TBR_MIN_BLOCKS
#define FRKC2_TBR_MIN_BLOCKS 2
#endif

__device__ __forceinline__ int wrap_r(int g, int n) {
  if (g >= 0 && g < n) return g;
  if (g < 0 && g >= -n) return g + n;
  if (g >= n && g < 2 * n) return g - n;
  const int r = g % n;
  return r < 0 ? r + n : r;
}

// a - b on both halves in one packed instruction (sm_100 family)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

template <bool PERIODIC>
__global__ void __launch_bounds__(RT_THREADS, FRKC2_TBR_MIN_BLOCKS) k_tb2d_reg(const PassArgs p) {
  __shared__ float4 sh_bot[2][2][16][16];  // [stage parity][U, V][ty][tx]: the thread's row 0
  __shared__ float4 sh_top[2][2][16][16];  // its row 3
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k = p.k;
  const int T = RT_R - 2 * k;
  const int x0 = blockIdx.x * T - k, y0 = blockIdx.y * T - k;
  const int nx = p.nx, ny = p.ny;
  // the next pass may be launched as soon as every CTA of this one is running (it then loads
  // its face conductivities, which no pass writes, and waits below for this pass's state)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const float* __restrict__ Uin = static_cast<const float*>(p.U_in);
  const float* __restrict__ Vin = static_cast<const float*>(p.V_in);
  const float* __restrict__ FX = static_cast<const float*>(p.fx);
  const float* __restrict__ FY = static_cast<const float*>(p.fy);

  // wrapped (periodic) or raw (Dirichlet) grid rows / columns of the thread's cells; the fifth
  // entry is the next row / column (north and east faces)
  int gyr[5], gxc[5];
  bool yin[5], xin[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int gx = x0 + 4 * tx + i, gy = y0 + 4 * ty + i;
    gxc[i] = PERIODIC ? wrap_r(gx, nx) : gx;
    gyr[i] = PERIODIC ? wrap_r(gy, ny) : gy;
    xin[i] = gx >= 0 && gx < nx;
    yin[i] = gy >= 0 && gy < ny;
  }
  // fx[r][c]: x face c of row r (the west face of cell c; c = 4 is the east face of cell 3);
  // fy[r][c]: y face r of column c (the south face of row r; r = 4 is the north face of row 3)
  float fx[4][5], fy[5][4];
  unsigned inside = 0;  // Dirichlet: bit 4r + c set if cell (r, c) lies in the grid
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (r < 4) {
        float v = 0.f;
        if (PERIODIC || (yin[r] && gxc[c] >= 0 && gxc[c] <= nx)) {
          const size_t fi = size_t(gyr[r]) * (nx + 1) + gxc[c];
          if (in_bounds(fi < size_t(ny) * (nx + 1), p.status)) v = FX[fi];
        }
        fx[r][c] = v;
      }
      if (c < 4) {
        float v = 0.f;
        if (PERIODIC || (xin[c] && gyr[r] >= 0 && gyr[r] <= ny)) {
          const size_t fi = size_t(gyr[r]) * nx + gxc[c];
          if (in_bounds(fi < size_t(ny + 1) * nx, p.status)) v = FY[fi];
        }
        fy[r][c] = v;
        if (r < 4 && xin[c] && yin[r]) inside |= 1u << (4 * r + c);
      }
    }
  }
  // the state as horizontal cell pairs: U2[r][h] = (U[r][2h], U[r][2h + 1]); the y faces too
  // the previous pass's state is complete and visible after this (a no-op for a launch
  // without the programmatic-serialization attribute)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  float2 U2[4][2], V2[4][2], FY2[5][2];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) FY2[r][h] = make_float2(fy[r][2 * h], fy[r][2 * h + 1]);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float uu = 0.f, vv = 0.f;
      if (PERIODIC || (inside & (1u << (4 * r + c)))) {
        const size_t g = size_t(gyr[r]) * nx + gxc[c];
        if (in_bounds(g < size_t(nx) * ny, p.status)) {
          uu = Uin[g];
          if (Vin) vv = Vin[g];
        }
      }
      if (c & 1) {
        U2[r][c >> 1].y = uu;
        V2[r][c >> 1].y = vv;
      } else {
        U2[r][c >> 1].x = uu;
        V2[r][c >> 1].x = vv;
      }
    }

  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = 0; j < k; ++j) {
    const int b = j & 1;
    sh_bot[b][0][ty][tx] = make_float4(U2[0][0].x, U2[0][0].y, U2[0][1].x, U2[0][1].y);
    sh_bot[b][1][ty][tx] = make_float4(V2[0][0].x, V2[0][0].y, V2[0][1].x, V2[0][1].y);
    sh_top[b][0][ty][tx] = make_float4(U2[3][0].x, U2[3][0].y, U2[3][1].x, U2[3][1].y);
    sh_top[b][1][ty][tx] = make_float4(V2[3][0].x, V2[3][0].y, V2[3][1].x, V2[3][1].y);
    __syncthreads();
    // the region's outermost thread rows have no neighbour row here: their edge goes stale
    const float4 su4 = ty > 0 ? sh_top[b][0][ty - 1][tx] : z4, sv4 = ty > 0 ? sh_top[b][1][ty - 1][tx] : z4;
    const float4 nu4 = ty < 15 ? sh_bot[b][0][ty + 1][tx] : z4, nv4 = ty < 15 ? sh_bot[b][1][ty + 1][tx] : z4;
    const float ca = p.caf[j], cb = p.cbf[j];
    const float2 ca2 = make_float2(ca, ca), cb2 = make_float2(cb, cb), ncb2 = make_float2(-cb, -cb);
    const float2 su2[2] = {make_float2(su4.x, su4.y), make_float2(su4.z, su4.w)};
    const float2 sv2[2] = {make_float2(sv4.x, sv4.y), make_float2(sv4.z, sv4.w)};
    const float2 nu2[2] = {make_float2(nu4.x, nu4.y), make_float2(nu4.z, nu4.w)};
    const float2 nv2[2] = {make_float2(nv4.x, nv4.y), make_float2(nv4.z, nv4.w)};
    // differences across the south faces of the current row: W(r) - W(r - 1)
    float2 dsU[2], dsV[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      dsU[h] = sub2(U2[0][h], su2[h]);
      dsV[h] = sub2(V2[0][h], sv2[h]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // columns beyond the thread's own, before this row is updated
      const float wU = __shfl_up_sync(0xffffffffu, U2[r][1].y, 1, 16);
      const float wV = __shfl_up_sync(0xffffffffu, V2[r][1].y, 1, 16);
      const float eU = __shfl_down_sync(0xffffffffu, U2[r][0].x, 1, 16);
      const float eV = __shfl_down_sync(0xffffffffu, V2[r][0].x, 1, 16);
      const float u[6] = {wU, U2[r][0].x, U2[r][0].y, U2[r][1].x, U2[r][1].y, eU};
      const float v[6] = {wV, V2[r][0].x, V2[r][0].y, V2[r][1].x, V2[r][1].y, eV};
      // dx[c]: across x face c, W(c) - W(c - 1), each formed once for the two cells of the face
      float dxU[5], dxV[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        dxU[c] = u[c + 1] - u[c];
        dxV[c] = v[c + 1] - v[c];
      }
      // x part of f per cell, written straight into the halves of the pairs
      float2 fU[2], fV[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 2 * h;
        fU[h].x = fx[r][c + 1] * dxU[c + 1] - fx[r][c] * dxU[c];
        fU[h].y = fx[r][c + 2] * dxU[c + 2] - fx[r][c + 1] * dxU[c + 1];
        fV[h].x = fx[r][c + 1] * dxV[c + 1] - fx[r][c] * dxV[c];
        fV[h].y = fx[r][c + 2] * dxV[c + 2] - fx[r][c + 1] * dxV[c + 1];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 nU = r < 3 ? U2[r + 1][h] : nu2[h];
        const float2 nV = r < 3 ? V2[r + 1][h] : nv2[h];
        const float2 dnU = sub2(nU, U2[r][h]), dnV = sub2(nV, V2[r][h]);
        // y part, two cells per instruction: f += k_n d_n - k_s d_s
        const float2 nks = make_float2(-FY2[r][h].x, -FY2[r][h].y);
        fU[h] = __ffma2_rn(nks, dsU[h], __ffma2_rn(FY2[r + 1][h], dnU, fU[h]));
        fV[h] = __ffma2_rn(nks, dsV[h], __ffma2_rn(FY2[r + 1][h], dnV, fV[h]));
        // W += (ca + i cb) f
        float2 un = __ffma2_rn(ncb2, fV[h], __ffma2_rn(ca2, fU[h], U2[r][h]));
        float2 vn = __ffma2_rn(cb2, fU[h], __ffma2_rn(ca2, fV[h], V2[r][h]));
        if (!PERIODIC) {
          if (!(inside & (1u << (4 * r + 2 * h)))) un.x = vn.x = 0.f;
          if (!(inside & (1u << (4 * r + 2 * h + 1)))) un.y = vn.y = 0.f;
        }
        U2[r][h] = un;
        V2[r][h] = vn;
        dsU[h] = dnU;
        dsV[h] = dnV;
      }
    }
  }

  // store the output tile: region cells at distance >= k from the region edge
  float* __restrict__ Uo = static_cast<float*>(p.U_out);
  float* __restrict__ Vo = static_cast<float*>(p.V_out);
  bool bad = false;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int ry = 4 * ty + r;
    const int gy = y0 + ry;
    if (ry < k || ry >= RT_R - k || gy >= ny) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int rx = 4 * tx + c;
      const int gx = x0 + rx;
      if (rx < k || rx >= RT_R - k || gx >= nx) continue;
      const size_t g = size_t(gy) * nx + gx;
      if (!in_bounds(g < size_t(nx) * ny, p.status)) continue;
      const float uu = (c & 1) ? U2[r][c >> 1].y : U2[r][c >> 1].x;
      Uo[g] = uu;
      if (Vo) Vo[g] = (c & 1) ? V2[r][c >> 1].y : V2[r][c >> 1].x;
      if (p.check_finite) bad |= (__float_as_uint(uu) & 0x7f800000u) == 0x7f800000u;
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

}  // namespace

bool tb2d_supported(const frkc2_problem& p, int k) {
  return p.ndim == 2 && p.precision == FRKC2_FP32 && p.kappa_kind != FRKC2_KAPPA_POWER && k >= 1 &&
         2 * k < RT_R;
}

cudaError_t launch_pass_tb2d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st, bool overlap_previous) {
  (void)p;
  const int T = RT_R - 2 * a.k;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((a.nx + T - 1) / T, (a.ny + T - 1) / T, 1);
  cfg.blockDim = dim3(RT_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap_previous ? 1 : 0;
  const cudaError_t e = a.bc == FRKC2_BC_PERIODIC ? cudaLaunchKernelEx(&cfg, k_tb2d_reg<true>, a)
                                                  : cudaLaunchKernelEx(&cfg, k_tb2d_reg<false>, a);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace frkc2
