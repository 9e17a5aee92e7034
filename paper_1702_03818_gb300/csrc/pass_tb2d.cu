// 2D temporally blocked pass for FP32 (fixed conductivity): k stages of Sec. 3, Eq. 13 per
// HBM round trip, the stages computed in shared memory and registers.
//
// A CTA of 16 x (64/PY) threads owns a 64 x 64 region: its output tile (64 - 2k)^2 plus a
// k-cell halo (recomputed redundantly).  Every stage updates every region cell; values near
// the region edge go stale one cell per stage, which never reaches the output tile.  Thread
// (tx, ty) owns the 4 x PY cells at columns 4tx..4tx+3, rows PY ty..PY ty+PY-1 (PY = 2 gives
// 512-thread CTAs and twice the resident warps of PY = 4, for the same shared memory):
//   - the state ping-pongs between two shared buffers; a thread reads its rows as float4,
//     walking up its 4 rows with the row below and above in registers;
//   - the x neighbours beyond its 4 columns come from the adjacent threads by 16-lane
//     shuffles (the region's outermost columns get wrapped-around values, which are stale
//     anyway);
//   - its face conductivities (5 x faces per row, 5 y faces per column) stay in registers
//     for all k stages;
//   - each face flux is formed once and used by both of its cells.
#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int TB_R = 64;          // region edge (cells)
constexpr int TB_ROWS = TB_R + 2; // shared rows: region rows at 1..64, zero rows 0 and 65
#ifndef FRKC2_TB_PY
#define FRKC2_TB_PY 4
#endif
constexpr int TB_PY = FRKC2_TB_PY;          // rows per thread
constexpr int TB_THREADS = 16 * (TB_R / TB_PY);

__device__ __forceinline__ int wrap_t(int g, int n) {
  if (g >= 0 && g < n) return g;
  if (g < 0 && g >= -n) return g + n;
  if (g >= n && g < 2 * n) return g - n;
  const int r = g % n;
  return r < 0 ? r + n : r;
}

template <bool PERIODIC>
__global__ void __launch_bounds__(TB_THREADS, 2) k_tb2d_f32(const PassArgs p) {
  constexpr int PY = TB_PY;
  extern __shared__ __align__(16) float tb_smem[];
  float* Ub[2] = {tb_smem, tb_smem + 2 * TB_ROWS * TB_R};
  float* Vb[2] = {tb_smem + TB_ROWS * TB_R, tb_smem + 3 * TB_ROWS * TB_R};
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k = p.k;
  const int T = TB_R - 2 * k;
  const int x0 = blockIdx.x * T - k, y0 = blockIdx.y * T - k;
  const int nx = p.nx, ny = p.ny;
  const float* __restrict__ Uin = static_cast<const float*>(p.U_in);
  const float* __restrict__ Vin = static_cast<const float*>(p.V_in);
  const float* __restrict__ FX = static_cast<const float*>(p.fx);
  const float* __restrict__ FY = static_cast<const float*>(p.fy);

  // wrapped (periodic) or raw (Dirichlet) grid rows / columns of the thread's 5 rows and
  // 5 columns (the fifth is the next row / column, for the north and east faces)
  int gyr[PY + 1], gxc[5];
  bool yin[PY + 1], xin[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int gx = x0 + 4 * tx + i;
    gxc[i] = PERIODIC ? wrap_t(gx, nx) : gx;
    xin[i] = gx >= 0 && gx < nx;
  }
#pragma unroll
  for (int i = 0; i <= PY; ++i) {
    const int gy = y0 + PY * ty + i;
    gyr[i] = PERIODIC ? wrap_t(gy, ny) : gy;
    yin[i] = gy >= 0 && gy < ny;
  }
  // faces in registers: fx[r][c] = west face of cell c (c = 4 is the east face of cell 3),
  // fy[r][c] = south face of row r (r = 4 is the north face of row 3)
  float fx[PY][5], fy[PY + 1][4];
  unsigned inside = 0;  // Dirichlet: bit r*4+c set if the cell lies in the grid
#pragma unroll
  for (int r = 0; r <= PY; ++r) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (r < PY) {
        float v = 0.f;
        if (PERIODIC) {
          // face index of the west face of the wrapped column (face nx equals face 0)
          v = FX[size_t(gyr[r]) * (nx + 1) + gxc[c]];
        } else if (yin[r] && gxc[c] >= 0 && gxc[c] <= nx) {
          v = FX[size_t(gyr[r]) * (nx + 1) + gxc[c]];
        }
        fx[r][c] = v;
      }
      if (c < 4) {
        float v = 0.f;
        if (PERIODIC) {
          v = FY[size_t(gyr[r]) * nx + gxc[c]];
        } else if (xin[c] && gyr[r] >= 0 && gyr[r] <= ny) {
          v = FY[size_t(gyr[r]) * nx + gxc[c]];
        }
        fy[r][c] = v;
        if (r < PY && xin[c] && yin[r]) inside |= 1u << (r * 4 + c);
      }
    }
  }
  // state into buffer 0; zero the border rows of both buffers
#pragma unroll
  for (int r = 0; r < PY; ++r) {
    float u4[4], v4[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float uu = 0.f, vv = 0.f;
      if (PERIODIC || (inside & (1u << (r * 4 + c)))) {
        const size_t g = size_t(gyr[r]) * nx + gxc[c];
        uu = Uin[g];
        if (Vin) vv = Vin[g];
      }
      u4[c] = uu;
      v4[c] = vv;
    }
    const int row = PY * ty + r + 1;
    *reinterpret_cast<float4*>(&Ub[0][row * TB_R + 4 * tx]) = make_float4(u4[0], u4[1], u4[2], u4[3]);
    *reinterpret_cast<float4*>(&Vb[0][row * TB_R + 4 * tx]) = make_float4(v4[0], v4[1], v4[2], v4[3]);
  }
  if (ty == 0) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      *reinterpret_cast<float4*>(&Ub[b][4 * tx]) = z;
      *reinterpret_cast<float4*>(&Vb[b][4 * tx]) = z;
      *reinterpret_cast<float4*>(&Ub[b][(TB_ROWS - 1) * TB_R + 4 * tx]) = z;
      *reinterpret_cast<float4*>(&Vb[b][(TB_ROWS - 1) * TB_R + 4 * tx]) = z;
    }
  }
  __syncthreads();

  for (int j = 0; j < k; ++j) {
    const float* us = Ub[j & 1];
    const float* vs = Vb[j & 1];
    float* ud = Ub[(j + 1) & 1];
    float* vd = Vb[(j + 1) & 1];
    const float ca = p.caf[j], cb = p.cbf[j];
    const int base = PY * ty * TB_R + 4 * tx;  // shared row PY ty (region row PY ty - 1)
    float4 s4 = *reinterpret_cast<const float4*>(&us[base]);
    float4 t4 = *reinterpret_cast<const float4*>(&vs[base]);
    float cu[4], cv[4];
    {
      const float4 a = *reinterpret_cast<const float4*>(&us[base + TB_R]);
      const float4 b = *reinterpret_cast<const float4*>(&vs[base + TB_R]);
      cu[0] = a.x; cu[1] = a.y; cu[2] = a.z; cu[3] = a.w;
      cv[0] = b.x; cv[1] = b.y; cv[2] = b.z; cv[3] = b.w;
    }
    // flux through the south face of the first row, into the cell
    float fsu[4], fsv[4];
    {
      const float su[4] = {s4.x, s4.y, s4.z, s4.w}, sv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        fsu[c] = fy[0][c] * (su[c] - cu[c]);
        fsv[c] = fy[0][c] * (sv[c] - cv[c]);
      }
    }
#pragma unroll
    for (int r = 0; r < PY; ++r) {
      const float4 a = *reinterpret_cast<const float4*>(&us[base + (r + 2) * TB_R]);
      const float4 b = *reinterpret_cast<const float4*>(&vs[base + (r + 2) * TB_R]);
      const float nu[4] = {a.x, a.y, a.z, a.w}, nv[4] = {b.x, b.y, b.z, b.w};
      // x neighbours beyond the thread's columns
      const float wu = __shfl_up_sync(0xffffffffu, cu[3], 1, 16);
      const float wv = __shfl_up_sync(0xffffffffu, cv[3], 1, 16);
      const float eu = __shfl_down_sync(0xffffffffu, cu[0], 1, 16);
      const float ev = __shfl_down_sync(0xffffffffu, cv[0], 1, 16);
      // g[c]: flux into cell c through its west face (g[4]: into the east neighbour)
      float gu[5], gv[5];
      gu[0] = fx[r][0] * (wu - cu[0]);
      gv[0] = fx[r][0] * (wv - cv[0]);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        gu[c] = fx[r][c] * (cu[c - 1] - cu[c]);
        gv[c] = fx[r][c] * (cv[c - 1] - cv[c]);
      }
      gu[4] = fx[r][4] * (cu[3] - eu);
      gv[4] = fx[r][4] * (cv[3] - ev);
      float ou[4], ov[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float fnu = fy[r + 1][c] * (nu[c] - cu[c]);
        const float fnv = fy[r + 1][c] * (nv[c] - cv[c]);
        const float fu = (gu[c] - gu[c + 1]) + (fnu + fsu[c]);
        const float fv = (gv[c] - gv[c + 1]) + (fnv + fsv[c]);
        float un = cu[c] + ca * fu - cb * fv;
        float vn = cv[c] + ca * fv + cb * fu;
        if (!PERIODIC && !(inside & (1u << (r * 4 + c)))) {
          un = 0.f;
          vn = 0.f;
        }
        ou[c] = un;
        ov[c] = vn;
        fsu[c] = -fnu;
        fsv[c] = -fnv;
        cu[c] = nu[c];
        cv[c] = nv[c];
      }
      *reinterpret_cast<float4*>(&ud[base + (r + 1) * TB_R]) = make_float4(ou[0], ou[1], ou[2], ou[3]);
      *reinterpret_cast<float4*>(&vd[base + (r + 1) * TB_R]) = make_float4(ov[0], ov[1], ov[2], ov[3]);
    }
    __syncthreads();
  }

  // store the output tile: region cells at distance >= k from the region edge
  const float* uf = Ub[k & 1];
  const float* vf = Vb[k & 1];
  float* __restrict__ Uo = static_cast<float*>(p.U_out);
  float* __restrict__ Vo = static_cast<float*>(p.V_out);
  bool bad = false;
#pragma unroll
  for (int r = 0; r < PY; ++r) {
    const int ry = PY * ty + r;
    const int gy = y0 + ry;
    if (ry < k || ry >= TB_R - k || gy >= ny) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int rx = 4 * tx + c;
      const int gx = x0 + rx;
      if (rx < k || rx >= TB_R - k || gx >= nx) continue;
      const size_t g = size_t(gy) * nx + gx;
      const float uu = uf[(ry + 1) * TB_R + rx];
      Uo[g] = uu;
      if (Vo) Vo[g] = vf[(ry + 1) * TB_R + rx];
      if (p.check_finite) bad |= (__float_as_uint(uu) & 0x7f800000u) == 0x7f800000u;
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

}  // namespace

size_t tb2d_smem_bytes() { return size_t(4) * TB_ROWS * TB_R * sizeof(float); }

bool tb2d_supported(const frkc2_problem& p, int k) {
  return p.ndim == 2 && p.precision == FRKC2_FP32 && p.kappa_kind != FRKC2_KAPPA_POWER && k >= 1 &&
         2 * k < TB_R;
}

#ifndef FRKC2_TB_REG
#define FRKC2_TB_REG 1
#endif

cudaError_t launch_pass_tb2d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st) {
  if (FRKC2_TB_REG) return launch_pass_tb2d_reg(p, a, st);  // state in registers
  const size_t smem = tb2d_smem_bytes();
  const int T = TB_R - 2 * a.k;
  dim3 grid((a.nx + T - 1) / T, (a.ny + T - 1) / T, 1);
  cudaError_t e;
  if (a.bc == FRKC2_BC_PERIODIC) {
    e = cudaFuncSetAttribute(k_tb2d_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_tb2d_f32<true><<<grid, TB_THREADS, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_tb2d_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_tb2d_f32<false><<<grid, TB_THREADS, smem, st>>>(a);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace frkc2
