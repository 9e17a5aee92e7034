// 2D temporally blocked pass for the DFLOAT precision (fixed conductivity): k stages of
// Sec. 3, Eq. 13 per HBM round trip, the float-pair state in registers.
//
// Same region scheme as the FP32 register-tiled pass: a CTA of 16 x 16 threads owns a 64 x 64
// region (output (64 - 2k)^2, k-cell recomputed halo), thread (tx, ty) the 4 x 4 cells at
// columns 4tx.., rows 4ty..  Each cell's state is two float pairs (U = Uh + Ul, V = Vh + Vl:
// 64 registers per thread); the thread's 40 face conductivities sit in its own slots of shared
// memory (written and read by that thread only, element-major so a warp hits 32 banks).  Per
// stage the thread's bottom and top rows go through shared memory (double-buffered, one barrier
// per stage), its edge columns come by 16-lane shuffles, neighbour differences are rounded to
// float from the pairs ((h_nb - h_c) + (l_nb - l_c)), f is formed in float with each difference
// shared inside the block, and the float increment is added to each pair by TwoSum and a fast
// renormalisation -- every operation on the FP32 pipe.  A step's first pass splits the caller's
// double state, its last pass writes hi + lo back as a double; in between the state is one
// float4 (Uh, Ul, Vh, Vl) per cell, as in the DFLOAT streaming pass.
#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "tb2d_region.cuh"

namespace frkc2 {
namespace {

constexpr int DT_FACES = 40;  // per thread: 4 rows x 5 x faces, 5 rows x 4 y faces

struct DfShared {
  float4 bot[2][4][16][16];  // [stage parity][Uh, Ul, Vh, Vl][ty][tx]: the thread's row 0
  float4 top[2][4][16][16];  // its row 3
  float faces[DT_FACES][RT_THREADS];
};

__device__ __forceinline__ void df_add2(float& h, float& l, float d) {
  const float s = h + d;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (d - bb);
  const float t = l + e;
  const float hi = s + t;
  l = t - (hi - s);
  h = hi;
}

__device__ __forceinline__ float dfd(float ah, float al, float bh, float bl) { return (ah - bh) + (al - bl); }

template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
__global__ void __launch_bounds__(RT_THREADS, 2) k_tb2d_df(const PassArgs p) {
  extern __shared__ __align__(16) unsigned char dt_smem[];
  DfShared& sh = *reinterpret_cast<DfShared*>(dt_smem);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int k = p.k;
  const int T = RT_R - 2 * k;
  const int x0 = blockIdx.x * T - k, y0 = blockIdx.y * T - k;
  const int nx = p.nx, ny = p.ny;
  const float* __restrict__ FX = static_cast<const float*>(p.fx);
  const float* __restrict__ FY = static_cast<const float*>(p.fy);
  float* myf = &sh.faces[0][tid];  // face e at myf[e * RT_THREADS]

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
  unsigned inside = 0;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (r < 4) {  // x face c of row r
        float v = 0.f;
        if (PERIODIC || (yin[r] && gxc[c] >= 0 && gxc[c] <= nx)) v = FX[size_t(gyr[r]) * (nx + 1) + gxc[c]];
        myf[(5 * r + c) * RT_THREADS] = v;
      }
      if (c < 4) {  // y face r of column c
        float v = 0.f;
        if (PERIODIC || (xin[c] && gyr[r] >= 0 && gyr[r] <= ny)) v = FY[size_t(gyr[r]) * nx + gxc[c]];
        myf[(20 + 4 * r + c) * RT_THREADS] = v;
        if (r < 4 && xin[c] && yin[r]) inside |= 1u << (4 * r + c);
      }
    }
  }
  float Uh[4][4], Ul[4][4], Vh[4][4], Vl[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (PERIODIC || (inside & (1u << (4 * r + c)))) {
        const size_t g = size_t(gyr[r]) * nx + gxc[c];
        if (IN_REAL) {
          const double u = static_cast<const double*>(p.U_in)[g];
          w.x = __double2float_rn(u);
          w.y = __double2float_rn(u - double(w.x));
        } else {
          w = static_cast<const float4*>(p.U_in)[g];
        }
      }
      Uh[r][c] = w.x;
      Ul[r][c] = w.y;
      Vh[r][c] = w.z;
      Vl[r][c] = w.w;
    }

  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = 0; j < k; ++j) {
    const int b = j & 1;
    sh.bot[b][0][ty][tx] = make_float4(Uh[0][0], Uh[0][1], Uh[0][2], Uh[0][3]);
    sh.bot[b][1][ty][tx] = make_float4(Ul[0][0], Ul[0][1], Ul[0][2], Ul[0][3]);
    sh.bot[b][2][ty][tx] = make_float4(Vh[0][0], Vh[0][1], Vh[0][2], Vh[0][3]);
    sh.bot[b][3][ty][tx] = make_float4(Vl[0][0], Vl[0][1], Vl[0][2], Vl[0][3]);
    sh.top[b][0][ty][tx] = make_float4(Uh[3][0], Uh[3][1], Uh[3][2], Uh[3][3]);
    sh.top[b][1][ty][tx] = make_float4(Ul[3][0], Ul[3][1], Ul[3][2], Ul[3][3]);
    sh.top[b][2][ty][tx] = make_float4(Vh[3][0], Vh[3][1], Vh[3][2], Vh[3][3]);
    sh.top[b][3][ty][tx] = make_float4(Vl[3][0], Vl[3][1], Vl[3][2], Vl[3][3]);
    __syncthreads();
    const float ca = p.caf[j], cb = p.cbf[j];
    // differences across the south faces of row 0 (the region's bottom thread row has none)
    float dsU[4], dsV[4];
    {
      const float4 a = ty > 0 ? sh.top[b][0][ty - 1][tx] : z4, bl = ty > 0 ? sh.top[b][1][ty - 1][tx] : z4;
      const float4 cvh = ty > 0 ? sh.top[b][2][ty - 1][tx] : z4, cvl = ty > 0 ? sh.top[b][3][ty - 1][tx] : z4;
      const float sUh[4] = {a.x, a.y, a.z, a.w}, sUl[4] = {bl.x, bl.y, bl.z, bl.w};
      const float sVh[4] = {cvh.x, cvh.y, cvh.z, cvh.w}, sVl[4] = {cvl.x, cvl.y, cvl.z, cvl.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        dsU[c] = dfd(Uh[0][c], Ul[0][c], sUh[c], sUl[c]);
        dsV[c] = dfd(Vh[0][c], Vl[0][c], sVh[c], sVl[c]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // columns beyond the thread's own, before this row is updated
      const float wUh = __shfl_up_sync(0xffffffffu, Uh[r][3], 1, 16);
      const float wUl = __shfl_up_sync(0xffffffffu, Ul[r][3], 1, 16);
      const float wVh = __shfl_up_sync(0xffffffffu, Vh[r][3], 1, 16);
      const float wVl = __shfl_up_sync(0xffffffffu, Vl[r][3], 1, 16);
      const float eUh = __shfl_down_sync(0xffffffffu, Uh[r][0], 1, 16);
      const float eUl = __shfl_down_sync(0xffffffffu, Ul[r][0], 1, 16);
      const float eVh = __shfl_down_sync(0xffffffffu, Vh[r][0], 1, 16);
      const float eVl = __shfl_down_sync(0xffffffffu, Vl[r][0], 1, 16);
      float dxU[5], dxV[5];
      dxU[0] = dfd(Uh[r][0], Ul[r][0], wUh, wUl);
      dxV[0] = dfd(Vh[r][0], Vl[r][0], wVh, wVl);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        dxU[c] = dfd(Uh[r][c], Ul[r][c], Uh[r][c - 1], Ul[r][c - 1]);
        dxV[c] = dfd(Vh[r][c], Vl[r][c], Vh[r][c - 1], Vl[r][c - 1]);
      }
      dxU[4] = dfd(eUh, eUl, Uh[r][3], Ul[r][3]);
      dxV[4] = dfd(eVh, eVl, Vh[r][3], Vl[r][3]);
      float dnU[4], dnV[4];
      if (r < 3) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          dnU[c] = dfd(Uh[r + 1 < 4 ? r + 1 : 3][c], Ul[r + 1 < 4 ? r + 1 : 3][c], Uh[r][c], Ul[r][c]);
          dnV[c] = dfd(Vh[r + 1 < 4 ? r + 1 : 3][c], Vl[r + 1 < 4 ? r + 1 : 3][c], Vh[r][c], Vl[r][c]);
        }
      } else {  // the north neighbour row (the region's top thread row has none)
        const float4 a = ty < 15 ? sh.bot[b][0][ty + 1][tx] : z4, bl = ty < 15 ? sh.bot[b][1][ty + 1][tx] : z4;
        const float4 cvh = ty < 15 ? sh.bot[b][2][ty + 1][tx] : z4, cvl = ty < 15 ? sh.bot[b][3][ty + 1][tx] : z4;
        const float nUh[4] = {a.x, a.y, a.z, a.w}, nUl[4] = {bl.x, bl.y, bl.z, bl.w};
        const float nVh[4] = {cvh.x, cvh.y, cvh.z, cvh.w}, nVl[4] = {cvl.x, cvl.y, cvl.z, cvl.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          dnU[c] = dfd(nUh[c], nUl[c], Uh[3][c], Ul[3][c]);
          dnV[c] = dfd(nVh[c], nVl[c], Vh[3][c], Vl[3][c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float kw = myf[(5 * r + c) * RT_THREADS], ke = myf[(5 * r + c + 1) * RT_THREADS];
        const float ks = myf[(20 + 4 * r + c) * RT_THREADS], kn = myf[(20 + 4 * (r + 1) + c) * RT_THREADS];
        const float fU = kn * dnU[c] - ks * dsU[c] + ke * dxU[c + 1] - kw * dxU[c];
        const float fV = kn * dnV[c] - ks * dsV[c] + ke * dxV[c + 1] - kw * dxV[c];
        df_add2(Uh[r][c], Ul[r][c], ca * fU - cb * fV);
        df_add2(Vh[r][c], Vl[r][c], ca * fV + cb * fU);
        if (!PERIODIC && !(inside & (1u << (4 * r + c)))) {
          Uh[r][c] = Ul[r][c] = Vh[r][c] = Vl[r][c] = 0.f;
        }
        dsU[c] = dnU[c];
        dsV[c] = dnV[c];
      }
    }
  }

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
      if (OUT_REAL) {
        const double u = double(Uh[r][c]) + double(Ul[r][c]);
        static_cast<double*>(p.U_out)[g] = u;
        if (p.check_finite) bad |= (__double2hiint(u) & 0x7ff00000) == 0x7ff00000;
      } else {
        static_cast<float4*>(p.U_out)[g] = make_float4(Uh[r][c], Ul[r][c], Vh[r][c], Vl[r][c]);
      }
    }
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
cudaError_t launch_t(const PassArgs& a, cudaStream_t st) {
  const auto kern = k_tb2d_df<PERIODIC, IN_REAL, OUT_REAL>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(DfShared)));
  if (attr != cudaSuccess) return attr;
  const int T = RT_R - 2 * a.k;
  kern<<<dim3((a.nx + T - 1) / T, (a.ny + T - 1) / T, 1), RT_THREADS, sizeof(DfShared), st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <bool PERIODIC>
cudaError_t launch_bc(const PassArgs& a, cudaStream_t st) {
  const bool in_real = a.in_mode == PASS_IO_REAL, out_real = a.out_mode == PASS_IO_REAL;
  if (in_real) return out_real ? launch_t<PERIODIC, true, true>(a, st) : launch_t<PERIODIC, true, false>(a, st);
  return out_real ? launch_t<PERIODIC, false, true>(a, st) : launch_t<PERIODIC, false, false>(a, st);
}

}  // namespace

cudaError_t launch_pass_tb2d_df(const frkc2_problem& p, const PassArgs& a, cudaStream_t st) {
  return p.bc == FRKC2_BC_PERIODIC ? launch_bc<true>(a, st) : launch_bc<false>(a, st);
}

}  // namespace frkc2
