// The DFLOAT register-tiled region (2D, fixed conductivity): one 64 x 64 region of kq stages
// of Sec. 3, Eq. 13 with the float-pair state in registers, shared by the single-problem DFLOAT
// pass (pass_tb2d_df.cu) and the batched launch's DFLOAT items (batched.cu).
//
// A CTA of 16 x 16 threads owns a 64 x 64 region (output (64 - 2k)^2, k-cell recomputed halo),
// thread (tx, ty) the 4 x 4 cells at columns 4tx.., rows 4ty..  Each cell's state is two float
// pairs (U = Uh + Ul, V = Vh + Vl: 64 registers per thread, held as horizontal cell pairs); the
// thread's 40 face conductivities sit in its own slots of shared memory (written and read by
// that thread only, element-major so a warp's accesses are conflict-free; the y faces as pairs
// of adjacent columns).  Per stage the thread's bottom and top rows go through shared memory
// (double-buffered, one barrier per stage), its edge columns come by 16-lane shuffles,
// neighbour differences are rounded to float from the pairs ((h_nb - h_c) + (l_nb - l_c)), f is
// formed in float with each difference shared inside the block, and the float increment is
// added to each pair by TwoSum and a fast renormalisation -- every operation on the FP32 pipe,
// and all of it but the x differences and x flux terms as packed two-lane instructions (add /
// fma .f32x2 of the sm_100 family) on two cells at once.  IN_REAL: the state comes as the
// double real state and is split; OUT_REAL: hi + lo goes out as a double; in between the state
// is one float4 (Uh, Ul, Vh, Vl) per cell, as in the DFLOAT streaming pass.
#pragma once

#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "tb2d_region.cuh"

namespace frkc2 {

struct DfShared {
  float4 bot[2][4][16][16];  // [stage parity][Uh, Ul, Vh, Vl][ty][tx]: the thread's row 0
  float4 top[2][4][16][16];  // its row 3
  float4 fx4[4][RT_THREADS];  // x faces 1..4 of row r (face c: west of cell c; 4 = east of 3)
  float4 fy4[5][RT_THREADS];  // y face r of columns 0..3 (face r: south of row r; 4 = north of 3)
};

// (h, l) += d on both halves: TwoSum of h and d, then the fast renormalisation with l
__device__ __forceinline__ void df_add2(float2& h, float2& l, float2 d) {
  const float2 s = __fadd2_rn(h, d);
  const float2 bb = sub2(s, h);
  const float2 e = __fadd2_rn(sub2(h, sub2(s, bb)), sub2(d, bb));
  const float2 t = __fadd2_rn(l, e);
  const float2 hi = __fadd2_rn(s, t);
  l = sub2(t, sub2(hi, s));
  h = hi;
}

// (ah + al) - (bh + bl) rounded to float
__device__ __forceinline__ float dfd(float ah, float al, float bh, float bl) { return (ah - bh) + (al - bl); }
__device__ __forceinline__ float2 dfd2(float2 ah, float2 al, float2 bh, float2 bl) {
  return __fadd2_rn(sub2(ah, bh), sub2(al, bl));
}

__device__ __forceinline__ float2 pair_of(float4 a, int h) { return h == 0 ? make_float2(a.x, a.y) : make_float2(a.z, a.w); }
__device__ __forceinline__ float half_of(float2 a, int i) { return i ? a.y : a.x; }

// One region: x0, y0 its corner (tile origin - k), kq <= k stages, coef(j, ca, cb) the float
// stage coefficients.  after_faces() runs between the face loads and the state loads (the
// single-problem pass waits there for the previous pass).  L1BYPASS: state loads through L2
// (buffers other CTAs of the same launch wrote).  Returns true if a stored value is not finite
// (when check_finite; OUT_REAL only).
template <bool PERIODIC, bool IN_REAL, bool OUT_REAL, bool L1BYPASS, class Coef, class AfterFaces>
__device__ __forceinline__ bool tb2d_df_region(DfShared& sh, int nx, int ny, int k, int kq, int x0, int y0,
                                               const void* in, void* out, const float* __restrict__ FX,
                                               const float* __restrict__ FY, Coef coef, bool check_finite,
                                               AfterFaces after_faces) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float4* myfx = &sh.fx4[0][tid];  // row r at myfx[r * RT_THREADS]
  float4* myfy = &sh.fy4[0][tid];

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
    float fxr[5], fyr[4];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (r < 4) {  // x face c of row r
        float v = 0.f;
        if (PERIODIC || (yin[r] && gxc[c] >= 0 && gxc[c] <= nx)) v = FX[size_t(gyr[r]) * (nx + 1) + gxc[c]];
        fxr[c] = v;
      }
      if (c < 4) {  // y face r of column c
        float v = 0.f;
        if (PERIODIC || (xin[c] && gyr[r] >= 0 && gyr[r] <= ny)) v = FY[size_t(gyr[r]) * nx + gxc[c]];
        fyr[c] = v;
        if (r < 4 && xin[c] && yin[r]) inside |= 1u << (4 * r + c);
      }
    }
    // face 0 of a row is the west neighbour's face 4: its flux term comes from there
    if (r < 4) myfx[r * RT_THREADS] = make_float4(fxr[1], fxr[2], fxr[3], fxr[4]);
    myfy[r * RT_THREADS] = make_float4(fyr[0], fyr[1], fyr[2], fyr[3]);
  }
  after_faces();
  // the state as horizontal cell pairs: Uh[r][h] = (Uh of cell (r, 2h), of cell (r, 2h + 1))
  float2 Uh[4][2], Ul[4][2], Vh[4][2], Vl[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float4 w[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int c = 2 * h + i;
        w[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (PERIODIC || (inside & (1u << (4 * r + c)))) {
          const size_t g = size_t(gyr[r]) * nx + gxc[c];
          if (IN_REAL) {
            const double u = L1BYPASS ? __ldcg(static_cast<const double*>(in) + g) : static_cast<const double*>(in)[g];
            w[i].x = __double2float_rn(u);
            w[i].y = __double2float_rn(u - double(w[i].x));
          } else {
            w[i] = L1BYPASS ? __ldcg(static_cast<const float4*>(in) + g) : static_cast<const float4*>(in)[g];
          }
        }
      }
      Uh[r][h] = make_float2(w[0].x, w[1].x);
      Ul[r][h] = make_float2(w[0].y, w[1].y);
      Vh[r][h] = make_float2(w[0].z, w[1].z);
      Vl[r][h] = make_float2(w[0].w, w[1].w);
    }

  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = 0; j < kq; ++j) {
    const int b = j & 1;
    sh.bot[b][0][ty][tx] = make_float4(Uh[0][0].x, Uh[0][0].y, Uh[0][1].x, Uh[0][1].y);
    sh.bot[b][1][ty][tx] = make_float4(Ul[0][0].x, Ul[0][0].y, Ul[0][1].x, Ul[0][1].y);
    sh.bot[b][2][ty][tx] = make_float4(Vh[0][0].x, Vh[0][0].y, Vh[0][1].x, Vh[0][1].y);
    sh.bot[b][3][ty][tx] = make_float4(Vl[0][0].x, Vl[0][0].y, Vl[0][1].x, Vl[0][1].y);
    sh.top[b][0][ty][tx] = make_float4(Uh[3][0].x, Uh[3][0].y, Uh[3][1].x, Uh[3][1].y);
    sh.top[b][1][ty][tx] = make_float4(Ul[3][0].x, Ul[3][0].y, Ul[3][1].x, Ul[3][1].y);
    sh.top[b][2][ty][tx] = make_float4(Vh[3][0].x, Vh[3][0].y, Vh[3][1].x, Vh[3][1].y);
    sh.top[b][3][ty][tx] = make_float4(Vl[3][0].x, Vl[3][0].y, Vl[3][1].x, Vl[3][1].y);
    __syncthreads();
    float ca, cb;
    coef(j, ca, cb);
    const float2 ca2 = make_float2(ca, ca), cb2 = make_float2(cb, cb), ncb2 = make_float2(-cb, -cb);
    // differences across the south faces of row 0 (the region's bottom thread row has none)
    float2 dsU[2], dsV[2];
    {
      const float4 a = ty > 0 ? sh.top[b][0][ty - 1][tx] : z4, bl = ty > 0 ? sh.top[b][1][ty - 1][tx] : z4;
      const float4 cvh = ty > 0 ? sh.top[b][2][ty - 1][tx] : z4, cvl = ty > 0 ? sh.top[b][3][ty - 1][tx] : z4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        dsU[h] = dfd2(Uh[0][h], Ul[0][h], pair_of(a, h), pair_of(bl, h));
        dsV[h] = dfd2(Vh[0][h], Vl[0][h], pair_of(cvh, h), pair_of(cvl, h));
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // the column east of the thread's own, before this row is updated
      const float eUh = __shfl_down_sync(0xffffffffu, Uh[r][0].x, 1, 16);
      const float eUl = __shfl_down_sync(0xffffffffu, Ul[r][0].x, 1, 16);
      const float eVh = __shfl_down_sync(0xffffffffu, Vh[r][0].x, 1, 16);
      const float eVl = __shfl_down_sync(0xffffffffu, Vl[r][0].x, 1, 16);
      const float uh[5] = {Uh[r][0].x, Uh[r][0].y, Uh[r][1].x, Uh[r][1].y, eUh};
      const float ul[5] = {Ul[r][0].x, Ul[r][0].y, Ul[r][1].x, Ul[r][1].y, eUl};
      const float vh[5] = {Vh[r][0].x, Vh[r][0].y, Vh[r][1].x, Vh[r][1].y, eVh};
      const float vl[5] = {Vl[r][0].x, Vl[r][0].y, Vl[r][1].x, Vl[r][1].y, eVl};
      // x flux terms k_c d_c of faces 1..4 (face c between cells c - 1 and c), each formed once;
      // face 0's is the west neighbour's face 4 (the region's west column goes stale)
      const float4 kx = myfx[r * RT_THREADS];
      const float kxa[4] = {kx.x, kx.y, kx.z, kx.w};
      float pU[5], pV[5];
#pragma unroll
      for (int c = 1; c < 5; ++c) {
        pU[c] = kxa[c - 1] * dfd(uh[c], ul[c], uh[c - 1], ul[c - 1]);
        pV[c] = kxa[c - 1] * dfd(vh[c], vl[c], vh[c - 1], vl[c - 1]);
      }
      pU[0] = __shfl_up_sync(0xffffffffu, pU[4], 1, 16);
      pV[0] = __shfl_up_sync(0xffffffffu, pV[4], 1, 16);
      // x part of f per cell, into the halves of the pairs
      float2 fU[2], fV[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 2 * h;
        fU[h] = make_float2(pU[c + 1] - pU[c], pU[c + 2] - pU[c + 1]);
        fV[h] = make_float2(pV[c + 1] - pV[c], pV[c + 2] - pV[c + 1]);
      }
      float2 dnU[2], dnV[2];
      if (r < 3) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rn = r + 1 < 4 ? r + 1 : 3;
          dnU[h] = dfd2(Uh[rn][h], Ul[rn][h], Uh[r][h], Ul[r][h]);
          dnV[h] = dfd2(Vh[rn][h], Vl[rn][h], Vh[r][h], Vl[r][h]);
        }
      } else {  // the north neighbour row (the region's top thread row has none)
        const float4 a = ty < 15 ? sh.bot[b][0][ty + 1][tx] : z4, bl = ty < 15 ? sh.bot[b][1][ty + 1][tx] : z4;
        const float4 cvh = ty < 15 ? sh.bot[b][2][ty + 1][tx] : z4, cvl = ty < 15 ? sh.bot[b][3][ty + 1][tx] : z4;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          dnU[h] = dfd2(pair_of(a, h), pair_of(bl, h), Uh[3][h], Ul[3][h]);
          dnV[h] = dfd2(pair_of(cvh, h), pair_of(cvl, h), Vh[3][h], Vl[3][h]);
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 ks4 = myfy[r * RT_THREADS], kn4 = myfy[(r + 1) * RT_THREADS];
        const float2 ks = pair_of(ks4, h), kn = pair_of(kn4, h);
        const float2 nks = make_float2(-ks.x, -ks.y);
        // y part, two cells per instruction: f += k_n d_n - k_s d_s
        fU[h] = __ffma2_rn(nks, dsU[h], __ffma2_rn(kn, dnU[h], fU[h]));
        fV[h] = __ffma2_rn(nks, dsV[h], __ffma2_rn(kn, dnV[h], fV[h]));
        // the float increments Re, Im of (ca + i cb) f, added to the pairs error-free
        df_add2(Uh[r][h], Ul[r][h], __ffma2_rn(ncb2, fV[h], __fmul2_rn(ca2, fU[h])));
        df_add2(Vh[r][h], Vl[r][h], __ffma2_rn(cb2, fU[h], __fmul2_rn(ca2, fV[h])));
        if (!PERIODIC) {
#pragma unroll
          for (int i = 0; i < 2; ++i)
            if (!(inside & (1u << (4 * r + 2 * h + i)))) {
              if (i) Uh[r][h].y = Ul[r][h].y = Vh[r][h].y = Vl[r][h].y = 0.f;
              else Uh[r][h].x = Ul[r][h].x = Vh[r][h].x = Vl[r][h].x = 0.f;
            }
        }
        dsU[h] = dnU[h];
        dsV[h] = dnV[h];
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
      const int h = c >> 1, i = c & 1;
      if (OUT_REAL) {
        const double u = double(half_of(Uh[r][h], i)) + double(half_of(Ul[r][h], i));
        static_cast<double*>(out)[g] = u;
        if (check_finite) bad |= (__double2hiint(u) & 0x7ff00000) == 0x7ff00000;
      } else {
        static_cast<float4*>(out)[g] =
            make_float4(half_of(Uh[r][h], i), half_of(Ul[r][h], i), half_of(Vh[r][h], i), half_of(Vl[r][h], i));
      }
    }
  }
  return bad;
}



}  // namespace frkc2
