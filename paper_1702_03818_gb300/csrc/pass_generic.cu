// Generic k-stage pass: the stage W <- W + dt a_l f(W) of Sec. 3, Eq. 13, applied k times
// to a tile held in shared memory, for every dimension, boundary kind, conductivity kind
// and precision.
//
// A CTA loads its output tile plus a halo of k cells along each present axis, then runs
// the k stages in shared memory; after stage j only the cells at distance >= j from the
// region edge are still exact, so the valid region shrinks by one cell per stage and ends
// as the output tile (temporal blocking with redundant halo recompute).  Two shared
// buffers ping-pong between stages.  With complex state W = U + iV and a_l = alpha_l +
// i beta_l the stage reads, in real arithmetic,
//   U' = U + ca f_R - cb f_I,  V' = V + ca f_I + cb f_R,   ca = dt alpha_l/dx^2, cb = dt beta_l/dx^2,
// where f_R + i f_I = dx^2 f(U + iV); for a fixed conductivity f_R = dx^2 f(U), f_I = dx^2 f(V).
// Optionally the pass also advances the embedded first-order solution of Eq. 14,
// What <- What + ca f_R (ca = dt Re(a_l)/dx^2), held in one more shared array.
#include <algorithm>

#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "frkc2_math.cuh"

namespace frkc2 {
namespace {

constexpr int GEN_THREADS = 256;

__device__ __forceinline__ int wrap_idx(int g, int n) {
  int r = g % n;
  return r < 0 ? r + n : r;
}

template <class S, class A, bool POWER>
__global__ void __launch_bounds__(GEN_THREADS) k_pass_generic(const PassArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int RX = p.tx + 2 * p.hx, RY = p.ty + 2 * p.hy, RZ = p.tz + 2 * p.hz;
  const int R = RX * RY * RZ;
  const int plane = RX * RY;
  S* ub[2];
  S* vb[2];
  ub[0] = reinterpret_cast<S*>(smem);
  vb[0] = ub[0] + R;
  ub[1] = vb[0] + R;
  vb[1] = ub[1] + R;
  A* f0 = reinterpret_cast<A*>(vb[1] + R);  // x faces, or Re kappa(W) for POWER
  A* f1 = f0 + R;                           // y faces, or Im kappa(W)
  A* f2 = f1 + R;                           // z faces
  const int nf = POWER ? 2 : p.ndim;
  // embedded solution (if H_out), 16-byte aligned after the face arrays
  S* hb = reinterpret_cast<S*>((reinterpret_cast<uintptr_t>(f0 + size_t(nf) * R) + 15) & ~uintptr_t(15));
  const bool hat = p.H_out != nullptr;
  const S* __restrict__ Hin = static_cast<const S*>(p.H_in);
  const bool periodic = p.bc == FRKC2_BC_PERIODIC;
  const int x0 = blockIdx.x * p.tx - p.hx;
  const int y0 = blockIdx.y * p.ty - p.hy;
  const int z0 = blockIdx.z * p.tz - p.hz;
  const S* __restrict__ Uin = static_cast<const S*>(p.U_in);
  const S* __restrict__ Vin = static_cast<const S*>(p.V_in);
  const A* __restrict__ FX = static_cast<const A*>(p.fx);
  const A* __restrict__ FY = static_cast<const A*>(p.fy);
  const A* __restrict__ FZ = static_cast<const A*>(p.fz);
  const int tid = threadIdx.x;

  // array sizes, for the bounds-checking build's index checks
  const size_t ncell = size_t(p.nz) * p.ny * p.nx;
  const size_t nfx = size_t(p.nz) * p.ny * (p.nx + 1), nfy = size_t(p.nz) * (p.ny + 1) * p.nx;
  const size_t nfz = size_t(p.nz + 1) * p.ny * p.nx;
  // ---- load the region: state, and the low-side face of every region cell ----
  for (int z = 0; z < RZ; ++z) {
    for (int idx = tid; idx < plane; idx += GEN_THREADS) {
      const int y = idx / RX, x = idx - y * RX;
      const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
      const int i = z * plane + idx;
      S uu = S(0), vv = S(0);
      A a0 = A(0), a1 = A(0), a2 = A(0);
      if (periodic) {
        const int wx = wrap_idx(gx, p.nx), wy = wrap_idx(gy, p.ny), wz = wrap_idx(gz, p.nz);
        const size_t g = (size_t(wz) * p.ny + wy) * p.nx + wx;
        if (in_bounds(g < ncell, p.status)) {
          uu = Uin[g];
          if (Vin) vv = Vin[g];
          if (hat) hb[i] = Hin[g];
        }
        if (!POWER) {
          const size_t f0 = (size_t(wz) * p.ny + wy) * (p.nx + 1) + wx;
          const size_t f1 = (size_t(wz) * (p.ny + 1) + wy) * p.nx + wx;
          const size_t f2 = (size_t(wz) * p.ny + wy) * p.nx + wx;
          if (in_bounds(f0 < nfx, p.status)) a0 = FX[f0];
          if (p.ndim >= 2 && in_bounds(f1 < nfy, p.status)) a1 = FY[f1];
          if (p.ndim >= 3 && in_bounds(f2 < nfz, p.status)) a2 = FZ[f2];
        }
      } else {
        const bool inx = gx >= 0 && gx < p.nx, iny = gy >= 0 && gy < p.ny, inz = gz >= 0 && gz < p.nz;
        if (hat) hb[i] = S(0);
        if (inx && iny && inz) {
          const size_t g = (size_t(gz) * p.ny + gy) * p.nx + gx;
          if (in_bounds(g < ncell, p.status)) {
            uu = Uin[g];
            if (Vin) vv = Vin[g];
            if (hat) hb[i] = Hin[g];
          }
        }
        if (!POWER) {
          if (iny && inz && gx >= 0 && gx <= p.nx) {
            const size_t f0 = (size_t(gz) * p.ny + gy) * (p.nx + 1) + gx;
            if (in_bounds(f0 < nfx, p.status)) a0 = FX[f0];
          }
          if (p.ndim >= 2 && inx && inz && gy >= 0 && gy <= p.ny) {
            const size_t f1 = (size_t(gz) * (p.ny + 1) + gy) * p.nx + gx;
            if (in_bounds(f1 < nfy, p.status)) a1 = FY[f1];
          }
          if (p.ndim >= 3 && inx && iny && gz >= 0 && gz <= p.nz) {
            const size_t f2 = (size_t(gz) * p.ny + gy) * p.nx + gx;
            if (in_bounds(f2 < nfz, p.status)) a2 = FZ[f2];
          }
        }
      }
      ub[0][i] = uu;
      vb[0][i] = vv;
      ub[1][i] = S(0);
      vb[1][i] = S(0);
      if (!POWER) {
        f0[i] = a0;
        if (p.ndim >= 2) f1[i] = a1;
        if (p.ndim >= 3) f2[i] = a2;
      }
    }
  }
  __syncthreads();

  const int sy = RX, sz = plane;
  for (int j = 1; j <= p.k; ++j) {
    const S* __restrict__ us = ub[(j - 1) & 1];
    const S* __restrict__ vs = vb[(j - 1) & 1];
    S* __restrict__ ud = ub[j & 1];
    S* __restrict__ vd = vb[j & 1];
    const int lx = p.hx ? j : 0, ly = p.hy ? j : 0, lz = p.hz ? j : 0;
    if (POWER) {
      // kappa(W) on every cell the stage reads: one cell wider than the updated range
      const int mx = p.hx ? j - 1 : 0, my = p.hy ? j - 1 : 0, mz = p.hz ? j - 1 : 0;
      const int wdt = RX - 2 * mx, hgt = RY - 2 * my;
      for (int z = mz; z < RZ - mz; ++z)
        for (int idx = tid; idx < wdt * hgt; idx += GEN_THREADS) {
          const int y = my + idx / wdt, x = mx + idx % wdt;
          const int i = z * plane + y * RX + x;
          A kr, ki;
          kappa_power<A>(A(us[i]), A(vs[i]), A(p.kc), A(p.kp), kr, ki);
          f0[i] = kr;
          f1[i] = ki;
        }
      __syncthreads();
    }
    const S ca = S(p.ca[j - 1]), cb = S(p.cb[j - 1]);
    const int wdt = RX - 2 * lx, hgt = RY - 2 * ly;
    for (int z = lz; z < RZ - lz; ++z) {
      for (int idx = tid; idx < wdt * hgt; idx += GEN_THREADS) {
        const int y = ly + idx / wdt, x = lx + idx % wdt;
        const int i = z * plane + y * RX + x;
        if (!periodic) {
          const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
          if (gx < 0 || gx >= p.nx || gy < 0 || gy >= p.ny || gz < 0 || gz >= p.nz) {
            ud[i] = S(0);
            vd[i] = S(0);
            continue;
          }
        }
        const S Uc = us[i], Vc = vs[i];
        A fR = A(0), fI = A(0);
        if (!POWER) {
          // face (i, i+s) has conductivity F[i+s]; face (i-s, i) has F[i]
          {
            const A fe = f0[i + 1], fw = f0[i];
            fR += fe * A(us[i + 1] - Uc) + fw * A(us[i - 1] - Uc);
            fI += fe * A(vs[i + 1] - Vc) + fw * A(vs[i - 1] - Vc);
          }
          if (p.ndim >= 2) {
            const A fn = f1[i + sy], fs = f1[i];
            fR += fn * A(us[i + sy] - Uc) + fs * A(us[i - sy] - Uc);
            fI += fn * A(vs[i + sy] - Vc) + fs * A(vs[i - sy] - Vc);
          }
          if (p.ndim >= 3) {
            const A fu = f2[i + sz], fd = f2[i];
            fR += fu * A(us[i + sz] - Uc) + fd * A(us[i - sz] - Uc);
            fI += fu * A(vs[i + sz] - Vc) + fd * A(vs[i - sz] - Vc);
          }
        } else {
          const A kr = f0[i], ki = f1[i];
          const int st[3] = {1, sy, sz};
          for (int d = 0; d < p.ndim; ++d) {
            for (int sgn = 0; sgn < 2; ++sgn) {
              const int nb = sgn ? i + st[d] : i - st[d];
              const A kfr = A(0.5) * (kr + f0[nb]), kfi = A(0.5) * (ki + f1[nb]);
              const A dr = A(us[nb] - Uc), di = A(vs[nb] - Vc);
              fR += kfr * dr - kfi * di;
              fI += kfr * di + kfi * dr;
            }
          }
        }
        ud[i] = Uc + ca * S(fR) - cb * S(fI);
        vd[i] = Vc + ca * S(fI) + cb * S(fR);
        if (hat) hb[i] += ca * S(fR);
      }
    }
    __syncthreads();
  }

  // ---- store the output tile ----
  const S* __restrict__ uf = ub[p.k & 1];
  const S* __restrict__ vf = vb[p.k & 1];
  S* __restrict__ Uout = static_cast<S*>(p.U_out);
  S* __restrict__ Vout = static_cast<S*>(p.V_out);
  const int ox = blockIdx.x * p.tx, oy = blockIdx.y * p.ty, oz = blockIdx.z * p.tz;
  const int ex = min(p.tx, p.nx - ox), ey = min(p.ty, p.ny - oy), ez = min(p.tz, p.nz - oz);
  bool bad = false;
  for (int z = 0; z < ez; ++z)
    for (int idx = tid; idx < ex * ey; idx += GEN_THREADS) {
      const int y = idx / ex, x = idx - y * ex;
      const int i = (z + p.hz) * plane + (y + p.hy) * RX + (x + p.hx);
      const size_t g = (size_t(oz + z) * p.ny + (oy + y)) * p.nx + (ox + x);
      if (!in_bounds(g < size_t(p.nz) * p.ny * p.nx, p.status)) continue;
      const S uu = uf[i];
      Uout[g] = uu;
      if (Vout) Vout[g] = vf[i];
      if (hat) static_cast<S*>(p.H_out)[g] = hb[i];
      if (p.check_finite && !isfinite(double(uu))) bad = true;
    }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

// sum over cells of e_i^2, e_i = |u_i - h_i| / (1 + max(|u_i|, |h_i|)) (Eq. 15 without TOL)
template <class S>
__global__ void k_err_sum(const S* __restrict__ u, const S* __restrict__ h, size_t n, double* out) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const double a = double(u[i]), b = double(h[i]);
    const double e = fabs(a - b) / (1.0 + fmax(fabs(a), fabs(b)));
    acc += e * e;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) part[w] = acc;
  __syncthreads();
  if (w == 0) {
    acc = lane < int(blockDim.x >> 5) ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(out, acc);
  }
}

}  // namespace

cudaError_t launch_err_sum(const frkc2_problem& p, const void* u, const void* h, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const size_t n = size_t(p.n[0]) * p.n[1] * p.n[2];
  const int threads = 256;
  const int blocks = int(std::min<size_t>((n + threads - 1) / threads, 152 * 8));
  if (state_bytes(p.precision) == 8)
    k_err_sum<double><<<blocks, threads, 0, st>>>(static_cast<const double*>(u), static_cast<const double*>(h), n, out);
  else
    k_err_sum<float><<<blocks, threads, 0, st>>>(static_cast<const float*>(u), static_cast<const float*>(h), n, out);
  count_launch();
  return cudaGetLastError();
}

size_t generic_smem_bytes(const frkc2_problem& pr, const PassArgs& a) {
  const size_t R = size_t(a.tx + 2 * a.hx) * (a.ty + 2 * a.hy) * (a.tz + 2 * a.hz);
  const size_t S = state_bytes(pr.precision), A = arith_bytes(pr.precision);
  const size_t nf = pr.kappa_kind == FRKC2_KAPPA_POWER ? 2 : size_t(pr.ndim);
  return R * (4 * S + nf * A) + (a.H_out ? R * S + 16 : 0);
}

template <class S, class A, bool POWER>
static cudaError_t launch_t(const PassArgs& a, size_t smem, cudaStream_t st) {
  auto kern = k_pass_generic<S, A, POWER>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.nx + a.tx - 1) / a.tx, (a.ny + a.ty - 1) / a.ty, (a.nz + a.tz - 1) / a.tz);
  kern<<<grid, GEN_THREADS, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pass_generic(const frkc2_problem& pr, const PassArgs& a, cudaStream_t st) {
  const size_t smem = generic_smem_bytes(pr, a);
  const bool power = pr.kappa_kind == FRKC2_KAPPA_POWER;
  switch (pr.precision) {
    case FRKC2_FP64:
      return power ? launch_t<double, double, true>(a, smem, st) : launch_t<double, double, false>(a, smem, st);
    case FRKC2_FP32:
      return power ? launch_t<float, float, true>(a, smem, st) : launch_t<float, float, false>(a, smem, st);
    default:
      return power ? launch_t<double, float, true>(a, smem, st) : launch_t<double, float, false>(a, smem, st);
  }
}

}  // namespace frkc2
