// 2D temporally blocked pass for FP32 (fixed conductivity): k stages of Sec. 3, Eq. 13 per
// HBM round trip, one 64 x 64 register-tiled region per CTA (tb2d_region.cuh).
#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "tb2d_region.cuh"

namespace frkc2 {
namespace {

#ifndef FRKC2_TBR_MIN_BLOCKS
#define FRKC2_TBR_MIN_BLOCKS 2
#endif

template <bool PERIODIC>
__global__ void __launch_bounds__(RT_THREADS, FRKC2_TBR_MIN_BLOCKS) k_tb2d_reg(const PassArgs p) {
  __shared__ RegionShared sh;
  const int T = RT_R - 2 * p.k;
  const int x0 = blockIdx.x * T - p.k, y0 = blockIdx.y * T - p.k;
  auto coef = [&](int j, float& ca, float& cb) {
    ca = p.caf[j];
    cb = p.cbf[j];
  };
  const bool bad = tb2d_region<PERIODIC, false>(
      sh, p.nx, p.ny, p.k, p.k, x0, y0, static_cast<const float*>(p.U_in), static_cast<const float*>(p.V_in),
      static_cast<float*>(p.U_out), static_cast<float*>(p.V_out), static_cast<const float*>(p.fx),
      static_cast<const float*>(p.fy), coef, p.check_finite != 0);
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

}  // namespace

bool tb2d_supported(const frkc2_problem& p, int k) {
  return p.ndim == 2 && p.precision == FRKC2_FP32 && p.kappa_kind != FRKC2_KAPPA_POWER && k >= 1 &&
         2 * k < RT_R;
}

cudaError_t launch_pass_tb2d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st) {
  (void)p;
  const int T = RT_R - 2 * a.k;
  dim3 grid((a.nx + T - 1) / T, (a.ny + T - 1) / T, 1);
  if (a.bc == FRKC2_BC_PERIODIC)
    k_tb2d_reg<true><<<grid, RT_THREADS, 0, st>>>(a);
  else
    k_tb2d_reg<false><<<grid, RT_THREADS, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace frkc2
