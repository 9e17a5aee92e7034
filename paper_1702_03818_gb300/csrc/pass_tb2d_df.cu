// 2D temporally blocked pass for the DFLOAT precision (fixed conductivity): k stages of
// Sec. 3, Eq. 13 per HBM round trip, the float-pair state in registers.
//
// Same region scheme as the FP32 register-tiled pass: a CTA of 16 x 16 threads owns a 64 x 64
// region (output (64 - 2k)^2, k-cell recomputed halo), thread (tx, ty) the 4 x 4 cells at
// columns 4tx.., rows 4ty..  Each cell's state is two float pairs (U = Uh + Ul, V = Vh + Vl:
// 64 registers per thread, held as horizontal cell pairs); the thread's 40 face conductivities
// sit in its own slots of shared memory (written and read by that thread only, element-major
// so a warp's accesses are conflict-free; the y faces as pairs of adjacent columns).  Per
// stage the thread's bottom and top rows go through shared memory (double-buffered, one barrier
// per stage), its edge columns come by 16-lane shuffles, neighbour differences are rounded to
// float from the pairs ((h_nb - h_c) + (l_nb - l_c)), f is formed in float with each difference
// shared inside the block, and the float increment is added to each pair by TwoSum and a fast
// renormalisation -- every operation on the FP32 pipe, and all of it but the x differences
// and x flux terms as packed two-lane instructions (add / fma .f32x2 of the sm_100 family) on
// two cells at once.  A step's first pass splits the caller's
// double state, its last pass writes hi + lo back as a double; in between the state is one
// float4 (Uh, Ul, Vh, Vl) per cell, as in the DFLOAT streaming pass.
#include <cuda_runtime.h>

#include "frkc2_internal.h"
#include "tb2d_df_region.cuh"

namespace frkc2 {
namespace {

template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
__global__ void __launch_bounds__(RT_THREADS, 2) k_tb2d_df(const PassArgs p) {
  extern __shared__ __align__(16) unsigned char dt_smem[];
  DfShared& sh = *reinterpret_cast<DfShared*>(dt_smem);
  const int k = p.k;
  const int T = RT_R - 2 * k;
  // the next pass may be launched as soon as every CTA of this one is running (it then stores
  // its face conductivities, which no pass writes, and waits for this pass's state)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  auto coef = [&](int j, float& ca, float& cb) {
    ca = p.caf[j];
    cb = p.cbf[j];
  };
  // the previous pass's state is complete and visible after the wait (a no-op for a launch
  // without the programmatic-serialization attribute)
  auto wait_prev = [] { asm volatile("griddepcontrol.wait;" ::: "memory"); };
  const bool bad = tb2d_df_region<PERIODIC, IN_REAL, OUT_REAL, false>(
      sh, p.nx, p.ny, k, k, int(blockIdx.x) * T - k, int(blockIdx.y) * T - k, p.U_in, p.U_out,
      static_cast<const float*>(p.fx), static_cast<const float*>(p.fy), coef, p.check_finite != 0, wait_prev);
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
cudaError_t launch_t(const PassArgs& a, cudaStream_t st, bool overlap_previous) {
  const auto kern = k_tb2d_df<PERIODIC, IN_REAL, OUT_REAL>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(DfShared)));
  if (attr != cudaSuccess) return attr;
  const int T = RT_R - 2 * a.k;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((a.nx + T - 1) / T, (a.ny + T - 1) / T, 1);
  cfg.blockDim = dim3(RT_THREADS, 1, 1);
  cfg.dynamicSmemBytes = sizeof(DfShared);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = overlap_previous ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <bool PERIODIC>
cudaError_t launch_bc(const PassArgs& a, cudaStream_t st, bool ov) {
  const bool in_real = a.in_mode == PASS_IO_REAL, out_real = a.out_mode == PASS_IO_REAL;
  if (in_real)
    return out_real ? launch_t<PERIODIC, true, true>(a, st, ov) : launch_t<PERIODIC, true, false>(a, st, ov);
  return out_real ? launch_t<PERIODIC, false, true>(a, st, ov) : launch_t<PERIODIC, false, false>(a, st, ov);
}

}  // namespace

cudaError_t launch_pass_tb2d_df(const frkc2_problem& p, const PassArgs& a, cudaStream_t st, bool overlap_previous) {
  return p.bc == FRKC2_BC_PERIODIC ? launch_bc<true>(a, st, overlap_previous)
                                   : launch_bc<false>(a, st, overlap_previous);
}

}  // namespace frkc2
