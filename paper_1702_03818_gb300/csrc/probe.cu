// FMA throughput probe: the FP64 and FP32 pipe rates the kernels' rooflines are stated against.
//
// Not part of the method.  Each thread runs `iters` rounds of eight independent fused
// multiply-add chains (enough independent work per warp to keep its pipe busy) and stores
// their sum, so nothing is optimised away.  The caller times the launch; the count of FMAs is
// grid x block x iters x 8.
#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The FP32 chains as packed two-lane FMAs: four float pairs, the same eight FMAs per round.
__global__ void __launch_bounds__(256) k_fma2_probe(float* __restrict__ out, int iters, float a, float b) {
  float2 x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = make_float2(float(threadIdx.x + 2 * i) * 1e-3f, float(threadIdx.x + 2 * i + 1) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += x[i].x + x[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" frkc2_status frkc2_fma_probe(int precision, int blocks, int iters, void* out, void* stream) {
  if (blocks < 1 || iters < 1 || !out ||
      (precision != FRKC2_FP64 && precision != FRKC2_FP32 && precision != (FRKC2_FP32 | FRKC2_PROBE_PACKED)))
    return FRKC2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a = 1 - 2^-20 and b small keep the chains bounded and away from subnormals
  if (precision == FRKC2_FP64)
    k_fma_probe<double><<<blocks, 256, 0, st>>>(static_cast<double*>(out), iters, 1.0 - 0x1p-20, 0x1p-10);
  else if (precision & FRKC2_PROBE_PACKED)
    k_fma2_probe<<<blocks, 256, 0, st>>>(static_cast<float*>(out), iters, 1.0f - 0x1p-20f, 0x1p-10f);
  else
    k_fma_probe<float><<<blocks, 256, 0, st>>>(static_cast<float*>(out), iters, 1.0f - 0x1p-20f, 0x1p-10f);
  frkc2::count_launch();
  return cudaGetLastError() == cudaSuccess ? FRKC2_OK : FRKC2_ECUDA;
}
