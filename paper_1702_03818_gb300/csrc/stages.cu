// frkc2_stages: a range of stages of one step (Sec. 3, Eq. 13) on a complex state, for callers
// that split the stage loop -- a grid decomposed into slabs whose halo rows are exchanged between
// groups of stages.
//
// The state is an interleaved (re, im) array, in and out.  Each stage runs the single-stage
// streaming pass (interleaved complex state, face pairs, every neighbour difference formed once);
// consecutive stages alternate between the workspace's two interleaved buffers, and the range's
// last stage writes the caller's array.  A range that starts a step (l0 == 0) first sets the
// imaginary parts to zero: every step starts from the real state W^0 = w^n.
#include <cmath>

#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"

namespace frkc2 {

frkc2_status validate_problem(const frkc2_problem* p);

namespace {

template <class S>
__global__ void k_zero_imag(S* __restrict__ w, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    w[2 * i + 1] = S(0);
}

}  // namespace
}  // namespace frkc2

using namespace frkc2;

extern "C" frkc2_status frkc2_stages(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int l0, int l1,
                                     void* w, void* ws, size_t ws_bytes, void* stream) {
  const frkc2::NvtxRange call_range("frkc2_stages");
  if (!plan || !w || !ws) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (prob->ndim != 2 || prob->kappa_kind == FRKC2_KAPPA_POWER || prob->precision == FRKC2_DFLOAT)
    return FRKC2_EUNSUPPORTED;
  if (!(dt > 0.0) || !std::isfinite(dt) || l0 < 0 || l1 <= l0 || l1 > plan->s) return FRKC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return FRKC2_EINVAL;
  const size_t sb = state_bytes(prob->precision);
  if (reinterpret_cast<uintptr_t>(w) & (2 * sb - 1)) return FRKC2_EINVAL;
  const frkc2_problem& p = *prob;
  const StepLayout L = step_layout(p);
  if (ws_bytes < L.total) return FRKC2_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  const size_t n = cells(p);
  if (l0 == 0) {
    const int threads = 256;
    const int blocks = int(std::min<size_t>((n + threads - 1) / threads, 152 * 8));
    if (sb == 8)
      k_zero_imag<double><<<blocks, threads, 0, st>>>(static_cast<double*>(w), n);
    else
      k_zero_imag<float><<<blocks, threads, 0, st>>>(static_cast<float*>(w), n);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return FRKC2_ECUDA;
  }
  if (launch_faces(p, base + L.fx, base + L.fy, base + L.fz, st) != cudaSuccess ||
      launch_face_pairs(p, base + L.fx, base + L.fy, base + L.fen, st) != cudaSuccess)
    return FRKC2_ECUDA;
  // interleaved buffers: ua with va, ub with vb
  void* ua = base + L.ua;
  void* ub = base + L.ub;
  const double h2 = p.dx * p.dx;
  PassArgs a{};
  a.ndim = 2;
  a.bc = p.bc;
  a.nx = int(p.n[0]);
  a.ny = int(p.n[1]);
  a.nz = 1;
  a.k = 1;
  a.hx = a.hy = 1;
  a.in_mode = a.out_mode = PASS_IO_COMPLEX;
  a.status = reinterpret_cast<unsigned*>(base + L.status);
  const void* cur = w;
  for (int l = l0; l < l1; ++l) {
    const bool last = l == l1 - 1;
    void* out = (last && cur != w) ? w : (cur == ua ? ub : ua);
    a.U_in = cur;
    a.U_out = out;
    a.V_in = a.V_out = nullptr;
    a.check_finite = last ? 1 : 0;
    a.ca[0] = dt * plan->a_re[l] / h2;
    a.cb[0] = dt * plan->a_im[l] / h2;
    a.caf[0] = float(a.ca[0]);
    a.cbf[0] = float(a.cb[0]);
    if (launch_pass_stream2d(p, a, base + L.fen, st) != cudaSuccess) return FRKC2_ECUDA;
    cur = out;
  }
  if (cur != w && cudaMemcpyAsync(w, cur, 2 * n * sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return FRKC2_ECUDA;
  return FRKC2_OK;
}
