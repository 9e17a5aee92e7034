// frkc2_step_noalloc: the forward step for callers that cannot allocate device memory.
//
// frkc2_step needs a caller-provided workspace (status word, face conductivities and the
// ping-pong stage buffers).  Some callers cannot provide one: a solver plugin whose host
// application owns every device allocation and forbids the plugin from calling the CUDA
// allocator, code that runs while a memory pool or allocator is locked by the caller, or a
// deployment with a fixed device-memory budget decided before the solver is loaded.  This
// entry point gives them the same step with the workspace taken from a fixed array that is
// part of the library image: nothing is allocated at call time.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library holds
// FRKC2_NOALLOC_SCRATCH_BYTES of device memory for it until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a host-side
// stand-in); every call obtains the device address with cudaGetSymbolAddress on the current
// device.  The address is not cached: after cudaDeviceReset, or when the primary context is
// destroyed and created again, the library's device code is loaded anew and the array may
// move, and a cached address would then point at freed memory.
#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FRKC2_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current device's context.  The lookup allocates
// nothing; the first one in a context may load the library's device code.
frkc2_status scratch_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FRKC2_ECUDA;
  *out = p;
  return FRKC2_OK;
}

}  // namespace

extern "C" frkc2_status frkc2_step_noalloc(frkc2_plan_t plan, const frkc2_problem* prob, double dt,
                                           int nsteps, double rho, void* u, void* stream) {
  if (!plan || !u || nsteps < 0) return FRKC2_EINVAL;
  size_t need = 0;
  const frkc2_status v = frkc2_workspace_size(prob, nullptr, &need);
  if (v != FRKC2_OK) return v;
  if (need > FRKC2_NOALLOC_SCRATCH_BYTES) return FRKC2_ENOMEM;  // problem too large for the array
  if (!(dt > 0.0) || (rho > 0.0 && dt * rho > plan->beta * (1.0 + 1e-12))) {
    return dt > 0.0 ? FRKC2_EUNSTABLE : FRKC2_EINVAL;
  }
  void* ws = nullptr;
  const frkc2_status a = scratch_address(&ws);
  if (a != FRKC2_OK) return a;
  // the status word must start at zero; the rest of the array is written before it is read
  if (cudaMemsetAsync(ws, 0, 256, static_cast<cudaStream_t>(stream)) != cudaSuccess) return FRKC2_ECUDA;
  return frkc2_step(plan, prob, dt, nsteps, rho, u, ws, FRKC2_NOALLOC_SCRATCH_BYTES, nullptr, stream);
}
