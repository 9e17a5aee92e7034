// Batched persistent forward step over many independent 2D problems.
#include "frkc2.h"
#include "frkc2_internal.h"

extern "C" {

frkc2_status frkc2_batch_workspace_size(int, const frkc2_plan_t*, const frkc2_problem*, const int*,
                                        const frkc2_tuning*, size_t*) {
  return FRKC2_EUNSUPPORTED;
}
frkc2_status frkc2_batch_prepare(int, const frkc2_plan_t*, const frkc2_problem*, const double*, const int*,
                                 void* const*, const frkc2_tuning*, void*, size_t, void*) {
  return FRKC2_EUNSUPPORTED;
}
frkc2_status frkc2_batch_launch(void*, void*) { return FRKC2_EUNSUPPORTED; }
frkc2_status frkc2_step_batched(int, const frkc2_plan_t*, const frkc2_problem*, const double*, const int*,
                                void* const*, const frkc2_tuning*, void*, size_t, void*) {
  return FRKC2_EUNSUPPORTED;
}

}  // extern "C"
