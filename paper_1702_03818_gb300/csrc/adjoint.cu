// Adjoint entry points (reverse replay of the FRKC2 stages).
#include "frkc2.h"
#include "frkc2_internal.h"

extern "C" {

frkc2_status frkc2_adjoint_workspace_size(const frkc2_plan_t, const frkc2_problem*, int, int, size_t*) {
  return FRKC2_EUNSUPPORTED;
}

frkc2_status frkc2_adjoint(frkc2_plan_t, const frkc2_problem*, double, int, int, const void*, const void*,
                           void*, void*, void*, size_t, void*) {
  return FRKC2_EUNSUPPORTED;
}

}  // extern "C"
