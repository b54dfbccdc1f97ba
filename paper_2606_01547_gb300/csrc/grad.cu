// Chi^2 log-likelihood and its hand-written adjoint (placeholder until the adjoint kernels land).
#include "kernels.h"
#include "lens_sim.h"
#include "sim_internal.h"

extern "C" int lens_sim_grad(lens_sim* s, const lens_system*, const float*, float, float, const float*, int,
                             float*, float*, void*) {
  if (!s) return LENS_ERR_INVALID_ARG;
  return ls::fail(s, LENS_ERR_UNSUPPORTED, "lens_sim_grad is not built yet");
}
