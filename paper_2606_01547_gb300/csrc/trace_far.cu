// Far-field instantiations of the fused image-simulation kernels (the optional interpolation of
// the subhalo sum at a unit's Chebyshev nodes; device code in trace_unit.cuh), compiled apart
// from the exact ones in trace.cu so that the two build in parallel.
#include "trace_unit.cuh"

namespace ls {

void launch_trace_far(const DevSystem& sys, int variant, int units, cudaStream_t st) {
  if (block_layout(sys.s)) launch_trace_form<true, true>(sys, variant, units, st);
  else launch_trace_form<true, false>(sys, variant, units, st);
}

void launch_trace_batch_far(BatchMeta* m, int form, int grid, cudaStream_t st) {
  launch_batch_form<true>(m, form, grid, st);
}

}  // namespace ls
