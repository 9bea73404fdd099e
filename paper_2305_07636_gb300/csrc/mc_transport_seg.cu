// Builds of the transport kernel (mc_transport.cuh) for FP32 tracking with segments scored apart
// from their flights: the 80- and 128-register budgets, each as one launch and as the two launches
// of a split run.
#include "mc_transport.cuh"

namespace mcgb {

const void* transport_fn_seg(bool wide, int mode) {
  if (mode == 1) return wide ? (const void*)k_transport<float, 2, false, true, 1> : (const void*)k_transport<float, 3, false, true, 1>;
  if (mode == 2) return wide ? (const void*)k_transport<float, 2, false, true, 2> : (const void*)k_transport<float, 3, false, true, 2>;
  return wide ? (const void*)k_transport<float, 2, false, true, 0> : (const void*)k_transport<float, 3, false, true, 0>;
}

}  // namespace mcgb
