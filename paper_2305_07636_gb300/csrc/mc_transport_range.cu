// Builds of the transport kernel (mc_transport.cuh) for FP32 tracking with the range walk of
// time-fine tallies: the 80- and 128-register budgets, each as one launch and as the two launches
// of a split run.
#include "mc_transport.cuh"

namespace mcgb {

const void* transport_fn_range(bool wide, int mode) {
  if (mode == 1) return wide ? (const void*)k_transport<float, 2, true, false, 1> : (const void*)k_transport<float, 3, true, false, 1>;
  if (mode == 2) return wide ? (const void*)k_transport<float, 2, true, false, 2> : (const void*)k_transport<float, 3, true, false, 2>;
  return wide ? (const void*)k_transport<float, 2, true, false, 0> : (const void*)k_transport<float, 3, true, false, 0>;
}

}  // namespace mcgb
