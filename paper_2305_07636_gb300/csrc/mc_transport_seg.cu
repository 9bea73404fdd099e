// Builds of the transport kernel (mc_transport.cuh) for FP32 tracking with segments scored apart
// from their flights: the 80- and 128-register budgets at 256 threads per CTA and the 96-register
// budget at 128 threads (5 CTAs per SM), each as one launch and as the two launches of a split run.
#include "mc_transport.cuh"

namespace mcgb {

const void* transport_fn_seg(bool wide, int block, int mode) {
  if (wide) {
    if (mode == 1) return (const void*)k_transport<float, 2, false, true, 1>;
    if (mode == 2) return (const void*)k_transport<float, 2, false, true, 2>;
    return (const void*)k_transport<float, 2, false, true, 0>;
  }
  if (block == 128) {
    if (mode == 1) return (const void*)k_transport<float, 5, false, true, 1>;
    if (mode == 2) return (const void*)k_transport<float, 5, false, true, 2>;
    return (const void*)k_transport<float, 5, false, true, 0>;
  }
  if (mode == 1) return (const void*)k_transport<float, 3, false, true, 1>;
  if (mode == 2) return (const void*)k_transport<float, 3, false, true, 2>;
  return (const void*)k_transport<float, 3, false, true, 0>;
}

}  // namespace mcgb
