// Sliced sweep kernels, reads of any length up to GK_SLICED_MAX_LEN (a test
// per position): the compiled ranges of shift counts, each filtered in one pass.
#include "sliced_kernels.cuh"

namespace gk {

cudaError_t launch_sliced_sweep_m0(int klo, const SlicedArgs &a, cudaStream_t stream) {
  switch (klo) {
    case 0: return launch_sliced_range<0, 5, 0>(a, stream);
    case 6: return launch_sliced_range<6, 10, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
