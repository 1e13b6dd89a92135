// Sliced filter kernels, read length any (runtime), shift counts K = 6..10.
#include "sliced_kernels.cuh"

namespace gk {

cudaError_t launch_sliced_m0_k6_10(int K, const SlicedArgs &a, cudaStream_t stream) {
  switch (K) {
    case 6: return launch_sliced_km<6, 0>(a, stream);
    case 7: return launch_sliced_km<7, 0>(a, stream);
    case 8: return launch_sliced_km<8, 0>(a, stream);
    case 9: return launch_sliced_km<9, 0>(a, stream);
    case 10: return launch_sliced_km<10, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
