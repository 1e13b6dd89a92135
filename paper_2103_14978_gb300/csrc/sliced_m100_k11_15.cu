// Sliced filter kernels, read length 100 bases, shift counts K = 11..15.
#include "sliced_kernels.cuh"

namespace gk {

cudaError_t launch_sliced_m100_k11_15(int K, const SlicedArgs &a, cudaStream_t stream) {
  switch (K) {
    case 11: return launch_sliced_km<11, 100>(a, stream);
    case 12: return launch_sliced_km<12, 100>(a, stream);
    case 13: return launch_sliced_km<13, 100>(a, stream);
    case 14: return launch_sliced_km<14, 100>(a, stream);
    case 15: return launch_sliced_km<15, 100>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
