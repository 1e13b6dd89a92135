// Sliced filter kernels, read length 100 bases, shift counts K = 0..5.
#include "sliced_kernels.cuh"

namespace gk {

cudaError_t launch_sliced_m100_k0_5(int K, const SlicedArgs &a, cudaStream_t stream) {
  switch (K) {
    case 0: return launch_sliced_km<0, 100>(a, stream);
    case 1: return launch_sliced_km<1, 100>(a, stream);
    case 2: return launch_sliced_km<2, 100>(a, stream);
    case 3: return launch_sliced_km<3, 100>(a, stream);
    case 4: return launch_sliced_km<4, 100>(a, stream);
    case 5: return launch_sliced_km<5, 100>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
