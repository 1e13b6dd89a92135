// Sliced filter kernels, read length 150 bases, shift counts K = 0..5.
#include "sliced_kernels.cuh"

namespace gk {

cudaError_t launch_sliced_m150_k0_5(int K, const SlicedArgs &a, cudaStream_t stream) {
  switch (K) {
    case 0: return launch_sliced_km<0, 150>(a, stream);
    case 1: return launch_sliced_km<1, 150>(a, stream);
    case 2: return launch_sliced_km<2, 150>(a, stream);
    case 3: return launch_sliced_km<3, 150>(a, stream);
    case 4: return launch_sliced_km<4, 150>(a, stream);
    case 5: return launch_sliced_km<5, 150>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
