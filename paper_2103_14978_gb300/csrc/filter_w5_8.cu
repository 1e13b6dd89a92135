// Instantiations of the plain filter kernel for W = 5..8 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w5_8(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 5: return variant == 3 ? launch_filter_variant<5, 3>(a, stream) : variant == 2 ? launch_filter_variant<5, 2>(a, stream) : variant == 1 ? launch_filter_variant<5, 1>(a, stream) : launch_filter_variant<5, 0>(a, stream);
    case 6: return variant == 3 ? launch_filter_variant<6, 3>(a, stream) : variant == 2 ? launch_filter_variant<6, 2>(a, stream) : variant == 1 ? launch_filter_variant<6, 1>(a, stream) : launch_filter_variant<6, 0>(a, stream);
    case 7: return variant == 3 ? launch_filter_variant<7, 3>(a, stream) : variant == 2 ? launch_filter_variant<7, 2>(a, stream) : variant == 1 ? launch_filter_variant<7, 1>(a, stream) : launch_filter_variant<7, 0>(a, stream);
    case 8: return variant == 3 ? launch_filter_variant<8, 3>(a, stream) : variant == 2 ? launch_filter_variant<8, 2>(a, stream) : variant == 1 ? launch_filter_variant<8, 1>(a, stream) : launch_filter_variant<8, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
