// Instantiations of the plain filter kernel for W = 1..4 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w1_4(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 1: return variant == 4 ? launch_filter_variant<1, 4>(a, stream) : variant == 3 ? launch_filter_variant<1, 3>(a, stream) : variant == 2 ? launch_filter_variant<1, 2>(a, stream) : variant == 1 ? launch_filter_variant<1, 1>(a, stream) : launch_filter_variant<1, 0>(a, stream);
    case 2: return variant == 4 ? launch_filter_variant<2, 4>(a, stream) : variant == 3 ? launch_filter_variant<2, 3>(a, stream) : variant == 2 ? launch_filter_variant<2, 2>(a, stream) : variant == 1 ? launch_filter_variant<2, 1>(a, stream) : launch_filter_variant<2, 0>(a, stream);
    case 3: return variant == 4 ? launch_filter_variant<3, 4>(a, stream) : variant == 3 ? launch_filter_variant<3, 3>(a, stream) : variant == 2 ? launch_filter_variant<3, 2>(a, stream) : variant == 1 ? launch_filter_variant<3, 1>(a, stream) : launch_filter_variant<3, 0>(a, stream);
    case 4: return variant == 4 ? launch_filter_variant<4, 4>(a, stream) : variant == 3 ? launch_filter_variant<4, 3>(a, stream) : variant == 2 ? launch_filter_variant<4, 2>(a, stream) : variant == 1 ? launch_filter_variant<4, 1>(a, stream) : launch_filter_variant<4, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
