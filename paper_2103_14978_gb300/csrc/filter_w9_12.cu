// Instantiations of the plain filter kernel for W = 9..12 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w9_12(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 9: return variant == 3 ? launch_filter_variant<9, 3>(a, stream) : variant == 2 ? launch_filter_variant<9, 2>(a, stream) : variant == 1 ? launch_filter_variant<9, 1>(a, stream) : launch_filter_variant<9, 0>(a, stream);
    case 10: return variant == 3 ? launch_filter_variant<10, 3>(a, stream) : variant == 2 ? launch_filter_variant<10, 2>(a, stream) : variant == 1 ? launch_filter_variant<10, 1>(a, stream) : launch_filter_variant<10, 0>(a, stream);
    case 11: return variant == 3 ? launch_filter_variant<11, 3>(a, stream) : variant == 2 ? launch_filter_variant<11, 2>(a, stream) : variant == 1 ? launch_filter_variant<11, 1>(a, stream) : launch_filter_variant<11, 0>(a, stream);
    case 12: return variant == 3 ? launch_filter_variant<12, 3>(a, stream) : variant == 2 ? launch_filter_variant<12, 2>(a, stream) : variant == 1 ? launch_filter_variant<12, 1>(a, stream) : launch_filter_variant<12, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
