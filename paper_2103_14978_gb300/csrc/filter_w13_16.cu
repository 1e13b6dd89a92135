// Instantiations of the plain filter kernel for W = 13..16 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w13_16(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 13: return variant == 3 ? launch_filter_variant<13, 3>(a, stream) : variant == 2 ? launch_filter_variant<13, 2>(a, stream) : variant == 1 ? launch_filter_variant<13, 1>(a, stream) : launch_filter_variant<13, 0>(a, stream);
    case 14: return variant == 3 ? launch_filter_variant<14, 3>(a, stream) : variant == 2 ? launch_filter_variant<14, 2>(a, stream) : variant == 1 ? launch_filter_variant<14, 1>(a, stream) : launch_filter_variant<14, 0>(a, stream);
    case 15: return variant == 3 ? launch_filter_variant<15, 3>(a, stream) : variant == 2 ? launch_filter_variant<15, 2>(a, stream) : variant == 1 ? launch_filter_variant<15, 1>(a, stream) : launch_filter_variant<15, 0>(a, stream);
    case 16: return variant == 3 ? launch_filter_variant<16, 3>(a, stream) : variant == 2 ? launch_filter_variant<16, 2>(a, stream) : variant == 1 ? launch_filter_variant<16, 1>(a, stream) : launch_filter_variant<16, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
