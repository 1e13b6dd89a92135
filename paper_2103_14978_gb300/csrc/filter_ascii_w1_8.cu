// Instantiations of the fused encode + filter kernel for W = 1..8 words per read.
#include "filter_ascii.cuh"

namespace gk {

cudaError_t launch_filter_ascii_w1_8(int W, int variant, const AsciiArgs &g, cudaStream_t stream) {
  switch (W) {
    case 1: return variant == 2 ? launch_filter_ascii_variant<1, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<1, 1>(g, stream) : launch_filter_ascii_variant<1, 0>(g, stream);
    case 2: return variant == 2 ? launch_filter_ascii_variant<2, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<2, 1>(g, stream) : launch_filter_ascii_variant<2, 0>(g, stream);
    case 3: return variant == 2 ? launch_filter_ascii_variant<3, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<3, 1>(g, stream) : launch_filter_ascii_variant<3, 0>(g, stream);
    case 4: return variant == 2 ? launch_filter_ascii_variant<4, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<4, 1>(g, stream) : launch_filter_ascii_variant<4, 0>(g, stream);
    case 5: return variant == 2 ? launch_filter_ascii_variant<5, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<5, 1>(g, stream) : launch_filter_ascii_variant<5, 0>(g, stream);
    case 6: return variant == 2 ? launch_filter_ascii_variant<6, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<6, 1>(g, stream) : launch_filter_ascii_variant<6, 0>(g, stream);
    case 7: return variant == 2 ? launch_filter_ascii_variant<7, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<7, 1>(g, stream) : launch_filter_ascii_variant<7, 0>(g, stream);
    case 8: return variant == 2 ? launch_filter_ascii_variant<8, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<8, 1>(g, stream) : launch_filter_ascii_variant<8, 0>(g, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
