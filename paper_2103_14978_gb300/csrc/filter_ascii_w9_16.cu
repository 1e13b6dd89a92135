// Instantiations of the fused encode + filter kernel for W = 9..16 words per read.
#include "filter_ascii.cuh"

namespace gk {

cudaError_t launch_filter_ascii_w9_16(int W, int variant, const AsciiArgs &g, cudaStream_t stream) {
  switch (W) {
    case 9: return variant == 2 ? launch_filter_ascii_variant<9, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<9, 1>(g, stream) : launch_filter_ascii_variant<9, 0>(g, stream);
    case 10: return variant == 2 ? launch_filter_ascii_variant<10, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<10, 1>(g, stream) : launch_filter_ascii_variant<10, 0>(g, stream);
    case 11: return variant == 2 ? launch_filter_ascii_variant<11, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<11, 1>(g, stream) : launch_filter_ascii_variant<11, 0>(g, stream);
    case 12: return variant == 2 ? launch_filter_ascii_variant<12, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<12, 1>(g, stream) : launch_filter_ascii_variant<12, 0>(g, stream);
    case 13: return variant == 2 ? launch_filter_ascii_variant<13, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<13, 1>(g, stream) : launch_filter_ascii_variant<13, 0>(g, stream);
    case 14: return variant == 2 ? launch_filter_ascii_variant<14, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<14, 1>(g, stream) : launch_filter_ascii_variant<14, 0>(g, stream);
    case 15: return variant == 2 ? launch_filter_ascii_variant<15, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<15, 1>(g, stream) : launch_filter_ascii_variant<15, 0>(g, stream);
    case 16: return variant == 2 ? launch_filter_ascii_variant<16, 2>(g, stream) : variant == 1 ? launch_filter_ascii_variant<16, 1>(g, stream) : launch_filter_ascii_variant<16, 0>(g, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
