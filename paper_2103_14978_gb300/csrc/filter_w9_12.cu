// Instantiations of the plain filter kernel for W = 9..12 words per read.
#include "filter.cuh"

namespace gk {

namespace {

template <int W, int VARIANT>
cudaError_t launch_one(const FilterArgs &a, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  filter_kernel<W, VARIANT><<<blocks, kFilterThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter_w9_12(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 9: return variant == 2 ? launch_one<9, 2>(a, stream) : variant == 1 ? launch_one<9, 1>(a, stream) : launch_one<9, 0>(a, stream);
    case 10: return variant == 2 ? launch_one<10, 2>(a, stream) : variant == 1 ? launch_one<10, 1>(a, stream) : launch_one<10, 0>(a, stream);
    case 11: return variant == 2 ? launch_one<11, 2>(a, stream) : variant == 1 ? launch_one<11, 1>(a, stream) : launch_one<11, 0>(a, stream);
    case 12: return variant == 2 ? launch_one<12, 2>(a, stream) : variant == 1 ? launch_one<12, 1>(a, stream) : launch_one<12, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
