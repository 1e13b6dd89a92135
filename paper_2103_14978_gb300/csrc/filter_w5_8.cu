// Instantiations of the plain filter kernel for W = 5..8 words per read.
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

cudaError_t launch_filter_w5_8(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 5: return variant == 2 ? launch_one<5, 2>(a, stream) : variant == 1 ? launch_one<5, 1>(a, stream) : launch_one<5, 0>(a, stream);
    case 6: return variant == 2 ? launch_one<6, 2>(a, stream) : variant == 1 ? launch_one<6, 1>(a, stream) : launch_one<6, 0>(a, stream);
    case 7: return variant == 2 ? launch_one<7, 2>(a, stream) : variant == 1 ? launch_one<7, 1>(a, stream) : launch_one<7, 0>(a, stream);
    case 8: return variant == 2 ? launch_one<8, 2>(a, stream) : variant == 1 ? launch_one<8, 1>(a, stream) : launch_one<8, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
