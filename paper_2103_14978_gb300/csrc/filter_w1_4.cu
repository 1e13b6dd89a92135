// Instantiations of the plain filter kernel for W = 1..4 words per read.
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

cudaError_t launch_filter_w1_4(int W, int variant, const FilterArgs &a, cudaStream_t stream) {
  switch (W) {
    case 1: return variant == 2 ? launch_one<1, 2>(a, stream) : variant == 1 ? launch_one<1, 1>(a, stream) : launch_one<1, 0>(a, stream);
    case 2: return variant == 2 ? launch_one<2, 2>(a, stream) : variant == 1 ? launch_one<2, 1>(a, stream) : launch_one<2, 0>(a, stream);
    case 3: return variant == 2 ? launch_one<3, 2>(a, stream) : variant == 1 ? launch_one<3, 1>(a, stream) : launch_one<3, 0>(a, stream);
    case 4: return variant == 2 ? launch_one<4, 2>(a, stream) : variant == 1 ? launch_one<4, 1>(a, stream) : launch_one<4, 0>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
