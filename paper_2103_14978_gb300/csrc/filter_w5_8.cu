// Instantiations of the plain filter kernel for W = 5..8 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w5_8(int W, const FilterArgs &a, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  switch (W) {
    case 5: filter_kernel<5><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 6: filter_kernel<6><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 7: filter_kernel<7><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 8: filter_kernel<8><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gk
