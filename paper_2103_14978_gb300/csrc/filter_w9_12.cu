// Instantiations of the plain filter kernel for W = 9..12 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w9_12(int W, const FilterArgs &a, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  switch (W) {
    case 9: filter_kernel<9><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 10: filter_kernel<10><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 11: filter_kernel<11><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 12: filter_kernel<12><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gk
