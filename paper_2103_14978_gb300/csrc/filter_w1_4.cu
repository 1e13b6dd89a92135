// Instantiations of the plain filter kernel for W = 1..4 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w1_4(int W, const FilterArgs &a, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  switch (W) {
    case 1: filter_kernel<1><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 2: filter_kernel<2><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 3: filter_kernel<3><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 4: filter_kernel<4><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gk
