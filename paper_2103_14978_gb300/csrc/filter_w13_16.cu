// Instantiations of the plain filter kernel for W = 13..16 words per read.
#include "filter.cuh"

namespace gk {

cudaError_t launch_filter_w13_16(int W, const FilterArgs &a, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  switch (W) {
    case 13: filter_kernel<13><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 14: filter_kernel<14><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 15: filter_kernel<15><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    case 16: filter_kernel<16><<<blocks, kFilterThreads, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gk
