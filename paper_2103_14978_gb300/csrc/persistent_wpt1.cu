// Persistent batched filter kernel, one pair per lane for reads up to 256
// bases (lane groups of 4 words per lane for longer reads).
#include "batched.cuh"

namespace gk {

cudaError_t launch_persistent_wpt1(const BatchArgs &a, uint32_t grid, uint32_t wpb, cudaStream_t s) {
  int fit = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, persistent_kernel<1>, 32 * (int)wpb, 0);
  if (err != cudaSuccess) return err;
  if (fit == 0) return cudaErrorInvalidConfiguration;  // block does not fit the register file
  persistent_kernel<1><<<grid, 32 * wpb, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gk
