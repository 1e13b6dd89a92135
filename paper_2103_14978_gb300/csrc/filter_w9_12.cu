// Instantiations of the plain filter kernel for W = 9..12 words per read.
#include "filter.cuh"

namespace gk {

namespace {

template <int W, int VARIANT>
cudaError_t launch_one(const FilterArgs &a, cudaStream_t stream) {
  unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  if (a.compact) {  // persistent warps: a few waves of resident blocks
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, filter_kernel<W, VARIANT, true>,
                                                                            kFilterThreads, 0);
      if (err != cudaSuccess) return err;
      if (per_sm < 1) per_sm = 1;
    }
    const uint64_t wave = 4ull * (uint64_t)sms * (uint64_t)per_sm;
    if (blocks > wave) blocks = (unsigned)wave;
  }
  if (a.compact)
    filter_kernel<W, VARIANT, true><<<blocks, kFilterThreads, 0, stream>>>(a);
  else
    filter_kernel<W, VARIANT, false><<<blocks, kFilterThreads, 0, stream>>>(a);
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
