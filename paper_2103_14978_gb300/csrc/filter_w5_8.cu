// Instantiations of the plain filter kernel for W = 5..8 words per read.
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
