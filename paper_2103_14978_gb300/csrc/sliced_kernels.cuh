// Sliced filter kernels: one thread per group of 32 pairs, one
// instantiation per range of shift counts KLO..KHI (KLO == KHI: one
// threshold) and read length M (M = 0: any length).  Each sliced_m*_k*.cu
// instantiates one M and a range of single shift counts; each
// sliced_sweep_m*.cu the sweep ranges of one M.
#pragma once

#include "sliced.cuh"

namespace gk {
namespace {

// Resident 128-thread blocks per SM the register budget is set for.  One
// threshold: the read ring takes 3 words per slot (16 slots up to K = 6, 24
// up to K = 10, 32 up to K = 14, 40 at K = 15).  Sweeps add the per-K
// erosion and count state (about 13 words per shift count).
template <int KLO, int KHI>
struct SlicedMinBlocks {
  static constexpr int value = KLO == KHI ? (KHI <= 3 ? 4 : (KHI <= 10 ? 3 : 2)) : 2;
};

template <int KLO, int KHI, int M>
__global__ void __launch_bounds__(kSlicedThreads, SlicedMinBlocks<KLO, KHI>::value)
    sliced_filter_kernel(const SlicedArgs a) {
  __shared__ uint32_t s_clr[SlicedCorr<KLO, KHI>::words * kSlicedThreads];
  const uint64_t g = (uint64_t)blockIdx.x * kSlicedThreads + threadIdx.x;
  if (g >= sliced_groups(a.n_pairs)) return;
  sliced_sweep_group<KLO, KHI, M>(a, g, s_clr + threadIdx.x, kSlicedThreads);
}

template <int KLO, int KHI, int M>
cudaError_t launch_sliced_range(const SlicedArgs &a, cudaStream_t stream) {
  const uint64_t groups = sliced_groups(a.n_pairs);
  const unsigned blocks = (unsigned)((groups + kSlicedThreads - 1) / kSlicedThreads);
  sliced_filter_kernel<KLO, KHI, M><<<blocks, kSlicedThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

template <int K, int M>
cudaError_t launch_sliced_km(const SlicedArgs &a, cudaStream_t stream) {
  return launch_sliced_range<K, K, M>(a, stream);
}

}  // namespace
}  // namespace gk
