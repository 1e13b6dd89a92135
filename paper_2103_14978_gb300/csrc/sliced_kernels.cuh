// Sliced filter kernels: one thread per group of 32 pairs, one
// instantiation per shift count K and read length M (M = 0: any length).
// Each sliced_m*_k*.cu instantiates one M and a range of K.
#pragma once

#include "sliced.cuh"

namespace gk {
namespace {

// Resident 128-thread blocks per SM the register budget is set for: the
// read ring takes 3 words per slot (16 slots up to K = 6, 24 up to K = 10,
// 32 up to K = 14, 40 at K = 15).
template <int K>
struct SlicedMinBlocks {
  static constexpr int value = K <= 3 ? 4 : (K <= 10 ? 3 : 2);
};

template <int K, int M>
__global__ void __launch_bounds__(kSlicedThreads, SlicedMinBlocks<K>::value) sliced_filter_kernel(const SlicedArgs a) {
  __shared__ uint32_t s_clr[(2 * K + 2) * kSlicedThreads];
  const uint64_t g = (uint64_t)blockIdx.x * kSlicedThreads + threadIdx.x;
  if (g >= sliced_groups(a.n_pairs)) return;
  sliced_group<K, M>(a, g, s_clr + threadIdx.x, kSlicedThreads);
}

template <int K, int M>
cudaError_t launch_sliced_km(const SlicedArgs &a, cudaStream_t stream) {
  const uint64_t groups = sliced_groups(a.n_pairs);
  const unsigned blocks = (unsigned)((groups + kSlicedThreads - 1) / kSlicedThreads);
  sliced_filter_kernel<K, M><<<blocks, kSlicedThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace gk
