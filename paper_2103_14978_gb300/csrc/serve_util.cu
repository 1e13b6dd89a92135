// Device support for continuous batching: a coalesced launch concatenates
// the pairs of many requests, whose read ids are relative to each request's
// own reads; this kernel moves them to the positions the reads were given in
// the launch's read buffer.
#include "gk_internal.cuh"

namespace {

__global__ void rebase_kernel(uint32_t *__restrict__ pair_read, uint8_t *__restrict__ pair_e, uint64_t n_pairs,
                              const uint64_t *__restrict__ seg_end, const int64_t *__restrict__ seg_delta,
                              const uint8_t *__restrict__ seg_e, uint32_t n_segs) {
  const uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  // first segment whose end exceeds p
  uint32_t lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (seg_end[mid] > p) hi = mid; else lo = mid + 1;
  }
  const int64_t v = (int64_t)pair_read[p] + seg_delta[lo];
  // Out-of-range results become an id no read has; the filter reports the
  // pair as invalid.
  pair_read[p] = (v < 0 || v > 0xFFFFFFFFll) ? 0xFFFFFFFFu : (uint32_t)v;
  if (pair_e) pair_e[p] = seg_e[lo];
}

}  // namespace

extern "C" int gk_rebase_pairs(uint32_t *pair_read, uint8_t *pair_e, uint64_t n_pairs, const uint64_t *seg_end,
                               const int64_t *seg_delta, const uint8_t *seg_e, uint32_t n_segs, void *stream) {
  gk::clear_error();
  if (n_pairs == 0) return GK_OK;
  if (!pair_read || !seg_end || !seg_delta || n_segs == 0 || (pair_e && !seg_e))
    return gk::fail(GK_EINVAL, "gk_rebase_pairs: null buffer or no segments");
  const int threads = 256;
  rebase_kernel<<<(unsigned)((n_pairs + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
      pair_read, pair_e, n_pairs, seg_end, seg_delta, seg_e, n_segs);
  return gk::cuda_check(cudaGetLastError(), "gk_rebase_pairs: launch");
}

extern "C" int gk_copy_many(void *const *dst, const void *const *src, const uint64_t *bytes, uint32_t n,
                            int kind, void *stream) {
  gk::clear_error();
  if (n == 0) return GK_OK;
  if (!dst || !src || !bytes) return gk::fail(GK_EINVAL, "gk_copy_many: null array");
  if (kind != 1 && kind != 2 && kind != 3) return gk::fail(GK_EINVAL, "gk_copy_many: kind must be 1, 2 or 3");
  const cudaMemcpyKind k = kind == 1 ? cudaMemcpyHostToDevice
                                     : (kind == 2 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  for (uint32_t i = 0; i < n; ++i) {
    if (bytes[i] == 0) continue;
    const cudaError_t err = cudaMemcpyAsync(dst[i], src[i], bytes[i], k, (cudaStream_t)stream);
    if (err != cudaSuccess) return gk::cuda_check(err, "gk_copy_many: cudaMemcpyAsync");
  }
  return GK_OK;
}
