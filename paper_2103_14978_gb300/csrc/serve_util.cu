// Device support for continuous batching: a coalesced launch concatenates
// the pairs of many requests, whose read ids are relative to each request's
// own reads; this kernel moves them to the positions the reads were given in
// the launch's read buffer.
#include <atomic>

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

// One thread per read of the launch (reads numbered across the segments):
// its segment by binary search, its slot, its pairs from the start offsets,
// clamped to the segment's pairs.
__global__ void expand_kernel(uint32_t *__restrict__ pair_read, uint8_t *__restrict__ pair_e,
                              const uint32_t *__restrict__ read_start, const uint64_t *__restrict__ seg_read_end,
                              const uint64_t *__restrict__ seg_pair_end, const uint64_t *__restrict__ seg_read_slot,
                              const uint32_t *__restrict__ seg_start_base, const uint8_t *__restrict__ seg_e,
                              const uint32_t *__restrict__ seg_read_info, uint16_t *__restrict__ read_len,
                              uint8_t *__restrict__ read_nflag, uint32_t n_segs, uint64_t n_vreads,
                              uint64_t n_pairs) {
  const uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (v >= n_vreads) return;
  uint32_t lo = 0, hi = n_segs - 1;  // first segment whose read end exceeds v
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (seg_read_end[mid] > v) hi = mid; else lo = mid + 1;
  }
  const uint64_t r0 = lo ? seg_read_end[lo - 1] : 0, p0 = lo ? seg_pair_end[lo - 1] : 0;
  const uint64_t np = seg_pair_end[lo] - p0;
  const uint64_t slot = seg_read_slot[lo] + (v - r0);
  const uint32_t base = seg_start_base[lo];
  const uint64_t a = (uint32_t)(read_start[slot] - base);
  const uint64_t b = v + 1 < seg_read_end[lo] ? (uint64_t)(uint32_t)(read_start[slot + 1] - base) : np;
  const uint64_t from = a < np ? a : np, to = b < np ? b : np;
  const uint32_t id = slot <= 0xFFFFFFFEull ? (uint32_t)slot : 0xFFFFFFFFu;
  const uint8_t e = seg_e[lo];
  if (seg_read_info) {  // one length and / or no N for the whole segment
    const uint32_t info = seg_read_info[lo];
    if ((info & 0xFFFFu) && read_len) read_len[slot] = (uint16_t)(info & 0xFFFFu);
    if ((info & GK_SEG_NO_N) && read_nflag) read_nflag[slot] = 0;
  }
  const uint64_t end = p0 + to < n_pairs ? p0 + to : n_pairs;  // never past the launch's pairs
  for (uint64_t j = p0 + from; j < end; ++j) {
    pair_read[j] = id;
    pair_e[j] = e;
  }
}

// One batch, one thread per read: pairs read_start[i] .. read_start[i+1]-1
// (the last read's through n_pairs-1) get id i, clamped to the batch.
__global__ void expand_rows_kernel(uint32_t *__restrict__ pair_read, uint64_t n_pairs,
                                   const uint32_t *__restrict__ read_start, uint64_t n_reads) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n_reads) return;
  const uint64_t a = read_start[i], b = i + 1 < n_reads ? (uint64_t)read_start[i + 1] : n_pairs;
  const uint64_t to = b < n_pairs ? b : n_pairs;
  for (uint64_t j = a; j < to; ++j) pair_read[j] = (uint32_t)i;
}

}  // namespace

namespace gk {

cudaError_t launch_expand_rows(uint32_t *pair_read, uint64_t n_pairs, const uint32_t *read_start, uint64_t n_reads,
                               cudaStream_t stream) {
  if (n_pairs == 0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(pair_read, 0xFF, n_pairs * sizeof(uint32_t), stream);
  if (err != cudaSuccess || n_reads == 0) return err;
  const int threads = 256;
  expand_rows_kernel<<<(unsigned)((n_reads + threads - 1) / threads), threads, 0, stream>>>(pair_read, n_pairs,
                                                                                          read_start, n_reads);
  return cudaGetLastError();
}

}  // namespace gk

extern "C" int gk_expand_pairs(uint32_t *pair_read, uint8_t *pair_e, uint64_t n_pairs, const uint32_t *read_start,
                               const uint64_t *seg_read_end, const uint64_t *seg_pair_end,
                               const uint64_t *seg_read_slot, const uint32_t *seg_start_base,
                               const uint8_t *seg_e, const uint32_t *seg_read_info, uint16_t *read_len,
                               uint8_t *read_nflag, uint32_t n_segs, uint64_t n_reads, void *stream) {
  gk::clear_error();
  if (n_pairs == 0 && !seg_read_info) return GK_OK;
  if (!pair_read || !pair_e || !read_start || !seg_read_end || !seg_pair_end || !seg_read_slot ||
      !seg_start_base || !seg_e || n_segs == 0)
    return gk::fail(GK_EINVAL, "gk_expand_pairs: null buffer or no segments");
  cudaStream_t st = (cudaStream_t)stream;
  // Pairs that no read claims stay invalid (an id no read has).
  if (n_pairs) {
    const cudaError_t err = cudaMemsetAsync(pair_read, 0xFF, n_pairs * sizeof(uint32_t), st);
    if (err != cudaSuccess) return gk::cuda_check(err, "gk_expand_pairs: fill");
  }
  if (n_reads == 0) return GK_OK;
  const int threads = 256;
  expand_kernel<<<(unsigned)((n_reads + threads - 1) / threads), threads, 0, st>>>(
      pair_read, pair_e, read_start, seg_read_end, seg_pair_end, seg_read_slot, seg_start_base, seg_e,
      seg_read_info, read_len, read_nflag, n_segs, n_reads, n_pairs);
  return gk::cuda_check(cudaGetLastError(), "gk_expand_pairs: launch");
}

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

namespace {

// Copies entry `at`: bytes[at] (<= GK_GATHER_MAX_BYTES) from src[at] to
// dst[at] with 16-byte accesses when both addresses share their offset
// modulo 16, else 4-byte accesses when they share it modulo 4, else bytes.
__device__ __forceinline__ void gather_entry(const uint64_t *__restrict__ dst, const uint64_t *__restrict__ src,
                                             const uint64_t *__restrict__ bytes, uint32_t at) {
  const uint64_t n = bytes[at];
  if (n == 0 || n > GK_GATHER_MAX_BYTES) return;
  uint8_t *d = reinterpret_cast<uint8_t *>(dst[at]);
  const uint8_t *s = reinterpret_cast<const uint8_t *>(src[at]);
  const uint32_t t = threadIdx.x, nt = blockDim.x;
  const uintptr_t rel = reinterpret_cast<uintptr_t>(s) ^ reinterpret_cast<uintptr_t>(d);
  const uint32_t unit = (rel & 15) == 0 ? 16u : ((rel & 3) == 0 ? 4u : 1u);
  // bytes before the first aligned unit, then whole units, then the tail
  uint64_t head = (unit - (reinterpret_cast<uintptr_t>(s) & (unit - 1))) & (unit - 1);
  if (head > n) head = n;
  const uint64_t body = (n - head) / unit;
  const uint64_t tail_at = head + body * unit;
  for (uint64_t i = t; i < head; i += nt) d[i] = s[i];
  if (unit == 16) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(s + head);
    uint4 *d4 = reinterpret_cast<uint4 *>(d + head);
    uint64_t i = t;
    for (; i + 3 * nt < body; i += 4 * nt) {  // four loads in flight per thread
      const uint4 a = s4[i], b = s4[i + nt], c = s4[i + 2 * nt], e = s4[i + 3 * nt];
      d4[i] = a;
      d4[i + nt] = b;
      d4[i + 2 * nt] = c;
      d4[i + 3 * nt] = e;
    }
    for (; i < body; i += nt) d4[i] = s4[i];
  } else if (unit == 4) {
    const uint32_t *s1 = reinterpret_cast<const uint32_t *>(s + head);
    uint32_t *d1 = reinterpret_cast<uint32_t *>(d + head);
    uint64_t i = t;
    for (; i + 3 * nt < body; i += 4 * nt) {
      const uint32_t a = s1[i], b = s1[i + nt], c = s1[i + 2 * nt], e = s1[i + 3 * nt];
      d1[i] = a;
      d1[i + nt] = b;
      d1[i + 2 * nt] = c;
      d1[i + 3 * nt] = e;
    }
    for (; i < body; i += nt) d1[i] = s1[i];
  } else {
    for (uint64_t i = t; i < body; i += nt) d[head + i] = s[head + i];
  }
  for (uint64_t i = tail_at + t; i < n; i += nt) d[i] = s[i];
}

// A few blocks per SM walk the entries: enough loads in flight to fill the
// host link without taking the SMs from a filter running on another stream.
__global__ void __launch_bounds__(256) gather_kernel(const uint64_t *__restrict__ dst, const uint64_t *__restrict__ src,
                                                     const uint64_t *__restrict__ bytes, uint32_t n) {
  for (uint32_t at = blockIdx.x; at < n; at += gridDim.x) gather_entry(dst, src, bytes, at);
}

}  // namespace

extern "C" int gk_gather(const uint64_t *dst, const uint64_t *src, const uint64_t *bytes, uint32_t n,
                         void *stream) {
  gk::clear_error();
  if (n == 0) return GK_OK;
  if (!dst || !src || !bytes) return gk::fail(GK_EINVAL, "gk_gather: null table");
  if (n > 0x7fffffffu) return gk::fail(GK_ERANGE, "gk_gather: too many entries");
  // SM count of the current device, looked up once per device.
  constexpr int kMaxDev = 64;
  static std::atomic<int> sm_count[kMaxDev];
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return gk::cuda_check(err, "gk_gather: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDev) return gk::fail(GK_ERANGE, "gk_gather: device index too large");
  int sms = sm_count[dev].load(std::memory_order_relaxed);
  if (sms == 0) {
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return gk::cuda_check(err, "gk_gather: cudaDeviceGetAttribute");
    if (sms < 1) sms = 1;
    sm_count[dev].store(sms, std::memory_order_relaxed);
  }
  const uint32_t grid = n < 2u * (uint32_t)sms ? n : 2u * (uint32_t)sms;
  gather_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(dst, src, bytes, n);
  return gk::cuda_check(cudaGetLastError(), "gk_gather: launch");
}
