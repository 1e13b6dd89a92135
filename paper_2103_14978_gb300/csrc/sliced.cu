// Bit-sliced filter: the slice kernel, the dispatch over the compiled shift
// counts and the C ABI (gk_sliced_bytes, gk_slice, gk_filter_sliced).  The
// per-group code and the buffer layout are in sliced.cuh.
#include "sliced.cuh"

namespace gk {
namespace {

// One thread per group of 32 pairs.  The block's 4096 pair ids are read
// coalesced into shared memory (rows of 33 words: conflict-free per-thread
// reads), then every thread gathers and transposes its group.
__global__ void __launch_bounds__(kSliceThreads) slice_kernel(const SliceArgs a, uint32_t *err_count) {
  __shared__ uint32_t s_rid[kSliceThreads * 33], s_off[kSliceThreads * 33];
  const uint64_t g0 = (uint64_t)blockIdx.x * kSliceThreads;
  for (int i = threadIdx.x; i < 32 * kSliceThreads; i += kSliceThreads) {
    const uint64_t p = g0 * 32 + (uint64_t)i;
    uint32_t rid = 0xffffffffu, off = 0xffffffffu;
    if (p < a.n_pairs) {
      rid = __ldg(a.pair_read + p);
      off = __ldg(a.pair_off + p);
    }
    s_rid[(i >> 5) * 33 + (i & 31)] = rid;
    s_off[(i >> 5) * 33 + (i & 31)] = off;
  }
  __syncthreads();
  const uint64_t g = g0 + threadIdx.x;
  if (g >= sliced_groups(a.n_pairs)) return;
  const uint64_t left = a.n_pairs - g * 32;
  const uint32_t n_here = left < 32 ? (uint32_t)left : 32u;
  const uint32_t n_inv = slice_group(a, g, s_rid + threadIdx.x * 33, s_off + threadIdx.x * 33, 1, n_here);
  if (n_inv && err_count) atomicAdd(err_count, n_inv);
}

}  // namespace

cudaError_t launch_slice(const SliceArgs &a, uint32_t *err_count, cudaStream_t stream) {
  const uint64_t groups = sliced_groups(a.n_pairs);
  const unsigned blocks = (unsigned)((groups + kSliceThreads - 1) / kSliceThreads);
  slice_kernel<<<blocks, kSliceThreads, 0, stream>>>(a, err_count);
  return cudaGetLastError();
}

// The read lengths of the paper's data sets (100, 150, 250 bp, Sec. 4) have
// kernels with the length compiled in; any other length takes the general
// ones.
cudaError_t launch_sliced_filter(int K, const SlicedArgs &a, cudaStream_t stream) {
  if (K < 0 || K > kSlicedMaxK) return cudaErrorInvalidValue;
  const bool lo = K <= 5;
  switch (a.m) {
    case 100: return lo ? launch_sliced_m100_k0_5(K, a, stream) : launch_sliced_m100_k6_10(K, a, stream);
    case 150: return lo ? launch_sliced_m150_k0_5(K, a, stream) : launch_sliced_m150_k6_10(K, a, stream);
    case 250: return lo ? launch_sliced_m250_k0_5(K, a, stream) : launch_sliced_m250_k6_10(K, a, stream);
    default: return lo ? launch_sliced_m0_k0_5(K, a, stream) : launch_sliced_m0_k6_10(K, a, stream);
  }
}

}  // namespace gk

using gk::fail;

namespace {
bool aligned_to(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
}  // namespace

extern "C" {

uint64_t gk_sliced_bytes(uint64_t n_pairs, uint32_t m) {
  if (n_pairs == 0 || m == 0 || m > gk::kSlicedMaxLen) return 0;
  return gk::sliced_bytes(n_pairs, m);
}

int gk_slice(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words, uint64_t n_reads,
             const uint8_t *read_nflag, uint32_t m, const uint32_t *pair_read, const uint32_t *pair_off,
             uint64_t n_pairs, void *sliced, uint64_t sliced_cap, uint32_t *err_count, void *stream) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_slice: null reference handle");
  if (m == 0 || m > gk::kSlicedMaxLen) return fail(GK_ERANGE, "gk_slice: m outside 1..255");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > (1ull << 40)) return fail(GK_ERANGE, "gk_slice: too many pairs");
  if (!reads || !pair_read || !pair_off || !sliced) return fail(GK_EINVAL, "gk_slice: null buffer");
  const uint32_t W = (m + 31) / 32;
  if (stride_words < W) return fail(GK_EINVAL, "gk_slice: stride_words < ceil(m/32)");
  if (!aligned_to(reads, 8)) return fail(GK_EINVAL, "gk_slice: reads must be 8-byte aligned");
  if (!aligned_to(sliced, 16)) return fail(GK_EINVAL, "gk_slice: sliced buffer must be 16-byte aligned");
  if (sliced_cap < gk::sliced_bytes(n_pairs, m)) return fail(GK_EINVAL, "gk_slice: sliced buffer too small");
  gk::SliceArgs a{};
  a.ref_hl = ref->hl;
  a.ref_nidx = ref->nidx;
  a.ref_len = ref->n_bases;
  a.reads = reinterpret_cast<const uint2 *>(reads);
  a.stride_words = stride_words;
  a.n_reads = n_reads;
  a.read_nflag = read_nflag;
  a.m = m;
  a.pair_read = pair_read;
  a.pair_off = pair_off;
  a.n_pairs = n_pairs;
  a.pitch = gk::sliced_pitch(n_pairs);
  a.rs = reinterpret_cast<uint2 *>(sliced);
  a.gs = a.rs + (uint64_t)m * a.pitch;
  a.st = a.gs + (uint64_t)m * a.pitch;
  return gk::cuda_check(gk::launch_slice(a, err_count, (cudaStream_t)stream), "gk_slice: launch");
}

int gk_filter_sliced(const void *sliced, uint64_t sliced_cap, uint64_t n_pairs, uint32_t m, uint32_t fixed_e,
                     int count_mode, uint32_t flags, uint8_t *accept_out, uint16_t *edits_out, void *stream) {
  gk::clear_error();
  if (m == 0 || m > gk::kSlicedMaxLen) return fail(GK_ERANGE, "gk_filter_sliced: m outside 1..255");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > (1ull << 40)) return fail(GK_ERANGE, "gk_filter_sliced: too many pairs");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE)) return fail(GK_EINVAL, "gk_filter_sliced: unknown flags");
  if (flags & GK_FLAG_NO_EDGE_FIX)
    return fail(GK_EINVAL, "gk_filter_sliced: computes the Sec. 3.4 edge OR only (use gk_filter without it)");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter_sliced: unknown count_mode");
  if (fixed_e > 255) return fail(GK_ERANGE, "gk_filter_sliced: fixed_e above 255");
  if (result_byte && fixed_e > 252) return fail(GK_ERANGE, "gk_filter_sliced: GK_FLAG_RESULT_BYTE needs fixed_e <= 252");
  const uint32_t K = fixed_e < m - 1 ? fixed_e : m - 1;
  if (K > (uint32_t)gk::kSlicedMaxK)
    return fail(GK_ERANGE, "gk_filter_sliced: min(e, m-1) above the compiled shift counts (10)");
  if (!sliced || !accept_out || (!edits_out && !result_byte)) return fail(GK_EINVAL, "gk_filter_sliced: null buffer");
  if (!aligned_to(sliced, 16)) return fail(GK_EINVAL, "gk_filter_sliced: sliced buffer must be 16-byte aligned");
  if (sliced_cap < gk::sliced_bytes(n_pairs, m)) return fail(GK_EINVAL, "gk_filter_sliced: sliced buffer too small");
  gk::SlicedArgs a{};
  a.pitch = gk::sliced_pitch(n_pairs);
  a.rs = reinterpret_cast<const uint2 *>(sliced);
  a.gs = a.rs + (uint64_t)m * a.pitch;
  a.st = a.gs + (uint64_t)m * a.pitch;
  a.n_pairs = n_pairs;
  a.m = m;
  a.e = fixed_e;
  a.runs4 = count_mode == GK_COUNT_RUNS4 ? 1u : 0u;
  a.result_byte = result_byte ? 1 : 0;
  a.vec_out = aligned_to(accept_out, 16) && (result_byte || aligned_to(edits_out, 16)) ? 1 : 0;
  a.accept = accept_out;
  a.edits = result_byte ? nullptr : edits_out;
  return gk::cuda_check(gk::launch_sliced_filter((int)K, a, (cudaStream_t)stream), "gk_filter_sliced: launch");
}

}  // extern "C"
