// C ABI of libgk: argument checks, error reporting, the resident reference
// and the launch of the filter kernels.  Declarations and contracts are in
// include/gk.h.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batched.cuh"
#include "filter_ascii.cuh"
#include "gk_internal.cuh"

namespace gk {

cudaError_t launch_filter_w1_4(int W, int variant, const FilterArgs &a, cudaStream_t stream);
cudaError_t launch_filter_w5_8(int W, int variant, const FilterArgs &a, cudaStream_t stream);
cudaError_t launch_filter_w9_12(int W, int variant, const FilterArgs &a, cudaStream_t stream);
cudaError_t launch_filter_w13_16(int W, int variant, const FilterArgs &a, cudaStream_t stream);
cudaError_t launch_filter_ascii_w1_8(int W, int variant, const AsciiArgs &g, cudaStream_t stream);
cudaError_t launch_filter_ascii_w9_16(int W, int variant, const AsciiArgs &g, cudaStream_t stream);

namespace {
thread_local std::string t_last_error;
}

int fail(int code, const std::string &msg) {
  t_last_error = msg;
  return code;
}

void clear_error() { t_last_error.clear(); }

int cuda_check(cudaError_t err, const char *what) {
  if (err == cudaSuccess) return GK_OK;
  return fail(GK_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

// Variant of the per-pair code for a launch: 2 deferred erosion, 1 exact
// with every shift below 32, 0 exact for any thresholds.
int filter_variant(const FilterArgs &a, bool pair_k) {
  if (a.out_stride != 0) return 3;  // a threshold sweep (gk_filter_sweep)
  // One threshold 0..2 below m, reads of at most 128 bases, no compaction:
  // the two-pairs-per-thread deferred kernel with the shift count fixed at
  // compile time (measured on GB300 at 100 bp against the exact one-pair
  // kernel at e = 0, 1 and the runtime-K form at e = 2).
  if (pair_k && a.edge_on && !a.pair_e && a.fixed_e <= 2 && a.m > a.fixed_e && a.m <= 128 && !a.compact) return 4;
  // Every shift count below 32 (one threshold under 32, or reads of at most
  // 32 bases): the edge vectors live in the end words only.
  const bool small = (!a.pair_e && a.fixed_e < 32) || a.m <= 32;
  // Deferred erosion: every shift count <= 30, edge OR on, and enough shifts
  // (e >= 2) to repay its once-per-pair corrections (measured on GB300: from
  // e = 2 it is as fast or faster at 100-300 bp).
  const bool deferred = a.edge_on && !a.pair_e && a.fixed_e >= 2 && (a.fixed_e <= 30 || a.m <= 31);
  return deferred ? 2 : (small ? 1 : 0);
}

cudaError_t launch_filter(int W, const FilterArgs &a, cudaStream_t stream) {
  const int variant = filter_variant(a, true);
  if (W >= 1 && W <= 4) return launch_filter_w1_4(W, variant, a, stream);
  if (W <= 8) return launch_filter_w5_8(W, variant, a, stream);
  if (W <= 12) return launch_filter_w9_12(W, variant, a, stream);
  if (W <= 16) return launch_filter_w13_16(W, variant, a, stream);
  return cudaErrorInvalidValue;
}

}  // namespace gk

using gk::fail;

namespace {

constexpr uint64_t kMaxRefBases = (1ull << 32) - (1ull << 16);
constexpr uint64_t kMaxPairs = (1ull << 31) * 128ull;  // grid x limit at 256 threads
constexpr uint64_t kMaxDeviceAsciiStride = 3072;      // encoder tile: >= 16 rows in 48 KiB of shared memory

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

struct DeviceBuffer {
  void *p = nullptr;
  ~DeviceBuffer() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" {

const char *gk_last_error(void) { return gk::t_last_error.c_str(); }

int gk_version(void) { return 100; }  // 0.1.0

int gk_encode(const uint8_t *ascii, uint64_t ascii_stride, const uint16_t *lens,
              uint16_t fixed_len, uint64_t n_seq, uint32_t *packed, uint32_t stride_words,
              uint8_t *nflag, int on_device, void *stream) {
  gk::clear_error();
  if (n_seq == 0) return GK_OK;
  if (!ascii || !packed || !nflag) return fail(GK_EINVAL, "gk_encode: null buffer");
  if (!lens && fixed_len > GK_MAX_LEN)
    return fail(GK_ERANGE, "gk_encode: fixed_len above GK_MAX_LEN");
  if (!lens && fixed_len > ascii_stride)
    return fail(GK_EINVAL, "gk_encode: fixed_len larger than ascii_stride");
  if (stride_words == 0 || stride_words > GK_MAX_LEN / 32)
    return fail(GK_EINVAL, "gk_encode: stride_words must be 1..GK_MAX_LEN/32");
  if (!lens && (uint32_t)fixed_len > 32u * stride_words)
    return fail(GK_EINVAL, "gk_encode: stride_words too small for fixed_len");
  if (ascii_stride == 0) return fail(GK_EINVAL, "gk_encode: ascii_stride is 0");
  if (!aligned(packed, 8)) return fail(GK_EINVAL, "gk_encode: packed must be 8-byte aligned");
  if (on_device) {
    if (ascii_stride > kMaxDeviceAsciiStride)
      return fail(GK_ERANGE, "gk_encode: device path needs ascii_stride <= 3072");
    cudaError_t err = gk::launch_encode_reads(ascii, ascii_stride, lens, fixed_len, n_seq, packed,
                                              stride_words, nflag, (cudaStream_t)stream);
    return gk::cuda_check(err, "gk_encode: launch");
  }
  gk::host_encode_reads(ascii, ascii_stride, lens, fixed_len, n_seq, packed, stride_words, nflag);
  return GK_OK;
}

int gk_load_reference(const uint8_t *ascii, uint64_t n_bases, int on_device, void *stream,
                      gk_ref_t *out) {
  gk::clear_error();
  if (!ascii || !out) return fail(GK_EINVAL, "gk_load_reference: null pointer");
  *out = nullptr;
  if (n_bases == 0 || n_bases >= kMaxRefBases)
    return fail(GK_EINVAL, "gk_load_reference: n_bases must be in 1..2^32-2^16");
  cudaStream_t s = (cudaStream_t)stream;
  gk_ref_s *ref = new (std::nothrow) gk_ref_s();
  if (!ref) return fail(GK_ENOMEM, "gk_load_reference: host allocation");
  int rc = GK_OK;
  const uint64_t n_words = (n_bases + 31) / 32;
  ref->n_bases = n_bases;
  ref->n_words = n_words;
  cudaGetDevice(&ref->device);
  DeviceBuffer staging, nbits_dev;
  std::vector<uint32_t> nbits;
  std::vector<uint2> nidx;
  const uint8_t *dev_ascii = ascii;
  do {
    if (cudaMalloc(&ref->hl, (n_words + 2) * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc(&nbits_dev.p, (n_words + 2) * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(GK_ENOMEM, "gk_load_reference: device allocation");
      break;
    }
    if (!on_device) {
      if (cudaMalloc(&staging.p, n_bases) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(GK_ENOMEM, "gk_load_reference: device staging allocation");
        break;
      }
      rc = gk::cuda_check(cudaMemcpyAsync(staging.p, ascii, n_bases, cudaMemcpyHostToDevice, s),
                          "gk_load_reference: copy to device");
      if (rc) break;
      dev_ascii = static_cast<const uint8_t *>(staging.p);
    }
    rc = gk::cuda_check(cudaMemsetAsync(ref->hl, 0, (n_words + 2) * sizeof(uint2), s),
                        "gk_load_reference: memset");
    if (rc) break;
    rc = gk::cuda_check(gk::launch_encode_contig(dev_ascii, n_bases, ref->hl,
                                                 static_cast<uint32_t *>(nbits_dev.p), s),
                        "gk_load_reference: encode");
    if (rc) break;
    // The N index: per word its N bits and the first N position at or after
    // the next word, so that one load answers "any N in [off, off+m)".
    nbits.resize(n_words);
    rc = gk::cuda_check(cudaMemcpyAsync(nbits.data(), nbits_dev.p, n_words * sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, s),
                        "gk_load_reference: copy N bits");
    if (rc) break;
    rc = gk::cuda_check(cudaStreamSynchronize(s), "gk_load_reference: synchronize");
    if (rc) break;
    uint64_t n_undef = 0;
    for (uint64_t w = 0; w < n_words; ++w) n_undef += (uint64_t)__builtin_popcount(nbits[w]);
    ref->n_undefined = n_undef;
    if (n_undef > 0) {
      nidx.resize(n_words + 2);
      uint32_t next = 0xffffffffu;  // first N position >= 32*(w+1)
      nidx[n_words] = make_uint2(0, next);
      nidx[n_words + 1] = make_uint2(0, next);
      for (uint64_t w = n_words; w-- > 0;) {
        nidx[w] = make_uint2(nbits[w], next);
        if (nbits[w]) next = (uint32_t)(32 * w + (uint64_t)__builtin_ctz(nbits[w]));
      }
      if (cudaMalloc(&ref->nidx, (n_words + 2) * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(GK_ENOMEM, "gk_load_reference: N index allocation");
        break;
      }
      rc = gk::cuda_check(cudaMemcpyAsync(ref->nidx, nidx.data(), (n_words + 2) * sizeof(uint2),
                                          cudaMemcpyHostToDevice, s),
                          "gk_load_reference: copy N index");
      if (rc) break;
    }
    rc = gk::cuda_check(cudaStreamSynchronize(s), "gk_load_reference: synchronize");
  } while (false);
  if (rc != GK_OK) {
    gk_free_reference(ref);
    return rc;
  }
  *out = ref;
  return GK_OK;
}

void gk_free_reference(gk_ref_t ref) {
  if (!ref) return;
  if (ref->hl) cudaFree(ref->hl);
  if (ref->nidx) cudaFree(ref->nidx);
  delete ref;
}

int gk_reference_info(gk_ref_t ref, uint64_t *n_bases, uint64_t *n_undefined) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_reference_info: null handle");
  if (n_bases) *n_bases = ref->n_bases;
  if (n_undefined) *n_undefined = ref->n_undefined;
  return GK_OK;
}

int gk_filter(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words, uint64_t n_reads,
              const uint8_t *read_nflag, uint32_t m, const uint32_t *pair_read,
              const uint32_t *pair_off, const uint8_t *pair_e, uint32_t fixed_e,
              uint64_t n_pairs, int count_mode, uint32_t flags, uint8_t *accept_out,
              uint16_t *edits_out, uint32_t *err_count, void *stream) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_filter: null reference handle");
  if (m > GK_MAX_LEN) return fail(GK_ERANGE, "gk_filter: m above GK_MAX_LEN");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > kMaxPairs) return fail(GK_ERANGE, "gk_filter: too many pairs for one launch");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (!pair_read || !pair_off || !accept_out || (!edits_out && !result_byte))
    return fail(GK_EINVAL, "gk_filter: null pair or output buffer");
  if (result_byte && pair_e)
    return fail(GK_EINVAL, "gk_filter: GK_FLAG_RESULT_BYTE needs one threshold (pair_e NULL)");
  if (result_byte && fixed_e > 252)
    return fail(GK_ERANGE, "gk_filter: GK_FLAG_RESULT_BYTE needs fixed_e <= 252");
  const uint32_t W = m == 0 ? 1 : (m + 31) / 32;
  if (m > 0 && (!reads || stride_words < W))
    return fail(GK_EINVAL, "gk_filter: reads missing or stride_words < ceil(m/32)");
  if (!pair_e && fixed_e > 255) return fail(GK_ERANGE, "gk_filter: fixed_e above 255");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter: unknown count_mode");
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE)) return fail(GK_EINVAL, "gk_filter: unknown flags");
  if (reads && !aligned(reads, 8)) return fail(GK_EINVAL, "gk_filter: reads must be 8-byte aligned");
  gk::FilterArgs a{};
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
  a.pair_e = pair_e;
  a.fixed_e = fixed_e;
  a.n_pairs = n_pairs;
  a.count_mode = count_mode;
  a.edge_on = (flags & GK_FLAG_NO_EDGE_FIX) ? 0 : 1;
  a.result_byte = result_byte ? 1 : 0;
  a.accept = accept_out;
  a.edits = edits_out;
  a.err_count = err_count;
  // A genome with N makes a share of windows undefined (about 1 - (1-r)^m
  // for an N density r): filter only the defined pairs, in full warps, when
  // that share (r*m >= 0.05) and the per-pair work repay the queueing.  The
  // thresholds are GB300 measurements on 10M pairs at 0.1% N in genome and
  // reads: the queue wins from e >= 1 at W >= 7 (200-300 bp), from e >= 3 at
  // W = 5 (150 bp) and from e >= 7 at W = 4 (100 bp); below them one thread
  // per pair is faster, its loads issued together.  Per-pair thresholds
  // always queue.
  const uint32_t e_queue = W >= 7 ? 1u : (W >= 5 ? 3u : 7u);
  const bool n_dense = (double)ref->n_undefined * (double)m >= 0.05 * (double)ref->n_bases;
  a.compact = (ref->n_undefined > 0 && n_pairs < (1ull << 32) && m > 0 &&
               (pair_e || (n_dense && fixed_e >= e_queue))) ? 1 : 0;
  return gk::cuda_check(gk::launch_filter((int)W, a, (cudaStream_t)stream), "gk_filter: launch");
}

int gk_filter_sweep(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words, uint64_t n_reads,
                    const uint8_t *read_nflag, uint32_t m, const uint32_t *pair_read, const uint32_t *pair_off,
                    uint32_t e_lo, uint32_t e_hi, uint64_t n_pairs, int count_mode, uint32_t flags,
                    uint8_t *accept_out, uint16_t *edits_out, uint64_t out_stride, uint32_t *err_count,
                    void *stream) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_filter_sweep: null reference handle");
  if (m > GK_MAX_LEN) return fail(GK_ERANGE, "gk_filter_sweep: m above GK_MAX_LEN");
  if (e_lo > e_hi) return fail(GK_EINVAL, "gk_filter_sweep: e_lo > e_hi");
  if (e_hi > 255) return fail(GK_ERANGE, "gk_filter_sweep: e_hi above 255");
  if (m > 0 && (e_hi < m - 1 ? e_hi : m - 1) > GK_SWEEP_MAX_SHIFT)
    return fail(GK_ERANGE, "gk_filter_sweep: min(e_hi, m-1) above GK_SWEEP_MAX_SHIFT");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > kMaxPairs) return fail(GK_ERANGE, "gk_filter_sweep: too many pairs for one launch");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE)) return fail(GK_EINVAL, "gk_filter_sweep: unknown flags");
  if (flags & GK_FLAG_NO_EDGE_FIX)
    return fail(GK_EINVAL, "gk_filter_sweep: computes the Sec. 3.4 edge OR only (use gk_filter without it)");
  if (result_byte && e_hi > 252) return fail(GK_ERANGE, "gk_filter_sweep: GK_FLAG_RESULT_BYTE needs e_hi <= 252");
  if (!pair_read || !pair_off || !accept_out || (!edits_out && !result_byte))
    return fail(GK_EINVAL, "gk_filter_sweep: null pair or output buffer");
  if (out_stride < n_pairs) return fail(GK_EINVAL, "gk_filter_sweep: out_stride < n_pairs");
  const uint32_t W = m == 0 ? 1 : (m + 31) / 32;
  if (m > 0 && (!reads || stride_words < W))
    return fail(GK_EINVAL, "gk_filter_sweep: reads missing or stride_words < ceil(m/32)");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter_sweep: unknown count_mode");
  if (reads && !aligned(reads, 8)) return fail(GK_EINVAL, "gk_filter_sweep: reads must be 8-byte aligned");
  gk::FilterArgs a{};
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
  a.fixed_e = e_lo;
  a.sweep_hi = e_hi;
  a.out_stride = out_stride;
  a.n_pairs = n_pairs;
  a.count_mode = count_mode;
  a.edge_on = 1;
  a.result_byte = result_byte ? 1 : 0;
  a.accept = accept_out;
  a.edits = edits_out;
  a.err_count = err_count;
  // As gk_filter: with a genome dense in N, persistent warps filter only
  // the defined pairs (a sweep is work enough to repay the queueing).
  const bool n_dense = (double)ref->n_undefined * (double)m >= 0.05 * (double)ref->n_bases;
  a.compact = (ref->n_undefined > 0 && n_pairs < (1ull << 32) && m > 0 && n_dense) ? 1 : 0;
  return gk::cuda_check(gk::launch_filter((int)W, a, (cudaStream_t)stream), "gk_filter_sweep: launch");
}

int gk_filter_ascii(gk_ref_t ref, const uint8_t *ascii, uint64_t ascii_stride, uint64_t n_reads, uint32_t m,
                    const uint32_t *pair_read, const uint32_t *pair_off, const uint8_t *pair_e, uint32_t fixed_e,
                    uint64_t n_pairs, int count_mode, uint32_t flags, uint8_t *accept_out, uint16_t *edits_out,
                    uint32_t *err_count, void *stream) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_filter_ascii: null reference handle");
  if (m > GK_MAX_LEN) return fail(GK_ERANGE, "gk_filter_ascii: m above GK_MAX_LEN");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > kMaxPairs) return fail(GK_ERANGE, "gk_filter_ascii: too many pairs for one launch");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (!pair_read || !pair_off || !accept_out || (!edits_out && !result_byte))
    return fail(GK_EINVAL, "gk_filter_ascii: null pair or output buffer");
  if (m > 0 && (!ascii || ascii_stride < m))
    return fail(GK_EINVAL, "gk_filter_ascii: ascii missing or ascii_stride < m");
  if (!pair_e && fixed_e > 255) return fail(GK_ERANGE, "gk_filter_ascii: fixed_e above 255");
  if (result_byte && pair_e)
    return fail(GK_EINVAL, "gk_filter_ascii: GK_FLAG_RESULT_BYTE needs one threshold (pair_e NULL)");
  if (result_byte && fixed_e > 252)
    return fail(GK_ERANGE, "gk_filter_ascii: GK_FLAG_RESULT_BYTE needs fixed_e <= 252");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter_ascii: unknown count_mode");
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE))
    return fail(GK_EINVAL, "gk_filter_ascii: unknown flags");
  gk::AsciiArgs g{};
  gk::FilterArgs &a = g.f;
  a.ref_hl = ref->hl;
  a.ref_nidx = ref->nidx;
  a.ref_len = ref->n_bases;
  a.n_reads = n_reads;
  a.m = m;
  a.pair_read = pair_read;
  a.pair_off = pair_off;
  a.pair_e = pair_e;
  a.fixed_e = fixed_e;
  a.n_pairs = n_pairs;
  a.count_mode = count_mode;
  a.edge_on = (flags & GK_FLAG_NO_EDGE_FIX) ? 0 : 1;
  a.result_byte = result_byte ? 1 : 0;
  a.accept = accept_out;
  a.edits = edits_out;
  a.err_count = err_count;
  g.ascii = ascii;
  g.ascii_stride = ascii_stride;
  g.rows_aligned = (aligned(ascii, 4) && ascii_stride % 4 == 0) ? 1 : 0;
  const int W = m == 0 ? 1 : (int)((m + 31) / 32);
  const int variant = gk::filter_variant(a, false);
  const cudaError_t err = W <= 8 ? gk::launch_filter_ascii_w1_8(W, variant, g, (cudaStream_t)stream)
                                 : gk::launch_filter_ascii_w9_16(W, variant, g, (cudaStream_t)stream);
  return gk::cuda_check(err, "gk_filter_ascii: launch");
}

uint64_t gk_filter_batched_workspace(uint64_t n_pairs) { return gk::batch_scratch_bytes(n_pairs); }

int gk_filter_batched(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words, uint64_t n_reads,
                      const uint16_t *read_len, const uint8_t *read_nflag, const uint32_t *pair_read,
                      const uint32_t *pair_off, const uint8_t *pair_e, uint32_t fixed_e, uint64_t n_pairs,
                      int count_mode, uint32_t flags, const gk_tiling_t *tiling, void *workspace,
                      uint64_t workspace_bytes, uint8_t *accept_out, uint16_t *edits_out,
                      uint32_t *err_count, void *stream) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_filter_batched: null reference handle");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs >= (1ull << 32)) return fail(GK_ERANGE, "gk_filter_batched: n_pairs must be < 2^32");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (!reads || !read_len || !pair_read || !pair_off || !accept_out || (!edits_out && !result_byte) || !tiling)
    return fail(GK_EINVAL, "gk_filter_batched: null buffer");
  if (stride_words == 0 || stride_words > GK_MAX_LEN / 32)
    return fail(GK_EINVAL, "gk_filter_batched: stride_words must be 1..GK_MAX_LEN/32");
  if (!aligned(reads, 8)) return fail(GK_EINVAL, "gk_filter_batched: reads must be 8-byte aligned");
  if (!pair_e && fixed_e > 255) return fail(GK_ERANGE, "gk_filter_batched: fixed_e above 255");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter_batched: unknown count_mode");
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE)) return fail(GK_EINVAL, "gk_filter_batched: unknown flags");
  const gk_tiling_t t = *tiling;
  if (!(t.words_per_thread == 1 || t.words_per_thread == 2 || t.words_per_thread == 3 ||
        t.words_per_thread == 4 || t.words_per_thread == 6 || t.words_per_thread == 8))
    return fail(GK_EINVAL, "gk_filter_batched: words_per_thread must be 1, 2, 3, 4, 6 or 8");
  if (t.tile_pairs < 32 || t.tile_pairs > 65536 || t.blocks_per_sm < 1 || t.blocks_per_sm > 32 ||
      t.warps_per_block < 1 || t.warps_per_block > 8)
    return fail(GK_EINVAL, "gk_filter_batched: tiling out of range");
  if (!workspace || !aligned(workspace, 256) || workspace_bytes < gk::batch_scratch_bytes(n_pairs))
    return fail(GK_EINVAL, "gk_filter_batched: workspace missing, unaligned or too small");
  gk::BatchArgs a{};
  a.f.ref_hl = ref->hl;
  a.f.ref_nidx = ref->nidx;
  a.f.ref_len = ref->n_bases;
  a.f.reads = reinterpret_cast<const uint2 *>(reads);
  a.f.stride_words = stride_words;
  a.f.n_reads = n_reads;
  a.f.read_nflag = read_nflag;
  a.f.m = 0;
  a.f.pair_read = pair_read;
  a.f.pair_off = pair_off;
  a.f.pair_e = pair_e;
  a.f.fixed_e = fixed_e;
  a.f.n_pairs = n_pairs;
  a.f.count_mode = count_mode;
  a.f.edge_on = (flags & GK_FLAG_NO_EDGE_FIX) ? 0 : 1;
  a.f.accept = accept_out;
  a.f.edits = edits_out;
  a.f.result_byte = result_byte ? 1 : 0;
  a.f.err_count = err_count;
  a.read_len = read_len;
  a.tile_pairs = t.tile_pairs;
  a.s = gk::batch_scratch_layout(workspace, n_pairs);
  return gk::cuda_check(gk::launch_batched((int)t.words_per_thread, a, t.blocks_per_sm, t.warps_per_block,
                                           (cudaStream_t)stream),
                        "gk_filter_batched: launch");
}

}  // extern "C"
