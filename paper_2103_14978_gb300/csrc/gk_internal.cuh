// Internal declarations shared by the libgk translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "gk.h"

struct gk_ref_s {
  int device = -1;
  uint64_t n_bases = 0;
  uint64_t n_words = 0;       // ceil(n_bases / 32)
  uint64_t n_undefined = 0;   // non-ACGT bases
  uint2 *hl = nullptr;        // {high, low} plane per word, n_words + 2 (zero tail)
  uint2 *nidx = nullptr;      // {N bits of the word, first N position >= 32(w+1)}
};

namespace gk {

__host__ __device__ __forceinline__ uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t min_i64(int64_t a, int64_t b) { return a < b ? a : b; }

// Sets the calling thread's error message and returns `code`.
int fail(int code, const std::string &msg);
// Clears the calling thread's error message.
void clear_error();
// Maps a CUDA error to GK_ECUDA with context; GK_OK for cudaSuccess.
int cuda_check(cudaError_t err, const char *what);

// 2-bit code of one ASCII byte (A=00 C=01 G=10 T=11, Sec. 2.1), case folded.
// Sets *undefined for any byte that is not A/C/G/T; its code is 00.
__host__ __device__ __forceinline__ void code_of(uint32_t c, uint32_t &hi, uint32_t &lo,
                                                 uint32_t &undefined) {
  const uint32_t u = c & 0xDFu;  // fold a-z onto A-Z; only 'a' and 'A' map to 'A'
  const uint32_t is_a = u == 'A', is_c = u == 'C', is_g = u == 'G', is_t = u == 'T';
  hi = is_g | is_t;
  lo = is_c | is_t;
  undefined = !(is_a | is_c | is_g | is_t);
}

struct FilterArgs {
  const uint2 *ref_hl;
  const uint2 *ref_nidx;  // nullptr when the reference holds no N
  uint64_t ref_len;
  const uint2 *reads;
  uint32_t stride_words;
  uint64_t n_reads;
  const uint8_t *read_nflag;  // nullable
  uint32_t m;
  const uint32_t *pair_read;
  const uint32_t *pair_off;
  const uint8_t *pair_e;  // nullable
  uint32_t fixed_e;
  uint64_t n_pairs;
  int count_mode;
  int edge_on;
  uint8_t *accept;
  uint16_t *edits;
  uint32_t *err_count;  // nullable
  int compact;          // plain filter: persistent warps that filter only defined pairs
  int result_byte;      // accept receives one result byte per pair (GK_FLAG_RESULT_BYTE)
  // Threshold sweep (gk_filter_sweep): thresholds fixed_e .. sweep_hi, the
  // results of threshold e at accept / edits + (e - fixed_e) * out_stride;
  // sweep_hi < fixed_e: one threshold.
  uint32_t sweep_hi;
  uint64_t out_stride;
};

// Launches the plain filter for words-per-read W = ceil(m/32) (1..16).
cudaError_t launch_filter(int W, const FilterArgs &a, cudaStream_t stream);

// Device encoders (encode.cu).
cudaError_t launch_encode_reads(const uint8_t *ascii, uint64_t ascii_stride,
                                const uint16_t *lens, uint16_t fixed_len, uint64_t n_seq,
                                uint32_t *packed, uint32_t stride_words, uint8_t *nflag,
                                cudaStream_t stream);
cudaError_t launch_encode_contig(const uint8_t *ascii, uint64_t n_bases, uint2 *hl,
                                 uint32_t *nbits, cudaStream_t stream);
// Read ids of one batch's pairs from its reads' starts (serve_util.cu):
// pairs start[i] .. start[i+1]-1 (the last read's through n_pairs-1) get id
// i, clamped to [0, n_pairs); pairs no read claims get 0xFFFFFFFF.
cudaError_t launch_expand_rows(uint32_t *pair_read, uint64_t n_pairs, const uint32_t *read_start,
                               uint64_t n_reads, cudaStream_t stream);
// Host encoder (multi-threaded).
void host_encode_reads(const uint8_t *ascii, uint64_t ascii_stride, const uint16_t *lens,
                       uint16_t fixed_len, uint64_t n_seq, uint32_t *packed,
                       uint32_t stride_words, uint8_t *nflag);

}  // namespace gk
