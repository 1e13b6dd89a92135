// 2-bit encoding of reads and of the reference (Sec. 3.3), device and host.
//
// Output layout: per 32-base word a {high plane, low plane} pair of uint32,
// base 32w+b in bit b; the code is A=00 C=01 G=10 T=11 (Sec. 2.1).  Bytes
// that are not A/C/G/T in either case are coded 00 and reported, per read as
// a flag and per reference word as a bit mask (Sec. 3.3, Sec. 3.5).
#include <algorithm>
#include <thread>
#include <vector>

#include "encode_core.cuh"
#include "gk_internal.cuh"

namespace gk {
namespace {

constexpr int kMaxTileSeqs = 256;  // reads staged in shared memory per block, at most
constexpr int kTileBytes = 32768;  // staged bytes per block aimed at (the tile shrinks for long rows)
constexpr int kEncThreads = 256;
constexpr int kTileSlack = 64;   // bytes past the tile an unaligned word gather may touch

// One block encodes tile_seqs (<= kMaxTileSeqs) consecutive reads.  The
// tile's bytes are one contiguous span of the input, staged into shared
// memory with 16-byte loads where the span is aligned (about 32 KiB per
// block, so every thread has several loads in flight); each thread then
// builds whole words from shared memory and the block ORs the undefined
// bits per read.
__global__ void __launch_bounds__(kEncThreads)
encode_reads_kernel(const uint8_t *__restrict__ ascii, uint64_t stride, const uint16_t *__restrict__ lens,
                    uint32_t fixed_len, uint64_t n_seq, uint32_t *__restrict__ packed,
                    uint32_t stride_words, uint8_t *__restrict__ nflag, uint32_t tile_seqs) {
  extern __shared__ __align__(16) uint8_t tile[];  // tile_seqs * stride bytes
  __shared__ uint32_t undef[kMaxTileSeqs];
  const uint64_t seq0 = (uint64_t)blockIdx.x * tile_seqs;
  const int nseq = (int)min_u64(tile_seqs, n_seq - seq0);
  const uint8_t *src = ascii + seq0 * stride;
  for (int i = threadIdx.x; i < nseq; i += blockDim.x) undef[i] = 0;
  // Bytes needed: up to the end of the last read's length (a length is never
  // taken past the stride, so the tile holds at most tile_seqs * stride).
  const uint32_t last_len = lens ? lens[seq0 + nseq - 1] : fixed_len;
  const uint64_t need = (uint64_t)(nseq - 1) * stride + min_u64(last_len, stride);
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0);
  if (aligned) {
    const uint64_t n16 = need / 16;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *t4 = reinterpret_cast<uint4 *>(tile);
    for (uint64_t i = threadIdx.x; i < n16; i += blockDim.x) t4[i] = s4[i];
    for (uint64_t i = n16 * 16 + threadIdx.x; i < need; i += blockDim.x) tile[i] = src[i];
  } else {
    for (uint64_t i = threadIdx.x; i < need; i += blockDim.x) tile[i] = src[i];
  }
  __syncthreads();
  const uint32_t *t32 = reinterpret_cast<const uint32_t *>(tile);
  const bool rows4 = (stride & 3) == 0;  // every word starts on 4 bytes: no byte shift
  auto encode_word = [&](int s, int w) {
    const uint32_t len = (uint32_t)min_u64(lens ? lens[seq0 + s] : fixed_len, stride);
    const int64_t rem = (int64_t)len - 32 * (int64_t)w;
    uint32_t hi = 0, lo = 0, nb = 0;
    if (rem > 0) {
      // the word's 32 bytes from 8 (9 when unaligned) shared-memory words
      const uint64_t o = (uint64_t)s * stride + 32u * (uint64_t)w;
      const uint32_t *src = t32 + (o >> 2);
      uint32_t wb[8];
      if (rows4) {
#pragma unroll
        for (int j = 0; j < 8; ++j) wb[j] = src[j];
      } else {
        const uint32_t sh = (uint32_t)(o & 3) * 8u;
#pragma unroll
        for (int j = 0; j < 8; ++j) wb[j] = __funnelshift_r(src[j], src[j + 1], sh);
      }
      const uint32_t nv = rem >= 32 ? 32u : (uint32_t)rem;
      encode32_any(wb, nv, hi, lo, nb);
      if (nb) encode32(wb, nv, hi, lo, nb);  // a non-ACGT byte: exact per-base path
    }
    uint32_t *out = packed + ((seq0 + s) * (uint64_t)stride_words + w) * 2;
    *reinterpret_cast<uint2 *>(out) = make_uint2(hi, lo);
    if (nb) atomicOr(&undef[s], 1u);
  };
  const int sw = (int)stride_words;
  if ((int)blockDim.x % sw == 0) {  // each thread keeps one word index: no division per word
    const int w = (int)threadIdx.x % sw, step = (int)blockDim.x / sw;
    for (int s = (int)threadIdx.x / sw; s < nseq; s += step) encode_word(s, w);
  } else {
    for (int t = threadIdx.x; t < nseq * sw; t += blockDim.x) {
      const int s = t / sw;
      encode_word(s, t - s * sw);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nseq; i += blockDim.x) nflag[seq0 + i] = (uint8_t)(undef[i] != 0);
}

// Reads of one length in rows starting on 4 bytes, with a power-of-two row
// of G <= 32 words: one thread per output word (G lanes per read, the lanes
// of a read in one warp), its 32 bytes read straight from global memory in
// 4-byte loads (the lanes of a warp cover consecutive rows, so the loads
// coalesce), no shared-memory staging.  Words past ceil(len/32) are written
// as zeros; the read's N flag is the OR over its lanes by shuffles.  Bytes
// past a read's length are never read.
__global__ void __launch_bounds__(kEncThreads)
encode_reads_words_kernel(const uint8_t *__restrict__ ascii, uint64_t stride, uint32_t len, uint64_t n_seq,
                          uint32_t *__restrict__ packed, uint32_t lg, uint8_t *__restrict__ nflag) {
  const uint64_t t = blockIdx.x * (uint64_t)kEncThreads + threadIdx.x;
  const uint32_t G = 1u << lg;
  const uint64_t r = t >> lg;
  const uint32_t w = (uint32_t)t & (G - 1);
  const bool active = r < n_seq;
  uint32_t hi = 0, lo = 0, bad = 0;
  const int64_t rem = (int64_t)len - 32 * (int64_t)w;
  if (active && rem > 0) {
    const uint32_t nv = rem >= 32 ? 32u : (uint32_t)rem;
    const uint8_t *row = ascii + r * stride + 32u * w;
    // Whole 4-byte groups as predicated loads, issued together, "AAAA" (code
    // 00, valid) past the read; the one partial group (m not a multiple of
    // 4) byte by byte afterwards.  Every lane then runs encode32_full.
    uint32_t wb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      wb[j] = 4u * j + 4 <= nv ? __ldg(reinterpret_cast<const uint32_t *>(row) + j) : 0x41414141u;
    if (nv & 3u) {
      const uint32_t j = nv >> 2;
      uint32_t v = 0x41414141u;
      for (uint32_t i = 4 * j; i < nv; ++i) {
        const uint32_t sh = 8 * (i - 4 * j);
        v = (v & ~(0xFFu << sh)) | ((uint32_t)__ldg(row + i) << sh);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if ((uint32_t)q == j) wb[q] = v;
    }
    encode32_full(wb, hi, lo, bad);
    if (bad) encode32(wb, nv, hi, lo, bad);  // a non-ACGT byte: exact per-base path
  }
  if (active) reinterpret_cast<uint2 *>(packed)[t] = make_uint2(hi, lo);
  for (uint32_t d = 1; d < G; d <<= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, d);
  if (active && w == 0) nflag[r] = (uint8_t)(bad != 0);
}

// One thread per 32-base word of a contiguous sequence (the reference): two
// 16-byte loads when the word is complete, byte loads for the tail word.
__global__ void encode_contig_kernel(const uint8_t *__restrict__ ascii, uint64_t n_bases,
                                     uint2 *__restrict__ hl, uint32_t *__restrict__ nbits,
                                     uint64_t n_words) {
  const uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (w >= n_words) return;
  const uint64_t b0 = w * 32;
  uint32_t hi = 0, lo = 0, nb = 0;
  uint32_t wb[8];
  if (b0 + 32 <= n_bases && (reinterpret_cast<uintptr_t>(ascii) & 15u) == 0) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(ascii + b0);
    const uint4 v0 = s4[0], v1 = s4[1];
    wb[0] = v0.x; wb[1] = v0.y; wb[2] = v0.z; wb[3] = v0.w;
    wb[4] = v1.x; wb[5] = v1.y; wb[6] = v1.z; wb[7] = v1.w;
    encode32(wb, 32u, hi, lo, nb);
  } else {
    const int n = (int)min_u64(32, n_bases - b0);
#pragma unroll
    for (int j = 0; j < 8; ++j) wb[j] = 0;
    for (int b = 0; b < n; ++b) wb[b >> 2] |= (uint32_t)ascii[b0 + b] << (8 * (b & 3));
    encode32(wb, (uint32_t)n, hi, lo, nb);
  }
  hl[w] = make_uint2(hi, lo);
  nbits[w] = nb;
}

}  // namespace

cudaError_t launch_encode_reads(const uint8_t *ascii, uint64_t ascii_stride, const uint16_t *lens,
                                uint16_t fixed_len, uint64_t n_seq, uint32_t *packed,
                                uint32_t stride_words, uint8_t *nflag, cudaStream_t stream) {
  if (n_seq == 0) return cudaSuccess;
  // One length, rows on 4 bytes, a power-of-two row of at most 32 words:
  // one thread per word, straight from global memory (measured on GB300 for
  // 5M reads of 100 bp: about half the time of the staged kernel).
  const uint32_t sw = stride_words;
  const bool pow2 = sw >= 1 && sw <= 32 && (sw & (sw - 1)) == 0;
  if (!lens && pow2 && (ascii_stride & 3) == 0 && (reinterpret_cast<uintptr_t>(ascii) & 3) == 0 &&
      (uint64_t)fixed_len <= ascii_stride) {
    uint32_t lg = 0;
    while ((1u << lg) < sw) ++lg;
    const uint64_t threads = n_seq << lg;
    encode_reads_words_kernel<<<(unsigned)((threads + kEncThreads - 1) / kEncThreads), kEncThreads, 0, stream>>>(
        ascii, ascii_stride, fixed_len, n_seq, packed, lg, nflag);
    return cudaGetLastError();
  }
  // about kTileBytes per block, 16..kMaxTileSeqs reads (ascii_stride <= 3072
  // keeps the largest tile at 48 KiB)
  uint64_t tile_seqs = kTileBytes / ascii_stride;
  tile_seqs = tile_seqs < 16 ? 16 : (tile_seqs > kMaxTileSeqs ? kMaxTileSeqs : tile_seqs);
  const uint64_t blocks = (n_seq + tile_seqs - 1) / tile_seqs;
  const size_t smem = (size_t)tile_seqs * ascii_stride + kTileSlack;
  if (smem > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(encode_reads_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  encode_reads_kernel<<<(unsigned)blocks, kEncThreads, smem, stream>>>(
      ascii, ascii_stride, lens, fixed_len, n_seq, packed, stride_words, nflag, (uint32_t)tile_seqs);
  return cudaGetLastError();
}

cudaError_t launch_encode_contig(const uint8_t *ascii, uint64_t n_bases, uint2 *hl, uint32_t *nbits,
                                 cudaStream_t stream) {
  const uint64_t n_words = (n_bases + 31) / 32;
  if (n_words == 0) return cudaSuccess;
  const int threads = 256;
  encode_contig_kernel<<<(unsigned)((n_words + threads - 1) / threads), threads, 0, stream>>>(
      ascii, n_bases, hl, nbits, n_words);
  return cudaGetLastError();
}

void host_encode_reads(const uint8_t *ascii, uint64_t ascii_stride, const uint16_t *lens,
                       uint16_t fixed_len, uint64_t n_seq, uint32_t *packed, uint32_t stride_words,
                       uint8_t *nflag) {
  auto work = [&](uint64_t lo_seq, uint64_t hi_seq) {
    for (uint64_t s = lo_seq; s < hi_seq; ++s) {
      const uint32_t len = (uint32_t)std::min<uint64_t>(lens ? lens[s] : fixed_len, ascii_stride);
      const uint8_t *p = ascii + s * ascii_stride;
      uint32_t any = 0;
      for (uint32_t w = 0; w < stride_words; ++w) {
        uint32_t hi = 0, lo = 0;
        for (uint32_t b = 0; b < 32 && w * 32 + b < len; ++b) {
          uint32_t h, l, u;
          code_of(p[w * 32 + b], h, l, u);
          hi |= h << b;
          lo |= l << b;
          any |= u;
        }
        uint32_t *out = packed + (s * stride_words + w) * 2;
        out[0] = hi;
        out[1] = lo;
      }
      nflag[s] = (uint8_t)(any != 0);
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const uint64_t nthreads = std::min<uint64_t>(hw, std::max<uint64_t>(1, n_seq / 4096));
  if (nthreads <= 1) {
    work(0, n_seq);
    return;
  }
  std::vector<std::thread> pool;
  const uint64_t chunk = (n_seq + nthreads - 1) / nthreads;
  for (uint64_t t = 0; t < nthreads; ++t) {
    const uint64_t a = std::min(n_seq, t * chunk), b = std::min(n_seq, a + chunk);
    pool.emplace_back(work, a, b);
  }
  for (auto &th : pool) th.join();
}

}  // namespace gk
