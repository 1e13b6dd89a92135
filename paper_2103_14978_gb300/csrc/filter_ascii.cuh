// Fused device encode + filter (the paper's device-encoded mode, Sec. 3.3):
// the reads arrive as ASCII rows and are 2-bit encoded inside the filter
// kernel, so no packed copy of them is written or read back.
//
// One thread per pair, as the plain filter.  The 32 pairs of a warp usually
// hold a few reads, each with several candidates side by side; the warp finds
// its distinct reads (runs of one read id among its valid pairs) and encodes
// each once, cooperatively: the (read, word) jobs are spread over the lanes,
// every job turns 32 ASCII bytes into one {high, low} word with the read
// encoder's word encoder, and the words land in shared memory, where each
// lane then picks up its read.  From there the pair is filtered exactly as
// by gk_filter (Sec. 2.1, 3.4).
#pragma once

#include "encode_core.cuh"
#include "filter.cuh"

namespace gk {

struct AsciiArgs {
  FilterArgs f;           // f.reads, f.stride_words and f.read_nflag are unused
  const uint8_t *ascii;   // read i at ascii + i * ascii_stride, m bytes used
  uint64_t ascii_stride;
  int rows_aligned;       // every row starts on 4 bytes: 4-byte loads
};

// Bytes [32w, 32w + nv) of an ASCII row as 8 little-endian words (zero past
// nv); reads no byte past row + 32w + nv.
__device__ __forceinline__ void load_word_bytes(const uint8_t *row, uint32_t w, uint32_t nv, bool aligned,
                                                uint32_t (&wb)[8]) {
  const uint8_t *b = row + 32u * w;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t lo = 4u * k;
    uint32_t v = 0x41414141u;
    if (aligned && lo + 4 <= nv) {
      v = *reinterpret_cast<const uint32_t *>(b + lo);
    } else {
      for (uint32_t i = lo; i < lo + 4 && i < nv; ++i) {
        const uint32_t sh = 8 * (i - lo);
        v = (v & ~(0xFFu << sh)) | ((uint32_t)b[i] << sh);
      }
    }
    wb[k] = v;
  }
}

// Resident blocks per SM: one fewer than the plain kernel's for W <= 4, which
// would spill with the encoder's registers.
template <int W>
struct MinBlocksAscii {
  static constexpr int value = W <= 2 ? 5 : (W <= 4 ? 4 : MinBlocks<W, false>::value);
};

template <int W, int VARIANT>
__global__ void __launch_bounds__(kFilterThreads, MinBlocksAscii<W>::value)
    filter_ascii_kernel(const AsciiArgs g) {
  const FilterArgs &a = g.f;
  __shared__ uint2 s_words[kFilterWarps][32][W];
  __shared__ uint32_t s_undef[kFilterWarps][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const bool active = p < a.n_pairs;

  PairData<W> x;
  x.status = 0;
  x.rid = 0xffffffffu;
  x.off = 0;
  x.e = a.fixed_e;
  x.m = a.m;
  x.nflag = 0;
  x.ni = make_uint2(0, 0xffffffffu);
  if (active) {
    x.rid = a.pair_read[p];
    x.off = a.pair_off[p];
    if (a.pair_e) x.e = a.pair_e[p];
    x.status = ((uint64_t)x.rid >= a.n_reads || (uint64_t)x.off + a.m > a.ref_len) ? 2 : 0;
  }
  if (a.err_count) {
    const unsigned bad = __ballot_sync(0xffffffffu, active && x.status == 2);
    if (bad && lane == 0) atomicAdd(a.err_count, (unsigned)__popc(bad));
  }
  const bool valid = active && x.status == 0 && a.m > 0;
  if (valid) {  // window words and N index word, in flight while the warp encodes
    if (a.ref_nidx) x.ni = a.ref_nidx[x.off >> 5];
    const uint2 *gp = a.ref_hl + (x.off >> 5);
#pragma unroll
    for (int w = 0; w <= W; ++w) x.g[w] = gp[w];
  }

  // The warp's distinct reads: a valid pair starts a run unless the lane
  // below holds a valid pair of the same read.
  const uint32_t below_rid = __shfl_up_sync(0xffffffffu, x.rid, 1);
  const int below_valid = __shfl_up_sync(0xffffffffu, valid ? 1 : 0, 1);
  const bool lead = valid && (lane == 0 || !below_valid || below_rid != x.rid);
  const unsigned runs = __ballot_sync(0xffffffffu, lead);
  const int n_runs = __popc(runs);
  const int my_run = valid ? __popc(runs & (0xffffffffu >> (31 - lane))) - 1 : 0;
  if (lane < n_runs) s_undef[wib][lane] = 0;
  __syncwarp();
  const uint32_t n_jobs = (uint32_t)n_runs * W;
  const bool aligned = g.rows_aligned != 0;
  for (uint32_t j0 = 0; j0 < n_jobs; j0 += 32) {  // warp-uniform trip count
    const uint32_t j = j0 + (uint32_t)lane;
    const bool has = j < n_jobs;
    const uint32_t r = has ? j / W : 0, w = has ? j % W : 0;
    const int src = has ? (int)__fns(runs, 0, (int)r + 1) : 0;  // the run's first lane
    const uint32_t rid = __shfl_sync(0xffffffffu, x.rid, src);
    if (has && 32u * w < a.m) {
      const uint32_t nv = min(32u, a.m - 32u * w);
      uint32_t wb[8];
      load_word_bytes(g.ascii + (uint64_t)rid * g.ascii_stride, w, nv, aligned, wb);
      uint32_t hi, lo, nb;
      encode32_full(wb, hi, lo, nb);
      if (nb) {
        encode32(wb, nv, hi, lo, nb);
        atomicOr(&s_undef[wib][r], 1u);
      }
      s_words[wib][r][w] = make_uint2(hi, lo);
    } else if (has) {
      s_words[wib][r][w] = make_uint2(0u, 0u);
    }
  }
  __syncwarp();
  if (!active) return;
  if (valid) {
#pragma unroll
    for (int w = 0; w < W; ++w) x.r[w] = s_words[wib][my_run][w];
    x.nflag = s_undef[wib][my_run];
  }
  const int status = pair_status<W>(a, x);
  if (status != 0 || a.m == 0) {
    write_trivial(a, p, status);
    return;
  }
  filter_and_write<W, VARIANT>(a, p, x);
}

template <int W, int VARIANT>
cudaError_t launch_filter_ascii_variant(const AsciiArgs &g, cudaStream_t stream) {
  const unsigned blocks = (unsigned)((g.f.n_pairs + kFilterThreads - 1) / kFilterThreads);
  filter_ascii_kernel<W, VARIANT><<<blocks, kFilterThreads, 0, stream>>>(g);
  return cudaGetLastError();
}

}  // namespace gk
