// Batched filter over pairs of mixed read lengths and per-pair thresholds
// (the paper batches many reads and candidates per launch, Sec. 3.3/3.5; here
// one persistent launch covers every length).
//
// Work is grouped by key = (W, K): W = ceil(m/32) words per read, K =
// min(e, 32W) shift steps.  A tile is up to tile_pairs pairs of one key, so a
// warp's control flow is uniform; persistent warps take tiles from one
// atomic counter, heaviest keys first.
#pragma once

#include "coop.cuh"
#include "filter.cuh"
#include "gk_internal.cuh"

namespace gk {

constexpr int kKeys = 16 * 256;  // W in 1..16, K in 0..255
constexpr uint16_t kNoKey = 0xFFFF;

__host__ __device__ __forceinline__ uint32_t key_of(uint32_t W, uint32_t K) { return (W - 1) * 256 + K; }
__host__ __device__ __forceinline__ uint32_t key_W(uint32_t key) { return key / 256 + 1; }
__host__ __device__ __forceinline__ uint32_t key_K(uint32_t key) { return key % 256; }

// Scratch of the batched path (all device memory, caller-provided).
struct BatchScratch {
  uint32_t *km;         // n_pairs: key | m << 16 (key kNoKey: result already written)
  uint4 *rec;           // n_pairs records grouped by key: {pair index, read id, offset, e | m << 16}
  uint32_t *hist;       // kKeys pair counts
  uint32_t *cursor;     // kKeys scatter cursors
  uint32_t *pair_base;  // kKeys + 1: first record slot of each key (descending key order)
  uint32_t *tile_base;  // kKeys + 1: first tile of each key (descending key order)
  uint32_t *counters;   // [0] next tile, [1] tile count, [2] [3] next tile of the W ranges 9-12, 13-16
};

constexpr uint64_t batch_up256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Byte size of the scratch for n_pairs pairs (one 256-aligned workspace).
constexpr uint64_t batch_scratch_size(uint64_t n_pairs) {
  return batch_up256(4 * n_pairs) + batch_up256(16 * n_pairs) + 2 * batch_up256(4 * kKeys) +
         2 * batch_up256(4 * (kKeys + 1)) + batch_up256(16);
}

struct BatchArgs {
  FilterArgs f;               // shared fields; f.m is unused (per-read lengths)
  const uint16_t *read_len;   // n_reads lengths
  uint32_t tile_pairs;
  BatchScratch s;
};

// batch_scratch_size at run time, and the layout inside one 256-aligned
// workspace.
uint64_t batch_scratch_bytes(uint64_t n_pairs);
BatchScratch batch_scratch_layout(void *base, uint64_t n_pairs);

cudaError_t launch_batched(int wpt, const BatchArgs &a, uint32_t blocks_per_sm, uint32_t warps_per_block,
                           cudaStream_t stream);

template <int WPT>
cudaError_t launch_persistent(const BatchArgs &a, uint32_t grid, uint32_t warps_per_block, cudaStream_t stream);

// One pair per lane over a tile of words-per-read W: the plain filter's
// per-thread code (deferred erosion when the tile's shift count is 2..30
// with the edge OR on, exact erosion otherwise), each pair with its own m.
// Every pair of a tile with K <= 30 has e = K; the code clamps the shift
// count to m - 1 per pair.  Records are read in slot order (coalesced).
template <int W>
__device__ __forceinline__ void tile_whole(const BatchArgs &a, uint32_t first, uint32_t end, uint32_t K,
                                           int lane) {
  const bool deferred = a.f.edge_on && K >= 2 && K <= 30;
  for (uint32_t base = first; base < end; base += 32) {
    const uint32_t slot = base + (uint32_t)lane;
    if (slot < end) {
      const uint4 rec = a.s.rec[slot];
      PairData<W> x;
      x.rid = rec.y;
      x.off = rec.z;
      x.e = rec.w & 0xFFFFu;
      x.m = rec.w >> 16;
      x.status = 0;
      load_words_wide<W>(a.f.reads, a.f.stride_words, a.f.ref_hl, x);
      const uint32_t count = deferred ? filter_loaded_deferred<W>(a.f, x)
                                      : (K < 32 ? filter_loaded<W, true>(a.f, x) : filter_loaded<W, false>(a.f, x));
      write_count(a.f, rec.x, count, x.e);
    }
  }
}

template <int W, int WHI>
__device__ __forceinline__ void dispatch_whole(const BatchArgs &a, uint32_t first, uint32_t end, uint32_t Wt,
                                               uint32_t K, int lane) {
  if (Wt == W) {
    tile_whole<W>(a, first, end, K, lane);
  } else if constexpr (W < WHI) {
    dispatch_whole<W + 1, WHI>(a, first, end, Wt, K, lane);
  }
}

// Key slot of tile t among slots [s_lo, s_hi): the last slot whose first tile
// is <= t (slots without tiles share their successor's tile_base).
__device__ __forceinline__ int slot_of_tile(const BatchArgs &a, uint32_t t, int s_lo, int s_hi) {
  int lo = s_lo, hi = s_hi - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.s.tile_base[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One pair per lane over the tiles whose W lies in [WLO, WHI].  In the
// descending key order those keys are the slots [kKeys - 256 WHI,
// kKeys - 256 (WLO - 1)), so their tiles form one contiguous range of
// tile_base; the range has its own tile counter, counters[CTR].  Register
// use follows the widest W of the range, so ranges are launched separately
// (widest first) rather than sharing one register budget.
template <int WLO, int WHI, int CTR>
__global__ void __launch_bounds__(256, WHI <= 8 ? 2 : 1) whole_kernel(const BatchArgs a) {
  const int lane = threadIdx.x & 31;
  constexpr int s_lo = kKeys - 256 * WHI, s_hi = kKeys - 256 * (WLO - 1);
  const uint32_t t_lo = a.s.tile_base[s_lo], t_hi = a.s.tile_base[s_hi];
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = t_lo + atomicAdd(&a.s.counters[CTR], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= t_hi) break;
    const int slot = slot_of_tile(a, t, s_lo, s_hi);
    const uint32_t key = (uint32_t)(kKeys - 1 - slot);
    const uint32_t first = a.s.pair_base[slot] + (t - a.s.tile_base[slot]) * a.tile_pairs;
    const uint32_t end = min(first + a.tile_pairs, a.s.pair_base[slot + 1]);
    dispatch_whole<WLO, WHI>(a, first, end, key_W(key), key_K(key), lane);
    __syncwarp();
  }
}

// Launches whole_kernel<WLO, WHI, CTR> on at most blocks_per_sm blocks per SM
// (fewer when the register file holds fewer).
template <int WLO, int WHI, int CTR>
cudaError_t launch_whole(const BatchArgs &a, uint32_t sms, uint32_t blocks_per_sm, uint32_t wpb,
                         cudaStream_t s) {
  int fit = 0;
  cudaError_t err =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, whole_kernel<WLO, WHI, CTR>, 32 * (int)wpb, 0);
  if (err != cudaSuccess) return err;
  if (fit == 0) return cudaErrorInvalidConfiguration;  // block does not fit the register file
  const uint32_t grid = sms * ((uint32_t)fit < blocks_per_sm ? (uint32_t)fit : blocks_per_sm);
  whole_kernel<WLO, WHI, CTR><<<grid, 32 * wpb, 0, s>>>(a);
  return cudaGetLastError();
}

template <int WPT>
__device__ __forceinline__ void tile_coop(const BatchArgs &a, uint32_t first, uint32_t end, uint32_t W, uint32_t K,
                                          int lane);

// Persistent filter body of the lane-group tilings: a pair spread over
// ceil(W / WPT) lanes.
template <int WPT>
__global__ void __launch_bounds__(256, 1) persistent_kernel(const BatchArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t n_tiles = a.s.counters[1];
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&a.s.counters[0], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_tiles) break;
    const int slot = slot_of_tile(a, t, 0, kKeys);
    const uint32_t key = (uint32_t)(kKeys - 1 - slot);  // slot 0 is the heaviest key
    const uint32_t W = key_W(key), K = key_K(key);
    const uint32_t first = a.s.pair_base[slot] + (t - a.s.tile_base[slot]) * a.tile_pairs;
    const uint32_t end = min(first + a.tile_pairs, a.s.pair_base[slot + 1]);
    tile_coop<WPT>(a, first, end, W, K, lane);
  }
}

template <int WPT>
__device__ __forceinline__ void tile_coop(const BatchArgs &a, uint32_t first, uint32_t end, uint32_t W, uint32_t K,
                                          int lane) {
  const bool edge_on = a.f.edge_on != 0;
  {
    Group g;
    g.L = (int)((W + WPT - 1) / WPT);
    const int ppw = 32 / g.L;
    const int grp = lane / g.L;
    g.lig = lane - grp * g.L;
    for (uint32_t base = first; base < end; base += (uint32_t)ppw) {
      const uint32_t slot = base + (uint32_t)grp;
      const bool valid = grp < ppw && slot < end;
      uint32_t rh[WPT], rl[WPT], gh[WPT], gl[WPT], vm[WPT];
      uint32_t p = 0, e = 0, m = 0;
#pragma unroll
      for (int j = 0; j < WPT; ++j) rh[j] = rl[j] = gh[j] = gl[j] = vm[j] = 0;
      if (valid) {
        const uint4 rec = a.s.rec[slot];
        p = rec.x;
        const uint32_t rid = rec.y;
        const uint32_t off = rec.z;
        e = rec.w & 0xFFFFu;
        m = rec.w >> 16;
        const uint2 *rp = a.f.reads + (uint64_t)rid * a.f.stride_words;
        const uint2 *gp = a.f.ref_hl + (off >> 5);
        const uint32_t sh = off & 31;
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
          const uint32_t w = (uint32_t)(g.lig * WPT + j);
          if (w < W) {
            const int64_t rem = (int64_t)m - 32 * (int64_t)w;
            vm[j] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
            const uint2 r = rp[w];
            rh[j] = r.x & vm[j];
            rl[j] = r.y & vm[j];
            const uint2 c0 = gp[w], c1 = gp[w + 1];
            gh[j] = __funnelshift_r(c0.x, c1.x, sh) & vm[j];
            gl[j] = __funnelshift_r(c0.y, c1.y, sh) & vm[j];
          }
        }
      }
      const uint32_t count = coop_filter<WPT>(rh, rl, gh, gl, vm, K, edge_on, a.f.count_mode, g);
      if (valid && g.lig == 0) {
        write_count(a.f, p, count, e);
      }
    }
  }
}

}  // namespace gk
