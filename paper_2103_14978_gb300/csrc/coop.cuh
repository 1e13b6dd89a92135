// Lane-group form of the filter for the batched path: a pair's W words are
// spread over L = ceil(W / WPT) consecutive lanes, WPT words per lane, and the
// bits that cross a lane boundary travel by warp shuffles.  The arithmetic is
// the plain kernel's (filter.cuh): incremental +k / -k read copies, mask =
// (high XOR) | (low XOR), amendment as a 3-base closing, edge bits OR-folded
// into the AND, window-run or popcount count (Sec. 2.1, 3.3, 3.4).
//
// Every lane of the warp executes every shuffle: the caller keeps control
// flow warp-uniform (one tile = one words-per-read class and one step count).
#pragma once

#include "gk_internal.cuh"

namespace gk {

struct Group {
  int lig;  // lane index inside the group, 0..L-1
  int L;    // lanes per pair
};

// The lane below's last word, or `fill` for the group's first lane.
__device__ __forceinline__ uint32_t from_below(uint32_t my_last, const Group &g, uint32_t fill) {
  const uint32_t v = __shfl_up_sync(0xffffffffu, my_last, 1);
  return g.lig == 0 ? fill : v;
}

// The lane above's first word, or `fill` for the group's last lane.
__device__ __forceinline__ uint32_t from_above(uint32_t my_first, const Group &g, uint32_t fill) {
  const uint32_t v = __shfl_down_sync(0xffffffffu, my_first, 1);
  return g.lig == g.L - 1 ? fill : v;
}

template <int WPT>
__device__ __forceinline__ void coop_amend_and(const uint32_t (&d)[WPT], uint32_t (&acc)[WPT],
                                               const uint32_t (&edge)[WPT], const Group &g) {
  const uint32_t dl = from_below(d[WPT - 1], g, 0u);
  const uint32_t dh = from_above(d[0], g, 0u);
  uint32_t dil[WPT];
#pragma unroll
  for (int w = 0; w < WPT; ++w) {
    const uint32_t below = __funnelshift_l(w > 0 ? d[w - 1] : dl, d[w], 1);
    const uint32_t above = __funnelshift_r(d[w], w + 1 < WPT ? d[w + 1] : dh, 1);
    dil[w] = d[w] | below | above;
  }
  // Beyond the vector the dilation is the end bit of d itself.
  const uint32_t il = from_below(dil[WPT - 1], g, d[0] << 31);
  const uint32_t ih = from_above(dil[0], g, d[WPT - 1] >> 31);
#pragma unroll
  for (int w = 0; w < WPT; ++w) {
    const uint32_t below = __funnelshift_l(w > 0 ? dil[w - 1] : il, dil[w], 1);
    const uint32_t above = __funnelshift_r(dil[w], w + 1 < WPT ? dil[w + 1] : ih, 1);
    acc[w] &= (dil[w] & below & above) | edge[w];
  }
}

// Filters one pair per lane group.  rh/rl/gh/gl hold this lane's words of the
// read and window planes (zero past m), vm the valid-bit masks (bits < m),
// K the number of shift steps (uniform over the warp; shifts past m - 1 are
// no-ops with the edge OR and repeat the fully vacated mask without it).
// Returns the group's count in lane lig == 0 (other lanes: partial sums).
template <int WPT>
__device__ __forceinline__ uint32_t coop_filter(const uint32_t (&rh)[WPT], const uint32_t (&rl)[WPT],
                                                const uint32_t (&gh)[WPT], const uint32_t (&gl)[WPT],
                                                const uint32_t (&vm)[WPT], uint32_t K, bool edge_on,
                                                int count_mode, const Group &g) {
  uint32_t acc[WPT], d[WPT], zero[WPT];
#pragma unroll
  for (int w = 0; w < WPT; ++w) {
    acc[w] = 0xffffffffu;
    zero[w] = 0;
    d[w] = (rh[w] ^ gh[w]) | (rl[w] ^ gl[w]);
  }
  coop_amend_and<WPT>(d, acc, zero, g);
  if (K > 0) {
    uint32_t ph[WPT], pl[WPT], nh[WPT], nl[WPT], lead[WPT], trail[WPT];
#pragma unroll
    for (int w = 0; w < WPT; ++w) {
      ph[w] = nh[w] = rh[w];
      pl[w] = nl[w] = rl[w];
      lead[w] = 0;
      trail[w] = edge_on ? ~vm[w] : 0u;
    }
    const uint32_t lead_fill = edge_on ? 0x80000000u : 0u;
    const uint32_t trail_fill = edge_on ? 0xffffffffu : 0u;
    for (uint32_t k = 1; k <= K; ++k) {
      const uint32_t bh = from_below(ph[WPT - 1], g, 0u);
      const uint32_t bl = from_below(pl[WPT - 1], g, 0u);
      const uint32_t bL = from_below(lead[WPT - 1], g, lead_fill);
#pragma unroll
      for (int w = WPT - 1; w >= 0; --w) {
        ph[w] = __funnelshift_l(w > 0 ? ph[w - 1] : bh, ph[w], 1);
        pl[w] = __funnelshift_l(w > 0 ? pl[w - 1] : bl, pl[w], 1);
        lead[w] = __funnelshift_l(w > 0 ? lead[w - 1] : bL, lead[w], 1);
      }
      const uint32_t ah = from_above(nh[0], g, 0u);
      const uint32_t al = from_above(nl[0], g, 0u);
      const uint32_t aT = from_above(trail[0], g, trail_fill);
#pragma unroll
      for (int w = 0; w < WPT; ++w) {
        nh[w] = __funnelshift_r(nh[w], w + 1 < WPT ? nh[w + 1] : ah, 1);
        nl[w] = __funnelshift_r(nl[w], w + 1 < WPT ? nl[w + 1] : al, 1);
        trail[w] = __funnelshift_r(trail[w], w + 1 < WPT ? trail[w + 1] : aT, 1);
      }
#pragma unroll
      for (int w = 0; w < WPT; ++w) d[w] = ((ph[w] ^ gh[w]) | (pl[w] ^ gl[w])) & vm[w];
      coop_amend_and<WPT>(d, acc, lead, g);
#pragma unroll
      for (int w = 0; w < WPT; ++w) d[w] = (nh[w] ^ gh[w]) | (nl[w] ^ gl[w]);
      coop_amend_and<WPT>(d, acc, trail, g);
    }
  }
  uint32_t count = 0;
  if (count_mode == GK_COUNT_POPCOUNT) {
#pragma unroll
    for (int w = 0; w < WPT; ++w) count += __popc(acc[w]);
  } else {
#pragma unroll
    for (int w = 0; w < WPT; ++w) count += __popc(acc[w] & ~((acc[w] << 1) & 0xEEEEEEEEu));
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_down_sync(0xffffffffu, count, off);
    if (g.lig + off < g.L) count += v;
  }
  return count;
}

}  // namespace gk
