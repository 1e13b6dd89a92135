// The plain GateKeeper-GPU filter kernel: one thread per (read, candidate)
// pair, every mask held in registers as W = ceil(m/32) 32-bit words.
//
// Per pair (arxiv 2103.14978):
//   - undefined pairs (a non-ACGT base in the read or the window) pass with
//     accept = 1 and no filtration (Sec. 3.3);
//   - the window's two bit planes are funnel-shifted out of the resident
//     reference at the candidate offset;
//   - mask s compares the read shifted by s bases with the window: per base,
//     (high XOR) | (low XOR) is 1 when the 2-bit codes differ, and shifted-in
//     bases are code 00 (Sec. 2.1, Sec. 3.4).  The shifted read is kept
//     incrementally: each step moves the +k copy up and the -k copy down by
//     one base, a funnel shift per word and plane;
//   - amendment (Sec. 2.1) flips 0-streaks of length 1-2 bounded by 1s.  On a
//     bit vector with zeros outside [0, m) this equals a morphological closing
//     with a 3-base window: dilate (x | x<<1 | x>>1), then erode (AND of the
//     dilation and its two 1-base shifts); the erosion reads the dilation one
//     base beyond each end, which is the mask's own end bit;
//   - the edge OR of Sec. 3.4 sets, after amendment, the k vacated positions
//     of mask +k (the low end) and of mask -k (the high end).  The vacated
//     sets are kept as two incremental bit vectors and folded into the AND:
//     acc &= eroded | edge is one 3-input logic op;
//   - the AND of the 2e+1 masks stays in registers; the count of the final
//     vector is per-window runs (a 1 starts a run unless the bit below it is
//     1 and in the same 4-base window) or a popcount (Sec. 2.1).
//
// A shift by k >= m vacates the whole mask, which the edge OR then fills with
// 1s, so only k <= m-1 are computed.  Without the edge OR (the original
// GateKeeper) such masks are the window compared with code 00, ANDed once.
#pragma once

#include "gk_internal.cuh"

namespace gk {

constexpr int kFilterThreads = 256;

template <int W>
__device__ __forceinline__ void amend_and(const uint32_t (&d)[W], uint32_t (&acc)[W],
                                          const uint32_t (&edge)[W]) {
  uint32_t dil[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t below = __funnelshift_l(w > 0 ? d[w - 1] : 0u, d[w], 1);      // bit i <- d[i-1]
    const uint32_t above = __funnelshift_r(d[w], w + 1 < W ? d[w + 1] : 0u, 1);  // bit i <- d[i+1]
    dil[w] = d[w] | below | above;
  }
#pragma unroll
  for (int w = 0; w < W; ++w) {
    // The dilation one base below position 0 is d[0]; one base above the
    // last word it is the last word's top bit of d.
    const uint32_t lo_in = w > 0 ? dil[w - 1] : (d[0] << 31);
    const uint32_t hi_in = w + 1 < W ? dil[w + 1] : (d[W - 1] >> 31);
    const uint32_t below = __funnelshift_l(lo_in, dil[w], 1);
    const uint32_t above = __funnelshift_r(dil[w], hi_in, 1);
    acc[w] &= (dil[w] & below & above) | edge[w];
  }
}

template <int W>
__device__ __forceinline__ void diff_mask(const uint32_t (&sh)[W], const uint32_t (&sl)[W],
                                          const uint32_t (&gh)[W], const uint32_t (&gl)[W],
                                          uint32_t lastmask, uint32_t (&d)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) d[w] = (sh[w] ^ gh[w]) | (sl[w] ^ gl[w]);
  d[W - 1] &= lastmask;
}

template <int W>
__global__ void __launch_bounds__(kFilterThreads) filter_kernel(const FilterArgs a) {
  const uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const bool active = p < a.n_pairs;
  uint32_t rid = 0, off = 0, e = 0;
  int status = 0;  // 0 filter, 1 undefined (N), 2 invalid
  if (active) {
    rid = a.pair_read[p];
    off = a.pair_off[p];
    e = a.pair_e ? (uint32_t)a.pair_e[p] : a.fixed_e;
    if ((uint64_t)rid >= a.n_reads || (uint64_t)off + a.m > a.ref_len) status = 2;
  }
  if (a.err_count) {
    const unsigned bad = __ballot_sync(0xffffffffu, status == 2);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(a.err_count, (unsigned)__popc(bad));
  }
  if (!active) return;
  const uint32_t m = a.m;
  if (status == 0 && m > 0) {
    if (a.read_nflag && a.read_nflag[rid]) {
      status = 1;
    } else if (a.ref_nidx) {
      const uint2 ni = a.ref_nidx[off >> 5];
      const uint32_t q = ni.x >> (off & 31);
      const uint64_t first = q ? (uint64_t)off + (uint32_t)(__ffs(q) - 1) : (uint64_t)ni.y;
      if (first < (uint64_t)off + m) status = 1;
    }
  }
  if (status != 0 || m == 0) {
    a.accept[p] = status != 2;
    a.edits[p] = status == 0 ? 0 : (status == 1 ? GK_EDITS_UNDEFINED : GK_EDITS_INVALID);
    return;
  }

  const uint32_t tail = m - 32u * (W - 1);  // 1..32 bases in the last word
  const uint32_t lastmask = tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u);

  // Read planes (zero past m).
  uint32_t rh[W], rl[W];
  const uint2 *rp = a.reads + (uint64_t)rid * a.stride_words;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint2 v = rp[w];
    rh[w] = v.x;
    rl[w] = v.y;
  }
  rh[W - 1] &= lastmask;
  rl[W - 1] &= lastmask;

  // Window planes: bases [off, off+m) funnel-shifted out of words off/32 ...
  uint32_t gh[W], gl[W];
  {
    const uint2 *gp = a.ref_hl + (off >> 5);
    const uint32_t sh = off & 31;
    uint2 cur = gp[0];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint2 nxt = gp[w + 1];
      gh[w] = __funnelshift_r(cur.x, nxt.x, sh);
      gl[w] = __funnelshift_r(cur.y, nxt.y, sh);
      cur = nxt;
    }
  }

  uint32_t acc[W], d[W], zero[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    acc[w] = 0xffffffffu;
    zero[w] = 0;
  }
  // Shift 0: the Hamming mask, amended, no edge.
  diff_mask<W>(rh, rl, gh, gl, lastmask, d);
  amend_and<W>(d, acc, zero);

  const uint32_t kmax = min(e, m - 1);
  if (kmax > 0) {
    uint32_t ph[W], pl[W], nh[W], nl[W], lead[W], trail[W];
    const bool edge_on = a.edge_on != 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      ph[w] = nh[w] = rh[w];
      pl[w] = nl[w] = rl[w];
      lead[w] = 0;
      trail[w] = 0;  // positions >= m - k (and above m, which acc already cleared)
    }
    if (edge_on) trail[W - 1] = ~lastmask;
    const uint32_t lead_fill = edge_on ? 0x80000000u : 0u;
    const uint32_t trail_fill = edge_on ? 0xffffffffu : 0u;
    for (uint32_t k = 1; k <= kmax; ++k) {
#pragma unroll
      for (int w = W - 1; w >= 0; --w) {  // +k copy: one base up
        ph[w] = __funnelshift_l(w > 0 ? ph[w - 1] : 0u, ph[w], 1);
        pl[w] = __funnelshift_l(w > 0 ? pl[w - 1] : 0u, pl[w], 1);
        lead[w] = __funnelshift_l(w > 0 ? lead[w - 1] : lead_fill, lead[w], 1);
      }
#pragma unroll
      for (int w = 0; w < W; ++w) {  // -k copy: one base down
        nh[w] = __funnelshift_r(nh[w], w + 1 < W ? nh[w + 1] : 0u, 1);
        nl[w] = __funnelshift_r(nl[w], w + 1 < W ? nl[w + 1] : 0u, 1);
        trail[w] = __funnelshift_r(trail[w], w + 1 < W ? trail[w + 1] : trail_fill, 1);
      }
      diff_mask<W>(ph, pl, gh, gl, lastmask, d);
      amend_and<W>(d, acc, lead);
      diff_mask<W>(nh, nl, gh, gl, lastmask, d);
      amend_and<W>(d, acc, trail);
    }
  }
  if (a.edge_on == 0 && e >= m) {
    // Fully vacated masks of the original GateKeeper: window vs code 00.
    uint32_t zh[W];
#pragma unroll
    for (int w = 0; w < W; ++w) zh[w] = 0;
    diff_mask<W>(zh, zh, gh, gl, lastmask, d);
    amend_and<W>(d, acc, zero);
  }

  uint32_t count = 0;
  if (a.count_mode == GK_COUNT_POPCOUNT) {
#pragma unroll
    for (int w = 0; w < W; ++w) count += __popc(acc[w]);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t f = acc[w];
      count += __popc(f & ~((f << 1) & 0xEEEEEEEEu));
    }
  }
  a.accept[p] = count <= e;
  a.edits[p] = (uint16_t)count;
}

}  // namespace gk
