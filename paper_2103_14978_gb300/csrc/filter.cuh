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
//     acc &= eroded | edge is one 3-input logic op.  With k < 32 the low set
//     lives in word 0 and the high set in the top two words only;
//   - the AND of the 2e+1 masks stays in registers; the count of the final
//     vector is per-window runs (a 1 starts a run unless the bit below it is
//     1 and in the same 4-base window) or a popcount (Sec. 2.1).
//
// A shift by k >= m vacates the whole mask, which the edge OR then fills with
// 1s, so only k <= m-1 are computed.  Without the edge OR (the original
// GateKeeper) such masks are the window compared with code 00, ANDed once.
#pragma once

#include <atomic>

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

// Inputs of one pair.
template <int W>
struct PairData {
  uint32_t rid, off, e, m;  // m: this pair's read length
  int status;     // 0 filter, 1 undefined, 2 invalid
  uint32_t nflag; // read's N flag
  uint2 ni;       // N index word of the window start
  uint2 r[W];     // read words
  uint2 g[W + 1]; // reference words covering the window
};

// Read words 0..W-1 of a valid pair (W = ceil(m/32) <= the row stride) in
// 16-byte loads, half the requests of 8-byte loads.  With a 16-byte aligned
// read buffer and an even row stride every read row starts on 16 bytes (an
// odd W is below the stride, so the extra word is row padding); otherwise
// the read takes 8-byte loads.
template <int W>
__device__ __forceinline__ void load_read_wide(const uint2 *reads, uint32_t stride_words, PairData<W> &x) {
  const uint2 *rp = reads + (uint64_t)x.rid * stride_words;
  if ((stride_words & 1u) == 0 && (reinterpret_cast<uintptr_t>(reads) & 15u) == 0) {
    const uint4 *rq = reinterpret_cast<const uint4 *>(rp);
#pragma unroll
    for (int i = 0; i < (W + 1) / 2; ++i) {
      const uint4 v = rq[i];
      x.r[2 * i] = make_uint2(v.x, v.y);
      if (2 * i + 1 < W) x.r[2 * i + 1] = make_uint2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) x.r[w] = rp[w];
  }
}

// Genome window words off/32 .. off/32 + W of a valid pair (off + m within
// the genome) in aligned 16-byte loads from the even word at or below
// off/32: ceil((W+1)/2) loads, one more when W and off/32 are both odd; the
// last word read is at most n_words + 1, inside the genome's two zero tail
// words.
template <int W>
__device__ __forceinline__ void load_window_wide(const uint2 *ref_hl, PairData<W> &x) {
  constexpr int NE = (W + 2) / 2;  // ceil((W + 1) / 2)
  const uint32_t s = x.off >> 5;
  const bool odd = (s & 1u) != 0;
  const uint4 *gq = reinterpret_cast<const uint4 *>(ref_hl + (s & ~1u));
  uint2 v[2 * NE + 2];
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const uint4 q = gq[i];
    v[2 * i] = make_uint2(q.x, q.y);
    v[2 * i + 1] = make_uint2(q.z, q.w);
  }
  v[2 * NE] = v[2 * NE + 1] = make_uint2(0u, 0u);
  if ((W & 1) && odd) {
    const uint4 q = gq[NE];
    v[2 * NE] = make_uint2(q.x, q.y);
  }
#pragma unroll
  for (int w = 0; w <= W; ++w) x.g[w] = odd ? v[w + 1] : v[w];
}

template <int W>
__device__ __forceinline__ void load_words_wide(const uint2 *reads, uint32_t stride_words, const uint2 *ref_hl,
                                                PairData<W> &x) {
  load_read_wide<W>(reads, stride_words, x);
  load_window_wide<W>(ref_hl, x);
}

// Window words off/32 .. off/32 + W of a valid pair in 8-byte loads: 40
// contiguous bytes, two 32-byte sectors.  SKIP_LAST: word off/32 + W only
// when the window reaches into it ((off mod 32) + m > 32W); otherwise its
// bits land past m, where the planes are masked (at 100 bp 29 pairs in 32
// skip it).  (A copy of the genome holding overlapping word pairs, read in
// 16-byte loads, measured 13% slower at e = 0: its three loads touch three
// sectors.)
template <int W, bool WIDE, bool SKIP_LAST = false>
__device__ __forceinline__ void load_window(const FilterArgs &a, PairData<W> &x) {
  if (WIDE) {
    load_window_wide<W>(a.ref_hl, x);
  } else {
    const uint2 *gp = a.ref_hl + (x.off >> 5);
#pragma unroll
    for (int w = 0; w < W; ++w) x.g[w] = gp[w];
    if (SKIP_LAST)
      x.g[W] = (x.off & 31u) + x.m > 32u * W ? gp[W] : make_uint2(0u, 0u);
    else
      x.g[W] = gp[W];
  }
}

// Loads pair p.  WIDE: read and window words in 16-byte loads.  The plain
// kernel keeps 8-byte loads: at e <= 2 (the launches waiting on loads) the
// wide form measured 2-6% slower at 100 and 150 bp.  share (nullable): a
// pair loaded before; when it is valid and has the same read, its read words
// and N flag are copied instead of loaded again.
template <int W, bool WIDE = false, bool SKIP_LAST = false>
__device__ __forceinline__ void load_pair(const FilterArgs &a, uint64_t p, PairData<W> &x,
                                          const PairData<W> *share = nullptr) {
  x.rid = a.pair_read[p];
  x.off = a.pair_off[p];
  x.e = a.pair_e ? (uint32_t)a.pair_e[p] : a.fixed_e;
  x.m = a.m;
  x.status = ((uint64_t)x.rid >= a.n_reads || (uint64_t)x.off + a.m > a.ref_len) ? 2 : 0;
  x.nflag = 0;
  x.ni = make_uint2(0, 0xffffffffu);
  if (x.status == 0 && a.m > 0) {
    if (a.ref_nidx) x.ni = a.ref_nidx[x.off >> 5];
    if (share && share->status == 0 && share->rid == x.rid) {
      x.nflag = share->nflag;
#pragma unroll
      for (int w = 0; w < W; ++w) x.r[w] = share->r[w];
    } else {
      if (a.read_nflag) x.nflag = a.read_nflag[x.rid];
      if (WIDE) {
        load_read_wide<W>(a.reads, a.stride_words, x);
      } else {
        const uint2 *rp = a.reads + (uint64_t)x.rid * a.stride_words;
#pragma unroll
        for (int w = 0; w < W; ++w) x.r[w] = rp[w];
      }
    }
    load_window<W, WIDE, SKIP_LAST>(a, x);
  }
}

// Filters one loaded pair; returns the count.
template <int W, bool SMALL_K>
__device__ __forceinline__ uint32_t filter_loaded(const FilterArgs &a, const PairData<W> &x) {
  const uint32_t m = x.m;
  const uint32_t tail = m - 32u * (W - 1);  // 1..32 bases in the last word
  const uint32_t lastmask = tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u);

  uint32_t rh[W], rl[W], gh[W], gl[W];
  const uint32_t sh = x.off & 31;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    rh[w] = x.r[w].x;
    rl[w] = x.r[w].y;
    gh[w] = __funnelshift_r(x.g[w].x, x.g[w + 1].x, sh);
    gl[w] = __funnelshift_r(x.g[w].y, x.g[w + 1].y, sh);
  }
  // Both sequences zero past m: the Hamming and -k masks need no masking.
  rh[W - 1] &= lastmask;
  rl[W - 1] &= lastmask;
  gh[W - 1] &= lastmask;
  gl[W - 1] &= lastmask;

  uint32_t acc[W], d[W], zero[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    acc[w] = 0xffffffffu;
    zero[w] = 0;
    d[w] = (rh[w] ^ gh[w]) | (rl[w] ^ gl[w]);
  }
  amend_and<W>(d, acc, zero);  // shift 0: the Hamming mask, no edge

  const uint32_t kmax = min(x.e, m - 1);
  const bool edge_on = a.edge_on != 0;
  if (kmax > 0) {
    uint32_t ph[W], pl[W], nh[W], nl[W], lead[W], trail[W];
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
        // vacated low positions [0, k): with k < 32 only word 0 holds them
        if (!SMALL_K || w == 0) lead[w] = __funnelshift_l(w > 0 ? lead[w - 1] : lead_fill, lead[w], 1);
      }
#pragma unroll
      for (int w = 0; w < W; ++w) {  // -k copy: one base down
        nh[w] = __funnelshift_r(nh[w], w + 1 < W ? nh[w + 1] : 0u, 1);
        nl[w] = __funnelshift_r(nl[w], w + 1 < W ? nl[w + 1] : 0u, 1);
        // vacated high positions [m-k, m): with k < 32 only the top two words
        if (!SMALL_K || w + 2 >= W) trail[w] = __funnelshift_r(trail[w], w + 1 < W ? trail[w + 1] : trail_fill, 1);
      }
#pragma unroll
      for (int w = 0; w < W; ++w) d[w] = (ph[w] ^ gh[w]) | (pl[w] ^ gl[w]);
      d[W - 1] &= lastmask;  // the +k copy carries read bases past m
      amend_and<W>(d, acc, lead);
#pragma unroll
      for (int w = 0; w < W; ++w) d[w] = (nh[w] ^ gh[w]) | (nl[w] ^ gl[w]);
      amend_and<W>(d, acc, trail);
    }
  }
  if (!edge_on && x.e >= m) {
    // Fully vacated masks of the original GateKeeper: window vs code 00.
#pragma unroll
    for (int w = 0; w < W; ++w) d[w] = gh[w] | gl[w];
    amend_and<W>(d, acc, zero);
  }

  uint32_t count = 0;
  if (a.count_mode == GK_COUNT_POPCOUNT) {
#pragma unroll
    for (int w = 0; w < W; ++w) count += __popc(acc[w]);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) count += __popc(acc[w] & ~((acc[w] << 1) & 0xEEEEEEEEu));
  }
  return count;
}

// Deferred-erosion form of filter_loaded for the edge OR on and every shift
// count k <= 30.  Erosion commutes with AND (the AND of erosions is the
// erosion of the AND), so the loop ANDs dilated masks only and erodes once at
// the end.  Mask +k is ORed with its dilated vacated set [-1, k] and mask -k
// with [m-k-1, m]; that agrees with "erode, then OR the vacated set" at every
// position except the two next to each vacated run (k and k+1, m-k-2 and
// m-k-1), where the erosion of the true mask needs two dilation bits the OR
// hid.  Those bits depend only on the read's first or last two bases against
// the window and on which window bases are 'A', so their corrections for all
// k are computed once per pair; so are the two values of the AND one base
// outside each end that the final erosion reads.
// Deferred-erosion counts of NP pairs that share one read and one shift
// count K, each against its own window: the read's +k and -k copies (4W
// funnel shifts per step) are built once for all NP windows.  rh/rl and
// gh/gl are the read's and the windows' planes, zero past m.
template <int W, int NP, bool DIRECT = false>
__device__ __forceinline__ void deferred_counts(const FilterArgs &a, uint32_t m, uint32_t K,
                                                const uint32_t (&rh)[W], const uint32_t (&rl)[W],
                                                const uint32_t (&gh)[NP][W], const uint32_t (&gl)[NP][W],
                                                uint32_t (&count)[NP]) {
  const uint32_t tail = m - 32u * (W - 1);  // 1..32 bases in the last word
  const uint32_t lastmask = tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u);

  uint32_t acc[NP][W], d[W], dn[W];
  // dilation of a mask: bit i <- d[i-1] | d[i] | d[i+1], zeros outside the words
  auto dil = [&](const uint32_t (&dd)[W], int w) -> uint32_t {
    const uint32_t below = __funnelshift_l(w > 0 ? dd[w - 1] : 0u, dd[w], 1);
    const uint32_t above = __funnelshift_r(dd[w], w + 1 < W ? dd[w + 1] : 0u, 1);
    return dd[w] | below | above;
  };
#pragma unroll
  for (int j = 0; j < NP; ++j) {
#pragma unroll
    for (int w = 0; w < W; ++w) d[w] = (rh[w] ^ gh[j][w]) | (rl[w] ^ gl[j][w]);
#pragma unroll
    for (int w = 0; w < W; ++w) acc[j][w] = dil(d, w);  // shift 0
  }
  {
    // DIRECT (a shift count fixed at compile time): the read's +k and -k
    // copies come straight from rh/rl by k-base funnel shifts, no copy carried
    // from step to step (fewer live registers: measured faster at K = 0..2);
    // otherwise each step moves the carried copies by one base (faster for a
    // runtime K and in the sweep).
    uint32_t ph[W], pl[W], nh[W], nl[W];
    if (!DIRECT) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        ph[w] = nh[w] = rh[w];
        pl[w] = nl[w] = rl[w];
      }
    }
    // The vacated positions of each shifted mask are ORed into its difference
    // vector before the dilation: dil(d | V) = dil(d) | dil(V), the mask ORed
    // with its dilated vacated set.
    uint32_t lead = 0u;               // mask +k: positions 0..k-1 (word 0)
    uint32_t tv_hi = ~lastmask;       // mask -k: positions >= m-k (and >= m), top word
    uint32_t tv_lo = 0u;              // and the word below it
    for (uint32_t k = 1; k <= K; ++k) {
      if (DIRECT) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          ph[w] = __funnelshift_l(w > 0 ? rh[w - 1] : 0u, rh[w], k);
          pl[w] = __funnelshift_l(w > 0 ? rl[w - 1] : 0u, rl[w], k);
          nh[w] = __funnelshift_r(rh[w], w + 1 < W ? rh[w + 1] : 0u, k);
          nl[w] = __funnelshift_r(rl[w], w + 1 < W ? rl[w + 1] : 0u, k);
        }
      } else {
#pragma unroll
        for (int w = W - 1; w >= 0; --w) {
          ph[w] = __funnelshift_l(w > 0 ? ph[w - 1] : 0u, ph[w], 1);
          pl[w] = __funnelshift_l(w > 0 ? pl[w - 1] : 0u, pl[w], 1);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
          nh[w] = __funnelshift_r(nh[w], w + 1 < W ? nh[w + 1] : 0u, 1);
          nl[w] = __funnelshift_r(nl[w], w + 1 < W ? nl[w + 1] : 0u, 1);
        }
      }
      lead = 2u * lead + 1u;
      tv_lo = __funnelshift_r(tv_lo, tv_hi, 1);
      tv_hi = __funnelshift_r(tv_hi, 0xffffffffu, 1);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const uint32_t vp = w == 0 ? lead : 0u;
          const uint32_t vn = w == W - 1 ? tv_hi : (w == W - 2 ? tv_lo : 0u);
          d[w] = (ph[w] ^ gh[j][w]) | vp | (pl[w] ^ gl[j][w]);
          dn[w] = (nh[w] ^ gh[j][w]) | vn | (nl[w] ^ gl[j][w]);
        }
        d[W - 1] &= lastmask;  // the +k copy carries read bases past m
#pragma unroll
        for (int w = 0; w < W; ++w) acc[j][w] &= dil(d, w) & dil(dn, w);
      }
    }
  }

  // ---- once per pair: end values of the AND, corrections, final erosion ----
  const uint32_t rangeK = (2u << K) - 1u;  // bits 0..K
  const uint32_t r1k = rangeK & ~1u;       // bits 1..K
  // The read's last 32 bases mirrored: bit j is position m-1-j (positions
  // below 0 read as code 00).  The high end's terms are the low end's
  // formulas on mirrored vectors, in 32-bit words.
  const uint32_t xrh = __funnelshift_rc(W >= 2 ? rh[W >= 2 ? W - 2 : 0] : 0u, rh[W - 1], tail);
  const uint32_t xrl = __funnelshift_rc(W >= 2 ? rl[W >= 2 ? W - 2 : 0] : 0u, rl[W - 1], tail);
  const uint32_t b0h = 0u - (xrh >> 31), b0l = 0u - (xrl >> 31);                // R[m-1]
  const uint32_t b1h = 0u - ((xrh >> 30) & 1u), b1l = 0u - ((xrl >> 30) & 1u);  // R[m-2]
  const uint32_t r0h = 0u - (rh[0] & 1u), r0l = 0u - (rl[0] & 1u);              // R[0]
  const uint32_t r1h = 0u - ((rh[0] >> 1) & 1u), r1l = 0u - ((rl[0] >> 1) & 1u);  // R[1]
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    // AND one base below position 0: every non-positive shift compares G[0]
    // with R[i], i = 0..K.
    const uint32_t g0h = 0u - (gh[j][0] & 1u), g0l = 0u - (gl[j][0] & 1u);
    const uint32_t q0 = (rh[0] ^ g0h) | (rl[0] ^ g0l);
    const uint32_t vlo = ((~q0 & rangeK) == 0) ? 1u : 0u;
    // The window's last 32 bases mirrored.
    const uint32_t mgh = __brev(__funnelshift_rc(W >= 2 ? gh[j][W >= 2 ? W - 2 : 0] : 0u, gh[j][W - 1], tail));
    const uint32_t mgl = __brev(__funnelshift_rc(W >= 2 ? gl[j][W >= 2 ? W - 2 : 0] : 0u, gl[j][W - 1], tail));
    // AND one base above position m-1, needed only when m fills the words:
    // every non-negative shift compares G[m-1] with R[m-1-i], i = 0..K.
    uint32_t vtop = 0u;
    if (tail == 32) {
      const uint32_t gmh = 0u - (mgh & 1u), gml = 0u - (mgl & 1u);
      const uint32_t qm = (__brev(xrh) ^ gmh) | (__brev(xrl) ^ gml);
      vtop = ((~qm & rangeK) == 0) ? 1u : 0u;
    }
    uint32_t f[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t lo_in = w > 0 ? acc[j][w - 1] : (vlo << 31);
      const uint32_t hi_in = w + 1 < W ? acc[j][w + 1] : vtop;
      f[w] = acc[j][w] & __funnelshift_l(lo_in, acc[j][w], 1) & __funnelshift_r(acc[j][w], hi_in, 1);
    }
    // Low-end corrections (positions 1..K+1, word 0).
    {
      const uint32_t v0 = W == 1 ? lastmask : 0xffffffffu;
      const uint32_t a0 = (gh[j][0] ^ r0h) | (gl[j][0] ^ r0l);
      const uint32_t a1 = ((gh[j][0] ^ r1h) | (gl[j][0] ^ r1l)) & v0;
      const uint32_t vac = gh[j][0] | gl[j][0];
      const uint32_t c1 = (vac << 2) | (vac << 1) | a0;
      const uint32_t c2 = (vac << 1) | a0 | (a1 >> 1);
      f[0] &= ~((~(c1 & c2) & r1k) | ((~c2 & r1k) << 1));
    }
    // High-end corrections (positions m-K-2..m-2), computed mirrored and
    // mapped back: mirrored bit j is position m-1-j.
    {
      const uint32_t a0 = (mgh ^ b0h) | (mgl ^ b0l);
      const uint32_t a1 = (mgh ^ b1h) | (mgl ^ b1l);
      const uint32_t vac = mgh | mgl;
      const uint32_t c1 = (vac << 2) | (vac << 1) | a0;
      const uint32_t c2 = (vac << 1) | a0 | (a1 >> 1);
      const uint32_t nc = __brev((~(c1 & c2) & r1k) | ((~c2 & r1k) << 1));  // bit b: position m-32+b
      f[W - 1] &= ~(nc >> (32u - tail));
      if (W >= 2 && tail < 32) f[W >= 2 ? W - 2 : 0] &= ~(nc << tail);
    }
    f[W - 1] &= lastmask;

    uint32_t c = 0;
    if (a.count_mode == GK_COUNT_POPCOUNT) {
#pragma unroll
      for (int w = 0; w < W; ++w) c += __popc(f[w]);
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w) c += __popc(f[w] & ~((f[w] << 1) & 0xEEEEEEEEu));
    }
    count[j] = c;
  }
}

template <int NP>
struct FinishPrep;
template <int W, int NP>
__device__ __forceinline__ void deferred_prep(int j, uint32_t tail, uint32_t lastmask, const uint32_t (&rh)[W],
                                              const uint32_t (&rl)[W], const uint32_t (&gh)[NP][W],
                                              const uint32_t (&gl)[NP][W], FinishPrep<NP> &pr);
template <int W, int NP>
__device__ __forceinline__ void deferred_finish(const FilterArgs &a, uint32_t K, uint32_t tail,
                                                uint32_t lastmask, const uint32_t (&acc)[NP][W],
                                                const FinishPrep<NP> &pr, uint32_t (&count)[NP]);

// deferred_counts at every shift count K = Klo .. K of a threshold sweep in
// one pass: the 2k+1 masks of shift count k are those of k-1 and the two
// shifted by k, so the running AND after step k is the AND of shift count k,
// and the once-per-pair finish (end values, erosion, corrections, count)
// runs on it at each k from Klo on; emit(k, count) receives the counts.  The
// finish's shift-independent terms are prepared once per pair.
template <int W, int NP, typename Emit>
__device__ __forceinline__ void deferred_sweep_counts(const FilterArgs &a, uint32_t m, uint32_t K,
                                                      const uint32_t (&rh)[W], const uint32_t (&rl)[W],
                                                      const uint32_t (&gh)[NP][W], const uint32_t (&gl)[NP][W],
                                                      uint32_t (&count)[NP], uint32_t Klo, Emit emit) {
  const uint32_t tail = m - 32u * (W - 1);  // 1..32 bases in the last word
  const uint32_t lastmask = tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u);

  uint32_t acc[NP][W], d[W], dn[W];
  FinishPrep<NP> pr;
#pragma unroll
  for (int j = 0; j < NP; ++j) deferred_prep<W, NP>(j, tail, lastmask, rh, rl, gh, gl, pr);
  auto finish = [&](uint32_t Kf) { deferred_finish<W, NP>(a, Kf, tail, lastmask, acc, pr, count); };
  // dilation of a mask: bit i <- d[i-1] | d[i] | d[i+1], zeros outside the words
  auto dil = [&](const uint32_t (&dd)[W], int w) -> uint32_t {
    const uint32_t below = __funnelshift_l(w > 0 ? dd[w - 1] : 0u, dd[w], 1);
    const uint32_t above = __funnelshift_r(dd[w], w + 1 < W ? dd[w + 1] : 0u, 1);
    return dd[w] | below | above;
  };
#pragma unroll
  for (int j = 0; j < NP; ++j) {
#pragma unroll
    for (int w = 0; w < W; ++w) d[w] = (rh[w] ^ gh[j][w]) | (rl[w] ^ gl[j][w]);
#pragma unroll
    for (int w = 0; w < W; ++w) acc[j][w] = dil(d, w);  // shift 0
  }
  if (Klo == 0) {
    finish(0);
    emit(0u, count);
  }
  {
    uint32_t ph[W], pl[W], nh[W], nl[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      ph[w] = nh[w] = rh[w];
      pl[w] = nl[w] = rl[w];
    }
    // The vacated positions of each shifted mask are ORed into its difference
    // vector before the dilation: dil(d | V) = dil(d) | dil(V), the mask ORed
    // with its dilated vacated set.
    uint32_t lead = 0u;               // mask +k: positions 0..k-1 (word 0)
    uint32_t tv_hi = ~lastmask;       // mask -k: positions >= m-k (and >= m), top word
    uint32_t tv_lo = 0u;              // and the word below it
    for (uint32_t k = 1; k <= K; ++k) {
#pragma unroll
      for (int w = W - 1; w >= 0; --w) {
        ph[w] = __funnelshift_l(w > 0 ? ph[w - 1] : 0u, ph[w], 1);
        pl[w] = __funnelshift_l(w > 0 ? pl[w - 1] : 0u, pl[w], 1);
      }
#pragma unroll
      for (int w = 0; w < W; ++w) {
        nh[w] = __funnelshift_r(nh[w], w + 1 < W ? nh[w + 1] : 0u, 1);
        nl[w] = __funnelshift_r(nl[w], w + 1 < W ? nl[w + 1] : 0u, 1);
      }
      lead = 2u * lead + 1u;
      tv_lo = __funnelshift_r(tv_lo, tv_hi, 1);
      tv_hi = __funnelshift_r(tv_hi, 0xffffffffu, 1);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const uint32_t vp = w == 0 ? lead : 0u;
          const uint32_t vn = w == W - 1 ? tv_hi : (w == W - 2 ? tv_lo : 0u);
          d[w] = (ph[w] ^ gh[j][w]) | vp | (pl[w] ^ gl[j][w]);
          dn[w] = (nh[w] ^ gh[j][w]) | vn | (nl[w] ^ gl[j][w]);
        }
        d[W - 1] &= lastmask;  // the +k copy carries read bases past m
#pragma unroll
        for (int w = 0; w < W; ++w) acc[j][w] &= dil(d, w) & dil(dn, w);
      }
      if (k >= Klo) {
        finish(k);
        emit(k, count);
      }
    }
  }
}

// The shift-count-independent terms of the once-per-pair end: per pair, the
// compare of window base 0 with the read's first bases (the AND one base
// below position 0), of window base m-1 with the read's last bases (the AND
// one base above m-1, when m fills the words), and the correction words at
// both ends before they are limited to the positions of a shift count.
template <int NP>
struct FinishPrep {
  // The AND one base below position 0 is 1 at shift count K iff K < t0 (t0:
  // the number of trailing 1s of the compare of window base 0 with the
  // read's first bases); likewise above m-1 with tm.
  uint32_t t0[NP], tm[NP];
  uint32_t lx[NP], ly[NP];  // low end: bit p set where a correction clears position p (from mask p) / p+1 (mask p-1)
  uint32_t hx[NP], hy[NP];  // high end, mirrored (bit j: position m-1-j), bit-reversed; hy pre-shifted by 1
};

// The high-end words are kept bit-reversed, so that each finish reverses one
// mask instead of one word per pair.
template <int W, int NP>
__device__ __forceinline__ void deferred_prep(int j, uint32_t tail, uint32_t lastmask, const uint32_t (&rh)[W],
                                              const uint32_t (&rl)[W], const uint32_t (&gh)[NP][W],
                                              const uint32_t (&gl)[NP][W], FinishPrep<NP> &pr) {
  // The read's last 32 bases mirrored: bit j is position m-1-j (positions
  // below 0 read as code 00).  The high end's terms are the low end's
  // formulas on mirrored vectors, in 32-bit words.
  const uint32_t xrh = __funnelshift_rc(W >= 2 ? rh[W >= 2 ? W - 2 : 0] : 0u, rh[W - 1], tail);
  const uint32_t xrl = __funnelshift_rc(W >= 2 ? rl[W >= 2 ? W - 2 : 0] : 0u, rl[W - 1], tail);
  const uint32_t b0h = 0u - (xrh >> 31), b0l = 0u - (xrl >> 31);                // R[m-1]
  const uint32_t b1h = 0u - ((xrh >> 30) & 1u), b1l = 0u - ((xrl >> 30) & 1u);  // R[m-2]
  const uint32_t r0h = 0u - (rh[0] & 1u), r0l = 0u - (rl[0] & 1u);              // R[0]
  const uint32_t r1h = 0u - ((rh[0] >> 1) & 1u), r1l = 0u - ((rl[0] >> 1) & 1u);  // R[1]
  {
    // Window base 0 against R[i] (bit i), every non-positive shift.
    const uint32_t g0h = 0u - (gh[j][0] & 1u), g0l = 0u - (gl[j][0] & 1u);
    pr.t0[j] = __ffs(~((rh[0] ^ g0h) | (rl[0] ^ g0l))) - 1u;  // 0xFFFFFFFF (all 1s): every K
    // The window's last 32 bases mirrored.
    const uint32_t mgh = __brev(__funnelshift_rc(W >= 2 ? gh[j][W >= 2 ? W - 2 : 0] : 0u, gh[j][W - 1], tail));
    const uint32_t mgl = __brev(__funnelshift_rc(W >= 2 ? gl[j][W >= 2 ? W - 2 : 0] : 0u, gl[j][W - 1], tail));
    // Window base m-1 against R[m-1-i] (bit i), every non-negative shift;
    // used only when m fills the words.
    pr.tm[j] = 0u;
    if (tail == 32) {
      const uint32_t gmh = 0u - (mgh & 1u), gml = 0u - (mgl & 1u);
      pr.tm[j] = __ffs(~((__brev(xrh) ^ gmh) | (__brev(xrl) ^ gml))) - 1u;
    }
    {  // low end (positions 1..K+1, word 0)
      const uint32_t v0 = W == 1 ? lastmask : 0xffffffffu;
      const uint32_t a0 = (gh[j][0] ^ r0h) | (gl[j][0] ^ r0l);
      const uint32_t a1 = ((gh[j][0] ^ r1h) | (gl[j][0] ^ r1l)) & v0;
      const uint32_t vac = gh[j][0] | gl[j][0];
      const uint32_t c1 = (vac << 2) | (vac << 1) | a0;
      const uint32_t c2 = (vac << 1) | a0 | (a1 >> 1);
      pr.lx[j] = ~(c1 & c2);
      pr.ly[j] = ~c2 << 1;  // applied one position up
    }
    {  // high end (positions m-K-2..m-2), mirrored; kept bit-reversed
      const uint32_t a0 = (mgh ^ b0h) | (mgl ^ b0l);
      const uint32_t a1 = (mgh ^ b1h) | (mgl ^ b1l);
      const uint32_t vac = mgh | mgl;
      const uint32_t c1 = (vac << 2) | (vac << 1) | a0;
      const uint32_t c2 = (vac << 1) | a0 | (a1 >> 1);
      pr.hx[j] = __brev(~(c1 & c2));
      pr.hy[j] = __brev(~c2) >> 1;  // applied one position down (mirrored)
    }
  }
}

// The once-per-pair end of deferred_sweep_counts for shift count K: the
// AND's values one base outside each end, the erosion, the corrections next
// to the vacated runs and the count (acc is read, not changed), as at the end
// of deferred_counts.
template <int W, int NP>
__device__ __forceinline__ void deferred_finish(const FilterArgs &a, uint32_t K, uint32_t tail,
                                                uint32_t lastmask, const uint32_t (&acc)[NP][W],
                                                const FinishPrep<NP> &pr, uint32_t (&count)[NP]) {
  // ---- once per pair: end values of the AND, corrections, final erosion ----
  const uint32_t r1k = (2u << K) - 2u;  // bits 1..K
  const uint32_t r2k = r1k << 1;         // bits 2..K+1
  const uint32_t r1kr = __brev(r1k);     // bits 1..K, mirrored
  const uint32_t r2kr = r1kr >> 1;       // bits 2..K+1, mirrored
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    // AND one base below position 0 (every non-positive shift compares G[0]
    // with R[i], i = 0..K) and, when m fills the words, above m-1.
    const uint32_t lo0 = K < pr.t0[j] ? 0x80000000u : 0u;
    const uint32_t vtop = (tail == 32 && K < pr.tm[j]) ? 1u : 0u;
    uint32_t f[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t lo_in = w > 0 ? acc[j][w - 1] : lo0;
      const uint32_t hi_in = w + 1 < W ? acc[j][w + 1] : vtop;
      f[w] = acc[j][w] & __funnelshift_l(lo_in, acc[j][w], 1) & __funnelshift_r(acc[j][w], hi_in, 1);
    }
    // Low-end corrections (positions 1..K+1, word 0).
    f[0] &= ~((pr.lx[j] & r1k) | (pr.ly[j] & r2k));
    // High-end corrections (positions m-K-2..m-2), mapped back from the
    // mirrored words: bit b of nc is position m-32+b; the last word also
    // drops the positions past m.
    {
      const uint32_t nc = (pr.hx[j] & r1kr) | (pr.hy[j] & r2kr);
      f[W - 1] &= ~(nc >> (32u - tail)) & lastmask;
      if (W >= 2 && tail < 32) f[W >= 2 ? W - 2 : 0] &= ~(nc << tail);
    }

    uint32_t c = 0;
    if (a.count_mode == GK_COUNT_POPCOUNT) {
#pragma unroll
      for (int w = 0; w < W; ++w) c += __popc(f[w]);
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w) c += __popc(f[w] & ~((f[w] << 1) & 0xEEEEEEEEu));
    }
    count[j] = c;
  }
}

// Read and window planes of a loaded pair, zero past m.
template <int W>
__device__ __forceinline__ void pair_planes(const PairData<W> &x, uint32_t (&rh)[W], uint32_t (&rl)[W],
                                            uint32_t (&gh)[W], uint32_t (&gl)[W]) {
  const uint32_t tail = x.m - 32u * (W - 1);
  const uint32_t lastmask = tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u);
  const uint32_t sh = x.off & 31;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    rh[w] = x.r[w].x;
    rl[w] = x.r[w].y;
    gh[w] = __funnelshift_r(x.g[w].x, x.g[w + 1].x, sh);
    gl[w] = __funnelshift_r(x.g[w].y, x.g[w + 1].y, sh);
  }
  rh[W - 1] &= lastmask;
  rl[W - 1] &= lastmask;
  gh[W - 1] &= lastmask;
  gl[W - 1] &= lastmask;
}

template <int W, bool DIRECT = false>
__device__ __forceinline__ uint32_t filter_loaded_deferred(const FilterArgs &a, const PairData<W> &x) {
  uint32_t rh[W], rl[W], gh[1][W], gl[1][W], count[1];
  pair_planes<W>(x, rh, rl, gh[0], gl[0]);
  deferred_counts<W, 1, DIRECT>(a, x.m, min(x.e, x.m - 1), rh, rl, gh, gl, count);
  return count[0];
}

// Resident blocks per SM the compiler must allow.  One thread per pair:
// small reads keep enough registers free for 40 warps per SM, which hides
// the dependent loads of a pair (ids, then read and window words); W = 5 and
// 6 fit 4 and 3 blocks without spilling (at 150 bp, e = 0..2, 4 blocks run
// 9-18% faster than 2).  The compacting loop stages its words with cp.async
// and carries a chunk pipeline, so it keeps fewer resident warps.
template <int W, bool COMPACT>
struct MinBlocks {
  static constexpr int value =
      COMPACT ? (W <= 2 ? 5 : (W <= 4 ? 4 : (W <= 6 ? 3 : (W <= 8 ? 2 : 1))))
              : (W <= 2 ? 6 : (W <= 4 ? 5 : (W == 5 ? 4 : (W == 6 ? 3 : (W <= 8 ? 2 : 1)))));
};

// Status of a loaded pair: 0 filter, 1 undefined (N in read or window),
// 2 invalid.
template <int W>
__device__ __forceinline__ int pair_status(const FilterArgs &a, const PairData<W> &x) {
  int status = x.status;
  if (status == 0 && a.m > 0) {
    if (x.nflag) {
      status = 1;
    } else {
      const uint32_t q = x.ni.x >> (x.off & 31);
      const uint64_t first = q ? (uint64_t)x.off + (uint32_t)(__ffs(q) - 1) : (uint64_t)x.ni.y;
      if (first < (uint64_t)x.off + a.m) status = 1;
    }
  }
  return status;
}

// SWEEP (VARIANT 3): the outcome goes to the row of every threshold.
template <bool SWEEP = false>
__device__ __forceinline__ void write_trivial(const FilterArgs &a, uint64_t p, int status) {
  const uint32_t rows = SWEEP ? a.sweep_hi - a.fixed_e + 1 : 1;
  uint8_t *acc = a.accept + p;
  if (a.result_byte) {
    const uint8_t b = status == 0 ? 0 : (status == 1 ? GK_RESULT_UNDEFINED : GK_RESULT_INVALID);
    for (uint32_t i = 0; i < rows; ++i, acc += a.out_stride) *acc = b;
    return;
  }
  uint16_t *ed = a.edits + p;
  const uint8_t acc_v = status != 2;
  const uint16_t ed_v = status == 0 ? 0 : (status == 1 ? GK_EDITS_UNDEFINED : GK_EDITS_INVALID);
  for (uint32_t i = 0; i < rows; ++i, acc += a.out_stride, ed += a.out_stride) {
    *acc = acc_v;
    *ed = ed_v;
  }
}

// The result of a filtered pair: accept bit and count, or the result byte.
__device__ __forceinline__ void write_count(const FilterArgs &a, uint64_t p, uint32_t count, uint32_t e) {
  if (a.result_byte) {
    a.accept[p] = (uint8_t)min(count, GK_RESULT_MAX_COUNT);
    return;
  }
  a.accept[p] = count <= e;
  a.edits[p] = (uint16_t)count;
}

// Threshold sweep of one loaded pair (VARIANT 3): thresholds e = a.fixed_e ..
// a.sweep_hi have shift counts K = min(e, m-1); the shift loop runs once to
// the largest and the results of each K go to its rows (every e >= m-1
// shares K = m-1).
template <int W>
__device__ __forceinline__ void sweep_and_write(const FilterArgs &a, uint64_t p, const PairData<W> &x) {
  uint32_t rh[W], rl[W], gh[1][W], gl[1][W], count[1];
  pair_planes<W>(x, rh, rl, gh[0], gl[0]);
  const uint32_t e_lo = a.fixed_e, e_hi = a.sweep_hi, kmax = x.m - 1;
  const uint32_t Klo = min(e_lo, kmax), Khi = min(e_hi, kmax);
  // The common case (K in e_lo..e_hi, below m-1) writes one row: its
  // pointers advance by a row per shift count.
  uint8_t *acc_row = a.accept + p;
  uint16_t *ed_row = a.edits + p;
  deferred_sweep_counts<W, 1>(a, x.m, Khi, rh, rl, gh, gl, count, Klo, [&](uint32_t K, const uint32_t (&c)[1]) {
    if (!a.result_byte && K >= e_lo && K < kmax) {
      *acc_row = c[0] <= K;
      *ed_row = (uint16_t)c[0];
      acc_row += a.out_stride;
      ed_row += a.out_stride;
      return;
    }
    const uint32_t first = K > e_lo ? K : e_lo, last = K == kmax ? e_hi : K;
    for (uint32_t e = first; e <= last; ++e) write_count(a, p + (uint64_t)(e - e_lo) * a.out_stride, c[0], e);
  });
}

template <int W, int VARIANT>
__device__ __forceinline__ void filter_and_write(const FilterArgs &a, uint64_t p, const PairData<W> &x) {
  if constexpr (VARIANT == 3) {
    sweep_and_write<W>(a, p, x);
  } else {
    const uint32_t count = VARIANT == 4   ? filter_loaded_deferred<W, true>(a, x)
                           : VARIANT == 2 ? filter_loaded_deferred<W>(a, x)
                                          : filter_loaded<W, VARIANT == 1>(a, x);
    write_count(a, p, count, x.e);
  }
}

// The classify phase of the compacting loop, in two steps so that the loads
// of one chunk are in flight while the warp works on another.
// ChunkLoads holds one lane's pair of a chunk: its ids and, for a valid pair,
// the read's N flag and the N index word of its window (loaded together).
struct ChunkLoads {
  uint32_t rid, off;
  uint32_t nflag;
  uint2 ni;
  int state;  // -1 no pair, 2 invalid, 3 empty read, 0 defined unless N
};

__device__ __forceinline__ void chunk_issue(const FilterArgs &a, ChunkLoads &x) {
  x.nflag = 0;
  x.ni = make_uint2(0u, 0xffffffffu);
  if (x.state < 0) return;
  if ((uint64_t)x.rid >= a.n_reads || (uint64_t)x.off + a.m > a.ref_len) {
    x.state = 2;
  } else if (a.m == 0) {
    x.state = 3;
  } else {
    x.state = 0;
    if (a.read_nflag) x.nflag = a.read_nflag[x.rid];
    if (a.ref_nidx) x.ni = a.ref_nidx[x.off >> 5];
  }
}

// 0 filter, 1 undefined, 2 invalid, 3 empty read, -1 no pair.
__device__ __forceinline__ int chunk_status(const FilterArgs &a, const ChunkLoads &x) {
  if (x.state != 0) return x.state;
  if (x.nflag) return 1;
  const uint32_t q = x.ni.x >> (x.off & 31);
  const uint64_t first = q ? (uint64_t)x.off + (uint32_t)(__ffs(q) - 1) : (uint64_t)x.ni.y;
  return first < (uint64_t)x.off + a.m ? 1 : 0;
}

__device__ __forceinline__ void chunk_ids(const FilterArgs &a, uint64_t c, uint64_t n_chunks, int lane,
                                          uint32_t &rid, uint32_t &off, int &state) {
  const uint64_t p = c * 32 + lane;
  state = -1;
  if (c < n_chunks && p < a.n_pairs) {
    rid = a.pair_read[p];
    off = a.pair_off[p];
    state = 0;
  }
}

// 8-byte asynchronous global -> shared copy (bypasses registers) and its
// group fences.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kFilterWarps = kFilterThreads / 32;

// Words of one staged batch (32 pairs): W read words and W + 1 window words
// per pair, stored word-major ([word][lane]) so that lanes touch consecutive
// 8-byte slots.  Two batches per warp are staged at a time.
template <int W>
constexpr int kStageWords = (2 * W + 1) * 32;
template <int W>
constexpr size_t compact_smem_bytes() {
  return (size_t)kFilterWarps * 2 * kStageWords<W> * sizeof(uint2);
}

// VARIANT 0: any thresholds; 1: every shift count of the launch is < 32;
// 2: edge OR on and one threshold in 2..30, deferred erosion; 3: edge OR on,
// a sweep of thresholds up to 30, deferred erosion (sweep_and_write).
//
// COMPACT false: one thread per pair.  COMPACT true (inputs with many
// undefined pairs): persistent warps take 32 pairs at a time (their ids
// loaded one chunk ahead), write the trivial outcomes at once and queue the
// pairs that need filtering in a 64-slot per-warp shared queue.  Each full
// batch of 32 queued pairs has its read and window words copied into shared
// memory by cp.async while the warp filters the previous batch, so that no
// lane idles next to an undefined pair and the word loads of one batch hide
// behind the arithmetic of the other.  Dynamic shared memory:
// compact_smem_bytes<W>().
template <int W, int VARIANT, bool COMPACT>
__global__ void __launch_bounds__(kFilterThreads, MinBlocks<W, COMPACT>::value) filter_kernel(const FilterArgs a) {
  if (!COMPACT) {
    const uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool active = p < a.n_pairs;
    PairData<W> cur;
    cur.status = 0;
    if (active) load_pair<W>(a, p, cur);
    if (a.err_count) {
      const unsigned bad = __ballot_sync(0xffffffffu, active && cur.status == 2);
      if (bad && (threadIdx.x & 31) == 0) atomicAdd(a.err_count, (unsigned)__popc(bad));
    }
    if (!active) return;
    const int status = pair_status<W>(a, cur);
    if (status != 0 || a.m == 0) {
      write_trivial<VARIANT == 3>(a, p, status);
      return;
    }
    filter_and_write<W, VARIANT>(a, p, cur);
    return;
  }
  extern __shared__ uint2 stage_all[];
  __shared__ uint32_t q_p[kFilterWarps][64], q_rid[kFilterWarps][64], q_off[kFilterWarps][64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint2 *stage = stage_all + wib * 2 * kStageWords<W>;
  const uint64_t n_chunks = (a.n_pairs + 31) / 32;
  const uint64_t n_warps = (uint64_t)gridDim.x * kFilterWarps;
  uint64_t c = blockIdx.x * (uint64_t)kFilterWarps + wib;
  // Load pipeline over this warp's chunks.  Wide reads (W >= 7, registers to
  // spare) run it two deep: while the warp classifies chunk c and filters,
  // the N information of its next chunk and the ids of the chunk after are
  // in flight.  Narrower reads keep one deep (the ids of the next chunk), as
  // two deep spills registers there and measured slower at 150 bp.
  constexpr bool kDeep = W >= 7;
  ChunkLoads cur;
  cur.rid = cur.off = 0;
  chunk_ids(a, c, n_chunks, lane, cur.rid, cur.off, cur.state);
  uint32_t next_rid = 0, next_off = 0;
  int next_state = -1;
  if (kDeep) {
    chunk_issue(a, cur);
    chunk_ids(a, c + n_warps, n_chunks, lane, next_rid, next_off, next_state);
  }
  uint32_t qn = 0;         // warp-uniform queue length
  int pend = -1;           // stage buffer of the batch in flight, or none
  bool pend_has = false;   // this lane holds a pair of that batch
  uint32_t pend_p = 0, pend_off = 0, pend_e = 0;
  auto filter_staged = [&]() {
    if (!pend_has) return;
    const uint2 *sb = stage + pend * kStageWords<W>;
    PairData<W> x;
    x.m = a.m;
    x.off = pend_off;
    x.e = pend_e;
    x.status = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) x.r[w] = sb[w * 32 + lane];
#pragma unroll
    for (int w = 0; w <= W; ++w) x.g[w] = sb[(W + w) * 32 + lane];
    filter_and_write<W, VARIANT>(a, pend_p, x);
  };
  for (;; c += n_warps) {
    const bool more = c < n_chunks;
    if (more) {
      const uint64_t p = c * 32 + lane;
      const bool active = p < a.n_pairs;
      int status;
      const uint32_t rid = cur.rid, off = cur.off;
      if (kDeep) {
        status = chunk_status(a, cur);
        cur.rid = next_rid;
        cur.off = next_off;
        cur.state = next_state;
        chunk_issue(a, cur);
        chunk_ids(a, c + 2 * n_warps, n_chunks, lane, next_rid, next_off, next_state);
      } else {
        ChunkLoads x = cur;
        chunk_ids(a, c + n_warps, n_chunks, lane, cur.rid, cur.off, cur.state);
        chunk_issue(a, x);
        status = chunk_status(a, x);
      }
      if (a.err_count) {
        const unsigned bad = __ballot_sync(0xffffffffu, status == 2);
        if (bad && lane == 0) atomicAdd(a.err_count, (unsigned)__popc(bad));
      }
      if (status > 0 && active) write_trivial<VARIANT == 3>(a, p, status == 3 ? 0 : status);
      const unsigned need = __ballot_sync(0xffffffffu, status == 0);
      if ((need >> lane) & 1u) {
        const uint32_t slot = qn + __popc(need & ((1u << lane) - 1u));
        q_p[wib][slot] = (uint32_t)p;
        q_rid[wib][slot] = rid;
        q_off[wib][slot] = off;
      }
      qn += __popc(need);
      __syncwarp();
    }
    while (qn >= 32 || (!more && qn > 0)) {
      const uint32_t take = qn < 32 ? qn : 32;
      const bool has = (uint32_t)lane < take;
      const int nb = pend == 0 ? 1 : 0;
      uint32_t np = 0, noff = 0, ne = a.fixed_e;
      if (has) {
        const uint32_t i = qn - take + lane;
        np = q_p[wib][i];
        const uint32_t rid = q_rid[wib][i];
        noff = q_off[wib][i];
        // a queued pair is valid: its read row holds W words and its window
        // words off/32 .. off/32 + W lie inside the genome's n_words + 2
        const uint2 *rp = a.reads + (uint64_t)rid * a.stride_words;
        const uint2 *gp = a.ref_hl + (noff >> 5);
        uint2 *sb = stage + nb * kStageWords<W>;
#pragma unroll
        for (int w = 0; w < W; ++w) cp_async8(sb + w * 32 + lane, rp + w);
#pragma unroll
        for (int w = 0; w <= W; ++w) cp_async8(sb + (W + w) * 32 + lane, gp + w);
        if (a.pair_e) ne = a.pair_e[np];
      }
      cp_async_commit();
      __syncwarp();
      qn -= take;
      if (pend >= 0) {
        cp_async_wait<1>();  // the previous batch's copies have landed
        filter_staged();
      }
      pend = nb;
      pend_has = has;
      pend_p = np;
      pend_off = noff;
      pend_e = ne;
    }
    if (!more) break;
  }
  if (pend >= 0) {
    cp_async_wait<0>();
    filter_staged();
  }
}

// The two-pairs-per-thread kernel gathers in 8-byte loads except at a
// compile-time shift count 0: 16-byte loads (load_words_wide) measured 2-4%
// slower at every other shift count at 100 bp.
constexpr bool kPair2Wide = false;

// Resident blocks per SM of the two-pairs-per-thread kernel: 4 (64 registers,
// a few spilled) measured faster than 3 (80 registers, no spill) at every
// threshold 1..10 and in the 0..10 sweep at 100 bp on GB300 (e = 2: 53.3 ->
// 57.5 Gpairs/s; the sweep 1.307 -> 1.280 ms), the same at e = 0.
template <int W>
struct MinBlocks2 {
  static constexpr int value = 4;
};

// Deferred erosion (VARIANT 2, or the sweep, VARIANT 3), two pairs per
// thread: pairs 2t and 2t+1.  When both are filtered and share their read
// (the candidates of one read usually sit next to each other), the read is
// loaded once and its shifted copies serve both windows: a shift step costs
// about 13W integer operations per pair instead of 15W.  Otherwise each pair
// is filtered on its own.  VARIANT 4: one threshold whose shift count KC
// (0..2, below m) is a compile-time constant, so the shift steps unroll and
// the end corrections of K = 0 vanish.
template <int W, int VARIANT, int KC = -1>
__global__ void __launch_bounds__(kFilterThreads, MinBlocks2<W>::value) filter_pair2_kernel(const FilterArgs a) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t p0 = 2 * t, p1 = p0 + 1;
  const bool act0 = p0 < a.n_pairs, act1 = p1 < a.n_pairs;
  PairData<W> x0, x1;
  x0.status = x1.status = 0;
  // Shift count 0: read and window in 16-byte loads (e0 82.3 -> 85.4 Gpairs/s
  // at 100 bp); 1 and 2: the window's last word loaded only when the window
  // reaches into it (e1 68.2 -> 70.1, e2 58.7 -> 59.4); each measured slower
  // with the other's choice.
  constexpr bool kWide = kPair2Wide || KC == 0, kSkipLast = KC >= 1;
  if (act0) load_pair<W, kWide, kSkipLast>(a, p0, x0);
  if (act1) load_pair<W, kWide, kSkipLast>(a, p1, x1, act0 ? &x0 : nullptr);
  if (a.err_count) {
    const unsigned b0 = __ballot_sync(0xffffffffu, act0 && x0.status == 2);
    const unsigned b1 = __ballot_sync(0xffffffffu, act1 && x1.status == 2);
    if ((b0 | b1) && (threadIdx.x & 31) == 0) atomicAdd(a.err_count, (unsigned)(__popc(b0) + __popc(b1)));
  }
  const int s0 = act0 ? pair_status<W>(a, x0) : -1;
  const int s1 = act1 ? pair_status<W>(a, x1) : -1;
  if (s0 > 0) write_trivial<VARIANT == 3>(a, p0, s0);
  if (s1 > 0) write_trivial<VARIANT == 3>(a, p1, s1);
  if (s0 == 0 && s1 == 0 && x0.rid == x1.rid) {
    uint32_t rh[W], rl[W], gh[2][W], gl[2][W], count[2];
    pair_planes<W>(x0, rh, rl, gh[0], gl[0]);
    {
      const uint32_t tail = a.m - 32u * (W - 1);
      const uint32_t lastmask = tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u);
      const uint32_t sh = x1.off & 31;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        gh[1][w] = __funnelshift_r(x1.g[w].x, x1.g[w + 1].x, sh);
        gl[1][w] = __funnelshift_r(x1.g[w].y, x1.g[w + 1].y, sh);
      }
      gh[1][W - 1] &= lastmask;
      gl[1][W - 1] &= lastmask;
    }
    if constexpr (VARIANT == 3) {
      const uint32_t e_lo = a.fixed_e, e_hi = a.sweep_hi, kmax = a.m - 1;
      // Pairs 2t and 2t+1 are adjacent in every row: one 2-byte and one
      // 4-byte store per threshold when the rows keep that alignment.
      const bool pack = (((uintptr_t)a.accept | (a.result_byte ? 0u : (uintptr_t)a.edits)) & 3u) == 0 &&
                        (a.out_stride & 1u) == 0;
      // The common case (K in e_lo..e_hi, below m-1) writes one row: its
      // accept and count pointers advance by a row per shift count.
      uint8_t *acc_row = a.accept + p0;
      uint16_t *ed_row = a.edits + p0;
      deferred_sweep_counts<W, 2>(a, a.m, min(e_hi, kmax), rh, rl, gh, gl, count, min(e_lo, kmax),
                                  [&](uint32_t K, const uint32_t (&c)[2]) {
                                    if (pack && !a.result_byte && K >= e_lo && K < kmax) {
                                      *reinterpret_cast<uint32_t *>(ed_row) = c[0] | (c[1] << 16);
                                      *reinterpret_cast<uint16_t *>(acc_row) =
                                          (uint16_t)((c[0] <= K ? 1u : 0u) | (c[1] <= K ? 0x100u : 0u));
                                      acc_row += a.out_stride;
                                      ed_row += a.out_stride;
                                      return;
                                    }
                                    const uint32_t first = K > e_lo ? K : e_lo, last = K == kmax ? e_hi : K;
                                    for (uint32_t e = first; e <= last; ++e) {
                                      const uint64_t o = (uint64_t)(e - e_lo) * a.out_stride;
                                      if (pack) {
                                        uint32_t b0, b1;
                                        if (a.result_byte) {
                                          b0 = min(c[0], GK_RESULT_MAX_COUNT);
                                          b1 = min(c[1], GK_RESULT_MAX_COUNT);
                                        } else {
                                          b0 = c[0] <= e;
                                          b1 = c[1] <= e;
                                          *reinterpret_cast<uint32_t *>(a.edits + o + p0) = c[0] | (c[1] << 16);
                                        }
                                        *reinterpret_cast<uint16_t *>(a.accept + o + p0) = (uint16_t)(b0 | (b1 << 8));
                                      } else {
                                        write_count(a, p0 + o, c[0], e);
                                        write_count(a, p1 + o, c[1], e);
                                      }
                                    }
                                  });
    } else {
      const uint32_t K = KC >= 0 ? (uint32_t)KC : min(a.fixed_e, a.m - 1);
      deferred_counts<W, 2, (KC >= 0)>(a, a.m, K, rh, rl, gh, gl, count);
      // The two pairs are adjacent: one 2-byte accept store and one 4-byte
      // count store when the buffers allow it.
      if (!a.result_byte && ((uintptr_t)a.accept & 1u) == 0 && ((uintptr_t)a.edits & 3u) == 0) {
        const uint32_t e = a.fixed_e;
        *reinterpret_cast<uint32_t *>(a.edits + p0) = count[0] | (count[1] << 16);
        *reinterpret_cast<uint16_t *>(a.accept + p0) =
            (uint16_t)((count[0] <= e ? 1u : 0u) | (count[1] <= e ? 0x100u : 0u));
      } else {
        write_count(a, p0, count[0], a.fixed_e);
        write_count(a, p1, count[1], a.fixed_e);
      }
    }
  } else {
    if (s0 == 0) filter_and_write<W, VARIANT>(a, p0, x0);
    if (s1 == 0) filter_and_write<W, VARIANT>(a, p1, x1);
  }
}

// Launches one instantiation of the plain filter over a.n_pairs pairs.
template <int W, int VARIANT>
cudaError_t launch_filter_variant(const FilterArgs &a, cudaStream_t stream) {
  unsigned blocks = (unsigned)((a.n_pairs + kFilterThreads - 1) / kFilterThreads);
  if (a.compact == 0) {
    // Two pairs per thread for W <= 4 only: at W = 5 (2 blocks per SM with
    // its registers unspilled) it measured 40% slower at e = 2, 150 bp.
    if constexpr ((VARIANT == 2 || VARIANT == 3 || VARIANT == 4) && W <= 4) {
      if (a.m > 0) {
        const uint64_t threads = (a.n_pairs + 1) / 2;
        const unsigned grid = (unsigned)((threads + kFilterThreads - 1) / kFilterThreads);
        if constexpr (VARIANT == 4) {
          // shift count = the threshold, 0..2, below m (checked by the caller)
          switch (a.fixed_e) {
            case 0: filter_pair2_kernel<W, 4, 0><<<grid, kFilterThreads, 0, stream>>>(a); break;
            case 1: filter_pair2_kernel<W, 4, 1><<<grid, kFilterThreads, 0, stream>>>(a); break;
            case 2: filter_pair2_kernel<W, 4, 2><<<grid, kFilterThreads, 0, stream>>>(a); break;
            default: return cudaErrorInvalidValue;
          }
        } else {
          filter_pair2_kernel<W, VARIANT><<<grid, kFilterThreads, 0, stream>>>(a);
        }
        return cudaGetLastError();
      }
    }
    if constexpr (VARIANT == 4) {
      return cudaErrorInvalidValue;  // VARIANT 4 is the two-pair kernel only
    } else {
      filter_kernel<W, VARIANT, false><<<blocks, kFilterThreads, 0, stream>>>(a);
      return cudaGetLastError();
    }
  }
  if constexpr (VARIANT == 4) {
    return cudaErrorInvalidValue;
  } else {
  // Persistent warps: a few waves of resident blocks.  The dynamic shared
  // memory limit and the occupancy are set up once per device (threads that
  // race here repeat the same idempotent setup; the block count is
  // published after the SM count).
  constexpr int kMaxDev = 64;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  static std::atomic<int> per_sm[kMaxDev], sms[kMaxDev];
  const size_t smem = compact_smem_bytes<W>();
  int blocks_per_sm = per_sm[dev].load(std::memory_order_acquire);
  if (blocks_per_sm == 0) {
    err = cudaFuncSetAttribute(filter_kernel<W, VARIANT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    int count = 0;
    err = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    int n = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, filter_kernel<W, VARIANT, true>, kFilterThreads, smem);
    if (err != cudaSuccess) return err;
    blocks_per_sm = n < 1 ? 1 : n;
    sms[dev].store(count, std::memory_order_relaxed);
    per_sm[dev].store(blocks_per_sm, std::memory_order_release);
  }
  const uint64_t wave = 4ull * (uint64_t)sms[dev].load(std::memory_order_relaxed) * (uint64_t)blocks_per_sm;
  if (blocks > wave) blocks = (unsigned)wave;
  filter_kernel<W, VARIANT, true><<<blocks, kFilterThreads, smem, stream>>>(a);
  return cudaGetLastError();
  }
}

}  // namespace gk
