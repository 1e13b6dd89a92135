// Bit-sliced form of the filter: 32 pairs per 32-bit word.
//
// The per-pair kernels hold a pair's masks as W words of 32 positions and
// pay, per shift step and word, funnel shifts for the read copies and for
// the dilation.  Here the bits of a word are 32 pairs instead ("a group"),
// and one word per base position holds that position of every pair of the
// group.  A shift by s bases is then a choice of register, not an
// instruction, and every mask costs four logic operations per position for
// 32 pairs: the difference (Sec. 2.1: high XOR, low XOR, OR), the AND of its
// dilation into the running vector and the carried OR for the next dilation.
//
// Two passes:
//   slice   once per batch of pairs, threshold-independent like the
//           encoding: gathers each group's read words and genome window
//           (funnel-shifted to the candidate offset) and transposes them
//           into position-major planes;
//   filter  once per threshold, or once per range of thresholds (a
//           sweep): streams the positions of a group in order, keeping the
//           read positions q-K .. q+K in a register ring.
//
// What is computed is the deferred-erosion form of the per-pair kernels
// (filter.cuh), restated per position: the AND over the 2K+1 masks of the
// dilated difference vectors, the vacated positions of each shifted mask set
// to 1 before the dilation (Sec. 3.4), one erosion of the AND, and the
// corrections at the two positions next to each vacated run, which depend on
// the read's first and last two bases and on which window bases are 'A'.
// Outside [0, m) a difference is 0, except for the -k masks past the read's
// end, which are vacated (1); the AND one base below position 0 and one base
// above m-1 then come out of the same recurrence.  The count is the windowed
// run count or the popcount of the eroded vector (Sec. 2.1).
//
// Layout of a sliced batch of n pairs and read length m, with
// G = ceil(n/32) groups and a pitch of G rounded up to 32 (uint2 = {high
// plane, low plane}, bit j of a word = pair 32g + j):
//   rs[q * pitch + g]   read position q of group g, q < m
//   gs[q * pitch + g]   window position q of group g, q < m
//   st[g]               {undefined pairs, invalid pairs} of group g
// in one buffer: rs and gs each with kSlicedPad rows past m (never
// written; the filter's prefetch reads them and discards what it reads),
// then st, then a 16-byte header {magic, m, n_pairs} that the filter checks
// against its arguments; (2(m + kSlicedPad) + 1) * pitch * 8 + 16 bytes.
#pragma once

#include "gk_internal.cuh"

namespace gk {

constexpr int kSliceThreads = 128;   // slice: four lanes per group, 32 groups per block
constexpr int kSlicedThreads = 128;  // filter: one thread per group
constexpr int kSlicedMaxK = (int)GK_SLICED_MAX_SHIFT;  // largest shift count with a compiled filter
constexpr uint32_t kSlicedMaxLen = GK_SLICED_MAX_LEN;
// Rows past m in each plane array: the ring's prefetch reads up to row
// m - 1 + (L - K - 1), at most m + 23 (K = 15: L = 40).
constexpr uint32_t kSlicedPad = 24;

__host__ __device__ __forceinline__ uint64_t sliced_groups(uint64_t n_pairs) { return (n_pairs + 31) / 32; }
__host__ __device__ __forceinline__ uint64_t sliced_pitch(uint64_t n_pairs) {
  return (sliced_groups(n_pairs) + 31) / 32 * 32;
}
__host__ __device__ __forceinline__ uint64_t sliced_bytes(uint64_t n_pairs, uint32_t m) {
  return (2ull * (m + kSlicedPad) + 1) * sliced_pitch(n_pairs) * 8ull + 16ull;
}

// ---- portable forms of the few intrinsics (host: a CPU check of this code) ----

__host__ __device__ __forceinline__ uint32_t bperm(uint32_t x, uint32_t y, uint32_t s) {
#ifdef __CUDA_ARCH__
  return __byte_perm(x, y, s);
#else
  const uint64_t v = ((uint64_t)y << 32) | x;
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((s >> (4 * i)) & 7))) & 0xFFu) << (8 * i);
  return r;
#endif
}

__host__ __device__ __forceinline__ uint32_t fshr(uint32_t lo, uint32_t hi, uint32_t sh) {
#ifdef __CUDA_ARCH__
  return __funnelshift_r(lo, hi, sh);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> (sh & 31));
#endif
}

__host__ __device__ __forceinline__ int ffs32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __ffs(x);
#else
  return __builtin_ffs((int)x);
#endif
}

// Per byte: 0xFF where a <= b, else 0.
__host__ __device__ __forceinline__ uint32_t cmple4(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __vcmpleu4(a, b);
#else
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) r |= (((a >> (8 * i)) & 0xFFu) <= ((b >> (8 * i)) & 0xFFu) ? 0xFFu : 0u) << (8 * i);
  return r;
#endif
}

__host__ __device__ __forceinline__ uint32_t min4(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __vminu4(a, b);
#else
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) {
    const uint32_t x = (a >> (8 * i)) & 0xFFu, y = (b >> (8 * i)) & 0xFFu;
    r |= (x < y ? x : y) << (8 * i);
  }
  return r;
#endif
}

__host__ __device__ __forceinline__ uint32_t popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__popc(x);
#else
  return (uint32_t)__builtin_popcount(x);
#endif
}

template <typename T>
__host__ __device__ __forceinline__ T ldro(const T *p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// ---- slice ----------------------------------------------------------------

struct SliceArgs {
  const uint2 *ref_hl;
  const uint2 *ref_nidx;  // nullable
  uint64_t ref_len;
  const uint2 *reads;
  uint32_t stride_words;
  uint64_t n_reads;
  const uint8_t *read_nflag;  // nullable
  uint32_t m;                 // 1..kSlicedMaxLen
  const uint32_t *pair_read;
  const uint32_t *pair_off;
  uint64_t n_pairs;
  uint64_t pitch;
  uint2 *rs, *gs, *st;
  uint4 *hdr;
};

// ---- filter -----------------------------------------------------------------

// Header written by the slice past the status words, {kSlicedMagic, m,
// n_pairs low, n_pairs high}: a filter launch whose arguments do not match
// it (a buffer sliced for another batch) writes the invalid sentinel for
// every pair instead of reading the planes at a wrong pitch.
constexpr uint32_t kSlicedMagic = 0x534B4731u;

struct SlicedArgs {
  const uint2 *rs, *gs, *st;
  const uint4 *hdr;
  uint64_t pitch;
  uint64_t n_pairs;
  uint32_t m;
  // Results are written for the shift counts K = k_first .. k_last (inside
  // the kernel's compiled range KLO..KHI); the threshold of K is
  // e + (K - k_first) and its results start (K - k_first) * out_stride
  // elements after accept / edits.  One threshold: k_first = k_last =
  // min(e, m-1).
  uint32_t e;
  uint32_t k_first, k_last;
  uint64_t out_stride;
  uint32_t runs4;    // 1: windowed run count, 0: popcount
  int result_byte;
  int vec_out;       // every result row 16-byte aligned: vector stores
  uint8_t *accept;
  uint16_t *edits;
  uint32_t *err_count;  // nullable: pairs of groups whose header does not match
};

// Register ring of the read positions: L slots (a multiple of 8, at least
// 2K+4), the read position q + K + D loaded while position q is filtered.
template <int K>
struct SlicedRing {
  static constexpr int L = (2 * K + 4 <= 16) ? 16 : ((2 * K + 4 + 7) / 8) * 8;
  static constexpr int D = L - 2 * K - 1;  // prefetch distance, >= 3
  static_assert(K + D <= (int)kSlicedPad, "the prefetch stays inside the padding rows");
};

// Positions per unrolled loop body.  The body indexes the ring with
// constants, so one ring period (L positions) is the natural unit; with a
// large period the warps stall on instruction fetch, and a body of 8
// positions that rotates the ring registers by 8 slots afterwards (3L moves,
// 9-15 per position) can run faster.  Which is faster was measured on GB300
// (20M pairs at 100 bp, 10M at 150 and 250 bp), and the rule follows it:
//   sweep of shift counts 6..10 (L = 24): rotate (0.60 against 0.75 ms at
//     100 bp, 0.48 / 0.60 at 150, 0.68 / 0.76 at 250);
//   sweep 0..5 (L = 16) and one shift count up to 10: one period (rotating
//     lost 0-18%);
//   one shift count 11..14 (L = 32): rotate at 100 bp (0.46-0.59 against
//     0.49-0.61 ms), one period at 150 and 250 bp (rotating lost 15-27%);
//   one shift count 15 (L = 40): rotate (0.60 / 0.96 at 100 bp, 0.45 / 0.52
//     at 150, 0.74 / 0.93 at 250).
template <int KLO, int KHI, int M>
struct SlicedBody {
  static constexpr int L = SlicedRing<KHI>::L;
  static constexpr bool rotate = KLO < KHI ? KHI >= 6 : (KHI >= 15 || (KHI >= 11 && M == 100));
  static constexpr int U = rotate ? 8 : L;
  static_assert(L % U == 0, "a chunk divides the ring period");
};

// Bit planes of count / 8 a group needs: the count is at most m (popcount;
// the windowed run count is at most m/2 + 2).
__host__ __device__ constexpr int sliced_count_planes(int M) {
  int v = (M > 0 ? M : (int)kSlicedMaxLen) / 8, b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b > 0 ? b : 1;
}

__host__ __device__ __forceinline__ void csa(uint32_t &acc, uint32_t x, uint32_t y, uint32_t &carry) {
  carry = (acc & x) | (acc & y) | (x & y);
  acc = acc ^ x ^ y;
}

__host__ __device__ __forceinline__ void add_plane(uint32_t (&c)[8], int w, uint32_t x) {
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < w) continue;
    const uint32_t t = c[b] & x;
    c[b] ^= x;
    x = t;
  }
}

// Writes the 32 results of group g (nvalid of them real pairs) from the
// count planes C (bit b of pair j: C[b] bit j), the status words and the
// threshold e: accept bytes + 16-bit counts, or result bytes.
__host__ __device__ __forceinline__ void sliced_store(const SlicedArgs &a, uint64_t pbase, uint32_t nvalid,
                                                      const uint32_t (&C)[8], uint2 stw, uint32_t e,
                                                      uint8_t *acc_out, uint16_t *ed_out) {
  const uint32_t e4 = (e > 255u ? 255u : e) * 0x01010101u;
  uint32_t outA[8], outE[16];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    uint32_t c4 = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) c4 |= ((((C[b] >> (4 * t)) & 0xFu) * 0x00204081u) & 0x01010101u) << b;
    const uint32_t um = ((((stw.x >> (4 * t)) & 0xFu) * 0x00204081u) & 0x01010101u) * 0xFFu;
    const uint32_t im = ((((stw.y >> (4 * t)) & 0xFu) * 0x00204081u) & 0x01010101u) * 0xFFu;
    if (a.result_byte) {
      const uint32_t r = min4(c4, GK_RESULT_MAX_COUNT * 0x01010101u);
      outA[t] = (r & ~(um | im)) | (um & (GK_RESULT_UNDEFINED * 0x01010101u)) | (im & (GK_RESULT_INVALID * 0x01010101u));
      outE[2 * t] = outE[2 * t + 1] = 0u;
    } else {
      const uint32_t acc4 = cmple4(c4, e4) & 0x01010101u;
      outA[t] = (acc4 & ~(um | im)) | (um & 0x01010101u);
      uint32_t lo = bperm(c4, 0u, 0x4140), hi = bperm(c4, 0u, 0x4342);
      const uint32_t ul = bperm(um, 0u, 0x1100), uh = bperm(um, 0u, 0x3322);
      const uint32_t il = bperm(im, 0u, 0x1100), ih = bperm(im, 0u, 0x3322);
      constexpr uint32_t kInv2 = GK_EDITS_INVALID * 0x00010001u;
      outE[2 * t] = (lo & ~(ul | il)) | ul | (il & kInv2);
      outE[2 * t + 1] = (hi & ~(uh | ih)) | uh | (ih & kInv2);
    }
  }
  if (nvalid == 32 && a.vec_out) {
    uint4 *pa = reinterpret_cast<uint4 *>(acc_out + pbase);
    pa[0] = make_uint4(outA[0], outA[1], outA[2], outA[3]);
    pa[1] = make_uint4(outA[4], outA[5], outA[6], outA[7]);
    if (!a.result_byte) {
      uint4 *pe = reinterpret_cast<uint4 *>(ed_out + pbase);
#pragma unroll
      for (int k = 0; k < 4; ++k) pe[k] = make_uint4(outE[4 * k], outE[4 * k + 1], outE[4 * k + 2], outE[4 * k + 3]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if ((uint32_t)j < nvalid) {
        acc_out[pbase + j] = (uint8_t)(outA[j >> 2] >> (8 * (j & 3)));
        if (!a.result_byte) ed_out[pbase + j] = (uint16_t)(outE[j >> 1] >> (16 * (j & 1)));
      }
    }
  }
}

// Correction words per end of a group for shift counts KLO..KHI.
template <int KLO, int KHI>
struct SlicedCorr {
  static constexpr int NZ = KHI;            // Z(p), p = 1..KHI
  static constexpr int NY = KHI - KLO + 1;  // Y(p), p = KLO+1..KHI+1
  static constexpr int words = 2 * (NZ + NY);
};

// Filters group g at every shift count K = KLO..KHI in one pass over its
// positions (a threshold sweep, Sec. 4: the 2K+1 masks of K are those of K-1
// and the two shifted by K, so the running AND of K is the one of K-1 ANDed
// with two more dilated masks), and writes the results of K = a.k_first ..
// a.k_last.  KLO == KHI is the filter at one threshold.
//
// clr: SlicedCorr<KLO, KHI>::words words at stride clr_stride, the end
// corrections.  At a position p next to a vacated run the true erosion of a
// shifted mask needs dilation bits that setting the vacated bits hid: the
// correction of K at p (1 <= p <= K+1) is Z(p) = X(p) | Y(p) for p <= K and
// Y(K+1) at p = K+1, where X(p) is the contribution of the mask shifted by p
// and Y(p) the one of the mask shifted by p-1; mirrored at the read's end.
//
// M > 0: the read length is M (a.m == M), known at compile time, so the
// positions run as whole ring periods and a fixed tail with no test per
// position.  M == 0: any length, with a test per position.
template <int KLO, int KHI, int M>
__host__ __device__ __forceinline__ void sliced_sweep_group(const SlicedArgs &a, uint64_t g, uint32_t *clr,
                                                            int clr_stride) {
  static_assert(0 <= KLO && KLO <= KHI, "shift count range");
  constexpr int L = SlicedRing<KHI>::L, D = SlicedRing<KHI>::D, NS = 2 * KHI + 1, NK = KHI - KLO + 1;
  constexpr int NZ = SlicedCorr<KLO, KHI>::NZ, NY = SlicedCorr<KLO, KHI>::NY;
  constexpr int NB = sliced_count_planes(M);
  const uint32_t m = M > 0 ? (uint32_t)M : a.m;
  const uint64_t P = a.pitch;
  const uint2 *rp = a.rs + g, *gp = a.gs + g;
  const uint2 z2 = make_uint2(0u, 0u);
  auto Rq = [&](int64_t q) -> uint2 { return (q >= 0 && q < (int64_t)m) ? ldro(rp + q * (int64_t)P) : z2; };
  auto Gq = [&](int64_t q) -> uint2 { return (q >= 0 && q < (int64_t)m) ? ldro(gp + q * (int64_t)P) : z2; };
  auto diff = [](uint2 x, uint2 y) -> uint32_t { return (x.x ^ y.x) | (x.y ^ y.y); };
  auto vacv = [](uint2 x) -> uint32_t { return x.x | x.y; };  // window base other than 'A'
  const uint64_t pbase = g * 32ull;
  const uint64_t left = a.n_pairs - pbase;
  const uint32_t nvalid = left < 32 ? (uint32_t)left : 32u;

  // ---- a buffer sliced for other arguments: every pair invalid ----
  {
    const uint4 h = ldro(a.hdr);
    if (h.x != kSlicedMagic || h.y != a.m || h.z != (uint32_t)a.n_pairs || h.w != (uint32_t)(a.n_pairs >> 32)) {
      uint32_t C[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) C[b] = 0u;
      const uint2 bad = make_uint2(0u, 0xffffffffu);
#pragma unroll
      for (int t = 0; t < NK; ++t) {
        const uint32_t K = (uint32_t)(KLO + t);
        if (K < a.k_first || K > a.k_last) continue;
        const uint64_t o = (uint64_t)(K - a.k_first) * a.out_stride;
        sliced_store(a, pbase, nvalid, C, bad, a.e + (K - a.k_first), a.accept + o,
                     a.result_byte ? nullptr : a.edits + o);
      }
#ifdef __CUDA_ARCH__
      if (a.err_count) atomicAdd(a.err_count, nvalid);
#endif
      return;
    }
  }

  // ---- end corrections (positions 1..KHI+1 and m-KHI-2..m-2) ----
  {
    const uint2 R0 = Rq(0), R1 = Rq(1), Rm1 = Rq((int64_t)m - 1), Rm2 = Rq((int64_t)m - 2);
    uint2 gl[KHI + 3];  // window positions 0 .. KHI+2
#pragma unroll
    for (int t = 0; t < KHI + 3; ++t) gl[t] = Gq(t);
    auto vlo = [&](int q) -> uint32_t { return q < 0 ? 0u : vacv(gl[q]); };
    auto a0 = [&](int q) -> uint32_t { return diff(gl[q], R0); };
    auto a1 = [&](int q) -> uint32_t { return (q < (int)m && q < 32) ? diff(gl[q], R1) : 0u; };
    auto c1 = [&](int q) -> uint32_t { return vlo(q - 2) | vlo(q - 1) | a0(q); };
    auto c2 = [&](int q) -> uint32_t { return vlo(q - 1) | a0(q) | a1(q + 1); };
    auto Y = [&](int p) -> uint32_t { return p >= 2 ? ~c2(p - 1) : 0u; };
#pragma unroll
    for (int p = 1; p <= KHI; ++p) clr[(p - 1) * clr_stride] = ~(c1(p) & c2(p)) | Y(p);
#pragma unroll
    for (int p = KLO + 1; p <= KHI + 1; ++p) clr[(NZ + p - KLO - 1) * clr_stride] = Y(p);
    // Mirrored about the read's end: j <-> position m-1-j.
    const int64_t hb = (int64_t)m - KHI - 3;
    uint2 gh[KHI + 4];  // window positions m-KHI-3 .. m
#pragma unroll
    for (int t = 0; t < KHI + 4; ++t) gh[t] = Gq(hb + t);
    auto G_of = [&](int j) -> uint2 { return gh[KHI + 2 - j]; };  // position m-1-j, j in -1 .. KHI+2
    auto vm = [&](int j) -> uint32_t { return vacv(G_of(j)); };
    auto a0m = [&](int j) -> uint32_t { return diff(G_of(j), Rm1); };
    auto a1m = [&](int j) -> uint32_t { return j < 32 ? diff(G_of(j), Rm2) : 0u; };
    auto c1m = [&](int j) -> uint32_t { return vm(j - 2) | vm(j - 1) | a0m(j); };
    auto c2m = [&](int j) -> uint32_t { return vm(j - 1) | a0m(j) | a1m(j + 1); };
    auto Ym = [&](int j) -> uint32_t { return j >= 2 ? ~c2m(j - 1) : 0u; };
    uint32_t *clh = clr + (NZ + NY) * clr_stride;
#pragma unroll
    for (int j = 1; j <= KHI; ++j) clh[(j - 1) * clr_stride] = ((int)m - 1 - j >= 0) ? (~(c1m(j) & c2m(j)) | Ym(j)) : 0u;
#pragma unroll
    for (int j = KLO + 1; j <= KHI + 1; ++j)
      clh[(NZ + j - KLO - 1) * clr_stride] = ((int)m - 1 - j >= 0) ? Ym(j) : 0u;
  }

  // ---- ring of read positions; slot of position r is r mod L ----
  uint32_t rh[L], rl[L], rx[L];  // rx: 1s where the position lies outside the read (vacated)
#pragma unroll
  for (int r = -KHI; r < KHI + D; ++r) {
    const int s = ((r % L) + L) % L;
    const uint2 v = Rq(r);
    rh[s] = v.x;
    rl[s] = v.y;
    rx[s] = (r >= 0 && r < (int)m) ? 0u : 0xffffffffu;
  }
  uint32_t wh[8], wl[8];  // window positions q .. q+7, slot q mod 8
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    const uint2 v = Gq(t);
    wh[t] = v.x;
    wl[t] = v.y;
  }
  const uint2 *rload = rp + (uint64_t)(KHI + D) * P;
  const uint2 *gload = gp + 7ull * P;

  uint32_t u[NS], dp[NS];  // per mask: d(q-2) | d(q-1), d(q-1)
#pragma unroll
  for (int i = 0; i < NS; ++i) u[i] = dp[i] = 0u;
  // Per shift count: acc(q-2); acc(q-3) & acc(q-2); f(p-1); the carry-save count.
  uint32_t aprev[NK], v[NK], fprev[NK], A0[NK], A1[NK], A2[NK], xa[NK], c1a[NK], c2a[NK], B[NK][NB];
#pragma unroll
  for (int t = 0; t < NK; ++t) {
    aprev[t] = v[t] = fprev[t] = A0[t] = A1[t] = A2[t] = xa[t] = c1a[t] = c2a[t] = 0u;
#pragma unroll
    for (int b = 0; b < NB; ++b) B[t][b] = 0u;
  }
  const uint32_t runs = a.runs4 ? 0xffffffffu : 0u;

  // Positions q0 .. q0+L-1 with an end correction (q in 3..KHI+3, the low
  // corrections at p = q-2 in 1..KHI+1, or q in m-KHI..m-1, the high ones):
  // one bit per position, so the other positions pay one bit test.
  static_assert(L <= 64, "one correction bit per position of a ring period");
  auto corr_bits = [&](uint32_t q0) -> uint64_t {
    auto range = [](int lo, int hi) -> uint64_t {
      lo = lo < 0 ? 0 : lo;
      hi = hi > L - 1 ? L - 1 : hi;
      if (hi < lo) return 0ull;
      return (hi == 63 ? ~0ull : ((2ull << hi) - 1ull)) & ~((1ull << lo) - 1ull);
    };
    return range(3 - (int)q0, KHI + 3 - (int)q0) | range((int)m - KHI - (int)q0, (int)m - 1 - (int)q0);
  };
  // The corrections of every shift count at p: Z(p) for K >= p, Y(p) for
  // K = p-1, at both ends.
  auto correct = [&](int p, uint32_t (&f)[NK]) {
    const bool zl = p >= 1 && p <= KHI, yl = p >= KLO + 1 && p <= KHI + 1;
    const uint32_t zlo = zl ? clr[(p - 1) * clr_stride] : 0u;
    const uint32_t ylo = yl ? clr[(NZ + p - KLO - 1) * clr_stride] : 0u;
    const int jj = (int)m - 1 - p;
    const uint32_t *clh = clr + (NZ + NY) * clr_stride;
    const bool zh = jj >= 1 && jj <= KHI, yh = jj >= KLO + 1 && jj <= KHI + 1;
    const uint32_t zhi = zh ? clh[(jj - 1) * clr_stride] : 0u;
    const uint32_t yhi = yh ? clh[(NZ + jj - KLO - 1) * clr_stride] : 0u;
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      const int K = KLO + t;
      const uint32_t cl = (p <= K) ? zlo : (p == K + 1 ? ylo : 0u);
      const uint32_t ch = (jj <= K) ? zhi : (jj == K + 1 ? yhi : 0u);
      f[t] &= ~(cl | ch);
    }
  };
  uint64_t cm = 0;
  // One position: q runs, j = q mod L is a constant after unrolling.
  auto step = [&](uint32_t q, int j) {
    // Read position q + KHI + D into the slot position q - KHI - 1 leaves,
    // and window position q + 7.  Past m the rows are padding: the shift
    // counts whose launches wait on memory (KHI <= 3) skip those loads, the
    // others read them unconditionally (the vacated flag masks the read;
    // window positions past m-1 are never used).
    {
      const int s = (j + KHI + D) % L;
      const bool in = q + KHI + D < m;
      const uint2 vv = (KHI > 3 || in) ? ldro(rload) : z2;
      rh[s] = vv.x;
      rl[s] = vv.y;
      rx[s] = in ? 0u : 0xffffffffu;
      rload += P;
    }
    {
      const int s = (j + 7) % 8;
      const uint2 vv = (KHI > 3 || q + 7 < m) ? ldro(gload) : z2;
      wh[s] = vv.x;
      wl[s] = vv.y;
      gload += P;
    }
    const uint32_t GH = wh[j % 8], GL = wl[j % 8];
    // The running AND over the masks |s| <= k, k = 0..KHI (acc(q-1) of K = k).
    uint32_t accn[NK];
    uint32_t run = 0xffffffffu;
#pragma unroll
    for (int k = 0; k <= KHI; ++k) {
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        if (k == 0 && sg == 1) continue;
        const int sh = sg ? -k : k;                 // mask s: read position q - s
        const int i = sh + KHI;
        const int sl = (((j - sh) % L) + L) % L;
        const uint32_t d = ((rh[sl] ^ GH) | rx[sl]) | (rl[sl] ^ GL);
        run &= u[i] | d;
        u[i] = dp[i] | d;
        dp[i] = d;
      }
      if (k >= KLO) accn[k - KLO] = run;
    }
    // f(p), p = q - 2: erosion of the AND, per shift count
    uint32_t f[NK];
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      f[t] = v[t] & accn[t];
      v[t] = aprev[t] & accn[t];
      aprev[t] = accn[t];
    }
    if ((cm >> j) & 1ull) correct((int)q - 2, f);  // an end correction at p = q - 2
    const int pm4 = (((j - 2) % 4) + 4) % 4, pm8 = (((j - 2) % 8) + 8) % 8;  // p mod 4, p mod 8
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      const uint32_t x = pm4 == 0 ? f[t] : (f[t] & ~(fprev[t] & runs));  // a run starts here
      fprev[t] = f[t];
      if ((pm8 & 1) == 0) {
        xa[t] = x;
      } else if (pm8 == 1 || pm8 == 5) {
        csa(A0[t], xa[t], x, c1a[t]);
        xa[t] = 0u;
      } else if (pm8 == 3) {
        uint32_t c1b;
        csa(A0[t], xa[t], x, c1b);
        csa(A1[t], c1a[t], c1b, c2a[t]);
        xa[t] = 0u;
        c1a[t] = 0u;
      } else {  // 7
        uint32_t c1b, c2b, c3;
        csa(A0[t], xa[t], x, c1b);
        csa(A1[t], c1a[t], c1b, c2b);
        csa(A2[t], c2a[t], c2b, c3);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint32_t tt = B[t][b] & c3;
          B[t][b] ^= c3;
          c3 = tt;
        }
        xa[t] = 0u;
        c1a[t] = 0u;
        c2a[t] = 0u;
      }
    }
  };
  uint32_t q0 = 0;
  if (M > 0) {
    // Chunks of U positions (SlicedBody); with U < L the ring is rotated by U
    // slots after each chunk, so that at every chunk start the slot of read
    // position r is (r - q0) mod L and the chunk's code indexes it with
    // constants.  (U is a multiple of 8: the window slots and the count's
    // position pattern need no rotation.)
    constexpr int U = SlicedBody<KLO, KHI, M>::U;
    constexpr int NFULL = M > 0 ? M / U : 0, TAIL = M > 0 ? M % U : 0;
#pragma unroll 1
    for (int it = 0; it < NFULL; ++it) {
      cm = corr_bits(q0);
#pragma unroll
      for (int j = 0; j < U; ++j) step(q0 + (uint32_t)j, j);
      q0 += U;
      if (U < L) {
        uint32_t th[L], tl[L], tx[L];
#pragma unroll
        for (int s = 0; s < L; ++s) {
          th[s] = rh[(s + U) % L];
          tl[s] = rl[(s + U) % L];
          tx[s] = rx[(s + U) % L];
        }
#pragma unroll
        for (int s = 0; s < L; ++s) {
          rh[s] = th[s];
          rl[s] = tl[s];
          rx[s] = tx[s];
        }
      }
    }
    cm = corr_bits(q0);
#pragma unroll
    for (int j = 0; j < TAIL; ++j) step(q0 + (uint32_t)j, j);
  } else {
    bool more = true;
    while (more) {
      cm = corr_bits(q0);
#pragma unroll
      for (int j = 0; j < L; ++j) {
        if (q0 + (uint32_t)j >= m) {
          more = false;
          break;
        }
        step(q0 + (uint32_t)j, j);
      }
      q0 += L;
    }
  }

  // ---- positions m-2 and m-1 (the two steps past the read's end), counts
  // and results, one shift count at a time ----
  const uint2 stw = ldro(a.st + g);
  uint32_t accm1 = 0xffffffffu, accm = 0xffffffffu;  // acc(m-1), acc(m): masks s >= 0 only, nested in K
#pragma unroll
  for (int k = 0; k <= KHI; ++k) {
    accm1 &= u[KHI + k];
    accm &= dp[KHI + k];
    if (k < KLO) continue;
    const int t = k - KLO;
    const uint32_t K = (uint32_t)k;
    if (K < a.k_first || K > a.k_last) continue;
    uint32_t fe[NK];
#pragma unroll
    for (int s = 0; s < NK; ++s) fe[s] = 0u;
    uint32_t C[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) C[b] = 0u;
#pragma unroll
    for (int b = 0; b < NB && 3 + b < 8; ++b) C[3 + b] = B[t][b];
    add_plane(C, 0, A0[t]);
    add_plane(C, 1, A1[t]);
    add_plane(C, 2, A2[t]);
    add_plane(C, 0, xa[t]);
    add_plane(C, 1, c1a[t]);
    add_plane(C, 2, c2a[t]);
    uint32_t fp = fprev[t];
    if (m >= 2) {
      const int pp = (int)m - 2;
      fe[t] = v[t] & accm1;  // f(m-2)
      correct(pp, fe);
      const uint32_t ff = fe[t];
      add_plane(C, 0, (pp % 4 == 0) ? ff : (ff & ~(fp & runs)));
      fp = ff;
    }
    {
      const int pp = (int)m - 1;
      fe[t] = (aprev[t] & accm1) & accm;  // f(m-1)
      correct(pp, fe);
      const uint32_t ff = fe[t];
      add_plane(C, 0, (pp % 4 == 0) ? ff : (ff & ~(fp & runs)));
    }
    const uint64_t o = (uint64_t)(K - a.k_first) * a.out_stride;
    sliced_store(a, pbase, nvalid, C, stw, a.e + (K - a.k_first), a.accept + o,
                 a.result_byte ? nullptr : a.edits + o);
  }
}

// Compiled ranges of shift counts of the sweep kernels (sliced_sweep_m*.cu).
__host__ __device__ __forceinline__ bool sliced_sweep_range(int klo, int khi) {
  return (klo == 0 && khi == 5) || (klo == 6 && khi == 10);
}
// The compiled range holding shift count K, if any.
__host__ __device__ __forceinline__ bool sliced_sweep_cover(int K, int *klo, int *khi) {
  if (K >= 0 && K <= 5) {
    *klo = 0;
    *khi = 5;
    return true;
  }
  if (K >= 6 && K <= 10) {
    *klo = 6;
    *khi = 10;
    return true;
  }
  return false;
}

// Launchers (sliced.cu, sliced_m*_k*.cu, sliced_sweep_m*.cu).
cudaError_t launch_slice(const SliceArgs &a, uint32_t *err_count, cudaStream_t stream);
// One threshold: shift count K = min(e, m-1).
cudaError_t launch_sliced_filter(int K, const SlicedArgs &a, cudaStream_t stream);
// A compiled range of shift counts [klo, khi] (sliced_sweep_ranges) with
// results for a.k_first .. a.k_last inside it.
cudaError_t launch_sliced_sweep(int klo, int khi, const SlicedArgs &a, cudaStream_t stream);
#define GK_SLICED_LAUNCHERS(M)                                                                  \
  cudaError_t launch_sliced_m##M##_k0_5(int K, const SlicedArgs &a, cudaStream_t stream);  \
  cudaError_t launch_sliced_m##M##_k6_10(int K, const SlicedArgs &a, cudaStream_t stream); \
  cudaError_t launch_sliced_m##M##_k11_15(int K, const SlicedArgs &a, cudaStream_t stream); \
  cudaError_t launch_sliced_sweep_m##M(int klo, const SlicedArgs &a, cudaStream_t stream);
GK_SLICED_LAUNCHERS(0)
GK_SLICED_LAUNCHERS(100)
GK_SLICED_LAUNCHERS(150)
GK_SLICED_LAUNCHERS(250)
#undef GK_SLICED_LAUNCHERS

}  // namespace gk
