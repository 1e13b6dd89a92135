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
//   filter  once per threshold: streams the positions of a group in order,
//           keeping the read positions q-K .. q+K in a register ring.
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
// then st; (2(m + kSlicedPad) + 1) * pitch * 8 bytes.
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
  return (2ull * (m + kSlicedPad) + 1) * sliced_pitch(n_pairs) * 8ull;
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
};

// ---- filter -----------------------------------------------------------------

struct SlicedArgs {
  const uint2 *rs, *gs, *st;
  uint64_t pitch;
  uint64_t n_pairs;
  uint32_t m;
  uint32_t e;        // the threshold accept compares with (K = min(e, m-1))
  uint32_t runs4;    // 1: windowed run count, 0: popcount
  int result_byte;
  int vec_out;       // accept (and edits) 16-byte aligned: vector stores
  uint8_t *accept;
  uint16_t *edits;
};

// Register ring of the read positions: L slots (a multiple of 8, at least
// 2K+4), the read position q + K + D loaded while position q is filtered.
template <int K>
struct SlicedRing {
  static constexpr int L = (2 * K + 4 <= 16) ? 16 : ((2 * K + 4 + 7) / 8) * 8;
  static constexpr int D = L - 2 * K - 1;  // prefetch distance, >= 3
  static_assert(K + D <= (int)kSlicedPad, "the prefetch stays inside the padding rows");
};

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

// Filters group g.  clr: 2K+2 words at stride clr_stride (the end
// corrections, low positions 1..K+1 then high positions m-2..m-K-2).
// M > 0: the read length is M (a.m == M), known at compile time, so the
// positions run as whole ring periods and a fixed tail with no test per
// position.  M == 0: any length, with a test per position.
template <int K, int M>
__host__ __device__ __forceinline__ void sliced_group(const SlicedArgs &a, uint64_t g, uint32_t *clr,
                                                      int clr_stride) {
  constexpr int L = SlicedRing<K>::L, D = SlicedRing<K>::D, NS = 2 * K + 1;
  const uint32_t m = M > 0 ? (uint32_t)M : a.m;
  const uint64_t P = a.pitch;
  const uint2 *rp = a.rs + g, *gp = a.gs + g;
  const uint2 z2 = make_uint2(0u, 0u);
  auto Rq = [&](int64_t q) -> uint2 { return (q >= 0 && q < (int64_t)m) ? ldro(rp + q * (int64_t)P) : z2; };
  auto Gq = [&](int64_t q) -> uint2 { return (q >= 0 && q < (int64_t)m) ? ldro(gp + q * (int64_t)P) : z2; };
  auto diff = [](uint2 x, uint2 y) -> uint32_t { return (x.x ^ y.x) | (x.y ^ y.y); };
  auto vacv = [](uint2 x) -> uint32_t { return x.x | x.y; };  // window base other than 'A'

  // ---- end corrections (positions 1..K+1 and m-K-2..m-2) ----
  {
    const uint2 R0 = Rq(0), R1 = Rq(1), Rm1 = Rq((int64_t)m - 1), Rm2 = Rq((int64_t)m - 2);
    uint2 gl[K + 3];  // window positions 0 .. K+2
#pragma unroll
    for (int t = 0; t < K + 3; ++t) gl[t] = Gq(t);
    auto vlo = [&](int q) -> uint32_t { return q < 0 ? 0u : vacv(gl[q]); };
    auto a0 = [&](int q) -> uint32_t { return diff(gl[q], R0); };
    auto a1 = [&](int q) -> uint32_t { return (q < (int)m && q < 32) ? diff(gl[q], R1) : 0u; };
    auto c1 = [&](int q) -> uint32_t { return vlo(q - 2) | vlo(q - 1) | a0(q); };
    auto c2 = [&](int q) -> uint32_t { return vlo(q - 1) | a0(q) | a1(q + 1); };
#pragma unroll
    for (int p = 1; p <= K + 1; ++p) {
      uint32_t c = 0;
      if (p <= K) c |= ~(c1(p) & c2(p));
      if (p - 1 >= 1) c |= ~c2(p - 1);
      clr[(p - 1) * clr_stride] = c;
    }
    // Mirrored about the read's end: j <-> position m-1-j.
    const int64_t hb = (int64_t)m - K - 3;
    uint2 gh[K + 4];  // window positions m-K-3 .. m
#pragma unroll
    for (int t = 0; t < K + 4; ++t) gh[t] = Gq(hb + t);
    auto G_of = [&](int j) -> uint2 { return gh[K + 2 - j]; };  // position m-1-j, j in -1 .. K+2
    auto vm = [&](int j) -> uint32_t { return vacv(G_of(j)); };
    auto a0m = [&](int j) -> uint32_t { return diff(G_of(j), Rm1); };
    auto a1m = [&](int j) -> uint32_t { return j < 32 ? diff(G_of(j), Rm2) : 0u; };
    auto c1m = [&](int j) -> uint32_t { return vm(j - 2) | vm(j - 1) | a0m(j); };
    auto c2m = [&](int j) -> uint32_t { return vm(j - 1) | a0m(j) | a1m(j + 1); };
#pragma unroll
    for (int j = 1; j <= K + 1; ++j) {
      uint32_t c = 0;
      if (j <= K) c |= ~(c1m(j) & c2m(j));
      if (j - 1 >= 1) c |= ~c2m(j - 1);
      clr[(K + j) * clr_stride] = ((int)m - 1 - j >= 0) ? c : 0u;
    }
  }

  // ---- ring of read positions; slot of position r is r mod L ----
  uint32_t rh[L], rl[L], rx[L];  // rx: 1s where the position lies outside the read (vacated)
#pragma unroll
  for (int r = -K; r < K + D; ++r) {
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
  const uint2 *rload = rp + (uint64_t)(K + D) * P;
  const uint2 *gload = gp + 7ull * P;

  uint32_t u[NS], dp[NS];  // per mask: d(q-2) | d(q-1), d(q-1)
#pragma unroll
  for (int i = 0; i < NS; ++i) u[i] = dp[i] = 0u;
  uint32_t aprev = 0u, v = 0u, fprev = 0u;          // acc(q-2); acc(q-3) & acc(q-2); f(p-1)
  uint32_t A0 = 0u, A1 = 0u, A2 = 0u, xa = 0u, c1a = 0u, c2a = 0u;  // carry-save count
  uint32_t B[5] = {0u, 0u, 0u, 0u, 0u};                              // count / 8
  const uint32_t runs = a.runs4 ? 0xffffffffu : 0u;

  // Positions q0 .. q0+L-1 with an end correction (q in 3..K+3, the low
  // corrections at p = q-2 in 1..K+1, or q in m-K..m-1, the high ones): one
  // bit per position, so the other positions pay one bit test.
  static_assert(L <= 64, "one correction bit per position of a ring period");
  auto corr_bits = [&](uint32_t q0) -> uint64_t {
    auto range = [](int lo, int hi) -> uint64_t {
      lo = lo < 0 ? 0 : lo;
      hi = hi > L - 1 ? L - 1 : hi;
      if (hi < lo) return 0ull;
      return (hi == 63 ? ~0ull : ((2ull << hi) - 1ull)) & ~((1ull << lo) - 1ull);
    };
    return range(3 - (int)q0, K + 3 - (int)q0) | range((int)m - K - (int)q0, (int)m - 1 - (int)q0);
  };
  uint64_t cm = 0;
  // One position: q runs, j = q mod L is a constant after unrolling.
  auto step = [&](uint32_t q, int j) {
    // Read position q + K + D into the slot position q - K - 1 leaves, and
    // window position q + 7.  Past m the rows are padding: the shift counts
    // whose launches wait on memory (K <= 3) skip those loads, the others
    // read them unconditionally (the vacated flag masks the read; window
    // positions past m-1 are never used).
    {
      const int s = (j + K + D) % L;
      const bool in = q + K + D < m;
      const uint2 vv = (K > 3 || in) ? ldro(rload) : z2;
      rh[s] = vv.x;
      rl[s] = vv.y;
      rx[s] = in ? 0u : 0xffffffffu;
      rload += P;
    }
    {
      const int s = (j + 7) % 8;
      const uint2 vv = (K > 3 || q + 7 < m) ? ldro(gload) : z2;
      wh[s] = vv.x;
      wl[s] = vv.y;
      gload += P;
    }
    const uint32_t GH = wh[j % 8], GL = wl[j % 8];
    uint32_t accn = 0xffffffffu;  // acc(q-1)
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      const int sh = i - K;                       // mask s: read position q - s
      const int sl = (((j - sh) % L) + L) % L;
      const uint32_t d = ((rh[sl] ^ GH) | rx[sl]) | (rl[sl] ^ GL);
      accn &= u[i] | d;
      u[i] = dp[i] | d;
      dp[i] = d;
    }
    // f(p), p = q - 2: erosion of the AND
    uint32_t f = v & accn;
    v = aprev & accn;
    aprev = accn;
    if ((cm >> j) & 1ull) {  // an end correction at p = q - 2
      const int p = (int)q - 2;
      if (p >= 1 && p <= K + 1) f &= ~clr[(p - 1) * clr_stride];
      const int jj = (int)m - 1 - p;
      if (jj >= 1 && jj <= K + 1) f &= ~clr[(K + jj) * clr_stride];
    }
    const int pm4 = (((j - 2) % 4) + 4) % 4, pm8 = (((j - 2) % 8) + 8) % 8;  // p mod 4, p mod 8
    const uint32_t x = pm4 == 0 ? f : (f & ~(fprev & runs));  // a run starts here
    fprev = f;
    if ((pm8 & 1) == 0) {
      xa = x;
    } else if (pm8 == 1 || pm8 == 5) {
      csa(A0, xa, x, c1a);
      xa = 0u;
    } else if (pm8 == 3) {
      uint32_t c1b;
      csa(A0, xa, x, c1b);
      csa(A1, c1a, c1b, c2a);
      xa = 0u;
      c1a = 0u;
    } else {  // 7
      uint32_t c1b, c2b, c3;
      csa(A0, xa, x, c1b);
      csa(A1, c1a, c1b, c2b);
      csa(A2, c2a, c2b, c3);
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const uint32_t t = B[b] & c3;
        B[b] ^= c3;
        c3 = t;
      }
      xa = 0u;
      c1a = 0u;
      c2a = 0u;
    }
  };
  uint32_t q0 = 0;
  if (M > 0) {
    constexpr int NFULL = M > 0 ? M / L : 0, TAIL = M > 0 ? M % L : 0;
#pragma unroll 1
    for (int it = 0; it < NFULL; ++it) {
      cm = corr_bits(q0);
#pragma unroll
      for (int j = 0; j < L; ++j) step(q0 + (uint32_t)j, j);
      q0 += L;
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

  // ---- positions m-2 and m-1: the two steps past the read's end ----
  uint32_t accm1 = 0xffffffffu, accm = 0xffffffffu;  // acc(m-1), acc(m): masks s >= 0 only
#pragma unroll
  for (int i = K; i < NS; ++i) {
    accm1 &= u[i];
    accm &= dp[i];
  }
  const uint32_t f_a = v & accm1;             // f(m-2)
  const uint32_t f_b = (aprev & accm1) & accm;  // f(m-1)
  uint32_t C[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) C[b] = 0u;
#pragma unroll
  for (int b = 0; b < 5; ++b) C[3 + b] = B[b];
  add_plane(C, 0, A0);
  add_plane(C, 1, A1);
  add_plane(C, 2, A2);
  add_plane(C, 0, xa);
  add_plane(C, 1, c1a);
  add_plane(C, 2, c2a);
  auto corrected = [&](int pp, uint32_t ff) -> uint32_t {
    if (pp >= 1 && pp <= K + 1) ff &= ~clr[(pp - 1) * clr_stride];
    const int jj = (int)m - 1 - pp;
    if (jj >= 1 && jj <= K + 1) ff &= ~clr[(K + jj) * clr_stride];
    return ff;
  };
  uint32_t fp = fprev;
  if (m >= 2) {
    const int pp = (int)m - 2;
    const uint32_t ff = corrected(pp, f_a);
    add_plane(C, 0, (pp % 4 == 0) ? ff : (ff & ~(fp & runs)));
    fp = ff;
  }
  {
    const int pp = (int)m - 1;
    const uint32_t ff = corrected(pp, f_b);
    add_plane(C, 0, (pp % 4 == 0) ? ff : (ff & ~(fp & runs)));
  }

  // ---- results: per pair byte counts, then accept/edits or result bytes ----
  const uint2 stw = ldro(a.st + g);
  const uint64_t pbase = g * 32ull;
  const uint64_t left = a.n_pairs - pbase;
  const uint32_t nvalid = left < 32 ? (uint32_t)left : 32u;
  const uint32_t e4 = (a.e > 255u ? 255u : a.e) * 0x01010101u;
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
    uint4 *pa = reinterpret_cast<uint4 *>(a.accept + pbase);
    pa[0] = make_uint4(outA[0], outA[1], outA[2], outA[3]);
    pa[1] = make_uint4(outA[4], outA[5], outA[6], outA[7]);
    if (!a.result_byte) {
      uint4 *pe = reinterpret_cast<uint4 *>(a.edits + pbase);
#pragma unroll
      for (int k = 0; k < 4; ++k) pe[k] = make_uint4(outE[4 * k], outE[4 * k + 1], outE[4 * k + 2], outE[4 * k + 3]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if ((uint32_t)j < nvalid) {
        a.accept[pbase + j] = (uint8_t)(outA[j >> 2] >> (8 * (j & 3)));
        if (!a.result_byte) a.edits[pbase + j] = (uint16_t)(outE[j >> 1] >> (16 * (j & 1)));
      }
    }
  }
}

// Launchers (sliced.cu, sliced_m*_k*.cu).
cudaError_t launch_slice(const SliceArgs &a, uint32_t *err_count, cudaStream_t stream);
cudaError_t launch_sliced_filter(int K, const SlicedArgs &a, cudaStream_t stream);
#define GK_SLICED_LAUNCHERS(M)                                                                  \
  cudaError_t launch_sliced_m##M##_k0_5(int K, const SlicedArgs &a, cudaStream_t stream);  \
  cudaError_t launch_sliced_m##M##_k6_10(int K, const SlicedArgs &a, cudaStream_t stream); \
  cudaError_t launch_sliced_m##M##_k11_15(int K, const SlicedArgs &a, cudaStream_t stream);
GK_SLICED_LAUNCHERS(0)
GK_SLICED_LAUNCHERS(100)
GK_SLICED_LAUNCHERS(150)
GK_SLICED_LAUNCHERS(250)
#undef GK_SLICED_LAUNCHERS

}  // namespace gk
