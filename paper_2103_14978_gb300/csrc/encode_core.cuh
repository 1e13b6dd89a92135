// Word encoders shared by the read encoder and the fused encode + filter
// kernel: 32 ASCII bytes -> one {high, low} word of the 2-bit code (A=00 C=01
// G=10 T=11, Sec. 2.1) and the bytes that are not A/C/G/T (Sec. 3.3).
#pragma once

#include <cstdint>

namespace gk {

// Four ASCII bytes -> 4 bits each of the high plane, the low plane and the
// undefined mask, the first `nvalid` bytes only.  In ASCII, bit 2 of A/C/G/T
// (either case) is the code's high bit and bit 1 XOR bit 2 its low bit
// (A=00 C=01 G=10 T=11, Sec. 2.1); a byte is valid iff it equals, case
// folded, the letter its code names (a byte_perm lookup).  The per-byte bits
// are gathered into a nibble with one multiply.
__device__ __forceinline__ void encode4(uint32_t c, uint32_t nvalid, uint32_t &hi4, uint32_t &lo4,
                                        uint32_t &n4) {
  const uint32_t hib = (c >> 2) & 0x01010101u;
  const uint32_t lob = ((c >> 1) ^ (c >> 2)) & 0x01010101u;
  const uint32_t code = ((c >> 1) & 0x02020202u) | lob;  // per byte 0..3
  uint32_t sel = (code | (code >> 4)) & 0x00FF00FFu;
  sel = (sel & 0xFFu) | ((sel >> 8) & 0xFF00u);
  const uint32_t expect = __byte_perm(0x54474341u, 0u, sel);  // 'A' 'C' 'G' 'T'
  const uint32_t bad = (c & 0xDFDFDFDFu) ^ expect;
  const uint32_t nz = (((bad & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | bad) & 0x80808080u;
  const uint32_t keep = nvalid >= 4 ? 0xFu : ((1u << nvalid) - 1u);
  n4 = (((nz >> 7) * 0x01020408u) >> 24) & keep;
  hi4 = (((hib * 0x01020408u) >> 24) & keep) & ~n4;
  lo4 = (((lob * 0x01020408u) >> 24) & keep) & ~n4;
}

// 32 bytes (8 little-endian words) -> one {high, low} word and its N bits.
__device__ __forceinline__ void encode32(const uint32_t (&wb)[8], uint32_t nvalid, uint32_t &hi, uint32_t &lo,
                                         uint32_t &nb) {
  hi = lo = nb = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int rem = (int)nvalid - 4 * j;
    uint32_t h, l, n;
    encode4(wb[j], rem <= 0 ? 0u : (uint32_t)rem, h, l, n);
    hi |= h << (4 * j);
    lo |= l << (4 * j);
    nb |= n << (4 * j);
  }
}

// A full word (32 bytes) -> its planes and whether any byte is not A/C/G/T
// (either case).  Per pair of 4-byte words, bit 2
// (high plane) and bit 1 XOR bit 2 (low plane) of each byte are gathered by
// one multiply each into the top byte of a product, the first word's 4 bits
// at bits 24..27 and the second's at 28..31 (the magic shifted by 4; no
// other partial product lands in that byte, so the two products are ORed);
// three byte permutes assemble the four top bytes into the plane word.
// Validity looks up the letter a byte's bits 2 and 1 name ("A", "C", "T",
// "G" for 00, 01, 10, 11) with two byte permutes and compares it with the
// case-folded byte.  bad != 0: re-encode with encode32 (codes 00 for the
// undefined bytes).
__device__ __forceinline__ void encode32_full(const uint32_t (&wb)[8], uint32_t &hi, uint32_t &lo, uint32_t &bad) {
  constexpr uint32_t kM = 0x00408102u;  // bit 2 of byte k -> bit 24 + k
  uint32_t yh[4], yl[4];
  bad = 0;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint32_t c0 = wb[2 * p], c1 = wb[2 * p + 1];
    yh[p] = ((c0 & 0x04040404u) * kM) | ((c1 & 0x04040404u) * (kM << 4));
    yl[p] = (((c0 ^ (c0 << 1)) & 0x04040404u) * kM) | (((c1 ^ (c1 << 1)) & 0x04040404u) * (kM << 4));
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t c = wb[2 * p + q];
      const uint32_t idx = (c >> 1) & 0x03030303u;
      const uint32_t sel = __byte_perm(idx | (idx >> 4), 0u, 0x4420u);
      const uint32_t expect = __byte_perm(0x47544341u, 0u, sel);  // 'A' 'C' 'T' 'G'
      bad |= (c ^ expect) & 0xDFDFDFDFu;
    }
  }
  hi = __byte_perm(__byte_perm(yh[0], yh[1], 0x0073u), __byte_perm(yh[2], yh[3], 0x0073u), 0x5410u);
  lo = __byte_perm(__byte_perm(yl[0], yl[1], 0x0073u), __byte_perm(yl[2], yl[3], 0x0073u), 0x5410u);
}

// Any word: the bytes past the first `nvalid` are replaced by 'A' (code 00,
// a valid letter), so that encode32_full gives the planes of the first
// `nvalid` bytes and flags only those.  Every lane of a warp runs the same
// instructions whatever its word's length (the last word of a read is
// usually short).  bad != 0: re-encode with encode32(wb, nvalid, ...).
__device__ __forceinline__ void encode32_any(uint32_t (&wb)[8], uint32_t nvalid, uint32_t &hi, uint32_t &lo,
                                             uint32_t &bad) {
  if (nvalid < 32) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int rem = (int)nvalid - 4 * j;
      const uint32_t keep = rem >= 4 ? 0xffffffffu : (rem <= 0 ? 0u : ((1u << (8 * rem)) - 1u));
      wb[j] = (wb[j] & keep) | (0x41414141u & ~keep);
    }
  }
  encode32_full(wb, hi, lo, bad);
}

}  // namespace gk
