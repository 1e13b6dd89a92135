// Bit-sliced filter: the slice kernel, the dispatch over the compiled shift
// counts and the C ABI (gk_sliced_bytes, gk_slice, gk_filter_sliced).  The
// per-group code and the buffer layout are in sliced.cuh.
#include "sliced.cuh"

namespace gk {
namespace {

constexpr int kSliceTpg = 4;                   // lanes per group
constexpr int kSliceRows = 32 / kSliceTpg;     // pairs (matrix rows) per lane
constexpr int kSliceGroups = kSliceThreads / kSliceTpg;

// Transposes a 32x32 bit matrix held by the kSliceTpg consecutive lanes of
// a group, kSliceRows rows each (lane part p: rows 8p .. 8p+7 in v[]; bit b
// of a row = column b).  Afterwards part p holds columns 8p .. 8p+7 (bit j =
// row j).  Recursive block swap as in a one-thread transpose: the 16- and
// 8-row stages pair rows held by different lanes (a shuffle and a byte
// permute per row, the selector picking the lane's half), the 4-, 2- and
// 1-row stages run in registers.
__device__ __forceinline__ void transpose_rows(uint32_t (&v)[kSliceRows], uint32_t part) {
#pragma unroll
  for (int k = 16; k >= kSliceRows; k >>= 1) {
    const int d = k / kSliceRows;  // lane distance of rows i and i+k
    const bool up = (part & (uint32_t)d) != 0;
    const uint32_t sel = k == 16 ? (up ? 0x3276u : 0x5410u) : (up ? 0x3715u : 0x6240u);
#pragma unroll
    for (int i = 0; i < kSliceRows; ++i) v[i] = __byte_perm(v[i], __shfl_xor_sync(0xffffffffu, v[i], d), sel);
  }
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int S = 4 >> st;
    const uint32_t M = st == 0 ? 0x0F0F0F0Fu : (st == 1 ? 0x33333333u : 0x55555555u);
#pragma unroll
    for (int i = 0; i < kSliceRows; ++i) {
      if (i & S) continue;
      const uint32_t x = v[i], y = v[i + S];
      v[i] = (x & M) | ((y << S) & ~M);
      v[i + S] = ((x >> S) & M) | (y & ~M);
    }
  }
}

// Stores the transposed word of positions 32w + 8p .. 32w + 8p + 7 (those
// below m) into plane rows (h, l) of group g.
__device__ __forceinline__ void store_rows(uint2 *plane, uint64_t pitch, uint64_t g, uint32_t q0, uint32_t m,
                                           const uint32_t (&h)[kSliceRows], const uint32_t (&l)[kSliceRows]) {
#pragma unroll
  for (int i = 0; i < kSliceRows; ++i)
    if (q0 + i < m) __stcs(plane + (uint64_t)(q0 + i) * pitch + g, make_uint2(h[i], l[i]));
}

// Four lanes per group of 32 pairs, 8 pairs per lane.  The block's pair ids
// come in coalesced through shared memory (rows of 33 words: the lanes'
// reads hit distinct banks); each lane reads its 8 pairs' words two per
// row at a time in 16-byte loads (a pair with the read of the pair before it
// reuses that read's words), the group's four lanes transpose them, and the
// planes are written with streaming stores, which leave the genome and the
// reads in L2.
__global__ void __launch_bounds__(kSliceThreads) slice_kernel(const SliceArgs a, uint32_t *err_count) {
  constexpr int R = kSliceRows;
  __shared__ uint32_t s_rid[kSliceGroups * 33], s_off[kSliceGroups * 33];
  const uint64_t groups = sliced_groups(a.n_pairs);
  const uint64_t g0 = (uint64_t)blockIdx.x * kSliceGroups;
  for (int i = threadIdx.x; i < 32 * kSliceGroups; i += kSliceThreads) {
    const uint64_t p = g0 * 32 + (uint64_t)i;
    uint32_t rid = 0xffffffffu, off = 0xffffffffu;
    if (p < a.n_pairs) {
      rid = ldro(a.pair_read + p);
      off = ldro(a.pair_off + p);
    }
    s_rid[(i >> 5) * 33 + (i & 31)] = rid;
    s_off[(i >> 5) * 33 + (i & 31)] = off;
  }
  __syncthreads();
  const uint32_t gl = threadIdx.x / kSliceTpg, part = threadIdx.x % kSliceTpg;
  const uint64_t g = g0 + gl;  // a group past the end runs on zeros (its lanes shuffle) and stores nothing
  const bool live = g < groups;
  const uint32_t *rid = s_rid + gl * 33 + part * R, *off = s_off + gl * 33 + part * R;
  const uint64_t first = g * 32 + part * R;
  const uint32_t n_here = first >= a.n_pairs ? 0u : (uint32_t)min_u64(R, a.n_pairs - first);

  // Status per pair: invalid (read id or window out of range), undefined (a
  // non-ACGT base in the read, from its flag, or in the window, from the
  // genome's N index, Sec. 3.3).  A pair with the previous pair's read
  // reuses that read's flag (and, below, its words).
  uint32_t und = 0, inv = 0, ok = 0, same = 0, prev = 0xffffffffu, prev_nf = 0;  // local bits j < R
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if ((uint32_t)j >= n_here) continue;
    const uint32_t r = rid[j], o = off[j];
    if ((uint64_t)r >= a.n_reads || (uint64_t)o + a.m > a.ref_len) {
      inv |= 1u << j;
      prev = 0xffffffffu;
      continue;
    }
    ok |= 1u << j;
    uint32_t nf;
    if (r == prev) {
      same |= 1u << j;
      nf = prev_nf;
    } else {
      nf = a.read_nflag ? (uint32_t)ldro(a.read_nflag + r) : 0u;
    }
    prev = r;
    prev_nf = nf;
    bool u = nf != 0;
    if (a.ref_nidx) {
      const uint2 ni = ldro(a.ref_nidx + (o >> 5));
      const uint32_t q = ni.x >> (o & 31);
      const uint64_t first = q ? (uint64_t)o + (uint32_t)(__ffs(q) - 1) : (uint64_t)ni.y;
      u = u || first < (uint64_t)o + a.m;
    }
    if (u) und |= 1u << j;
  }
  if (inv && err_count) atomicAdd(err_count, popc32(inv));
  if (blockIdx.x == 0 && threadIdx.x == 0)
    *a.hdr = make_uint4(kSlicedMagic, a.m, (uint32_t)a.n_pairs, (uint32_t)(a.n_pairs >> 32));
  uint32_t gund = und << (part * R), ginv = inv << (part * R);
#pragma unroll
  for (int d = 1; d < kSliceTpg; d <<= 1) {
    gund |= __shfl_xor_sync(0xffffffffu, gund, d);
    ginv |= __shfl_xor_sync(0xffffffffu, ginv, d);
  }
  if (live && part == 0) a.st[g] = make_uint2(gund, ginv);

  const uint32_t m = a.m, W = (m + 31) / 32;
  const bool wide = (a.stride_words & 1u) == 0 && (reinterpret_cast<uintptr_t>(a.reads) & 15u) == 0;
  for (uint32_t w = 0; w < W; w += 2) {
    const bool two = w + 1 < W;
    uint32_t h0[R], l0[R], h1[R], l1[R];
    {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (((ok & ~same) >> j) & 1u) {
          const uint2 *row = a.reads + (uint64_t)rid[j] * a.stride_words + w;
          if (wide) {
            v = ldro(reinterpret_cast<const uint4 *>(row));
          } else {
            const uint2 x = ldro(row), y = two ? ldro(row + 1) : make_uint2(0u, 0u);
            v = make_uint4(x.x, x.y, y.x, y.y);
          }
        } else if (!((same >> j) & 1u)) {
          v = make_uint4(0u, 0u, 0u, 0u);
        }
        h0[j] = v.x;
        l0[j] = v.y;
        h1[j] = v.z;
        l1[j] = v.w;
      }
    }
    const uint32_t q0 = 32 * w + part * R;
    transpose_rows(h0, part);
    transpose_rows(l0, part);
    if (live) store_rows(a.rs, a.pitch, g, q0, m, h0, l0);
    if (two) {  // warp-uniform
      transpose_rows(h1, part);
      transpose_rows(l1, part);
      if (live) store_rows(a.rs, a.pitch, g, q0 + 32, m, h1, l1);
    }
    // Window words w, w+1: genome words t, t+1, t+2 (t = off/32 + w) from
    // the aligned 16-byte loads at the even word at or below t; the last word
    // read is at most off/32 + W + 1 <= n_words + 1, inside the genome's two
    // zero tail words.
#pragma unroll
    for (int j = 0; j < R; ++j) {
      uint32_t a0 = 0, b0 = 0, a1 = 0, b1 = 0;
      if ((ok >> j) & 1u) {
        const uint32_t o = off[j];
        const uint32_t t = (o >> 5) + w;
        const uint4 *gq = reinterpret_cast<const uint4 *>(a.ref_hl + (t & ~1u));
        const uint4 A = ldro(gq);
        uint2 x0, x1, x2 = make_uint2(0u, 0u);
        if ((t & 1u) == 0) {
          x0 = make_uint2(A.x, A.y);
          x1 = make_uint2(A.z, A.w);
          if (two) {
            const uint4 B = ldro(gq + 1);
            x2 = make_uint2(B.x, B.y);
          }
        } else {
          const uint4 B = ldro(gq + 1);
          x0 = make_uint2(A.z, A.w);
          x1 = make_uint2(B.x, B.y);
          x2 = make_uint2(B.z, B.w);
        }
        const uint32_t sh = o & 31;
        a0 = __funnelshift_r(x0.x, x1.x, sh);
        b0 = __funnelshift_r(x0.y, x1.y, sh);
        a1 = __funnelshift_r(x1.x, x2.x, sh);
        b1 = __funnelshift_r(x1.y, x2.y, sh);
      }
      h0[j] = a0;
      l0[j] = b0;
      h1[j] = a1;
      l1[j] = b1;
    }
    transpose_rows(h0, part);
    transpose_rows(l0, part);
    if (live) store_rows(a.gs, a.pitch, g, q0, m, h0, l0);
    if (two) {
      transpose_rows(h1, part);
      transpose_rows(l1, part);
      if (live) store_rows(a.gs, a.pitch, g, q0 + 32, m, h1, l1);
    }
  }
}

}  // namespace

cudaError_t launch_slice(const SliceArgs &a, uint32_t *err_count, cudaStream_t stream) {
  const uint64_t blocks = (sliced_groups(a.n_pairs) + kSliceGroups - 1) / kSliceGroups;
  slice_kernel<<<(unsigned)blocks, kSliceThreads, 0, stream>>>(a, err_count);
  return cudaGetLastError();
}

// The read lengths of the paper's data sets (100, 150, 250 bp, Sec. 4) have
// kernels with the length compiled in; any other length takes the general
// ones.
cudaError_t launch_sliced_filter(int K, const SlicedArgs &a, cudaStream_t stream) {
  if (K < 0 || K > kSlicedMaxK) return cudaErrorInvalidValue;
#define GK_SLICED_PICK(M) \
  (K <= 5 ? launch_sliced_m##M##_k0_5(K, a, stream)  \
          : (K <= 10 ? launch_sliced_m##M##_k6_10(K, a, stream) : launch_sliced_m##M##_k11_15(K, a, stream)))
  switch (a.m) {
    case 100: return GK_SLICED_PICK(100);
    case 150: return GK_SLICED_PICK(150);
    case 250: return GK_SLICED_PICK(250);
    default: return GK_SLICED_PICK(0);
  }
#undef GK_SLICED_PICK
}

cudaError_t launch_sliced_sweep(int klo, int khi, const SlicedArgs &a, cudaStream_t stream) {
  if (!sliced_sweep_range(klo, khi)) return cudaErrorInvalidValue;
  switch (a.m) {
    case 100: return launch_sliced_sweep_m100(klo, a, stream);
    case 150: return launch_sliced_sweep_m150(klo, a, stream);
    case 250: return launch_sliced_sweep_m250(klo, a, stream);
    default: return launch_sliced_sweep_m0(klo, a, stream);
  }
}

}  // namespace gk

using gk::fail;

namespace {
bool aligned_to(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Arguments shared by every filter launch over one sliced buffer.
gk::SlicedArgs sliced_args(const void *sliced, uint64_t n_pairs, uint32_t m, int count_mode, bool result_byte,
                           uint32_t *err_count) {
  gk::SlicedArgs a{};
  a.pitch = gk::sliced_pitch(n_pairs);
  a.rs = reinterpret_cast<const uint2 *>(sliced);
  a.gs = a.rs + (uint64_t)(m + gk::kSlicedPad) * a.pitch;
  a.st = a.gs + (uint64_t)(m + gk::kSlicedPad) * a.pitch;
  a.hdr = reinterpret_cast<const uint4 *>(a.st + a.pitch);
  a.n_pairs = n_pairs;
  a.m = m;
  a.runs4 = count_mode == GK_COUNT_RUNS4 ? 1u : 0u;
  a.result_byte = result_byte ? 1 : 0;
  a.err_count = err_count;
  return a;
}
}  // namespace

extern "C" {

uint64_t gk_sliced_bytes(uint64_t n_pairs, uint32_t m) {
  if (n_pairs == 0 || m == 0 || m > gk::kSlicedMaxLen) return 0;
  return gk::sliced_bytes(n_pairs, m);
}

int gk_slice(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words, uint64_t n_reads,
             const uint8_t *read_nflag, uint32_t m, const uint32_t *pair_read, const uint32_t *pair_off,
             uint64_t n_pairs, void *sliced, uint64_t sliced_cap, uint32_t *err_count, void *stream) {
  gk::clear_error();
  if (!ref) return fail(GK_EINVAL, "gk_slice: null reference handle");
  if (m == 0 || m > gk::kSlicedMaxLen) return fail(GK_ERANGE, "gk_slice: m outside 1..255");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > (1ull << 40)) return fail(GK_ERANGE, "gk_slice: too many pairs");
  if (!reads || !pair_read || !pair_off || !sliced) return fail(GK_EINVAL, "gk_slice: null buffer");
  const uint32_t W = (m + 31) / 32;
  if (stride_words < W) return fail(GK_EINVAL, "gk_slice: stride_words < ceil(m/32)");
  if (!aligned_to(reads, 8)) return fail(GK_EINVAL, "gk_slice: reads must be 8-byte aligned");
  if (!aligned_to(sliced, 16)) return fail(GK_EINVAL, "gk_slice: sliced buffer must be 16-byte aligned");
  if (sliced_cap < gk::sliced_bytes(n_pairs, m)) return fail(GK_EINVAL, "gk_slice: sliced buffer too small");
  gk::SliceArgs a{};
  a.ref_hl = ref->hl;
  a.ref_nidx = ref->nidx;
  a.ref_len = ref->n_bases;
  a.reads = reinterpret_cast<const uint2 *>(reads);
  a.stride_words = stride_words;
  a.n_reads = n_reads;
  a.read_nflag = read_nflag;
  a.m = m;
  a.pair_read = pair_read;
  a.pair_off = pair_off;
  a.n_pairs = n_pairs;
  a.pitch = gk::sliced_pitch(n_pairs);
  a.rs = reinterpret_cast<uint2 *>(sliced);
  a.gs = a.rs + (uint64_t)(m + gk::kSlicedPad) * a.pitch;
  a.st = a.gs + (uint64_t)(m + gk::kSlicedPad) * a.pitch;
  a.hdr = reinterpret_cast<uint4 *>(a.st + a.pitch);
  return gk::cuda_check(gk::launch_slice(a, err_count, (cudaStream_t)stream), "gk_slice: launch");
}

int gk_filter_sliced(const void *sliced, uint64_t sliced_cap, uint64_t n_pairs, uint32_t m, uint32_t fixed_e,
                     int count_mode, uint32_t flags, uint8_t *accept_out, uint16_t *edits_out, void *stream) {
  gk::clear_error();
  if (m == 0 || m > gk::kSlicedMaxLen) return fail(GK_ERANGE, "gk_filter_sliced: m outside 1..255");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > (1ull << 40)) return fail(GK_ERANGE, "gk_filter_sliced: too many pairs");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE)) return fail(GK_EINVAL, "gk_filter_sliced: unknown flags");
  if (flags & GK_FLAG_NO_EDGE_FIX)
    return fail(GK_EINVAL, "gk_filter_sliced: computes the Sec. 3.4 edge OR only (use gk_filter without it)");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter_sliced: unknown count_mode");
  if (fixed_e > 255) return fail(GK_ERANGE, "gk_filter_sliced: fixed_e above 255");
  if (result_byte && fixed_e > 252) return fail(GK_ERANGE, "gk_filter_sliced: GK_FLAG_RESULT_BYTE needs fixed_e <= 252");
  const uint32_t K = fixed_e < m - 1 ? fixed_e : m - 1;
  if (K > (uint32_t)gk::kSlicedMaxK)
    return fail(GK_ERANGE, "gk_filter_sliced: min(e, m-1) above the compiled shift counts (GK_SLICED_MAX_SHIFT)");
  if (!sliced || !accept_out || (!edits_out && !result_byte)) return fail(GK_EINVAL, "gk_filter_sliced: null buffer");
  if (!aligned_to(sliced, 16)) return fail(GK_EINVAL, "gk_filter_sliced: sliced buffer must be 16-byte aligned");
  if (sliced_cap < gk::sliced_bytes(n_pairs, m)) return fail(GK_EINVAL, "gk_filter_sliced: sliced buffer too small");
  gk::SlicedArgs a = sliced_args(sliced, n_pairs, m, count_mode, result_byte, nullptr);
  a.e = fixed_e;
  a.k_first = a.k_last = K;
  a.out_stride = 0;
  a.vec_out = aligned_to(accept_out, 16) && (result_byte || aligned_to(edits_out, 16)) ? 1 : 0;
  a.accept = accept_out;
  a.edits = result_byte ? nullptr : edits_out;
  return gk::cuda_check(gk::launch_sliced_filter((int)K, a, (cudaStream_t)stream), "gk_filter_sliced: launch");
}

int gk_filter_sliced_sweep(const void *sliced, uint64_t sliced_cap, uint64_t n_pairs, uint32_t m, uint32_t e_lo,
                           uint32_t e_hi, int count_mode, uint32_t flags, uint8_t *accept_out, uint16_t *edits_out,
                           uint64_t out_stride, uint32_t *err_count, void *stream) {
  gk::clear_error();
  if (m == 0 || m > gk::kSlicedMaxLen) return fail(GK_ERANGE, "gk_filter_sliced_sweep: m outside 1..255");
  if (e_lo > e_hi) return fail(GK_EINVAL, "gk_filter_sliced_sweep: e_lo > e_hi");
  if (e_hi > 255) return fail(GK_ERANGE, "gk_filter_sliced_sweep: e_hi above 255");
  if (n_pairs == 0) return GK_OK;
  if (n_pairs > (1ull << 40)) return fail(GK_ERANGE, "gk_filter_sliced_sweep: too many pairs");
  const bool result_byte = (flags & GK_FLAG_RESULT_BYTE) != 0;
  if (flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE))
    return fail(GK_EINVAL, "gk_filter_sliced_sweep: unknown flags");
  if (flags & GK_FLAG_NO_EDGE_FIX)
    return fail(GK_EINVAL, "gk_filter_sliced_sweep: computes the Sec. 3.4 edge OR only (use gk_filter without it)");
  if (count_mode != GK_COUNT_RUNS4 && count_mode != GK_COUNT_POPCOUNT)
    return fail(GK_EINVAL, "gk_filter_sliced_sweep: unknown count_mode");
  if (result_byte && e_hi > 252)
    return fail(GK_ERANGE, "gk_filter_sliced_sweep: GK_FLAG_RESULT_BYTE needs e_hi <= 252");
  const uint32_t k_hi = e_hi < m - 1 ? e_hi : m - 1;
  if (k_hi > (uint32_t)gk::kSlicedMaxK)
    return fail(GK_ERANGE, "gk_filter_sliced_sweep: min(e_hi, m-1) above the compiled shift counts (GK_SLICED_MAX_SHIFT)");
  if (!sliced || !accept_out || (!edits_out && !result_byte))
    return fail(GK_EINVAL, "gk_filter_sliced_sweep: null buffer");
  if (out_stride < n_pairs) return fail(GK_EINVAL, "gk_filter_sliced_sweep: out_stride < n_pairs");
  if (!aligned_to(sliced, 16)) return fail(GK_EINVAL, "gk_filter_sliced_sweep: sliced buffer must be 16-byte aligned");
  if (sliced_cap < gk::sliced_bytes(n_pairs, m))
    return fail(GK_EINVAL, "gk_filter_sliced_sweep: sliced buffer too small");
  gk::SlicedArgs a = sliced_args(sliced, n_pairs, m, count_mode, result_byte, err_count);
  a.out_stride = out_stride;
  const bool rows16 = (out_stride % 16) == 0;
  a.vec_out = rows16 && aligned_to(accept_out, 16) && (result_byte || aligned_to(edits_out, 16)) ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  // Thresholds e <= m-1 have the shift count K = e: each compiled range of
  // shift counts filters its part of [e_lo, e_hi] in one pass (the K below
  // that part are computed and not written), a K outside every range has
  // its own launch.  Thresholds above m-1 share K = m-1 and have one launch
  // each.
  uint32_t e = e_lo;
  while (e <= e_hi) {
    const uint32_t K = e < m - 1 ? e : m - 1;
    int klo = -1, khi = -1;
    uint32_t last = e;
    if (e <= m - 1 && gk::sliced_sweep_cover((int)K, &klo, &khi)) {
      last = (uint32_t)khi;
      if (last > e_hi) last = e_hi;
      if (last > m - 1) last = m - 1;
    }
    if (last == e) klo = khi = -1;  // one threshold: the single-count kernel is cheaper
    a.e = e;
    a.k_first = K;
    a.k_last = K + (last - e);
    a.accept = accept_out + (uint64_t)(e - e_lo) * out_stride;
    a.edits = result_byte ? nullptr : edits_out + (uint64_t)(e - e_lo) * out_stride;
    const cudaError_t err = klo >= 0 ? gk::launch_sliced_sweep(klo, khi, a, st) : gk::launch_sliced_filter((int)K, a, st);
    const int rc = gk::cuda_check(err, "gk_filter_sliced_sweep: launch");
    if (rc != GK_OK) return rc;
    e = last + 1;
  }
  return GK_OK;
}

}  // extern "C"
