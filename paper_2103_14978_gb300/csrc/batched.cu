// Planning kernels of the batched filter: classify pairs (trivial outcomes
// written at once, the rest keyed by (W, K)), scan the key histogram into
// record slots and tiles (heaviest key first), scatter pair records by key.
#include "batched.cuh"

namespace gk {

namespace {

constexpr int kPlanThreads = 256;
constexpr int kScatterChunk = 2048;  // pairs per scatter block

constexpr int kClassifyChunk = 2048;  // pairs per classify block

// kClassifyChunk pairs per block, kClassifyChunk / kPlanThreads per thread.
// Invalid, undefined (N) and zero-length pairs get their result here (Sec.
// 3.3 pass-through, the invalid sentinel) and key kNoKey; the others get key
// (W, K) and are counted in the block-local histogram.  Each thread first
// loads the ids of all its pairs, then every per-read and per-window word
// they need (length, N flag, N index word; each only when its index is in
// range), and only then decides: two rounds of independent loads instead of
// a chain of dependent ones per pair.
__global__ void __launch_bounds__(kPlanThreads) classify_kernel(const BatchArgs a) {
  constexpr int R = kClassifyChunk / kPlanThreads;
  __shared__ uint32_t hist[kKeys];
  for (int i = threadIdx.x; i < kKeys; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kClassifyChunk + threadIdx.x;
  uint32_t rid[R], off[R], e[R], m[R], nf[R];
  uint2 ni[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t p = base + (uint64_t)r * kPlanThreads;
    rid[r] = 0xFFFFFFFFu;
    off[r] = 0;
    e[r] = a.f.fixed_e;
    if (p < a.f.n_pairs) {
      rid[r] = a.f.pair_read[p];
      off[r] = a.f.pair_off[p];
      if (a.f.pair_e) e[r] = a.f.pair_e[p];
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    m[r] = 0;
    nf[r] = 0;
    ni[r] = make_uint2(0u, 0xFFFFFFFFu);
    if ((uint64_t)rid[r] < a.f.n_reads) {
      m[r] = a.read_len[rid[r]];
      if (a.f.read_nflag) nf[r] = a.f.read_nflag[rid[r]];
    }
    if (a.f.ref_nidx && (uint64_t)off[r] < a.f.ref_len) ni[r] = a.f.ref_nidx[off[r] >> 5];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t p = base + (uint64_t)r * kPlanThreads;
    const bool active = p < a.f.n_pairs;
    int status = 0;  // 0 filter, 1 undefined, 2 invalid, 3 empty read
    uint32_t key = kNoKey;
    if (active) {
      const uint32_t mm = m[r];
      if ((uint64_t)rid[r] >= a.f.n_reads || mm > GK_MAX_LEN || mm > 32u * a.f.stride_words ||
          (uint64_t)off[r] + mm > a.f.ref_len)
        status = 2;
      if (status == 0 && mm == 0) status = 3;
      if (status == 0) {
        if (nf[r]) {
          status = 1;
        } else if (a.f.ref_nidx) {
          const uint32_t q = ni[r].x >> (off[r] & 31);
          const uint64_t firstN = q ? (uint64_t)off[r] + (uint32_t)(__ffs(q) - 1) : (uint64_t)ni[r].y;
          if (firstN < (uint64_t)off[r] + mm) status = 1;
        }
      }
      if (status == 0) {
        const uint32_t W = (mm + 31) / 32;
        const uint32_t K = min(e[r], 32u * W);
        key = key_of(W, min(K, 255u));
        atomicAdd(&hist[key], 1u);
      } else {
        write_trivial(a.f, p, status == 3 ? 0 : status);  // an empty read: count 0, accepted
      }
      a.s.km[p] = key | (mm << 16);
    }
    if (a.f.err_count) {
      const unsigned bad = __ballot_sync(0xffffffffu, status == 2);
      if ((threadIdx.x & 31) == 0 && bad) atomicAdd(a.f.err_count, (unsigned)__popc(bad));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kKeys; i += blockDim.x)
    if (hist[i]) atomicAdd(&a.s.hist[i], hist[i]);
}

// One block: exclusive scans over the key slots in descending key order.
__global__ void __launch_bounds__(1024) scan_kernel(const BatchArgs a) {
  constexpr int kPer = kKeys / 1024;  // slots per thread
  __shared__ uint32_t part_pairs[1024], part_tiles[1024];
  const int t = threadIdx.x;
  uint32_t np[kPer], nt[kPer];
  uint32_t sp = 0, st = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int slot = t * kPer + j;
    np[j] = a.s.hist[kKeys - 1 - slot];
    nt[j] = (np[j] + a.tile_pairs - 1) / a.tile_pairs;
    sp += np[j];
    st += nt[j];
  }
  part_pairs[t] = sp;
  part_tiles[t] = st;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan
    uint32_t vp = 0, vt = 0;
    if (t >= off) {
      vp = part_pairs[t - off];
      vt = part_tiles[t - off];
    }
    __syncthreads();
    part_pairs[t] += vp;
    part_tiles[t] += vt;
    __syncthreads();
  }
  uint32_t bp = part_pairs[t] - sp, bt = part_tiles[t] - st;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int slot = t * kPer + j;
    a.s.pair_base[slot] = bp;
    a.s.tile_base[slot] = bt;
    a.s.cursor[kKeys - 1 - slot] = bp;
    bp += np[j];
    bt += nt[j];
  }
  if (t == 1023) {
    a.s.pair_base[kKeys] = bp;
    a.s.tile_base[kKeys] = bt;
    a.s.counters[0] = 0;
    a.s.counters[1] = bt;
    a.s.counters[2] = 0;
    a.s.counters[3] = 0;
  }
}

// Each block takes kScatterChunk pairs: a block histogram reserves one range
// per key in the global cursors, then every pair writes its record (pair
// index, read id, offset, e and m) to a slot in its range, so the filter
// reads pair data in slot order.
__global__ void __launch_bounds__(kPlanThreads) scatter_kernel(const BatchArgs a) {
  __shared__ uint32_t local[kKeys];
  for (int i = threadIdx.x; i < kKeys; i += blockDim.x) local[i] = 0;
  __syncthreads();
  constexpr int R = kScatterChunk / kPlanThreads;
  const uint64_t p0 = (uint64_t)blockIdx.x * kScatterChunk + threadIdx.x;
  uint32_t km[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t p = p0 + (uint64_t)r * kPlanThreads;
    km[r] = p < a.f.n_pairs ? a.s.km[p] : (uint32_t)kNoKey;
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if ((km[r] & 0xFFFFu) != kNoKey) atomicAdd(&local[km[r] & 0xFFFFu], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kKeys; i += blockDim.x)
    if (local[i]) local[i] = atomicAdd(&a.s.cursor[i], local[i]);
  __syncthreads();
  uint32_t rid[R], off[R], e[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t p = p0 + (uint64_t)r * kPlanThreads;
    if ((km[r] & 0xFFFFu) != kNoKey) {
      rid[r] = a.f.pair_read[p];
      off[r] = a.f.pair_off[p];
      e[r] = a.f.pair_e ? (uint32_t)a.f.pair_e[p] : min(a.f.fixed_e, 0xFFFFu);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t k = km[r] & 0xFFFFu;
    if (k != kNoKey) {
      const uint64_t p = p0 + (uint64_t)r * kPlanThreads;
      a.s.rec[atomicAdd(&local[k], 1u)] = make_uint4((uint32_t)p, rid[r], off[r], e[r] | (km[r] & 0xFFFF0000u));
    }
  }
}

}  // namespace

uint64_t batch_scratch_bytes(uint64_t n_pairs) { return batch_scratch_size(n_pairs); }

BatchScratch batch_scratch_layout(void *base, uint64_t n_pairs) {
  auto up = [](uint64_t x) { return (x + 255) & ~uint64_t(255); };
  char *b = static_cast<char *>(base);
  BatchScratch s;
  s.km = reinterpret_cast<uint32_t *>(b);
  b += up(4 * n_pairs);
  s.rec = reinterpret_cast<uint4 *>(b);
  b += up(16 * n_pairs);
  s.hist = reinterpret_cast<uint32_t *>(b);
  b += up(4 * kKeys);
  s.cursor = reinterpret_cast<uint32_t *>(b);
  b += up(4 * kKeys);
  s.pair_base = reinterpret_cast<uint32_t *>(b);
  b += up(4 * (kKeys + 1));
  s.tile_base = reinterpret_cast<uint32_t *>(b);
  b += up(4 * (kKeys + 1));
  s.counters = reinterpret_cast<uint32_t *>(b);
  return s;
}

cudaError_t launch_whole_w1_8(const BatchArgs &a, uint32_t sms, uint32_t bpsm, uint32_t wpb, cudaStream_t s);
cudaError_t launch_whole_w9_12(const BatchArgs &a, uint32_t sms, uint32_t bpsm, uint32_t wpb, cudaStream_t s);
cudaError_t launch_whole_w13_16(const BatchArgs &a, uint32_t sms, uint32_t bpsm, uint32_t wpb, cudaStream_t s);
cudaError_t launch_persistent_wpt2(const BatchArgs &a, uint32_t grid, uint32_t wpb, cudaStream_t s);
cudaError_t launch_persistent_wpt3(const BatchArgs &a, uint32_t grid, uint32_t wpb, cudaStream_t s);
cudaError_t launch_persistent_wpt4(const BatchArgs &a, uint32_t grid, uint32_t wpb, cudaStream_t s);
cudaError_t launch_persistent_wpt6(const BatchArgs &a, uint32_t grid, uint32_t wpb, cudaStream_t s);
cudaError_t launch_persistent_wpt8(const BatchArgs &a, uint32_t grid, uint32_t wpb, cudaStream_t s);

cudaError_t launch_batched(int wpt, const BatchArgs &a, uint32_t blocks_per_sm, uint32_t warps_per_block,
                           cudaStream_t stream) {
  if (a.f.n_pairs == 0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(a.s.hist, 0, sizeof(uint32_t) * kKeys, stream);
  if (err != cudaSuccess) return err;
  const unsigned cblocks = (unsigned)((a.f.n_pairs + kClassifyChunk - 1) / kClassifyChunk);
  classify_kernel<<<cblocks, kPlanThreads, 0, stream>>>(a);
  scan_kernel<<<1, 1024, 0, stream>>>(a);
  const unsigned sblocks = (unsigned)((a.f.n_pairs + kScatterChunk - 1) / kScatterChunk);
  scatter_kernel<<<sblocks, kPlanThreads, 0, stream>>>(a);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t grid = (uint32_t)sms * blocks_per_sm;
  if (wpt == 1) {
    // One pair per lane: three W ranges, widest first; each launch drains its
    // own range of tiles.
    const uint32_t n = (uint32_t)sms;
    err = launch_whole_w13_16(a, n, blocks_per_sm, warps_per_block, stream);
    if (err == cudaSuccess) err = launch_whole_w9_12(a, n, blocks_per_sm, warps_per_block, stream);
    if (err == cudaSuccess) err = launch_whole_w1_8(a, n, blocks_per_sm, warps_per_block, stream);
    return err;
  }
  switch (wpt) {
    case 2: return launch_persistent_wpt2(a, grid, warps_per_block, stream);
    case 3: return launch_persistent_wpt3(a, grid, warps_per_block, stream);
    case 4: return launch_persistent_wpt4(a, grid, warps_per_block, stream);
    case 6: return launch_persistent_wpt6(a, grid, warps_per_block, stream);
    case 8: return launch_persistent_wpt8(a, grid, warps_per_block, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gk
