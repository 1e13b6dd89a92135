// Integer-pipe throughput probe (include/gk_probe.h): 64 independent ops per
// iteration, written as inline PTX so the compiler keeps exactly these
// instructions (lop3.b32 / shf.l.wrap.b32).
#include "gk_internal.cuh"
#include "gk_probe.h"

namespace {

__device__ __forceinline__ uint32_t lop3_xor_or(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  // (a ^ b) | c
  asm volatile("lop3.b32 %0, %1, %2, %3, 0xBE;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint32_t shf_l(uint32_t lo, uint32_t hi, uint32_t n) {
  uint32_t d;
  asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(lo), "r"(hi), "r"(n));
  return d;
}

template <int KIND>
__global__ void probe_kernel(uint32_t iters, uint32_t seed, uint32_t *sink) {
  constexpr int kChains = 16;
  uint32_t x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed ^ (threadIdx.x * 2654435761u + i * 40503u);
  const uint32_t k1 = seed | 1u, k2 = seed * 3u + 7u, sh = (seed & 15u) + 1u;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if (KIND == GK_PROBE_LOP3) {
          x[i] = lop3_xor_or(x[i], k1, k2 + r);
        } else if (KIND == GK_PROBE_SHF) {
          x[i] = shf_l(x[(i + 1) % kChains], x[i], sh);
        } else {
          x[i] = (r & 1) ? shf_l(x[(i + 1) % kChains], x[i], sh) : lop3_xor_or(x[i], k1, k2);
        }
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc ^= x[i];
  if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);  // practically never taken, not provably so
}

}  // namespace

extern "C" int gk_probe_alu(int kind, uint32_t iters, uint32_t blocks, uint32_t threads,
                            uint32_t *sink, void *stream) {
  gk::clear_error();
  if (!sink || blocks == 0 || threads == 0 || threads > 1024 || (threads % 32) != 0)
    return gk::fail(GK_EINVAL, "gk_probe_alu: bad launch shape or null sink");
  cudaStream_t s = (cudaStream_t)stream;
  switch (kind) {
    case GK_PROBE_LOP3: probe_kernel<GK_PROBE_LOP3><<<blocks, threads, 0, s>>>(iters, 0x1234567u, sink); break;
    case GK_PROBE_SHF: probe_kernel<GK_PROBE_SHF><<<blocks, threads, 0, s>>>(iters, 0x1234567u, sink); break;
    case GK_PROBE_MIX: probe_kernel<GK_PROBE_MIX><<<blocks, threads, 0, s>>>(iters, 0x1234567u, sink); break;
    default: return gk::fail(GK_EINVAL, "gk_probe_alu: unknown kind");
  }
  return gk::cuda_check(cudaGetLastError(), "gk_probe_alu: launch");
}
