// gk_filter_batched_noalloc: the batched filter running on scratch memory
// that is part of the library image instead of a caller-provided workspace.
//
// Who needs this: callers that cannot allocate device memory at the point
// where they filter, e.g. a plugin inside a host application whose device
// memory all belongs to the application's own pool, or a latency-bound thread
// that must not call cudaMalloc because it can synchronise the whole device.
// They pass inputs and outputs only; the scratch is a fixed-size array that
// every GPU loading the library keeps until the process exits.
#include <mutex>

#include "batched.cuh"
#include "gk_internal.cuh"

namespace {

constexpr uint64_t kNoallocMaxPairs = GK_NOALLOC_MAX_PAIRS;
// Same layout as the caller-provided workspace of gk_filter_batched.
constexpr uint64_t kNoallocBytes = gk::batch_scratch_size(kNoallocMaxPairs);

// The scratch itself.  Host code must not use this name as an address: it
// stands for the host-side shadow; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Per device: the scratch address and the unique ID of the context it was
// looked up in.  A device reset (cudaDeviceReset) or a released and re-created
// primary context gives a new context ID, and the address is looked up again.
void *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Driver calls through the runtime's entry-point table, so the library needs
// no link against libcuda (the CPU-only build and tests load it without a
// driver).  Signatures as cuda.h declares them; CUcontext is an opaque pointer.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

// Unique ID of the calling thread's current context, or 0 when none is
// current or the driver does not offer the query.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // under g_mutex
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    looked_up = true;
  }
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch on the current device, looked up with that
// device current on the first call and again whenever the device's context
// has changed since (ID 0, unknown, always looks up).
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return gk::cuda_check(err, "gk_filter_batched_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return gk::fail(GK_ERANGE, "gk_filter_batched_noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return gk::cuda_check(err, "gk_filter_batched_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = current_context_id();  // the lookup made the primary context current
  }
  *out = g_scratch_addr[dev];
  return GK_OK;
}

}  // namespace

extern "C" int gk_filter_batched_noalloc(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words,
                                         uint64_t n_reads, const uint16_t *read_len, const uint8_t *read_nflag,
                                         const uint32_t *pair_read, const uint32_t *pair_off,
                                         const uint8_t *pair_e, uint32_t fixed_e, uint64_t n_pairs,
                                         int count_mode, uint32_t flags, const gk_tiling_t *tiling,
                                         uint8_t *accept_out, uint16_t *edits_out, uint32_t *err_count,
                                         void *stream) {
  gk::clear_error();
  if (n_pairs > kNoallocMaxPairs)
    return gk::fail(GK_ERANGE, "gk_filter_batched_noalloc: n_pairs above GK_NOALLOC_MAX_PAIRS (1000000); "
                               "use gk_filter_batched with a workspace");
  if (n_pairs == 0) return GK_OK;
  void *scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != GK_OK) return rc;
  // The pipeline clears what must start at zero on every call (the key
  // histogram by a memset, the tile counter in its scan kernel) and writes
  // every other scratch word before reading it, so a previous call's contents
  // do no harm.
  return gk_filter_batched(ref, reads, stride_words, n_reads, read_len, read_nflag, pair_read, pair_off, pair_e,
                           fixed_e, n_pairs, count_mode, flags, tiling, scratch, kNoallocBytes, accept_out,
                           edits_out, err_count, stream);
}
