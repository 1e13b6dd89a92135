// Streamed host pipeline (gk_pipe_*): batches of fixed-length reads and their
// candidate pairs are copied in, encoded and filtered at every threshold of
// the pipe, and their results copied out, with n_slots batches in flight on
// three streams (Sec. 3.3, Sec. 3.5: host batches, one synchronisation point
// per batch).
//
// Ordering, per slot s (batches i, i + n_slots, ... use slot i mod n_slots):
//   copy-in of batch i   waits for run_done of batch i - n_slots (inputs consumed)
//   run of batch i       waits for in_done of batch i and out_done of batch
//                        i - n_slots (its result buffers read out)
//   copy-out of batch i  waits for run_done of batch i
// Each stream is in order, so batch i's out_done also marks every earlier
// batch's results as delivered.
#include <vector>

#include "gk_internal.cuh"

namespace {

constexpr uint32_t kMaxSlots = 4;
constexpr uint32_t kMaxThresholds = 64;

struct Slot {
  uint8_t *ascii = nullptr;
  uint32_t *pair_read = nullptr;
  uint32_t *read_start = nullptr;  // the batch's per-read starts (GK_PIPE_READ_STARTS)
  uint32_t *pair_off = nullptr;
  uint32_t *packed = nullptr;
  uint8_t *nflag = nullptr;
  uint8_t *accept = nullptr;
  uint16_t *edits = nullptr;
  uint8_t *sliced = nullptr;  // the batch in bit-sliced form (when the pipe slices)
  cudaEvent_t in_done = nullptr, run_done = nullptr, out_done = nullptr;
  bool used = false;
};

// Makes `dev` current for the lifetime of the guard, then restores the
// caller's device.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

struct gk_pipe_s {
  int device = -1;
  gk_ref_t ref = nullptr;
  uint64_t max_reads = 0, ascii_stride = 0, max_pairs = 0;
  uint32_t read_len = 0, stride_words = 0, n_slots = 0;
  std::vector<uint8_t> thresholds;
  int count_mode = GK_COUNT_RUNS4;
  uint32_t flags = 0;
  bool read_starts = false;  // pairs name their reads by per-read starts (GK_PIPE_READ_STARTS)
  uint64_t sliced_cap = 0;  // > 0: every batch is sliced once and filtered by gk_filter_sliced
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  Slot slot[kMaxSlots];
  uint64_t next_ticket = 0;
  int sticky = GK_OK;  // set by the first failure after work was enqueued
};

namespace {

void release(gk_pipe_s *p) {
  for (Slot &s : p->slot) {
    cudaFree(s.ascii);
    cudaFree(s.pair_read);
    cudaFree(s.read_start);
    cudaFree(s.pair_off);
    cudaFree(s.packed);
    cudaFree(s.nflag);
    cudaFree(s.accept);
    cudaFree(s.edits);
    cudaFree(s.sliced);
    if (s.in_done) cudaEventDestroy(s.in_done);
    if (s.run_done) cudaEventDestroy(s.run_done);
    if (s.out_done) cudaEventDestroy(s.out_done);
  }
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_run) cudaStreamDestroy(p->s_run);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  delete p;
}

template <typename T>
bool alloc(T **ptr, uint64_t bytes) {
  return cudaMalloc(reinterpret_cast<void **>(ptr), bytes ? bytes : 16) == cudaSuccess;
}

// Marks the pipe failed and returns the code.
int broken(gk_pipe_s *p, int code, const std::string &msg) {
  p->sticky = code;
  return gk::fail(code, msg);
}

}  // namespace

extern "C" {

int gk_pipe_create(gk_ref_t ref, const gk_pipe_desc_t *d, gk_pipe_t *out) {
  gk::clear_error();
  if (!ref || !d || !out) return gk::fail(GK_EINVAL, "gk_pipe_create: null argument");
  *out = nullptr;
  if (d->read_len == 0 || d->read_len > GK_MAX_LEN)
    return gk::fail(GK_ERANGE, "gk_pipe_create: read_len must be 1..GK_MAX_LEN");
  if (d->ascii_stride < d->read_len) return gk::fail(GK_EINVAL, "gk_pipe_create: ascii_stride < read_len");
  if (d->max_reads == 0 || d->max_pairs == 0 || d->max_pairs >= (1ull << 32))
    return gk::fail(GK_EINVAL, "gk_pipe_create: max_reads must be >= 1 and max_pairs 1..2^32-1");
  if (d->n_thresholds == 0 || d->n_thresholds > kMaxThresholds || !d->thresholds)
    return gk::fail(GK_EINVAL, "gk_pipe_create: n_thresholds must be 1..64 with a threshold array");
  if (d->count_mode != GK_COUNT_RUNS4 && d->count_mode != GK_COUNT_POPCOUNT)
    return gk::fail(GK_EINVAL, "gk_pipe_create: unknown count_mode");
  if (d->flags & ~(GK_FLAG_NO_EDGE_FIX | GK_FLAG_RESULT_BYTE | GK_PIPE_SLICED | GK_PIPE_READ_STARTS))
    return gk::fail(GK_EINVAL, "gk_pipe_create: unknown flags");
  if (d->flags & GK_FLAG_RESULT_BYTE)
    for (uint32_t i = 0; i < d->n_thresholds; ++i)
      if (d->thresholds[i] > 252) return gk::fail(GK_ERANGE, "gk_pipe_create: GK_FLAG_RESULT_BYTE needs e <= 252");
  if (d->n_slots < 2 || d->n_slots > kMaxSlots) return gk::fail(GK_EINVAL, "gk_pipe_create: n_slots must be 2..4");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return gk::fail(GK_ECUDA, "gk_pipe_create: cudaGetDevice failed");
  if (dev != ref->device)
    return gk::fail(GK_EINVAL, "gk_pipe_create: the reference lives on another device than the current one");

  gk_pipe_s *p = new gk_pipe_s;
  p->device = dev;
  p->ref = ref;
  p->max_reads = d->max_reads;
  p->ascii_stride = d->ascii_stride;
  p->max_pairs = d->max_pairs;
  p->read_len = d->read_len;
  p->stride_words = (d->read_len + 31) / 32;
  p->n_slots = d->n_slots;
  p->thresholds.assign(d->thresholds, d->thresholds + d->n_thresholds);
  p->count_mode = d->count_mode;
  p->flags = d->flags & ~(GK_PIPE_SLICED | GK_PIPE_READ_STARTS);  // the filters' flags
  p->read_starts = (d->flags & GK_PIPE_READ_STARTS) != 0;
  const uint64_t n_th = d->n_thresholds;
  // The bit-sliced filter when the pipe asks for it (GK_PIPE_SLICED) and it
  // covers the read length and every threshold (edge OR on, min(e, m-1)
  // within the compiled shift counts).
  bool slice = (d->flags & GK_PIPE_SLICED) && !(d->flags & GK_FLAG_NO_EDGE_FIX) && d->read_len >= 1 &&
               d->read_len <= GK_SLICED_MAX_LEN && d->max_pairs > 0;
  for (uint32_t i = 0; slice && i < d->n_thresholds; ++i)
    slice = (d->thresholds[i] < d->read_len - 1 ? d->thresholds[i] : d->read_len - 1) <= GK_SLICED_MAX_SHIFT;
  p->sliced_cap = slice ? gk_sliced_bytes(d->max_pairs, d->read_len) : 0;
  bool ok = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->s_run, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) == cudaSuccess;
  for (uint32_t i = 0; ok && i < p->n_slots; ++i) {
    Slot &s = p->slot[i];
    ok = alloc(&s.ascii, p->max_reads * p->ascii_stride) && alloc(&s.pair_read, 4 * p->max_pairs) &&
         (!p->read_starts || alloc(&s.read_start, 4 * p->max_reads)) &&
         alloc(&s.pair_off, 4 * p->max_pairs) && alloc(&s.packed, 8ull * p->stride_words * p->max_reads) &&
         alloc(&s.nflag, p->max_reads) && alloc(&s.accept, n_th * p->max_pairs) &&
         ((p->flags & GK_FLAG_RESULT_BYTE) || alloc(&s.edits, 2 * n_th * p->max_pairs)) &&
         (p->sliced_cap == 0 || alloc(&s.sliced, p->sliced_cap)) &&
         cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.run_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();  // clear a failed allocation
    release(p);
    return gk::fail(GK_ENOMEM, "gk_pipe_create: device allocation or stream/event creation failed");
  }
  *out = p;
  return GK_OK;
}

int gk_pipe_submit(gk_pipe_t p, const uint8_t *ascii, uint64_t n_reads, const uint32_t *pair_read,
                   const uint32_t *pair_off, uint64_t n_pairs, uint8_t *accept_out, uint16_t *edits_out,
                   uint64_t *ticket) {
  gk::clear_error();
  if (!p || !ticket) return gk::fail(GK_EINVAL, "gk_pipe_submit: null pipe or ticket");
  if (p->sticky != GK_OK) return gk::fail(p->sticky, "gk_pipe_submit: the pipe failed earlier");
  if (n_reads > p->max_reads || n_pairs > p->max_pairs)
    return gk::fail(GK_ERANGE, "gk_pipe_submit: batch larger than the pipe's max_reads / max_pairs");
  const bool result_byte = (p->flags & GK_FLAG_RESULT_BYTE) != 0;
  if ((n_reads && !ascii) || (n_pairs && (!pair_read || !pair_off || !accept_out || (!edits_out && !result_byte))))
    return gk::fail(GK_EINVAL, "gk_pipe_submit: null host buffer");
  DeviceGuard guard(p->device);
  if (guard.err != cudaSuccess) return broken(p, GK_ECUDA, "gk_pipe_submit: cannot make the pipe's device current");

  const uint64_t t = p->next_ticket;
  Slot &s = p->slot[t % p->n_slots];
  const uint64_t n_th = p->thresholds.size();
  auto cuda = [&](cudaError_t err, const char *what) {
    if (err == cudaSuccess) return true;
    broken(p, GK_ECUDA, std::string("gk_pipe_submit: ") + what + ": " + cudaGetErrorString(err));
    return false;
  };
  // copy in
  if (s.used && !cuda(cudaStreamWaitEvent(p->s_in, s.run_done, 0), "wait for the slot's inputs")) return p->sticky;
  if (n_reads && !cuda(cudaMemcpyAsync(s.ascii, ascii, n_reads * p->ascii_stride, cudaMemcpyHostToDevice, p->s_in),
                       "copy of the reads"))
    return p->sticky;
  if (n_pairs &&
      !((p->read_starts
             ? (n_reads == 0 ||
                cuda(cudaMemcpyAsync(s.read_start, pair_read, 4 * n_reads, cudaMemcpyHostToDevice, p->s_in),
                     "copy of the read starts"))
             : cuda(cudaMemcpyAsync(s.pair_read, pair_read, 4 * n_pairs, cudaMemcpyHostToDevice, p->s_in),
                    "copy of the read ids")) &&
        cuda(cudaMemcpyAsync(s.pair_off, pair_off, 4 * n_pairs, cudaMemcpyHostToDevice, p->s_in),
             "copy of the offsets")))
    return p->sticky;
  if (!cuda(cudaEventRecord(s.in_done, p->s_in), "event")) return p->sticky;
  // run
  if (!cuda(cudaStreamWaitEvent(p->s_run, s.in_done, 0), "wait for the copy-in")) return p->sticky;
  if (s.used && !cuda(cudaStreamWaitEvent(p->s_run, s.out_done, 0), "wait for the slot's results")) return p->sticky;
  if (n_reads) {
    const int rc = gk_encode(s.ascii, p->ascii_stride, nullptr, (uint16_t)p->read_len, n_reads, s.packed,
                             p->stride_words, s.nflag, 1, p->s_run);
    if (rc != GK_OK) return broken(p, rc, std::string("gk_pipe_submit: ") + gk_last_error());
  }
  if (p->read_starts && n_pairs &&
      !cuda(gk::launch_expand_rows(s.pair_read, n_pairs, s.read_start, n_reads, p->s_run), "read ids from the starts"))
    return p->sticky;
  if (p->sliced_cap && n_pairs) {
    const int rc = gk_slice(p->ref, s.packed, p->stride_words, n_reads, s.nflag, p->read_len, s.pair_read,
                            s.pair_off, n_pairs, s.sliced, p->sliced_cap, nullptr, p->s_run);
    if (rc != GK_OK) return broken(p, rc, std::string("gk_pipe_submit: ") + gk_last_error());
  }
  for (uint64_t i = 0; i < n_th && n_pairs;) {
    // Every run of consecutive thresholds (e, e+1, ...) is one sweep launch
    // when the sweep covers it (edge OR on, shift counts within the
    // sweep's limit), sliced when the pipe slices, per pair otherwise.
    const bool sweep_ok = !(p->flags & GK_FLAG_NO_EDGE_FIX);
    uint64_t j = i;
    if (sweep_ok || p->sliced_cap)
      while (j + 1 < n_th && p->thresholds[j + 1] == p->thresholds[j] + 1 &&
             (p->sliced_cap || (p->thresholds[j + 1] < p->read_len - 1 ? p->thresholds[j + 1] : p->read_len - 1) <=
                                   GK_SWEEP_MAX_SHIFT))
        ++j;
    const uint32_t ki = p->thresholds[i] < p->read_len - 1 ? p->thresholds[i] : p->read_len - 1;
    int rc;
    if (p->sliced_cap)
      rc = gk_filter_sliced_sweep(s.sliced, p->sliced_cap, n_pairs, p->read_len, p->thresholds[i], p->thresholds[j],
                                  p->count_mode, p->flags, s.accept + i * n_pairs,
                                  result_byte ? nullptr : s.edits + i * n_pairs, n_pairs, nullptr, p->s_run);
    else if (sweep_ok && ki <= GK_SWEEP_MAX_SHIFT)
      rc = gk_filter_sweep(p->ref, s.packed, p->stride_words, n_reads, s.nflag, p->read_len, s.pair_read, s.pair_off,
                           p->thresholds[i], p->thresholds[j], n_pairs, p->count_mode, p->flags,
                           s.accept + i * n_pairs, result_byte ? nullptr : s.edits + i * n_pairs, n_pairs, nullptr,
                           p->s_run);
    else
      rc = gk_filter(p->ref, s.packed, p->stride_words, n_reads, s.nflag, p->read_len, s.pair_read, s.pair_off,
                     nullptr, p->thresholds[i], n_pairs, p->count_mode, p->flags, s.accept + i * n_pairs,
                     result_byte ? nullptr : s.edits + i * n_pairs, nullptr, p->s_run);
    if (rc != GK_OK) return broken(p, rc, std::string("gk_pipe_submit: ") + gk_last_error());
    i = j + 1;
  }
  if (!cuda(cudaEventRecord(s.run_done, p->s_run), "event")) return p->sticky;
  // copy out
  if (!cuda(cudaStreamWaitEvent(p->s_out, s.run_done, 0), "wait for the run")) return p->sticky;
  if (n_pairs && !(cuda(cudaMemcpyAsync(accept_out, s.accept, n_th * n_pairs, cudaMemcpyDeviceToHost, p->s_out),
                        "copy of the accept bits") &&
                   (result_byte ||
                    cuda(cudaMemcpyAsync(edits_out, s.edits, 2 * n_th * n_pairs, cudaMemcpyDeviceToHost, p->s_out),
                         "copy of the edit counts"))))
    return p->sticky;
  if (!cuda(cudaEventRecord(s.out_done, p->s_out), "event")) return p->sticky;
  s.used = true;
  p->next_ticket = t + 1;
  *ticket = t;
  return GK_OK;
}

int gk_pipe_wait(gk_pipe_t p, uint64_t ticket) {
  gk::clear_error();
  if (!p) return gk::fail(GK_EINVAL, "gk_pipe_wait: null pipe");
  if (ticket >= p->next_ticket) return gk::fail(GK_EINVAL, "gk_pipe_wait: ticket not submitted");
  if (p->sticky != GK_OK) return gk::fail(p->sticky, "gk_pipe_wait: the pipe failed earlier");
  DeviceGuard guard(p->device);
  if (guard.err != cudaSuccess) return broken(p, GK_ECUDA, "gk_pipe_wait: cannot make the pipe's device current");
  // The slot now holds `ticket` or a later batch; the copy-out stream is in
  // order, so that batch's out_done covers `ticket` too.
  const cudaError_t err = cudaEventSynchronize(p->slot[ticket % p->n_slots].out_done);
  if (err != cudaSuccess)
    return broken(p, GK_ECUDA, std::string("gk_pipe_wait: ") + cudaGetErrorString(err));
  return GK_OK;
}

void gk_pipe_destroy(gk_pipe_t p) {
  if (!p) return;
  DeviceGuard guard(p->device);
  if (p->s_in) cudaStreamSynchronize(p->s_in);
  if (p->s_run) cudaStreamSynchronize(p->s_run);
  if (p->s_out) cudaStreamSynchronize(p->s_out);
  release(p);
}

}  // extern "C"
