/*
 * gk.h -- C ABI of the GateKeeper-GPU pre-alignment filter for sm_103a.
 *
 * The filter (arxiv 2103.14978) decides, for each pair of a read and a
 * candidate reference segment of the same length m, whether the pair can be
 * within e edits.  Per pair it builds the Hamming mask and the 2e masks of
 * the read shifted by 1..e bases each way (Sec. 2.1), amends 0-streaks of
 * length 1-2 bounded by 1s (Sec. 2.1), sets each shifted mask's vacated edge
 * bits after amendment (Sec. 3.4), ANDs the 2e+1 masks and counts the errors
 * of the result with a 4-base window table (Sec. 2.1); the pair is accepted
 * iff the count is at most e.  Pairs whose read or window holds a base other
 * than A/C/G/T pass without filtration (Sec. 3.3).
 *
 * Conventions shared by every entry point:
 *   - return 0 (GK_OK) on success or a negative GK_E* code; the thread's last
 *     message is in gk_last_error();
 *   - device pointers are plain CUDA device addresses (e.g. torch tensors'
 *     data pointers) of the current device; the library never frees memory it
 *     did not allocate;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); work is
 *     enqueued asynchronously and results are valid once the stream has
 *     reached the point of the call (the one sync point of Sec. 3.5);
 *   - no kernel traps or spins: bad per-pair input yields a sentinel and a
 *     counted device error, never a fault.
 *
 * Packed layout ("2-bit planes"): a sequence of m bases is W = ceil(m/32)
 * words; word w is two uint32 stored adjacently, first the high bit plane
 * then the low bit plane of the 2-bit codes A=00 C=01 G=10 T=11 (Sec. 2.1)
 * for bases 32w..32w+31, base 32w+b in bit b.  Bits of bases >= m are 0.  A
 * base that is not A/C/G/T (either case) is stored as 00 and flagged.
 */
#ifndef GK_H
#define GK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GK_MAX_LEN 512 /* longest read / reference window, in bases */

#define GK_OK 0
#define GK_EINVAL (-1)  /* a null pointer, size or stride that cannot be right */
#define GK_ERANGE (-2)  /* a length above GK_MAX_LEN or a count too large */
#define GK_ENOMEM (-3)  /* a library allocation failed */
#define GK_ECUDA (-4)   /* a CUDA call or kernel launch failed */

#define GK_COUNT_RUNS4 0    /* runs of 1s per 4-base window (default) */
#define GK_COUNT_POPCOUNT 1 /* number of 1s in the final vector */

#define GK_FLAG_NO_EDGE_FIX 1u /* skip the Sec. 3.4 improvement (the original
                                  GateKeeper), for accuracy comparisons */
#define GK_FLAG_RESULT_BYTE 2u /* one result byte per pair in accept_out (no
                                  edits_out): see gk_filter */

/* Result bytes of GK_FLAG_RESULT_BYTE: a filtered pair's count capped at
 * GK_RESULT_MAX_COUNT, or one of the two sentinels.  With a threshold
 * e <= 252 the pair is accepted iff byte <= e or byte == GK_RESULT_UNDEFINED. */
#define GK_RESULT_MAX_COUNT 253u
#define GK_RESULT_UNDEFINED 254u /* non-ACGT base in the read or window: accepted */
#define GK_RESULT_INVALID 255u   /* read id or window out of range: rejected */

#define GK_EDITS_UNDEFINED 0xFFFFu /* pair holds a non-ACGT base: accept = 1 */
#define GK_EDITS_INVALID 0xFFFEu   /* read id or window out of range: accept = 0 */

typedef struct gk_ref_s *gk_ref_t;

/* Message of the calling thread's last failed call ("" if none).  The
 * pointer stays valid until that thread's next gk_* call. */
const char *gk_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int gk_version(void);

/*
 * gk_encode -- 2-bit encoding of reads (Sec. 3.3: encode once, 16 bases per
 * 32-bit word in the paper; here two 32-base bit planes per word pair).
 *
 *   ascii        n_seq sequences, sequence i starting at ascii + i*ascii_stride
 *   ascii_stride bytes between sequence starts (>= the longest length)
 *   lens         per-sequence lengths (uint16, each <= GK_MAX_LEN), or NULL
 *                to use fixed_len for all
 *   packed       output, n_seq * stride_words * 2 uint32: sequence i's word w
 *                at packed[(i*stride_words + w)*2 + {0: high, 1: low}];
 *                words past ceil(len/32) are zeroed
 *   stride_words words per sequence, >= ceil(longest length / 32)
 *   nflag        output, n_seq bytes: 1 if the sequence holds a non-ACGT
 *                byte within its length, else 0
 *   on_device    1: every pointer is device memory and the work is a kernel
 *                on `stream`; 0: every pointer is host memory and the call
 *                encodes on the host threads before returning
 * Caller owns all buffers.  Bytes past a sequence's length are never read.
 */
int gk_encode(const uint8_t *ascii, uint64_t ascii_stride, const uint16_t *lens,
              uint16_t fixed_len, uint64_t n_seq, uint32_t *packed,
              uint32_t stride_words, uint8_t *nflag, int on_device, void *stream);

/*
 * gk_load_reference -- encode a reference genome once and keep it resident
 * on the current device (Sec. 3.5: the reference is encoded and loaded once,
 * and the positions of 'N' are recorded while encoding).
 *
 *   ascii     n_bases ASCII bytes (host memory if on_device == 0, else
 *             device memory); n_bases < 2^32 - 2^16
 *   out       receives the handle
 * The handle owns device buffers of about n_bases/4 + n_bases/4 bytes (the
 * two planes plus an N index); the call returns once they are filled.
 * Free with gk_free_reference.  Errors: GK_EINVAL (null pointer, empty or too
 * long reference), GK_ENOMEM, GK_ECUDA.
 */
int gk_load_reference(const uint8_t *ascii, uint64_t n_bases, int on_device,
                      void *stream, gk_ref_t *out);

/* Release a handle and its device buffers (NULL is ignored).  The caller
 * guarantees no enqueued filter still reads it. */
void gk_free_reference(gk_ref_t ref);

/* Length in bases and number of non-ACGT bases of a loaded reference. */
int gk_reference_info(gk_ref_t ref, uint64_t *n_bases, uint64_t *n_undefined);

/*
 * gk_filter -- filter n_pairs (read, candidate offset) pairs of one read
 * length m against a loaded reference (Sec. 2.1, Sec. 3.3, Sec. 3.4; one
 * result per pair as in Sec. 3.5).
 *
 *   ref          handle from gk_load_reference (same device)
 *   reads        packed reads (device), n_reads * stride_words * 2 uint32,
 *                as written by gk_encode
 *   stride_words words per packed read, >= ceil(m/32)
 *   n_reads      number of packed reads
 *   read_nflag   device, n_reads bytes (non-zero: the read holds a non-ACGT
 *                base), or NULL when no read does
 *   m            read length of every pair, 0..GK_MAX_LEN
 *   pair_read    device, n_pairs uint32 read ids
 *   pair_off     device, n_pairs uint32 reference offsets: the segment is
 *                bases [off, off+m) of the reference
 *   pair_e       device, n_pairs uint8 thresholds, or NULL to use fixed_e
 *   fixed_e      threshold for every pair when pair_e is NULL (0..255)
 *   count_mode   GK_COUNT_RUNS4 or GK_COUNT_POPCOUNT
 *   flags        0, GK_FLAG_NO_EDGE_FIX and/or GK_FLAG_RESULT_BYTE
 *   accept_out   device, n_pairs uint8: 1 accept, 0 reject; with
 *                GK_FLAG_RESULT_BYTE instead the pair's result byte: its
 *                count capped at GK_RESULT_MAX_COUNT, GK_RESULT_UNDEFINED or
 *                GK_RESULT_INVALID (a third of the bytes to move; it needs
 *                pair_e NULL and fixed_e <= 252, else GK_EINVAL / GK_ERANGE)
 *   edits_out    device, n_pairs uint16: the error count (not clamped at e),
 *                GK_EDITS_UNDEFINED or GK_EDITS_INVALID; unused (may be NULL)
 *                with GK_FLAG_RESULT_BYTE
 *   err_count    device uint32 or NULL: incremented once per invalid pair
 *                (read id >= n_reads or off + m > reference length)
 * Asynchronous on `stream`; n_pairs == 0 enqueues nothing.  Host-side
 * argument errors return GK_EINVAL / GK_ERANGE before any work is enqueued.
 */
int gk_filter(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words,
              uint64_t n_reads, const uint8_t *read_nflag, uint32_t m,
              const uint32_t *pair_read, const uint32_t *pair_off,
              const uint8_t *pair_e, uint32_t fixed_e, uint64_t n_pairs,
              int count_mode, uint32_t flags, uint8_t *accept_out,
              uint16_t *edits_out, uint32_t *err_count, void *stream);

/*
 * gk_filter_sweep -- gk_filter at every threshold e = e_lo .. e_hi (the
 * paper's threshold sweeps, Sec. 4) in one launch, each result equal to
 * gk_filter's at that e with the edge OR on.  The 2K+1 masks of shift count
 * K are those of K-1 and the two shifted by K, so each pair's running AND is
 * built once up to min(e_hi, m-1) and finished (erosion, end corrections,
 * count) at every threshold: one pass instead of e_hi - e_lo + 1.  Pairs
 * with a non-ACGT base are skipped once for all thresholds.
 *
 * Arguments as gk_filter, except:
 *   e_lo, e_hi   thresholds, e_lo <= e_hi <= 255 and min(e_hi, m-1) <=
 *                GK_SWEEP_MAX_SHIFT (the deferred-erosion form's limit)
 *   flags        0 or GK_FLAG_RESULT_BYTE (e_hi <= 252); GK_FLAG_NO_EDGE_FIX
 *                is GK_EINVAL
 *   accept_out   device, the results of threshold e at accept_out +
 *                (e - e_lo) * out_stride (n_pairs each)
 *   edits_out    likewise (uint16 elements); unused with GK_FLAG_RESULT_BYTE
 *   out_stride   elements between consecutive thresholds' rows, >= n_pairs
 * Asynchronous on `stream`; argument errors before any work.
 */
#define GK_SWEEP_MAX_SHIFT 30u
int gk_filter_sweep(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words,
                    uint64_t n_reads, const uint8_t *read_nflag, uint32_t m,
                    const uint32_t *pair_read, const uint32_t *pair_off, uint32_t e_lo,
                    uint32_t e_hi, uint64_t n_pairs, int count_mode, uint32_t flags,
                    uint8_t *accept_out, uint16_t *edits_out, uint64_t out_stride,
                    uint32_t *err_count, void *stream);

/*
 * gk_filter_ascii -- gk_filter on reads given as ASCII rows, encoded inside
 * the filter kernel (the paper's device-encoded mode, Sec. 3.3, without a
 * separate encoding pass or a packed copy of the reads).  The warp encodes
 * each distinct read among its 32 pairs once (runs of one read id), so
 * candidates of a read should sit side by side; any order is correct.
 * Same results as gk_encode + gk_filter on the same reads.
 *
 * Arguments as gk_filter, except:
 *   ascii        device, n_reads rows of ascii_stride bytes (read i at
 *                ascii + i*ascii_stride); only the first m bytes of a row are
 *                read; a byte other than A/C/G/T (either case) makes the
 *                read undefined (Sec. 3.3)
 *   ascii_stride bytes between rows, >= m (rows on 4-byte boundaries are
 *                loaded 4 bytes at a time)
 * Errors as gk_filter (GK_EINVAL for a null ascii with m > 0 or a stride
 * below m).
 */
int gk_filter_ascii(gk_ref_t ref, const uint8_t *ascii, uint64_t ascii_stride,
                    uint64_t n_reads, uint32_t m, const uint32_t *pair_read,
                    const uint32_t *pair_off, const uint8_t *pair_e,
                    uint32_t fixed_e, uint64_t n_pairs, int count_mode,
                    uint32_t flags, uint8_t *accept_out, uint16_t *edits_out,
                    uint32_t *err_count, void *stream);

/*
 * Bit-sliced batches: the same filter (Sec. 2.1, Sec. 3.3, Sec. 3.4) for a
 * batch filtered at several thresholds, as in the paper's threshold sweeps
 * (Sec. 4).  gk_slice gathers every pair's read and genome window once and
 * stores them position-major, 32 pairs per 32-bit word (one word per base
 * position and bit plane); each gk_filter_sliced call then filters the whole
 * batch at one threshold from that buffer.  Results equal gk_filter's with
 * the edge OR on (flags without GK_FLAG_NO_EDGE_FIX), bit for bit.
 * Limits: 1 <= m <= GK_SLICED_MAX_LEN, min(e, m-1) <= GK_SLICED_MAX_SHIFT.
 */
#define GK_SLICED_MAX_LEN 255u
#define GK_SLICED_MAX_SHIFT 15u

/* Bytes of the sliced buffer of n_pairs pairs of read length m:
 * (2(m + 24) + 1) * 8 * (ceil(n_pairs/32) rounded up to 32) + 16 (the last 16
 * bytes: a header recording m and n_pairs); 0 when n_pairs is 0 or m is
 * outside 1..GK_SLICED_MAX_LEN. */
uint64_t gk_sliced_bytes(uint64_t n_pairs, uint32_t m);

/*
 * gk_slice -- fill a sliced buffer from the pairs (arguments as gk_filter).
 *   sliced       device, caller-owned, 16-byte aligned, sliced_cap bytes
 *                (at least gk_sliced_bytes(n_pairs, m)); holds the batch
 *                until overwritten
 *   err_count    device uint32 or NULL: incremented once per invalid pair
 * Each pair's status is decided here: invalid (read id >= n_reads or
 * off + m > reference length) and undefined (a non-ACGT base in the read or
 * the window) pairs get their fixed results from every gk_filter_sliced.
 * Asynchronous on `stream`; GK_EINVAL / GK_ERANGE before any work for bad
 * arguments.
 */
int gk_slice(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words,
             uint64_t n_reads, const uint8_t *read_nflag, uint32_t m,
             const uint32_t *pair_read, const uint32_t *pair_off,
             uint64_t n_pairs, void *sliced, uint64_t sliced_cap,
             uint32_t *err_count, void *stream);

/*
 * gk_filter_sliced -- filter a sliced batch at threshold fixed_e.
 *   sliced, sliced_cap  a buffer filled by gk_slice with the same n_pairs
 *                       and m; the kernel compares both with the header
 *                       gk_slice wrote, and on a mismatch (a buffer sliced
 *                       for another batch, or never sliced) writes the
 *                       invalid result (accept 0, GK_EDITS_INVALID or
 *                       GK_RESULT_INVALID) for every pair
 *   fixed_e             0..255; min(fixed_e, m-1) <= GK_SLICED_MAX_SHIFT
 *   count_mode          GK_COUNT_RUNS4 or GK_COUNT_POPCOUNT
 *   flags               0 or GK_FLAG_RESULT_BYTE (fixed_e <= 252);
 *                       GK_FLAG_NO_EDGE_FIX is GK_EINVAL
 *   accept_out, edits_out  as gk_filter (16-byte aligned buffers take
 *                       vector stores)
 * Asynchronous on `stream`.
 */
int gk_filter_sliced(const void *sliced, uint64_t sliced_cap, uint64_t n_pairs,
                     uint32_t m, uint32_t fixed_e, int count_mode,
                     uint32_t flags, uint8_t *accept_out, uint16_t *edits_out,
                     void *stream);

/*
 * gk_filter_sliced_sweep -- filter a sliced batch at every threshold
 * e = e_lo .. e_hi (the paper's threshold sweeps, Sec. 4), each result the
 * same as gk_filter_sliced's at that e.  The 2K+1 masks of shift count K are
 * those of K-1 plus the two shifted by K, so the running AND of every K
 * comes out of one pass over the batch's positions: each compiled range of
 * shift counts (0..5 and 6..10) is one launch that reads the planes once;
 * a shift count outside the ranges, or a range holding one threshold of the
 * sweep, takes the single-threshold kernel.
 *   sliced, sliced_cap, n_pairs, m, count_mode   as gk_filter_sliced
 *   e_lo, e_hi   thresholds, e_lo <= e_hi <= 255, min(e_hi, m-1) <=
 *                GK_SLICED_MAX_SHIFT
 *   flags        0 or GK_FLAG_RESULT_BYTE (e_hi <= 252)
 *   accept_out   device, the results of threshold e at accept_out +
 *                (e - e_lo) * out_stride (n_pairs bytes each)
 *   edits_out    device, likewise (uint16 elements); unused (may be NULL)
 *                with GK_FLAG_RESULT_BYTE
 *   out_stride   elements between the rows of consecutive thresholds,
 *                >= n_pairs (a multiple of 16 with 16-byte aligned
 *                buffers gives vector stores)
 *   err_count    device uint32 or NULL: incremented by the pairs of every
 *                launch whose buffer header does not match (m, n_pairs)
 * Asynchronous on `stream`; GK_EINVAL / GK_ERANGE before any work for bad
 * arguments.
 */
int gk_filter_sliced_sweep(const void *sliced, uint64_t sliced_cap, uint64_t n_pairs,
                           uint32_t m, uint32_t e_lo, uint32_t e_hi, int count_mode,
                           uint32_t flags, uint8_t *accept_out, uint16_t *edits_out,
                           uint64_t out_stride, uint32_t *err_count, void *stream);

/* Tiling of the batched filter (chosen by the autotuner). */
typedef struct {
  uint32_t words_per_thread; /* words of a pair held per lane: 2, 3, 4, 6 or 8;
                                1 = a whole pair per lane for reads up to 256
                                bases (4 words per lane above) */
  uint32_t tile_pairs;       /* pairs per tile (work unit of a warp), 32..65536 */
  uint32_t blocks_per_sm;    /* persistent grid = SM count x this, 1..32 */
  uint32_t warps_per_block;  /* 1..8 */
} gk_tiling_t;

/* Workspace bytes gk_filter_batched needs for n_pairs pairs (20 bytes per
 * pair plus 80 KiB). */
uint64_t gk_filter_batched_workspace(uint64_t n_pairs);

/*
 * gk_filter_batched -- filter pairs of mixed read lengths and per-pair
 * thresholds in one persistent launch (the paper batches many reads and their
 * candidates per kernel call, Sec. 3.3 and Sec. 3.5; same per-pair result as
 * gk_filter, Sec. 2.1/3.3/3.4).
 *
 * Arguments as gk_filter, except:
 *   read_len    device, n_reads uint16 lengths (each read may differ; a read
 *               longer than GK_MAX_LEN or than 32*stride_words makes its
 *               pairs invalid)
 *   flags       GK_FLAG_RESULT_BYTE is allowed with pair_e: accept_out gets
 *               the result bytes (edits_out may be NULL); a pair's decision
 *               reads from its byte only for thresholds <= 252, which the
 *               caller keeps (the bytes themselves are defined for any e)
 *   tiling      host pointer, see gk_tiling_t
 *   workspace   device scratch of at least gk_filter_batched_workspace(
 *               n_pairs) bytes, 256-byte aligned, owned by the caller; its
 *               contents need no initialisation and are garbage afterwards;
 *               two calls in flight at once need two workspaces
 * Enqueues a memset, three planning kernels (classify, scan, scatter) and the
 * persistent filter kernel on `stream`; everything is stream-ordered and can
 * be captured in a CUDA graph.  n_pairs must be < 2^32.
 */
int gk_filter_batched(gk_ref_t ref, const uint32_t *reads, uint32_t stride_words,
                      uint64_t n_reads, const uint16_t *read_len,
                      const uint8_t *read_nflag, const uint32_t *pair_read,
                      const uint32_t *pair_off, const uint8_t *pair_e,
                      uint32_t fixed_e, uint64_t n_pairs, int count_mode,
                      uint32_t flags, const gk_tiling_t *tiling, void *workspace,
                      uint64_t workspace_bytes, uint8_t *accept_out,
                      uint16_t *edits_out, uint32_t *err_count, void *stream);

/*
 * gk_rebase_pairs -- read-id rebasing for coalesced launches.  When the pairs
 * of several requests are concatenated into one launch (continuous batching;
 * the paper fills one batch with many reads and their candidates, Sec. 3.5),
 * each request's read ids are relative to its own reads; this adds a
 * per-request offset in place and, optionally, writes each request's
 * threshold into every one of its pairs.
 *
 *   pair_read  device, n_pairs uint32, rewritten in place
 *   pair_e     device, n_pairs uint8 written from seg_e, or NULL
 *   seg_end    device, n_segs uint64: cumulative pair counts (request i owns
 *              pairs [seg_end[i-1], seg_end[i]), the last value >= n_pairs)
 *   seg_delta  device, n_segs int64: offset added to request i's read ids
 *   seg_e      device, n_segs uint8 thresholds (needed when pair_e is set)
 * A result outside 0..2^32-1 becomes 0xFFFFFFFF, which the filters report as
 * an invalid pair.  Asynchronous on `stream`.
 */
int gk_rebase_pairs(uint32_t *pair_read, uint8_t *pair_e, uint64_t n_pairs,
                    const uint64_t *seg_end, const int64_t *seg_delta,
                    const uint8_t *seg_e, uint32_t n_segs, void *stream);

/*
 * gk_expand_pairs -- per-pair read ids and thresholds of a coalesced launch
 * from per-read start offsets, so that a request's candidates travel as
 * their offsets plus one 32-bit start per read (CSR rows: read k's
 * candidates are pairs start[k] .. start[k+1]-1 of its request) instead of
 * one read id per pair (the paper's batches hold each read with its
 * candidate locations, Sec. 3.5).
 *
 * The launch covers pairs [0, n_pairs) of pair_read / pair_e and n_reads
 * reads numbered across n_segs segments (requests):
 *   seg_read_end   device, n_segs uint64: cumulative read counts (segment i
 *                  owns reads [seg_read_end[i-1], seg_read_end[i]))
 *   seg_pair_end   device, n_segs uint64: cumulative pair counts (segment i
 *                  owns pairs [seg_pair_end[i-1], seg_pair_end[i]))
 *   seg_read_slot  device, n_segs uint64: the read-buffer row of segment i's
 *                  first read (its reads occupy consecutive rows)
 *   seg_start_base device, n_segs uint32: subtracted (mod 2^32) from segment
 *                  i's start values, so that a request cut from a larger
 *                  numbering needs no rewriting
 *   seg_e          device, n_segs uint8 thresholds
 *   read_start     device, uint32 per read-buffer row: the start value of the
 *                  read in that row
 *   seg_read_info  device, n_segs uint32, or NULL: bits 0..15 a read length
 *                  shared by all of segment i's reads (0: lengths given per
 *                  read), bit GK_SEG_NO_N set when none of them holds a
 *                  non-ACGT base; for those segments the kernel writes
 *                  read_len / read_nflag (device, uint16 / uint8 per
 *                  read-buffer row; NULL when no segment needs them), so
 *                  such requests need not send these per-read arrays
 * Writes pair_read[j] = the row of the read owning pair j and pair_e[j] =
 * its segment's threshold.  Starts are clamped to the segment's pairs; a
 * pair that no read claims (before the first read's start) gets id
 * 0xFFFFFFFF, which the filters report as an invalid pair; with decreasing
 * starts a pair may be claimed by two reads and gets one of them.
 * Asynchronous on `stream`.
 */
#define GK_SEG_NO_N 0x10000u

int gk_expand_pairs(uint32_t *pair_read, uint8_t *pair_e, uint64_t n_pairs, const uint32_t *read_start,
                    const uint64_t *seg_read_end, const uint64_t *seg_pair_end, const uint64_t *seg_read_slot,
                    const uint32_t *seg_start_base, const uint8_t *seg_e, const uint32_t *seg_read_info,
                    uint16_t *read_len, uint8_t *read_nflag, uint32_t n_segs, uint64_t n_reads, void *stream);

/*
 * gk_copy_many -- n asynchronous copies on `stream`, one cudaMemcpyAsync
 * each (kind 1: host to device, 2: device to host, 3: device to device), so
 * that a coalesced launch moves many requests' inputs with one call.  Host
 * buffers should be pinned for the copies to be asynchronous.  Stops at the
 * first failing copy with GK_ECUDA.
 */
int gk_copy_many(void *const *dst, const void *const *src, const uint64_t *bytes,
                 uint32_t n, int kind, void *stream);

/*
 * gk_gather -- n copies done by one kernel instead of the copy engines, so
 * that a coalesced launch moves many requests' small inputs without one
 * copy-engine transfer per array (the continuous-batching analogue of the
 * paper filling one batch from many reads, Sec. 3.5).  Two blocks per SM
 * walk the entries; entry i copies bytes[i] bytes from src[i] to dst[i], with
 * 16-byte accesses when both addresses have the same offset modulo 16, else
 * 4-byte or 1-byte ones.
 *   dst, src   n addresses the device can access: device memory, or
 *              page-locked host memory (with unified addressing its host
 *              pointer is valid on the device and the kernel reads it over
 *              the host link)
 *   bytes      n sizes, each at most GK_GATHER_MAX_BYTES (larger entries
 *              are skipped: split them)
 *   The three tables are read by the kernel, so they must be device memory
 *   or page-locked host memory and stay unchanged until the kernel has run.
 *   Overlapping source and destination ranges give undefined contents.
 *   Asynchronous on `stream`.
 */
#define GK_GATHER_MAX_BYTES 65536u
int gk_gather(const uint64_t *dst, const uint64_t *src, const uint64_t *bytes,
              uint32_t n, void *stream);

/*
 * gk_filter_batched_noalloc -- gk_filter_batched for callers that cannot
 * allocate device memory when they filter: for example a plugin inside a host
 * application whose device memory is all owned by the application's own
 * pool, or a latency-bound thread that must not call cudaMalloc because it can
 * synchronise the whole device.  The paper has no counterpart; this is a
 * deployment convenience.
 *
 * Same arguments and results as gk_filter_batched, without the workspace:
 * the scratch is a fixed array inside the library image (about 19.1 MiB per
 * GPU, held by every GPU that loads the library until the process exits).
 * The call allocates nothing.
 *   - n_pairs is limited to GK_NOALLOC_MAX_PAIRS; larger batches return
 *     GK_ERANGE with a message (use gk_filter_batched then).
 *   - The first call on each device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     The address is kept per device together with the ID of the context it
 *     belongs to: after a cudaDeviceReset (or a released and re-created
 *     primary context) the next call sees a new context and looks the
 *     address up again, so make that call before any capture too.
 *   - All calls share the one array and each call overwrites it.  Calls whose
 *     work overlaps on the GPU (e.g. on two streams without ordering) race
 *     and give wrong results: keep them ordered on one stream or serialise
 *     them.
 */
#define GK_NOALLOC_MAX_PAIRS 1000000u

int gk_filter_batched_noalloc(gk_ref_t ref, const uint32_t *reads,
                              uint32_t stride_words, uint64_t n_reads,
                              const uint16_t *read_len, const uint8_t *read_nflag,
                              const uint32_t *pair_read, const uint32_t *pair_off,
                              const uint8_t *pair_e, uint32_t fixed_e,
                              uint64_t n_pairs, int count_mode, uint32_t flags,
                              const gk_tiling_t *tiling, uint8_t *accept_out,
                              uint16_t *edits_out, uint32_t *err_count,
                              void *stream);

/*
 * Streamed host pipeline.  The paper's host program sends reads and
 * candidates to the device in batches and reads the results back, with one
 * synchronisation point per batch (Sec. 3.3, Sec. 3.5).  A pipe keeps
 * n_slots batches in flight on three streams of its own, so the host-to-
 * device copy of batch i+1 and the device-to-host copy of batch i-1 overlap
 * the encoding and filtering of batch i:
 *   copy in   ASCII reads and pairs (waits until the slot's previous batch
 *             has been filtered)
 *   run       gk_encode on the device, then the filter at every threshold
 *             (waits for its copy-in and for the slot's previous copy-out):
 *             one gk_filter_sweep per run of consecutive thresholds (e,
 *             e+1, ...) whose shift counts it covers (edge OR on), else
 *             gk_filter per threshold; with GK_PIPE_SLICED, gk_slice once
 *             and gk_filter_sliced_sweep per run when the sliced filter
 *             covers the pipe (edge OR on, read_len <= GK_SLICED_MAX_LEN,
 *             every min(e, read_len-1) <= GK_SLICED_MAX_SHIFT)
 *   copy out  accept and edit counts of every threshold
 * Batches hold fixed-length reads (the read length of the pipe).  The pipe
 * owns its device buffers (n_slots * about max_reads * (ascii_stride +
 * 8 * ceil(read_len/32) + 1) + max_pairs * (8 + 3 * n_thresholds) bytes,
 * plus gk_sliced_bytes(max_pairs, read_len) per slot when it slices),
 * streams and events, all on the device current at creation; every call
 * makes that device current and restores the caller's.  One pipe must not
 * be used from two threads at once.
 */
typedef struct gk_pipe_s *gk_pipe_t;

#define GK_PIPE_SLICED 4u /* pipe flag: run the sliced filter (gk_slice +
                             gk_filter_sliced_sweep) where it covers the pipe */
#define GK_PIPE_READ_STARTS 8u /* pipe flag: gk_pipe_submit's pair_read holds
                                  one start per read (CSR), not a read id per
                                  pair */

typedef struct {
  uint64_t max_reads;          /* reads per batch, at most (>= 1) */
  uint64_t ascii_stride;       /* bytes between read starts in a batch's ASCII, >= read_len */
  uint32_t read_len;           /* length of every read, 1..GK_MAX_LEN */
  uint64_t max_pairs;          /* pairs per batch, at most (1 .. 2^32 - 1) */
  uint32_t n_thresholds;       /* filter passes per batch, 1..64 */
  const uint8_t *thresholds;   /* host, n_thresholds values of e (copied at creation) */
  int count_mode;              /* GK_COUNT_RUNS4 or GK_COUNT_POPCOUNT */
  uint32_t flags;              /* 0, GK_FLAG_NO_EDGE_FIX, GK_FLAG_RESULT_BYTE
                                  (then every threshold <= 252), GK_PIPE_SLICED,
                                  GK_PIPE_READ_STARTS */
  uint32_t n_slots;            /* batches in flight, 2..4 */
} gk_pipe_desc_t;

/* Create a pipe against a loaded reference (which must outlive it).
 * Errors: GK_EINVAL (null pointer, a field out of range), GK_ENOMEM,
 * GK_ECUDA. */
int gk_pipe_create(gk_ref_t ref, const gk_pipe_desc_t *desc, gk_pipe_t *out);

/*
 * Enqueue one batch and return at once.
 *   ascii       host, n_reads * ascii_stride bytes (read i at i*ascii_stride)
 *   pair_read   host, n_pairs uint32 read ids (within this batch); with
 *               GK_PIPE_READ_STARTS instead n_reads uint32 starts: read i's
 *               candidates are pairs pair_read[i] .. pair_read[i+1]-1 (the
 *               last read's through n_pairs-1), a quarter of the bytes at 4
 *               candidates per read (pairs before the first read's start are
 *               invalid; with decreasing starts a pair claimed by two reads
 *               gets one of them)
 *   pair_off    host, n_pairs uint32 reference offsets
 *   accept_out  host, n_thresholds * n_pairs uint8, threshold-major (the
 *               result bytes with GK_FLAG_RESULT_BYTE)
 *   edits_out   host, n_thresholds * n_pairs uint16, threshold-major; unused
 *               (may be NULL) with GK_FLAG_RESULT_BYTE
 *   ticket      receives the batch's number (0, 1, 2, ... per pipe)
 * Results are in accept_out / edits_out once gk_pipe_wait(ticket) returns;
 * all five host buffers must stay valid and unchanged until then.  Copies
 * overlap other work only from page-locked host memory (cudaHostAlloc or
 * cudaHostRegister).  Errors: GK_EINVAL / GK_ERANGE (sizes above the pipe's
 * maxima) before anything is enqueued; GK_ECUDA, after which the pipe only
 * reports the error.
 */
int gk_pipe_submit(gk_pipe_t pipe, const uint8_t *ascii, uint64_t n_reads,
                   const uint32_t *pair_read, const uint32_t *pair_off,
                   uint64_t n_pairs, uint8_t *accept_out, uint16_t *edits_out,
                   uint64_t *ticket);

/* Block until batch `ticket` (and every earlier one) has its results in the
 * host buffers.  Errors: GK_EINVAL (a ticket not yet submitted), GK_ECUDA. */
int gk_pipe_wait(gk_pipe_t pipe, uint64_t ticket);

/* Wait for every submitted batch, then release the pipe (NULL is ignored). */
void gk_pipe_destroy(gk_pipe_t pipe);

#ifdef __cplusplus
}
#endif

#endif /* GK_H */
