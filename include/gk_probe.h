/*
 * gk_probe.h -- measurement kernels shipped with libgk.
 *
 * The filter of arxiv 2103.14978 is bitwise integer work (Sec. 2.1: shifts,
 * XOR, OR, AND and a window count), so its roofline is set by the SM's
 * integer logic and shift throughput rather than by a tensor or FP unit.
 * gk_probe_alu measures that throughput on the device at hand with
 * dependency-free, unrolled chains of the instructions the filter issues.
 */
#ifndef GK_PROBE_H
#define GK_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GK_PROBE_LOP3 0  /* 3-input logic ops */
#define GK_PROBE_SHF 1   /* funnel shifts */
#define GK_PROBE_MIX 2   /* the filter's mix: ~1 funnel shift per logic op */

/*
 * Launches `blocks` x `threads` threads, each running `iters` iterations of
 * 64 independent integer ops of the kind `kind` (so the launch issues
 * blocks*threads*iters*64 ops).  `sink` (device, >= 1 uint32) receives a
 * value derived from every result so the work cannot be elided.  Time the
 * launch with events on `stream`.  Returns GK_OK or a GK_E* code (gk.h).
 */
int gk_probe_alu(int kind, uint32_t iters, uint32_t blocks, uint32_t threads,
                 uint32_t *sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GK_PROBE_H */
