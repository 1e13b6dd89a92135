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
#define GK_PROBE_IMAD 3  /* integer multiply-add (runtime multiplier) */
#define GK_PROBE_LOP3_IMAD 4 /* logic ops and multiply-adds, one to one */
#define GK_PROBE_IADD 5  /* integer adds */
#define GK_PROBE_LOP3_IADD 6 /* logic ops and adds, one to one */
#define GK_PROBE_SHF_IMAD 7  /* funnel shifts and multiply-adds, one to one */
#define GK_PROBE_ADDC 8      /* 4-word add-with-carry chains (x + x: shift by 1) */
#define GK_PROBE_LOP3_ADDC 9 /* logic ops and add-with-carry, one to one */
#define GK_PROBE_WIDE 10     /* 32x32->64 multiply-adds */
#define GK_PROBE_LOP3_WIDE 11 /* logic ops and wide multiply-adds, one to one */
#define GK_PROBE_LOP3_WIDE_2 12 /* logic ops and wide multiply-adds, two to one */
#define GK_PROBE_MULHI 13    /* high half of 32x32 products */
#define GK_PROBE_FUNNEL_FMA 14 /* funnel shift as mad.hi + mad.lo, mixed 1:1 with logic ops */

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
