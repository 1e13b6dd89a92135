/*
 * oracle.c -- plain, slow CPU restatement of the GateKeeper-GPU filter decision.
 *
 * TEST INFRASTRUCTURE ONLY.  The product library never links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * path.
 *
 * Every sequence is handled one base per byte (ASCII), one step at a time, in
 * the order the paper describes the method (arxiv 2103.14978):
 *
 *   1. a pair whose read or reference segment holds a base other than
 *      A/C/G/T is passed with no filtration ("undefined")        Sec. 3.3
 *   2. bases are coded on 2 bits, A=00 C=01 G=10 T=11              Sec. 2.1
 *   3. the Hamming mask (shift 0) and the 2e masks of the read
 *      shifted by 1..e bases in both directions; each base's
 *      2-bit XOR is OR-folded to one bit (1 = differ); bases
 *      shifted in from outside the read are zero codes            Sec. 2.1, 3.4
 *   4. every mask is amended: a streak of one or two 0s with a 1
 *      on both sides becomes 1s                                    Sec. 2.1
 *   5. after amendment, the positions a shift left vacant are set
 *      to 1 (the leading/trailing improvement)                     Sec. 3.4
 *   6. the 2e+1 masks are ANDed                                    Sec. 2.1
 *   7. errors in the final vector are counted with a 4-base
 *      window table; the pair is accepted iff count <= e          Sec. 2.1
 *
 * Readings taken where the text is silent or garbled (the paper's worked
 * figures are not available):
 *   - the window table counts the maximal runs of 1s inside each 4-base
 *     window, windows starting at base 0, the last one padded with 0s
 *     (mode GKO_RUNS4, the default); a plain popcount (GKO_POPCOUNT) and a
 *     whole-vector run count (GKO_RUNS) are kept for comparison;
 *   - a 0-streak touching either end of the mask is not amended;
 *   - vacated positions hold the comparison against code 00 ('A') while
 *     amending and are forced to 1 only afterwards;
 *   - the shift-0 mask is amended like the others;
 *   - lower-case bases are folded to upper case, every other byte is
 *     treated like 'N';
 *   - an undefined pair reports accept=1, edits=0xFFFF; a pair whose
 *     read id or reference window is out of range reports accept=0,
 *     edits=0xFFFE;
 *   - the count is reported in full, never clamped at e.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GKO_RUNS4 0
#define GKO_POPCOUNT 1
#define GKO_RUNS 2

#define GKO_FLAG_NO_EDGE_FIX 1 /* original GateKeeper: skip step 5 */

#define GKO_UNDEFINED 0xFFFFu
#define GKO_INVALID 0xFFFEu

/* Step 2: the 2-bit code of a base, or -1 for anything that is not A/C/G/T
 * in either case (Sec. 2.1, Sec. 3.3). */
int gko_code(unsigned char c) {
  switch (c) {
  case 'A': case 'a': return 0;
  case 'C': case 'c': return 1;
  case 'G': case 'g': return 2;
  case 'T': case 't': return 3;
  default: return -1;
  }
}

/* Step 1: 1 if the sequence holds a byte that is not A/C/G/T (Sec. 3.3). */
int gko_has_undefined(const char *S, int m) {
  for (int i = 0; i < m; i++)
    if (gko_code((unsigned char)S[i]) < 0) return 1;
  return 0;
}

/* Step 3: the mask for shift s (Sec. 2.1, Sec. 3.4).
 * M[i] = 1 iff the code of the shifted read at position i differs from the
 * code of the reference segment at i.  The shifted read at i is R[i - s]
 * when that index lies inside the read; otherwise the position was vacated
 * by the shift and holds the zero code (the code of 'A').  Folding the two
 * XOR bits with OR is the same as asking whether the codes differ. */
void gko_shifted_mask(const char *R, const char *G, int m, int s,
                      unsigned char *M) {
  for (int i = 0; i < m; i++) {
    int j = i - s;
    int read_code = (j >= 0 && j < m) ? gko_code((unsigned char)R[j]) : 0;
    int ref_code = gko_code((unsigned char)G[i]);
    int x = read_code ^ ref_code;
    int hi = (x >> 1) & 1, lo = x & 1;
    M[i] = (unsigned char)(hi | lo);
  }
}

/* Step 4: amendment (Sec. 2.1).  Each maximal run of 0s of length 1 or 2
 * that has a 1 immediately before and immediately after it, both inside the
 * mask, becomes 1s.  Flipping such a run never changes the 1s that bound
 * another run, so scanning left to right equals applying the rule to all
 * runs at once. */
void gko_amend(unsigned char *M, int m) {
  int i = 0;
  while (i < m) {
    if (M[i] != 0) { i++; continue; }
    int j = i;
    while (j < m && M[j] == 0) j++;         /* run is [i, j) */
    int len = j - i;
    int bounded_left = (i - 1 >= 0) && M[i - 1] == 1;
    int bounded_right = (j < m) && M[j] == 1;
    if (len <= 2 && bounded_left && bounded_right)
      for (int k = i; k < j; k++) M[k] = 1;
    i = j;
  }
}

/* Step 5: the leading/trailing improvement (Sec. 3.4).  After amendment the
 * positions that the shift left vacant are set to 1: the first s positions
 * when the read moved to higher indices (s > 0), the last |s| positions when
 * it moved to lower indices (s < 0). */
void gko_edge_fix(unsigned char *M, int m, int s) {
  if (s > 0) {
    for (int i = 0; i < s && i < m; i++) M[i] = 1;
  } else if (s < 0) {
    for (int i = m + s; i < m; i++)
      if (i >= 0) M[i] = 1;
  }
}

/* Step 7: the error count of the final vector (Sec. 2.1). */
int gko_count(const unsigned char *F, int m, int mode) {
  int count = 0;
  if (mode == GKO_POPCOUNT) {
    for (int i = 0; i < m; i++) count += F[i];
  } else if (mode == GKO_RUNS) {
    for (int i = 0; i < m; i++)
      if (F[i] && (i == 0 || !F[i - 1])) count++;
  } else { /* GKO_RUNS4: runs of 1s inside each 4-base window */
    for (int w = 0; w < m; w += 4) {
      int prev = 0;
      for (int i = w; i < w + 4; i++) {
        int bit = (i < m) ? F[i] : 0;
        if (bit && !prev) count++;
        prev = bit;
      }
    }
  }
  return count;
}

/* Steps 3-6 for one pair.  F receives the final vector.  Returns 1 (and
 * leaves F untouched) when the pair is undefined, else 0. */
int gko_final_vector(const char *R, const char *G, int m, int e, int flags,
                     unsigned char *F) {
  if (gko_has_undefined(R, m) || gko_has_undefined(G, m)) return 1;
  unsigned char *M = (unsigned char *)malloc(m > 0 ? (size_t)m : 1);
  for (int i = 0; i < m; i++) F[i] = 1;
  for (int s = -e; s <= e; s++) {
    gko_shifted_mask(R, G, m, s, M);
    gko_amend(M, m);
    if (!(flags & GKO_FLAG_NO_EDGE_FIX)) gko_edge_fix(M, m, s);
    for (int i = 0; i < m; i++) F[i] = (unsigned char)(F[i] & M[i]);
  }
  free(M);
  return 0;
}

/* The whole filter decision for one pair (Sec. 2.1, Sec. 3.3, Sec. 3.4). */
void gko_filter_pair(const char *R, const char *G, int m, int e, int mode,
                     int flags, unsigned char *accept, unsigned short *edits) {
  unsigned char *F = (unsigned char *)malloc(m > 0 ? (size_t)m : 1);
  if (gko_final_vector(R, G, m, e, flags, F)) {
    *accept = 1;
    *edits = (unsigned short)GKO_UNDEFINED;
  } else {
    int c = gko_count(F, m, mode);
    *edits = (unsigned short)c;
    *accept = (unsigned char)(c <= e);
  }
  free(F);
}

/* ---- batch driver: the same per-pair function over many pairs ---------- */

typedef struct {
  const char *reads;
  const uint64_t *read_start;
  const uint16_t *read_len;
  uint64_t n_reads;
  const char *ref;
  uint64_t ref_len;
  const uint32_t *pair_read;
  const uint32_t *pair_off;
  const uint8_t *pair_e; /* NULL: fixed_e for every pair */
  int fixed_e;
  int mode, flags;
  uint8_t *accept;
  uint16_t *edits;
  uint64_t lo, hi;
} gko_job;

static void *gko_run_job(void *arg) {
  gko_job *J = (gko_job *)arg;
  for (uint64_t p = J->lo; p < J->hi; p++) {
    uint32_t r = J->pair_read[p];
    if ((uint64_t)r >= J->n_reads) {
      J->accept[p] = 0;
      J->edits[p] = (uint16_t)GKO_INVALID;
      continue;
    }
    int m = J->read_len[r];
    uint64_t off = J->pair_off[p];
    if (off + (uint64_t)m > J->ref_len) {
      J->accept[p] = 0;
      J->edits[p] = (uint16_t)GKO_INVALID;
      continue;
    }
    int e = J->pair_e ? J->pair_e[p] : J->fixed_e;
    unsigned char a;
    unsigned short ed;
    gko_filter_pair(J->reads + J->read_start[r], J->ref + off, m, e, J->mode,
                    J->flags, &a, &ed);
    J->accept[p] = a;
    J->edits[p] = ed;
  }
  return NULL;
}

/* Filters n_pairs pairs (read id, reference offset, e) with n_threads POSIX
 * threads, each taking a contiguous slice of the pairs.  Read r is the
 * read_len[r] bytes at reads + read_start[r].  Returns the thread count used. */
int gko_filter_batch(const char *reads, const uint64_t *read_start,
                     const uint16_t *read_len, uint64_t n_reads,
                     const char *ref, uint64_t ref_len,
                     const uint32_t *pair_read, const uint32_t *pair_off,
                     const uint8_t *pair_e, int fixed_e, uint64_t n_pairs,
                     int mode, int flags, uint8_t *accept, uint16_t *edits,
                     int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n_pairs) n_threads = n_pairs > 0 ? (int)n_pairs : 1;
  gko_job *jobs = (gko_job *)calloc((size_t)n_threads, sizeof(gko_job));
  pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  uint64_t chunk = (n_pairs + (uint64_t)n_threads - 1) / (uint64_t)n_threads;
  for (int t = 0; t < n_threads; t++) {
    gko_job *J = &jobs[t];
    J->reads = reads; J->read_start = read_start; J->read_len = read_len;
    J->n_reads = n_reads; J->ref = ref; J->ref_len = ref_len;
    J->pair_read = pair_read; J->pair_off = pair_off; J->pair_e = pair_e;
    J->fixed_e = fixed_e; J->mode = mode; J->flags = flags;
    J->accept = accept; J->edits = edits;
    J->lo = chunk * (uint64_t)t;
    if (J->lo > n_pairs) J->lo = n_pairs;
    J->hi = J->lo + chunk < n_pairs ? J->lo + chunk : n_pairs;
  }
  for (int t = 1; t < n_threads; t++)
    pthread_create(&tid[t], NULL, gko_run_job, &jobs[t]);
  gko_run_job(&jobs[0]);
  for (int t = 1; t < n_threads; t++) pthread_join(tid[t], NULL);
  free(jobs);
  free(tid);
  return n_threads;
}

/* ---- ground truth: Levenshtein distance (Sec. 4.4 uses a global edit
 * distance as the truth) -- the textbook dynamic programme, unit costs. ---- */
int gko_levenshtein(const char *a, int n, const char *b, int k) {
  int *prev = (int *)malloc(sizeof(int) * (size_t)(k + 1));
  int *cur = (int *)malloc(sizeof(int) * (size_t)(k + 1));
  for (int j = 0; j <= k; j++) prev[j] = j;
  for (int i = 1; i <= n; i++) {
    cur[0] = i;
    for (int j = 1; j <= k; j++) {
      int sub = prev[j - 1] + (a[i - 1] != b[j - 1]);
      int del = prev[j] + 1;
      int ins = cur[j - 1] + 1;
      int best = sub < del ? sub : del;
      cur[j] = best < ins ? best : ins;
    }
    int *t = prev; prev = cur; cur = t;
  }
  int d = prev[k];
  free(prev);
  free(cur);
  return d;
}

typedef struct {
  const char *reads; const uint64_t *read_start; const uint16_t *read_len;
  const char *ref; const uint32_t *pair_read; const uint32_t *pair_off;
  int32_t *dist; uint64_t lo, hi;
} gko_lev_job;

static void *gko_run_lev(void *arg) {
  gko_lev_job *J = (gko_lev_job *)arg;
  for (uint64_t p = J->lo; p < J->hi; p++) {
    uint32_t r = J->pair_read[p];
    int m = J->read_len[r];
    J->dist[p] = gko_levenshtein(J->reads + J->read_start[r], m,
                                 J->ref + J->pair_off[p], m);
  }
  return NULL;
}

/* Edit distance between each read and its m-base reference window, over
 * n_threads threads.  The caller guarantees every pair is in range. */
int gko_levenshtein_batch(const char *reads, const uint64_t *read_start,
                          const uint16_t *read_len, const char *ref,
                          const uint32_t *pair_read, const uint32_t *pair_off,
                          uint64_t n_pairs, int32_t *dist, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n_pairs) n_threads = n_pairs > 0 ? (int)n_pairs : 1;
  gko_lev_job *jobs = (gko_lev_job *)calloc((size_t)n_threads, sizeof(gko_lev_job));
  pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  uint64_t chunk = (n_pairs + (uint64_t)n_threads - 1) / (uint64_t)n_threads;
  for (int t = 0; t < n_threads; t++) {
    gko_lev_job *J = &jobs[t];
    J->reads = reads; J->read_start = read_start; J->read_len = read_len;
    J->ref = ref; J->pair_read = pair_read; J->pair_off = pair_off; J->dist = dist;
    J->lo = chunk * (uint64_t)t;
    if (J->lo > n_pairs) J->lo = n_pairs;
    J->hi = J->lo + chunk < n_pairs ? J->lo + chunk : n_pairs;
  }
  for (int t = 1; t < n_threads; t++)
    pthread_create(&tid[t], NULL, gko_run_lev, &jobs[t]);
  gko_run_lev(&jobs[0]);
  for (int t = 1; t < n_threads; t++) pthread_join(tid[t], NULL);
  free(jobs);
  free(tid);
  return n_threads;
}
