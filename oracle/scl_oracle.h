/*
 * scl_oracle.h -- plain sequential CPU replay of Scalene's memory sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference the
 * CUDA library is checked against.  It shares no code, header, table or helper
 * with the CUDA path; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it.
 *
 * Method followed (arXiv 2212.07597):
 *   Section 3.2  threshold-based sampling: counters A (bytes allocated) and F
 *                (bytes freed); when |A - F| >= T a sample is taken and the
 *                counters are reset.
 *   Section 3.3  each sample carries the allocation / free totals, the Python
 *                share of them and the source line current when it fires;
 *                the footprint is recorded at every crossing.
 *   Section 3.4  leak detection: a growth sample that reaches a new footprint
 *                high-water mark starts tracking the sampled allocation;
 *                every free compares its pointer against it; at the next
 *                high-water crossing the site's (frees, mallocs) pair is
 *                updated; leak likelihood = 1 - (frees+1)/(mallocs-frees+2).
 *   Section 3.5  copy volume: memcpy bytes are counted and a sample is written
 *                each time a threshold amount has been copied; the copy
 *                threshold is a multiple of the allocation threshold.
 */
#ifndef SCL_ORACLE_H
#define SCL_ORACLE_H
#include <stdint.h>

typedef struct {
    int64_t threshold;          /* T >= 1 */
    uint64_t copy_threshold;    /* T_c >= 1 */
    uint64_t copy_phase;        /* initial copy counter, in [0, T_c) */
    int64_t initial_footprint;  /* F0 */
    uint32_t n_lines;           /* L */
    uint32_t leak_rule;         /* 0: as printed in Section 3.4, 1: Laplace's textbook form */
} orc_config;

typedef struct {
    uint64_t idx;               /* event index within the trace */
    int64_t A, F, A_py, F_py;   /* window totals since the previous sample */
    int64_t footprint;          /* F0 + sum of all deltas up to and including idx */
    uint32_t line;              /* line of the triggering event */
    int8_t kind;                /* +1 growth, -1 shrink */
    uint8_t is_python;          /* flag of the triggering event */
    uint8_t is_hwm;             /* 1 if this sample started tracking a new object */
    uint8_t pad;
} orc_sample;

typedef struct {
    uint64_t n_growth, n_shrink;
    int64_t A, F, A_py, F_py, net;
    uint64_t mallocs, frees;
    uint64_t copy_samples[2], copy_bytes[2];  /* index: is_python */
} orc_line;

typedef struct {
    orc_config cfg;
    int64_t c, A, F, A_py, F_py;   /* sampler counter and open-window totals */
    int64_t footprint, hwm;
    int32_t tracked_valid, tracked_reclaimed;
    uint64_t tracked_addr, tracked_idx;
    uint32_t tracked_line, pad;
    uint64_t n_events, n_copies, copy_counter;
    orc_line *lines;
    orc_sample *samples;
    uint64_t n_samples, cap_samples;
} orc_state;

int orc_init(orc_state *st, const orc_config *cfg);
void orc_free(orc_state *st);
/* returns 0, -1 on a line id >= L, -2 on allocation failure, -3 on int64 overflow */
int orc_replay_events(orc_state *st, const int64_t *delta, const uint64_t *addr,
                      const uint32_t *line, const uint8_t *is_python, uint64_t n);
int orc_replay_copies(orc_state *st, const uint64_t *size, const uint32_t *line,
                      const uint8_t *is_python, uint64_t m);
/* leak likelihood of one line as an unreduced fraction num/den */
void orc_leak_score(const orc_state *st, uint32_t line, int64_t *num, int64_t *den);

/* Rate-based sampling (Section 3.2, the baseline the threshold sampler is compared with):
 * every byte allocated or freed is a Bernoulli trial; the sampled bytes sit at cumulative
 * byte positions B_k = gap[0] - consumed + gap[1] + ... + gap[k] (gaps >= 1 are given).
 * Event i, moving |delta[i]| bytes, takes one sample per B_k in its byte range, counted in
 * counts[2 * line[i] + (is_python[i] != 0)].  state[0] = samples, state[1] = gaps used up,
 * state[2] = bytes of the next gap consumed, state[3] = flags (1 gaps exhausted, 2 line id
 * >= n_lines, 4 byte count overflow).  counts[2 * n_lines] is cleared first. */
void orc_rate_samples(const int64_t *delta, const uint32_t *line, const uint8_t *is_python, uint64_t n,
                      const uint64_t *gap, uint64_t n_gaps, uint64_t consumed, uint32_t n_lines,
                      uint64_t *counts, uint64_t *state);

#endif
