/*
 * scl_oracle.c -- plain sequential CPU replay of Scalene's memory sampler.
 *
 * TEST INFRASTRUCTURE ONLY (see scl_oracle.h).  One event at a time, in trace
 * order, exactly the steps of Sections 3.2-3.5 of arXiv 2212.07597.  Readings
 * of points the paper leaves open are marked "reading:" inline.
 */
#include "scl_oracle.h"
#include <stdlib.h>
#include <string.h>

int orc_init(orc_state *st, const orc_config *cfg) {
    memset(st, 0, sizeof *st);
    if (!cfg || cfg->threshold < 1 || cfg->copy_threshold < 1 || cfg->n_lines == 0 ||
        cfg->copy_phase >= cfg->copy_threshold)
        return -1;
    st->cfg = *cfg;
    st->footprint = cfg->initial_footprint;
    st->hwm = cfg->initial_footprint;          /* reading: the high-water mark starts at F0 */
    st->copy_counter = cfg->copy_phase;
    st->lines = (orc_line *)calloc(cfg->n_lines, sizeof(orc_line));
    return st->lines ? 0 : -2;
}

void orc_free(orc_state *st) {
    free(st->lines);
    free(st->samples);
    memset(st, 0, sizeof *st);
}

static int add_ovf(int64_t a, int64_t b, int64_t *out) { return __builtin_add_overflow(a, b, out); }

static int push_sample(orc_state *st, const orc_sample *s) {
    if (st->n_samples == st->cap_samples) {
        uint64_t nc = st->cap_samples ? st->cap_samples * 2 : 1024;
        orc_sample *ns = (orc_sample *)realloc(st->samples, nc * sizeof(orc_sample));
        if (!ns) return -2;
        st->samples = ns;
        st->cap_samples = nc;
    }
    st->samples[st->n_samples++] = *s;
    return 0;
}

int orc_replay_events(orc_state *st, const int64_t *delta, const uint64_t *addr,
                      const uint32_t *line, const uint8_t *is_python, uint64_t n) {
    const int64_t T = st->cfg.threshold;
    for (uint64_t i = 0; i < n; ++i) {
        const int64_t d = delta[i];
        const uint64_t g = st->n_events + i;        /* index within the whole trace */
        if (line[i] >= st->cfg.n_lines) return -1;
        if (d == INT64_MIN) return -3;

        /* the footprint follows every allocation and free (Section 3.3) */
        if (add_ovf(st->footprint, d, &st->footprint)) return -3;

        /* Section 3.2: A counts bytes allocated, F bytes freed; Section 3.3:
         * the Python share of each is kept alongside. */
        if (d > 0) {
            if (add_ovf(st->A, d, &st->A)) return -3;
            if (is_python[i] && add_ovf(st->A_py, d, &st->A_py)) return -3;
        } else if (d < 0) {
            if (add_ovf(st->F, -d, &st->F)) return -3;
            if (is_python[i] && add_ovf(st->F_py, -d, &st->F_py)) return -3;
        }

        /* Section 3.4: every free compares its pointer with the tracked object */
        if (d < 0 && st->tracked_valid && addr[i] == st->tracked_addr) st->tracked_reclaimed = 1;

        /* Section 3.2: sample once |A - F| >= T (A - F kept as one counter c) */
        if (add_ovf(st->c, d, &st->c)) return -3;
        int64_t mag = st->c < 0 ? -st->c : st->c;
        if (mag >= T) {
            orc_sample s;
            memset(&s, 0, sizeof s);
            s.idx = g;
            s.kind = st->c > 0 ? 1 : -1;
            s.A = st->A; s.F = st->F; s.A_py = st->A_py; s.F_py = st->F_py;
            s.footprint = st->footprint;                 /* Section 3.3: footprint at the crossing */
            s.line = line[i];                            /* reading: line of the triggering event */
            s.is_python = is_python[i];

            /* Section 3.3: the sample is attributed to its line */
            orc_line *L = &st->lines[line[i]];
            if (s.kind > 0) L->n_growth++; else L->n_shrink++;
            L->A += s.A; L->F += s.F; L->A_py += s.A_py; L->F_py += s.F_py; L->net += s.A - s.F;

            /* Section 3.4: a growth sample that sets a new high-water mark
             * closes the previous tracked object's trial and tracks the
             * sampled allocation instead.  reading: the mark is the largest
             * footprint seen at a growth sample, compared strictly. */
            if (s.kind > 0 && st->footprint > st->hwm) {
                if (st->tracked_valid) st->lines[st->tracked_line].frees += (uint64_t)st->tracked_reclaimed;
                st->tracked_valid = 1;
                st->tracked_addr = addr[i];
                st->tracked_line = line[i];
                st->tracked_idx = g;
                st->tracked_reclaimed = 0;
                st->lines[line[i]].mallocs++;
                st->hwm = st->footprint;
                s.is_hwm = 1;
            }
            int rc = push_sample(st, &s);
            if (rc) return rc;

            /* Section 3.2: reset the counters.  reading: the excess over T is
             * discarded, not carried. */
            st->c = 0; st->A = 0; st->F = 0; st->A_py = 0; st->F_py = 0;
        }
    }
    st->n_events += n;
    return 0;
}

int orc_replay_copies(orc_state *st, const uint64_t *size, const uint32_t *line,
                      const uint8_t *is_python, uint64_t m) {
    const uint64_t Tc = st->cfg.copy_threshold;
    for (uint64_t j = 0; j < m; ++j) {
        if (line[j] >= st->cfg.n_lines) return -1;
        /* Section 3.5: count copied bytes; one sample per T_c bytes copied.
         * reading: a deterministic countdown that keeps the remainder. */
        uint64_t total;
        if (__builtin_add_overflow(st->copy_counter, size[j], &total)) return -3;
        uint64_t q = total / Tc;
        st->copy_counter = total % Tc;
        orc_line *L = &st->lines[line[j]];
        int f = is_python[j] ? 1 : 0;
        L->copy_samples[f] += q;
        L->copy_bytes[f] += q * Tc;
    }
    st->n_copies += m;
    return 0;
}

void orc_leak_score(const orc_state *st, uint32_t line, int64_t *num, int64_t *den) {
    const orc_line *L = &st->lines[line];
    int64_t m = (int64_t)L->mallocs, f = (int64_t)L->frees;
    if (st->cfg.leak_rule == 0) {
        /* Section 3.4 as printed: 1 - (frees + 1) / (mallocs - frees + 2) */
        *den = m - f + 2;
        *num = *den - (f + 1);
    } else {
        /* Laplace's rule of succession: 1 - (frees + 1) / (mallocs + 2) */
        *den = m + 2;
        *num = *den - (f + 1);
    }
}

/* Section 3.2, rate-based sampling: a countdown of bytes to the next sampled byte,
 * decremented by each allocation and free; each time it runs out, a sample, and the
 * countdown restarts from the next gap.  Reading: every sampled byte is a sample, so an
 * event spanning several sampled bytes takes several. */
void orc_rate_samples(const int64_t *delta, const uint32_t *line, const uint8_t *is_python, uint64_t n,
                      const uint64_t *gap, uint64_t n_gaps, uint64_t consumed, uint32_t n_lines,
                      uint64_t *counts, uint64_t *state) {
    memset(counts, 0, sizeof(uint64_t) * 2 * (size_t)n_lines);
    uint64_t samples = 0, k = 0, flags = 0;
    /* left = bytes until (and including) the next sampled byte */
    uint64_t left = n_gaps ? gap[0] - consumed : 0;
    for (uint64_t i = 0; i < n; ++i) {
        const int64_t d = delta[i];
        uint64_t b = d < 0 ? (uint64_t)0 - (uint64_t)d : (uint64_t)d;
        while (b > 0) {
            if (k >= n_gaps) { flags |= 1; break; }
            if (b < left) { left -= b; b = 0; break; }
            /* the sampled byte falls in this event */
            b -= left;
            if (line[i] < n_lines) counts[2 * (size_t)line[i] + (is_python[i] ? 1 : 0)] += 1;
            else flags |= 2;
            ++samples;
            ++k;
            left = k < n_gaps ? gap[k] : 0;
        }
    }
    state[0] = samples;
    state[1] = k;
    state[2] = k < n_gaps ? gap[k] - left : 0;
    state[3] = flags;
}
