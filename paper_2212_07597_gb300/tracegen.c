/*
 * tracegen.c -- seeded synthetic allocation / free / memcpy event traces.
 *
 * These traces stand in for the allocator activity of the profiled Python
 * programs of the paper's evaluation (Section 6, the pyperformance suite),
 * whose allocation traces are not available.  The generator knows nothing
 * about sampling, footprints or leak scores: it only draws events.  Both the
 * CPU oracle (through the tests) and the CUDA library consume its output, and
 * neither links against the other.
 *
 * Layout produced (structure of arrays, one entry per event i):
 *   delta[i]  int64   signed byte count: > 0 malloc, < 0 free of exactly the
 *                     size that was allocated at that address
 *   addr[i]   uint64  address of the block (bump allocated, 16-byte aligned)
 *   line[i]   uint32  source line id in [0, n_lines), Zipf distributed
 *   py[i]     uint8   1 = allocation made by Python, 0 = native
 * and, for the memcpy stream, size[j] uint64 / line[j] / py[j].
 *
 * Randomness: one splitmix64 stream per trace (seed mixed with the trace id).
 * Floating-point draws use only +, *, and hand-written exp/log series below,
 * compiled with -ffp-contract=off, so the same seed gives the same trace on
 * x86_64 and aarch64 hosts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- random numbers ---------------- */

static inline uint64_t sm64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline double u01(uint64_t *s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) by the high half of a 64x64 product */
static inline uint64_t below(uint64_t *s, uint64_t n) {
    return (uint64_t)(((unsigned __int128)sm64(s) * n) >> 64);
}

static uint64_t mix_seed(uint64_t seed, uint64_t trace) {
    uint64_t s = seed ^ (0xD1B54A32D192ED03ull * (trace + 1));
    (void)sm64(&s);
    return s;
}

/* ---------------- deterministic exp / log (host only) ---------------- */

#define LN2 0.69314718055994530942

/* e^y: y = k*ln2 + r with |r| <= ln2/2, Taylor series of e^r to degree 22 */
static double det_exp(double y) {
    double kf = y / LN2;
    long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
    double r = y - (double)k * LN2;
    double term = 1.0, sum = 1.0;
    for (int n = 1; n <= 22; ++n) { term = term * r / (double)n; sum = sum + term; }
    while (k > 0) { sum = sum * 2.0; --k; }
    while (k < 0) { sum = sum * 0.5; ++k; }
    return sum;
}

/* ln x for x > 0: x = m * 2^e with m in [1/sqrt2, sqrt2), ln m = 2 atanh((m-1)/(m+1)) */
static double det_log(double x) {
    int e = 0;
    while (x >= 1.4142135623730951) { x = x * 0.5; ++e; }
    while (x < 0.7071067811865476) { x = x * 2.0; --e; }
    double t = (x - 1.0) / (x + 1.0), t2 = t * t, pw = t, sum = 0.0;
    for (int n = 1; n <= 61; n += 2) { sum = sum + pw / (double)n; pw = pw * t2; }
    return 2.0 * sum + (double)e * LN2;
}

/* floor(lo * (hi/lo)^u) for u uniform in [0,1): log-uniform on [lo, hi);
 * lnr = ln(hi/lo), computed once by the caller */
static uint64_t log_uniform(uint64_t *s, uint64_t lo, uint64_t hi, double lnr) {
    double u = u01(s);
    double v = (double)lo * det_exp(u * lnr);
    uint64_t x = (uint64_t)v;
    if (x < lo) x = lo;
    if (x >= hi) x = hi - 1;
    return x;
}

/* ---------------- Zipf line ids ---------------- */

typedef struct { uint32_t n; double *cdf; } zipf_t;

static int zipf_init(zipf_t *z, uint32_t n, double s) {
    z->n = n;
    z->cdf = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!z->cdf) return -1;
    double acc = 0.0;
    for (uint32_t i = 0; i < n; ++i) { acc = acc + det_exp(-s * det_log((double)(i + 1))); z->cdf[i] = acc; }
    for (uint32_t i = 0; i < n; ++i) z->cdf[i] = z->cdf[i] / acc;
    return 0;
}

static uint32_t zipf_draw(const zipf_t *z, uint64_t *s) {
    double u = u01(s);
    uint32_t lo = 0, hi = z->n - 1;
    while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (z->cdf[mid] > u) hi = mid; else lo = mid + 1; }
    return lo;
}

/* ---------------- event traces ---------------- */

typedef struct {
    uint64_t n;              /* events to produce */
    uint32_t n_lines;        /* line ids in [0, n_lines) */
    uint32_t addr_reuse;     /* 1: a malloc reuses the most recently freed address (LIFO) */
    double p_malloc;         /* probability an event is a malloc (forced when nothing is live) */
    double p_python;         /* probability the event is attributed to Python */
    double zipf_s;           /* Zipf exponent of line ids */
    uint64_t size_lo, size_hi;          /* log-uniform malloc sizes [lo, hi) */
    uint32_t n_leak_lines;              /* designated leaking lines (<= 16) */
    uint32_t leak_lines[16];
    double p_leak_unfreed;              /* a malloc on a leaking line is never freed with this probability */
    uint64_t leak_lo, leak_hi;          /* its size distribution */
    uint64_t ramp_count, ramp_size;     /* that many never-freed mallocs of ramp_size, evenly spaced */
    uint32_t ramp_line;
    uint64_t big_count, big_size;       /* that many mallocs of big_size (freeable), evenly spaced */
} tg_params;

typedef struct { uint64_t addr; int64_t size; } live_t;

/* returns 0, or -1 on allocation failure / bad parameters */
int tg_events(const tg_params *p, uint64_t seed, uint64_t trace,
              int64_t *delta, uint64_t *addr, uint32_t *line, uint8_t *py) {
    if (!p || p->n_lines == 0 || p->size_lo == 0 || p->size_hi <= p->size_lo) return -1;
    uint64_t s = mix_seed(seed, trace);
    zipf_t z;
    if (zipf_init(&z, p->n_lines, p->zipf_s)) return -1;
    uint64_t cap = 1024;
    live_t *live = (live_t *)malloc(sizeof(live_t) * cap);
    uint64_t nlive = 0;
    uint64_t *freed = NULL, nfreed = 0, capf = 0;
    if (p->addr_reuse) { capf = 1024; freed = (uint64_t *)malloc(sizeof(uint64_t) * capf); }
    uint8_t leakmask_small[4096];
    memset(leakmask_small, 0, sizeof leakmask_small);
    uint8_t *leakmask = p->n_lines <= 4096 ? leakmask_small : (uint8_t *)calloc(p->n_lines, 1);
    for (uint32_t k = 0; k < p->n_leak_lines && k < 16; ++k)
        if (p->leak_lines[k] < p->n_lines) leakmask[p->leak_lines[k]] = 1;
    uint64_t bump = 0x100000;
    const double ln_size = det_log((double)p->size_hi / (double)p->size_lo);
    const double ln_leak = p->leak_hi > p->leak_lo ? det_log((double)p->leak_hi / (double)p->leak_lo) : 0.0;
    uint64_t next_ramp = p->ramp_count ? (p->n / p->ramp_count) / 2 : UINT64_MAX, ramp_i = 0;
    uint64_t next_big = p->big_count ? (p->n / p->big_count) / 2 : UINT64_MAX, big_i = 0;
    int rc = 0;
    if (!live || (p->addr_reuse && !freed) || !leakmask) { rc = -1; goto out; }

    for (uint64_t i = 0; i < p->n; ++i) {
        uint32_t ln = zipf_draw(&z, &s);
        uint8_t isp = u01(&s) < p->p_python;
        double ukind = u01(&s);
        int forced = 0;
        int64_t sz = 0;
        int keep_live = 1;
        if (i == next_ramp) {
            forced = 1; sz = (int64_t)p->ramp_size; keep_live = 0; ln = p->ramp_line % p->n_lines;
            ++ramp_i; next_ramp = ramp_i < p->ramp_count ? (p->n / p->ramp_count) * ramp_i + (p->n / p->ramp_count) / 2 : UINT64_MAX;
        } else if (i == next_big) {
            forced = 1; sz = (int64_t)p->big_size;
            ++big_i; next_big = big_i < p->big_count ? (p->n / p->big_count) * big_i + (p->n / p->big_count) / 2 : UINT64_MAX;
        }
        if (forced || nlive == 0 || ukind < p->p_malloc) {
            if (!forced) {
                if (leakmask[ln] && p->leak_hi > p->leak_lo) {
                    sz = (int64_t)log_uniform(&s, p->leak_lo, p->leak_hi, ln_leak);
                    if (u01(&s) < p->p_leak_unfreed) keep_live = 0;
                } else {
                    sz = (int64_t)log_uniform(&s, p->size_lo, p->size_hi, ln_size);
                }
            }
            uint64_t a;
            if (p->addr_reuse && nfreed) a = freed[--nfreed];
            else { a = bump; bump += ((uint64_t)sz + 15u) & ~(uint64_t)15u; }
            if (keep_live) {
                if (nlive == cap) {
                    cap *= 2;
                    live_t *nl = (live_t *)realloc(live, sizeof(live_t) * cap);
                    if (!nl) { rc = -1; goto out; }
                    live = nl;
                }
                live[nlive].addr = a; live[nlive].size = sz; ++nlive;
            }
            delta[i] = sz; addr[i] = a;
        } else {
            uint64_t k = below(&s, nlive);
            live_t v = live[k];
            live[k] = live[--nlive];
            delta[i] = -v.size; addr[i] = v.addr;
            if (p->addr_reuse) {
                if (nfreed == capf) {
                    capf *= 2;
                    uint64_t *nf = (uint64_t *)realloc(freed, sizeof(uint64_t) * capf);
                    if (!nf) { rc = -1; goto out; }
                    freed = nf;
                }
                freed[nfreed++] = v.addr;
            }
        }
        line[i] = ln; py[i] = isp;
    }
out:
    free(live); free(freed); free(z.cdf);
    if (leakmask != leakmask_small) free(leakmask);
    return rc;
}

/* memcpy stream: sizes log-uniform [lo, hi), Zipf lines, Bernoulli python flag */
int tg_copies(uint64_t m, uint32_t n_lines, double zipf_s, double p_python, uint64_t lo, uint64_t hi,
              uint64_t seed, uint64_t trace, uint64_t *size, uint32_t *line, uint8_t *py) {
    if (n_lines == 0 || lo == 0 || hi <= lo) return -1;
    uint64_t s = mix_seed(seed ^ 0x5bd1e9955bd1e995ull, trace);
    zipf_t z;
    if (zipf_init(&z, n_lines, zipf_s)) return -1;
    const double lnr = det_log((double)hi / (double)lo);
    for (uint64_t j = 0; j < m; ++j) {
        line[j] = zipf_draw(&z, &s);
        py[j] = u01(&s) < p_python;
        size[j] = log_uniform(&s, lo, hi, lnr);
    }
    free(z.cdf);
    return 0;
}

/* alternating +(T-1) / -(T-1) deltas with a +1 event every `period` events (0: never) */
int tg_adversarial(uint64_t n, int64_t T, uint64_t period, uint32_t n_lines, uint64_t seed, uint64_t trace,
                   int64_t *delta, uint64_t *addr, uint32_t *line, uint8_t *py) {
    if (T < 2 || n_lines == 0) return -1;
    uint64_t s = mix_seed(seed ^ 0xA5A5A5A5ull, trace);
    uint64_t bump = 0x100000, last = 0;
    int up = 1;
    for (uint64_t i = 0; i < n; ++i) {
        line[i] = (uint32_t)below(&s, n_lines);
        py[i] = (uint8_t)(sm64(&s) & 1);
        if (period && i % period == period - 1) { delta[i] = 1; addr[i] = bump; bump += 16; continue; }
        if (up) { delta[i] = T - 1; addr[i] = last = bump; bump += ((uint64_t)(T - 1) + 15u) & ~(uint64_t)15u; }
        else { delta[i] = -(T - 1); addr[i] = last; }
        up = !up;
    }
    return 0;
}

/* malloc-only trace of constant size */
int tg_constant(uint64_t n, int64_t size, uint32_t n_lines, uint64_t seed, uint64_t trace,
                int64_t *delta, uint64_t *addr, uint32_t *line, uint8_t *py) {
    if (size <= 0 || n_lines == 0) return -1;
    uint64_t s = mix_seed(seed ^ 0x3C3C3C3Cull, trace);
    uint64_t bump = 0x100000;
    for (uint64_t i = 0; i < n; ++i) {
        delta[i] = size; addr[i] = bump; bump += ((uint64_t)size + 15u) & ~(uint64_t)15u;
        line[i] = (uint32_t)below(&s, n_lines);
        py[i] = (uint8_t)(sm64(&s) & 1);
    }
    return 0;
}

/* log-uniform integer lengths (e.g. trace lengths of a batch) */
int tg_lengths(uint64_t count, uint64_t lo, uint64_t hi, uint64_t seed, uint64_t *out) {
    if (lo == 0 || hi <= lo) return -1;
    uint64_t s = mix_seed(seed ^ 0x7777ull, 0);
    const double lnr = det_log((double)hi / (double)lo);
    for (uint64_t i = 0; i < count; ++i) out[i] = log_uniform(&s, lo, hi, lnr);
    return 0;
}

/* Poisson arrival times: exponential gaps with the given mean, in integer nanoseconds */
int tg_arrivals(uint64_t count, double mean_gap_ns, uint64_t seed, uint64_t *out_ns) {
    uint64_t s = mix_seed(seed ^ 0x9999ull, 0);
    double t = 0.0;
    for (uint64_t i = 0; i < count; ++i) {
        double u = u01(&s);
        t = t - mean_gap_ns * det_log(1.0 - u);
        out_ns[i] = (uint64_t)t;
    }
    return 0;
}

/* Gaps between sampled bytes of a rate-based sampler with one sample per `mean` bytes on
 * average: each byte is a Bernoulli trial with p = 1/mean, so the gap (bytes from one
 * sampled byte to the next, >= 1) is geometric: 1 + floor(ln(U) / ln(1 - p)) for U in (0, 1]. */
int tg_gaps(uint64_t count, double mean, uint64_t seed, uint64_t *out) {
    if (!(mean >= 1.0)) return -1;
    uint64_t s = mix_seed(seed ^ 0x6A09E667F3BCC909ull, 0);
    const double l1p = mean > 1.0 ? det_log(1.0 - 1.0 / mean) : -1.0;
    for (uint64_t i = 0; i < count; ++i) {
        const double u = 1.0 - u01(&s);   /* (0, 1] */
        double g = mean > 1.0 ? det_log(u) / l1p : 0.0;
        if (g > 9.0e18) g = 9.0e18;
        out[i] = 1u + (uint64_t)g;
    }
    return 0;
}

/* test hooks for the deterministic helpers */
double tg_det_exp(double y) { return det_exp(y); }
double tg_det_log(double x) { return det_log(x); }
