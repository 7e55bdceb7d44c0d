/*
 * scl.h -- C ABI of libscl: GB300 (sm_103a) replay of the memory-profiling
 * hot path of Scalene (Berger, Stern, Altmayer Pizzorno, arXiv 2212.07597).
 *
 * A trace is the stream of allocation, free and memcpy events one profiled
 * process would have sent through Scalene's allocator shim (Section 3.1).  The
 * library replays traces through
 *   - the threshold sampler (Section 3.2): counters A and F of bytes allocated
 *     and freed; when |A - F| >= T a sample is taken and both are reset;
 *   - sample records and per-line attribution (Section 3.3): each sample holds
 *     the window's allocation and free totals, their Python share, the
 *     footprint at the crossing and the line current when it fired;
 *   - the leak detector (Section 3.4): a growth sample that sets a new
 *     footprint high-water mark tracks the sampled block; frees compare their
 *     pointer with it; at the next mark the site's (frees, mallocs) pair is
 *     updated; likelihood = 1 - (frees + 1) / (mallocs - frees + 2);
 *   - the copy-volume sampler (Section 3.5): one sample per T_c bytes copied,
 *     T_c a multiple of T.
 *
 * Every trace has resident state on the device (counter, open-window totals,
 * footprint, high-water mark, tracked block, per-line tables, copy counter), so
 * a trace may arrive in any number of segments: replaying the pieces in order
 * gives exactly the result of replaying the whole.
 *
 * Conventions
 *   - Every int-returning call returns SCL_OK (0) or a negative SCL_E* code;
 *     scl_last_error() then holds a one-line message.
 *   - "device pointer": memory the CUDA device can read (cudaMalloc, torch).
 *     Event arrays stay owned by the caller and must stay valid until the
 *     stream work of the call has finished.  Each array must be 16-byte
 *     aligned when its segment holds >= 1024 events (SCL_EINVAL otherwise).
 *   - Replay calls are asynchronous on the caller's stream; query calls
 *     synchronise that stream first and report any error a kernel recorded.
 *   - Query outputs are caller-owned host arrays; when `cap` is too small the
 *     call stores the needed count in *n_out and returns SCL_ERANGE.
 *   - All arithmetic is exact 64-bit integer arithmetic.  The caller keeps the
 *     running sums of a trace's deltas inside int64 (the library does not
 *     check every event); a memcpy whose size plus the running copy counter
 *     (below T_c) passes 2^64, and record space that runs out, are reported as
 *     SCL_EOVERFLOW.
 *   - Line ids are read, and checked, where the method uses them: at the
 *     events that trigger a sample and at memcpy events.
 *   - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef SCL_H
#define SCL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCL_OK 0
#define SCL_EINVAL (-1)     /* bad argument, descriptor, alignment or trace id */
#define SCL_ENOMEM (-2)     /* device or pinned host allocation failed */
#define SCL_ECUDA (-3)      /* a CUDA runtime call failed */
#define SCL_ETIMEOUT (-4)   /* a bounded device wait gave up (see spin_limit) */
#define SCL_EOVERFLOW (-5)  /* an int64 sum would overflow, or a record buffer overflowed */
#define SCL_ERANGE (-6)     /* a line id >= n_lines was seen, or an output cap is too small */
#define SCL_EINTERNAL (-7)  /* an internal consistency check failed (a library bug) */

typedef struct scl_ctx scl_ctx;

/* One trace segment of allocation events, structure of arrays (Section 3.1-3.2).
 * delta[i] > 0 is a malloc of delta[i] bytes, delta[i] < 0 a free of -delta[i]
 * bytes, 0 is allowed and never samples.  addr[i] is the block address (only
 * compared for equality, Section 3.4).  line[i] < n_lines is the source line the
 * shim attributes the call to, is_python[i] = 1 for Python's allocator and 0 for
 * native code (Section 3.1).  All four are device pointers of length n. */
typedef struct {
    const int64_t *delta;
    const uint64_t *addr;
    const uint32_t *line;
    const uint8_t *is_python;
    uint64_t n;
} scl_events;

/* memcpy events of the same segment (Section 3.5): bytes copied, line, flag.
 * Device pointers of length n; n may be 0. */
typedef struct {
    const uint64_t *size;
    const uint32_t *line;
    const uint8_t *is_python;
    uint64_t n;
} scl_copies;

typedef struct {
    int64_t threshold;            /* T >= 1 (Section 3.2: a prime just above 10 MB, 10485767 by default) */
    uint32_t copy_multiple;       /* T_c = copy_multiple * T (Section 3.5), >= 1, default 2 */
    uint32_t n_lines;             /* L: line ids are < L, default 256 */
    uint64_t copy_phase;          /* copy counter at trace start, in [0, T_c), default 0 */
    int64_t initial_footprint;    /* F0: footprint and first high-water mark at trace start */
    uint32_t max_traces;          /* resident trace slots, ids 0 .. max_traces-1, default 1 */
    uint32_t leak_rule;           /* 0: likelihood as printed in Section 3.4 (default);
                                     1: Laplace's rule, 1 - (frees+1)/(mallocs+2) */
    uint64_t spin_limit;          /* iterations before a device wait reports SCL_ETIMEOUT (0: 1<<26) */
    uint64_t sample_log_capacity; /* samples kept per trace for scl_samples (0: keep none) */
    uint32_t sample_budget_shift; /* record space per work unit = (events >> shift) + 64; 0 never
                                     overflows; default SCL_BUDGET_AUTO: floor(log2 T) - 16, clamped
                                     to 0..4 (0 for T < 2^17, so T = 1 never overflows); a batch whose
                                     records overflow returns SCL_EOVERFLOW, and the context doubles the
                                     space of later batches (shift - 1, down to 0) */
    uint32_t unit_events;         /* events per work unit (multiple of 1024; 0: one unit per resident warp) */
} scl_config;

#define SCL_BUDGET_AUTO 0xffffffffu   /* sample_budget_shift picked from T */

/* Fill *cfg with the defaults listed above. */
int scl_config_default(scl_config *cfg);

/* One segment of trace `trace_id` (< max_traces). */
typedef struct {
    uint32_t trace_id;
    uint32_t reserved;
    scl_events ev;
    scl_copies cp;
} scl_segment;

/* One sample-file entry (Section 3.3): 56 bytes. */
typedef struct {
    uint64_t idx;         /* event index within the trace (counted over all its segments) */
    int64_t A, F;         /* bytes allocated / freed in the window that closed here */
    int64_t A_py, F_py;   /* the Python part of A and F */
    int64_t footprint;    /* F0 + all deltas up to and including idx */
    uint32_t line;        /* line of the event that crossed the threshold */
    int8_t kind;          /* +1 growth (A - F >= T), -1 shrink (A - F <= -T) */
    uint8_t is_python;    /* flag of that event */
    uint8_t is_hwm;       /* 1: this sample set a new high-water mark and started tracking its block */
    uint8_t reserved;
} scl_sample;

/* Per-line totals over all samples of a trace (Sections 3.3 and 3.5), row = line id. */
typedef struct {
    uint64_t n_growth, n_shrink;        /* samples attributed to the line */
    int64_t A, F, A_py, F_py;           /* sums of the window totals of those samples */
    int64_t net;                        /* sum of A - F over those samples */
    uint64_t copy_samples[2];           /* copy-volume samples, index = is_python */
    uint64_t copy_bytes[2];             /* copy_samples * T_c */
} scl_line_stat;

/* Per-line leak score (Section 3.4) as an unreduced fraction num/den. */
typedef struct {
    uint32_t line;
    uint32_t reserved;
    uint64_t mallocs;   /* tracked blocks sampled at this line (incremented when tracking starts) */
    uint64_t frees;     /* of those whose trial has closed, the ones freed inside their window */
    int64_t num, den;   /* likelihood = num / den under the configured leak_rule; den >= 2 */
} scl_leak_score;

/* Leak report row (Section 3.4, "Leak Report Filtering and Prioritization").  A line is
 * reported when its leak likelihood exceeds 95% (20 num > 19 den, exactly) and the trace's
 * memory grew by at least 1% (100 (footprint - F0) >= high-water mark > 0).  Its leak rate
 * -- bytes allocated in the windows attributed to the line per elapsed time, with the event
 * count as time -- is the exact fraction rate_num / rate_den; sort reported rows by it. */
typedef struct {
    uint32_t line;
    uint8_t reported;   /* likely && growth */
    uint8_t likely;     /* likelihood > 95% */
    uint8_t growth;     /* the trace's footprint grew by >= 1% (the same for every line) */
    uint8_t reserved;
    uint64_t mallocs, frees;
    int64_t num, den;   /* likelihood, as scl_leak_score */
    int64_t rate_num;   /* bytes allocated in the line's sample windows */
    uint64_t rate_den;  /* events elapsed */
} scl_leak_report_row;

/* Resident sampler state of one trace. */
typedef struct {
    uint64_t n_events, n_copies, n_samples;
    int64_t c;                          /* A - F of the open window */
    int64_t A, F, A_py, F_py;           /* open-window totals */
    int64_t footprint, hwm;
    uint64_t tracked_addr, tracked_idx; /* block tracked since the last high-water crossing */
    uint32_t tracked_line;
    uint8_t tracked_valid, tracked_reclaimed, reserved[2];
    uint64_t copy_counter;              /* bytes copied since the last copy sample, < T_c */
} scl_trace_info;

/* Create a context: validates *cfg, allocates the resident state of max_traces
 * traces on the current CUDA device.  The library owns *out until scl_replay_free. */
int scl_replay_init(scl_ctx **out, const scl_config *cfg);
void scl_replay_free(scl_ctx *ctx);
const char *scl_last_error(const scl_ctx *ctx);

/* Append each segment to its trace's resident state (Sections 3.2-3.5).
 * segs: host array of nsegs descriptors holding device pointers.  Segments of
 * the same trace are applied in array order.  Asynchronous on cuda_stream
 * (a cudaStream_t; NULL = legacy default stream).  Returns SCL_EINVAL on a bad
 * descriptor; errors found by kernels (line id >= L -> SCL_ERANGE, int64
 * overflow / record space -> SCL_EOVERFLOW, wait limit -> SCL_ETIMEOUT) are
 * reported by the next query or scl_sync, and the affected results are invalid. */
int scl_replay_batch(scl_ctx *ctx, const scl_segment *segs, uint32_t nsegs, void *cuda_stream);

/* Same as scl_replay_batch but the event arrays are in HOST memory: the library
 * copies them to its own device staging buffers on cuda_stream first, in pieces over
 * several copy streams (pinned host memory makes those copies asynchronous).  An event
 * line column in pinned, device-mapped memory is not copied: the kernels read it in
 * place at the events that sample.  Host arrays must stay valid until the stream work
 * of the call has finished. */
int scl_replay_batch_host(scl_ctx *ctx, const scl_segment *segs, uint32_t nsegs, void *cuda_stream);

/* Wait for the work of the last replay call; return the first recorded device error. */
int scl_sync(scl_ctx *ctx);

/* Queries (synchronise first).  scl_samples returns the trace's retained samples
 * in order; *n_out = all samples ever taken; if more were taken than
 * sample_log_capacity, the first sample_log_capacity are returned and the call
 * returns SCL_EOVERFLOW.  scl_line_stats / scl_leak_scores return n_lines rows. */
int scl_samples(scl_ctx *ctx, uint32_t trace, scl_sample *out, uint64_t cap, uint64_t *n_out);
int scl_line_stats(scl_ctx *ctx, uint32_t trace, scl_line_stat *out, uint32_t cap, uint32_t *n_out);
/* Footprint timeline of one line (Section 3.3's memory-trend feed): the event index and
 * footprint of every retained sample attributed to `line`, in trace order, into host arrays
 * idx_out / fp_out of cap entries; *n_out = the number of such samples (SCL_ERANGE when cap
 * is smaller; SCL_EOVERFLOW when the log did not retain every sample).  The paper's
 * downsampling of the plotted trend is not applied. */
int scl_line_timeline(scl_ctx *ctx, uint32_t trace, uint32_t line, uint64_t *idx_out, int64_t *fp_out, uint64_t cap,
                      uint64_t *n_out);
int scl_leak_scores(scl_ctx *ctx, uint32_t trace, scl_leak_score *out, uint32_t cap, uint32_t *n_out);
/* The same rows for ntr consecutive traces trace0 .. trace0 + ntr - 1 in one call (one
 * synchronisation, rows formed on the device, one copy): trace-major, row l of trace
 * trace0 + i at out[i * n_lines + l]; cap counts rows; *n_out = ntr * n_lines (SCL_ERANGE when
 * cap is smaller, SCL_EINVAL when the range passes max_traces).  out may be pinned or pageable
 * host memory.  Grows one device buffer of the context to ntr * n_lines rows. */
int scl_line_stats_range(scl_ctx *ctx, uint32_t trace0, uint32_t ntr, scl_line_stat *out, uint64_t cap,
                         uint64_t *n_out);
int scl_leak_scores_range(scl_ctx *ctx, uint32_t trace0, uint32_t ntr, scl_leak_score *out, uint64_t cap,
                          uint64_t *n_out);
int scl_trace_state(scl_ctx *ctx, uint32_t trace, scl_trace_info *out);
int scl_leak_report(scl_ctx *ctx, uint32_t trace, scl_leak_report_row *out, uint32_t cap, uint32_t *n_out);

/* Checkpoint / resume of one trace's resident state (counter, window totals,
 * footprint, mark, tracked block, per-line tables, copy counter; not the sample
 * log).  Export with buf == NULL stores the needed size in *n_out.  Import
 * replaces the trace's state; a state exported from a context with other
 * threshold, n_lines, copy_multiple or leak_rule is rejected (SCL_EINVAL). */
int scl_state_export(scl_ctx *ctx, uint32_t trace, void *buf, uint64_t cap, uint64_t *n_out);
int scl_state_import(scl_ctx *ctx, uint32_t trace, const void *buf, uint64_t n);

/* Return a trace to its initial state (F0, counters 0, empty tables and log);
 * trace = SCL_ALL_TRACES resets every trace slot in one launch. */
#define SCL_ALL_TRACES 0xffffffffu
int scl_trace_reset(scl_ctx *ctx, uint32_t trace, void *cuda_stream);

/* Tuning: events per work unit (the chunk of a trace whose entering counter the sketch
 * speculates), first-unit length, warps per block of phase 1 and of the exact replay,
 * warm-up events, fix-up strategy.  scl_autotune times scl_replay_batch on the given
 * segments (a warm-up call, then the mean of three calls issued back to back, so that each
 * call's host-side planning overlaps the previous call's device work as in repeated use;
 * the results of these calls are discarded) and searches one setting at a time,
 * twice over: unit 32k/64k/128k/256k/512k/1M/2M, first unit unit/512k/768k/1M/1.25M/1.5M,
 * phase-1 warps 8/12/16, replay warps 10/12/14, warm-up 16k/32k, fix-up 0/1, replay pieces
 * 32k/64k/128k/4M.  It restores the
 * touched traces' state before every run and at the end, keeps the fastest setting in the
 * context (read it back with scl_tuning_get), and allocates one device buffer for the
 * saved states. */
typedef struct {
    uint32_t unit_events;    /* events per work unit (multiple of 1024; 0 = one unit per resident warp) */
    uint32_t warps_per_block;/* sketch warps per thread block (1..16) */
    uint32_t ext_events;     /* warm-up events each unit's candidates run before the unit (multiple of 256; 0 = 32768) */
    uint32_t final_warps;    /* exact-replay warps per thread block (1..14) */
    uint32_t first_events;   /* length of each trace's first unit, replayed exactly in one pass from the
                                trace's resident state (multiple of 1024; 0 = unit_events); with fewer
                                traces than SMs a first unit is one warm-up long instead */
    uint32_t fixup;          /* how the exact replay of a sketched unit finds its samples once its entry is
                                known: 0 = from every reset the sketch listed for that run (default),
                                1 = by searching each step's prefix sums for crossings */
    uint32_t piece_events;   /* the exact replay of a sketched unit whose resets are listed is cut into
                                pieces replayed in parallel, each ending at the first listed reset past
                                the next multiple of piece_events (after a reset the counter and the
                                window restart from zero); multiple of 256; 0 = 65536 */
} scl_tuning;
int scl_tuning_get(const scl_ctx *ctx, scl_tuning *out);
int scl_tuning_set(scl_ctx *ctx, const scl_tuning *t);
int scl_autotune(scl_ctx *ctx, const scl_segment *segs, uint32_t nsegs, void *cuda_stream,
                 scl_tuning *best_out, double *best_ms_out);

/* Graph replay: with on != 0, a replay call on a non-default stream whose plan (segment
 * pointers and lengths, trace states' event counts, tuning, buffers) is byte-identical to
 * the previous call's is relaunched as one captured CUDA graph; any other call captures a
 * new graph.  Not used while profiling is enabled.  Default off. */
int scl_graph_enable(scl_ctx *ctx, int on);

/* Per-kernel device time of replay calls, for measurement.  When enabled, each
 * replay call records CUDA events around its kernels on its stream; scl_kernel_times
 * synchronises and returns, for each kernel name, the summed milliseconds and the
 * number of launches since the last reset.  names[i] point to static strings. */
int scl_profile_enable(scl_ctx *ctx, int on);
int scl_kernel_times(scl_ctx *ctx, const char **names, double *ms, uint64_t *launches,
                     uint32_t cap, uint32_t *n_out);
int scl_profile_reset(scl_ctx *ctx);

/* How the last replay call found each unit's entering counter (for tuning): units
 * whose true run matched no warm-up candidate are walked on demand, and stop as soon as
 * they share a reset with one of the unit's candidates. */
typedef struct {
    uint64_t units;             /* work units of the last batch */
    uint64_t walked;            /* units walked on demand by the per-trace chain */
    uint64_t walked_merged;     /* ... of which stopped early by merging into a candidate */
    uint64_t explicit_entries;  /* units entered with a counter no candidate carried */
    uint64_t transparent;       /* ... of which held no sample (skipped in O(1)) */
    uint64_t unit_events;       /* tuned events per unit (0: sized per batch) */
    uint64_t walked_events;     /* events the chain's walks covered before merging (or to the unit end) */
    uint64_t searched;          /* units replayed exactly without a reset list (crossings searched) */
    uint64_t first_events;      /* events of the traces' first units (replayed exactly from the resident state) */
    uint64_t sketch_events;     /* events the candidate counters streamed: the other units and their warm-ups */
} scl_batch_info;
int scl_batch_stats(scl_ctx *ctx, scl_batch_info *out);

/* Serving loop (Section 3.1 deployment: one profiler process per profiled process, each
 * streaming its events).  Requests are segments of many traces in HOST memory (pinned for
 * asynchronous copies), each with an offered arrival time; requests of one trace appear
 * in arrival order.  scl_serve admits arrived requests into a batch while its device
 * staging slot has room (three slots sized from the budget), copies a slot's arrays to
 * the device on a copy stream while the previous batch replays on a compute stream (a
 * pinned event line column is read in place instead), and
 * replays each batch with scl_replay_batch; a trace's results equal those of replaying
 * its requests alone, in order.  The call returns when every request has been replayed
 * (then scl_sync's status). */
typedef struct {
    uint32_t trace_id;    /* trace slot of the process (< max_traces) */
    uint32_t reserved;
    uint64_t arrival_ns;  /* offered arrival, ns after the call starts (used when realtime) */
    scl_events ev;        /* HOST pointers */
    scl_copies cp;        /* HOST pointers */
} scl_request;

typedef struct {
    uint64_t hbm_budget;  /* device staging bytes for the three slots (0: half the free HBM, <= 8 GiB);
                             SCL_ENOMEM if a slot cannot hold the largest request */
    uint32_t max_batch;   /* requests per batch (0: 256) */
    uint32_t realtime;    /* 1: admit a request only after its arrival time; 0: all arrived at start */
} scl_serve_opts;

typedef struct {
    uint64_t done_ns;     /* when its batch's replay was seen complete, ns after the call started */
    uint64_t latency_ns;  /* done_ns - arrival_ns (realtime), else done_ns */
    uint32_t batch;       /* index of the batch that replayed it */
    uint32_t reserved;
} scl_request_result;

typedef struct {
    uint64_t requests, batches, events;
    uint64_t staging_bytes; /* device bytes held by the staging slots */
    double wall_s;          /* from the first arrival to the last completion */
} scl_serve_summary;

int scl_serve(scl_ctx *ctx, const scl_request *reqs, uint32_t n, const scl_serve_opts *opts,
              scl_request_result *out, scl_serve_summary *summary);

/* Rate-based sampling (Section 3.2): the conventional sampler the paper compares threshold
 * sampling with (its Table 2).  Every byte allocated or freed is a Bernoulli trial; the
 * sampled bytes sit at cumulative byte positions B_k = gap[0] - consumed + gap[1] + ... +
 * gap[k], where gap[] (device, n_gaps values >= 1) are the caller's draws -- geometric with
 * mean T for the paper's sampler -- and consumed (< gap[0]) is how far the previous call got
 * into gap[0].  Event i of delta/line/is_python (device, n events) moves |delta[i]| bytes and
 * takes one sample per B_k in its byte range (a large event can take several), counted in
 * counts_out[2 * line + (is_python != 0)] (device, 2 * n_lines, cleared by the call).
 * state_out (device, 4): samples taken, gaps used up (continue with gap + that count),
 * bytes of the next gap consumed (the next call's `consumed`), flags (1: the gaps ran out
 * before the bytes did, 2: a sampled event's line id >= n_lines, not counted, 4: the byte
 * count passed 2^64).  Asynchronous on cuda_stream; scratch comes from the context. */
int scl_rate_samples(scl_ctx *ctx, const int64_t *delta, const uint32_t *line, const uint8_t *is_python, uint64_t n,
                     const uint64_t *gap, uint64_t n_gaps, uint64_t consumed, uint64_t *counts_out,
                     uint64_t *state_out, void *cuda_stream);

/* Python vs native time (Section 2.2): n CPU-timer interrupts, vtime[k] the virtual time
 * (ns, non-decreasing) at interrupt k and line[k] the interrupted line (device arrays).  The
 * elapsed time T since the previous interrupt (t_prev before the first) goes to the line's
 * Python counter up to the quantum q and to its native counter beyond it: python += min(T, q),
 * native += T - min(T, q).  python_out / native_out (device, n_lines each) and flags_out
 * (device, 1: 1 time went backwards, 2 a line id >= n_lines; such interrupts are skipped)
 * are cleared by the call.  Pass vtime[n-1] as the next call's t_prev. */
int scl_cpu_attribution(scl_ctx *ctx, const int64_t *vtime, const uint32_t *line, uint64_t n, int64_t quantum,
                        int64_t t_prev, int64_t *python_out, int64_t *native_out, uint64_t *flags_out,
                        void *cuda_stream);

/* Failure-detection self test (no counterpart in the paper): launches one warp that
 * waits, with the same bounded wait the walker uses, on a barrier nothing arrives at.
 * The wait gives up after `limit` polls and the call returns SCL_ETIMEOUT; the
 * context's error word is cleared afterwards, so the context stays usable. */
int scl_selftest_wait(scl_ctx *ctx, uint64_t limit, void *cuda_stream);

/* Copy-volume sampler for callers that cannot allocate device memory.  The paper has
 * no counterpart for this entry point: it is the copy sampler of scl_replay_batch
 * (Section 3.5) packaged for code that must not call cudaMalloc -- code running
 * inside an allocation hook (a profiler's interposition layer cannot re-enter the
 * allocator it intercepts), processes whose device memory belongs to a caching
 * allocator or a quota, and latency-bound callers (cudaMalloc synchronises).
 *
 * It allocates nothing.  Its only scratch, one 64-bit sum per 4,096 memcpy events,
 * is a static 128 KiB device array that every GPU loading this library holds until
 * the process exits; hence m <= 67,108,864 (SCL_EINVAL beyond).  All calls share that
 * array: calls that overlap on the GPU (on different streams, or from several host
 * threads) race on it and give wrong results; calls ordered on one stream are fine.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture on the device.
 *
 * Inputs (device pointers, length m): size, line (< n_lines; others are skipped and
 * counted), is_python.  copy_threshold = T_c >= 1; counter_in in [0, T_c) is the
 * running copy count carried from earlier memcpys (0 or copy_phase for a new trace).
 * Outputs (device pointers, caller-owned, cleared by the call, asynchronous on
 * cuda_stream): samples_out[2*n_lines] and bytes_out[2*n_lines], indexed
 * 2*line + is_python, the same values as scl_line_stat.copy_samples / copy_bytes of
 * a trace whose only events are these memcpys; state_out[3] = { counter after the
 * memcpys (< T_c), memcpys skipped for a line id >= n_lines, 1 if the byte count
 * overflowed uint64 }.  Returns SCL_EINVAL on bad arguments, SCL_ECUDA if a launch
 * or the address lookup fails. */
int scl_copy_volume_noalloc(const uint64_t *size, const uint32_t *line, const uint8_t *is_python, uint64_t m,
                            uint64_t copy_threshold, uint64_t counter_in, uint32_t n_lines, uint64_t *samples_out,
                            uint64_t *bytes_out, uint64_t *state_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SCL_H */
