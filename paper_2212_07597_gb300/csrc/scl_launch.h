// scl_launch.h -- host-side launchers of the libscl kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "scl_internal.cuh"

namespace scl {

// device counters of a batch: units walked, walked and merged, explicit entries,
// transparent, events walked (k_chain); units replayed with the crossing search (k_final)
constexpr int NSTATS = 6;
constexpr int PHASE1_MAX_WARPS = 16;   // k_phase1 warps per block (its launch bound)
constexpr int SKETCH_TILE = 512;       // sketch events per staged tile (warm-ups start on one)

struct LaunchSketch {
    const Unit *units;
    int nunits;
    const BTrace *bts;
    int nbt;
    UnitSum *usum;
    Cand *cand;
    SRes *lists;
    FRec *recs;          // first units: their records and outputs (k_phase1 replays them exactly)
    UnitOut *uout;
    uint8_t *match;
    Walk *uwalk;
    UnitTrue *utrue;
    uint32_t *umode;
    int64_t *uexp;
    const DevTrace *traces;
    int64_t T;
    uint32_t warmup;
    const uint32_t *order;   // phase-1 work: unit indices, longest work first
    int nitems;
    unsigned *queue;     // [0] phase 1, [2] final
    ErrWord *err;
    unsigned long long spin;
    unsigned long long *stats;   // NSTATS counters of the batch, see NSTATS
    int blocks, warps_per_block, num_sms;
};

struct LaunchFinal {
    unsigned long long *stats;   // [5]: units replayed with the crossing search
    const Unit *units;
    int nunits;
    const FItem *items;          // the pieces, in the order warps take them
    int nitems;
    uint32_t *phit;              // per piece: what k_mark applies (0 nothing, PHIT_ENTER, 1 + record)
    uint64_t piece;              // events per piece (cut at the next listed reset)
    const UnitTrue *utrue;
    const UnitPlan *uplan;
    const SRes *lists;
    FRec *recs;
    UnitOut *uout;
    int64_t T;
    unsigned *queue;
    ErrWord *err;
    unsigned long long spin;
    int blocks, warps_per_block;
};

struct LaunchCopy {           // the copy-volume sampler (scl_copy.cu)
    const CopyTile *ctiles;      // in the order blocks take them (rounds over the traces)
    int nctiles;
    void *cstatus;               // look-back state per tile, cleared before the batch
    const DevTrace *traces;
    BTraceRes *btres;
    unsigned long long *copies;  // resident copy-volume samples [trace][line][flag]
    uint32_t n_lines;
    uint64_t Tc;
    unsigned *queue;             // tile tickets
    ErrWord *err;
    unsigned long long spin;
    int num_sms;
};

struct CompactGroup {
    uint32_t u0, nu;
};

struct LaunchPost {
    const Unit *units;
    int nunits;
    const BTrace *bts;
    int nbt;
    const UnitSum *usum;
    const UnitTrue *utrue;
    UnitPlan *uplan;
    UnitOut *uout;
    BTraceRes *btres;
    FRec *recs;
    int64_t *pref;         // per unit: exclusive prefix of (totA, totApy, totSpy) within its trace
    DevTrace *traces;
    LineRow *lines;
    Sample *log;
    uint64_t log_cap;
    uint32_t n_lines;
    int64_t T;
    uint64_t Tc;
    const CompactGroup *groups;
    int ngroups;
    const uint32_t *phit;  // k_final's per-piece reports (see LaunchFinal)
    ErrWord *err;
};


int phase1_occupancy(int warps_per_block, int *blocks_per_sm);
int final_occupancy(int warps_per_block, int *blocks_per_sm);
cudaError_t launch_phase1(const LaunchSketch &a, cudaStream_t s);
size_t copy_status_bytes(size_t ntiles);   // look-back state of the copy-volume tiles
cudaError_t launch_copy(const LaunchCopy &a, cudaStream_t s);
cudaError_t launch_match(const LaunchSketch &a, cudaStream_t s);
cudaError_t launch_chain(const LaunchSketch &a, cudaStream_t s);
cudaError_t launch_totals(const LaunchSketch &a, cudaStream_t s);
cudaError_t launch_final(const LaunchFinal &a, cudaStream_t s);

cudaError_t launch_wait_selftest(ErrWord *err, unsigned long long limit, cudaStream_t s);

cudaError_t launch_scan(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_compact(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_mark(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_epi(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_state(const LaunchPost &a, cudaStream_t s);

cudaError_t launch_reset(DevTrace *traces, LineRow *lines, unsigned long long *copies, uint32_t trace0,
                         uint32_t ntr, uint32_t n_lines, int64_t F0, uint64_t phase, cudaStream_t s);
// the range queries' rows (scl_line_stat / scl_leak_score layouts), trace-major from trace0
cudaError_t launch_stat_rows(const LineRow *lines, const unsigned long long *copies, uint32_t trace0, uint64_t nrows,
                             uint32_t n_lines, uint64_t Tc, void *out, int num_sms, cudaStream_t s);
cudaError_t launch_score_rows(const LineRow *lines, uint32_t trace0, uint64_t nrows, uint32_t n_lines, uint32_t rule,
                              void *out, int num_sms, cudaStream_t s);
cudaError_t launch_scores(const LineRow *lines, uint32_t trace, uint32_t n_lines, uint32_t rule, void *out,
                          cudaStream_t s);
cudaError_t launch_timeline(const Sample *log, uint64_t n, uint32_t line, void *scratch, uint64_t cap,
                            uint64_t *idx_out, int64_t *fp_out, cudaStream_t s);
cudaError_t launch_report(const LineRow *lines, const DevTrace *traces, uint32_t trace, uint32_t n_lines,
                          uint32_t rule, int64_t F0, void *out, cudaStream_t s);

}  // namespace scl

// rate-based sampling (scl_rate.cu): scratch bytes and the launch sequence
namespace scl {
size_t rate_scratch_bytes(uint64_t n, uint64_t ng);
cudaError_t launch_rate(const int64_t *delta, const uint32_t *line, const uint8_t *py, uint64_t n,
                        const uint64_t *gap, uint64_t ng, uint64_t consumed, uint32_t n_lines, uint64_t *counts,
                        uint64_t *state, void *scratch, cudaStream_t s);
cudaError_t launch_cpu_attr(const int64_t *vt, const uint32_t *line, uint64_t n, int64_t q, int64_t t_prev,
                            uint32_t n_lines, int64_t *py, int64_t *nat, uint64_t *flags, int sms, cudaStream_t s);
}  // namespace scl

// context facts the serving loop needs (scl_serve.cu); defined in scl_host.cu
struct scl_ctx;
uint32_t scl_ctx_max_traces(const scl_ctx *c);
int scl_ctx_device(const scl_ctx *c);
int scl_ctx_fail(scl_ctx *c, int code, const char *msg);
void scl_ctx_forget_stream(scl_ctx *c);   // the last replay stream is about to be destroyed
