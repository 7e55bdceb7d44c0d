// scl_launch.h -- host-side launchers of the libscl kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "scl_internal.cuh"

namespace scl {

struct LaunchWalk {
    const Unit *units;
    int nunits;
    UnitRes *ures;
    Rec *recs;
    uint32_t *pub;
    uint32_t *bits;
    const DevTrace *traces;
    int64_t T;
    uint32_t ext_cap;
    unsigned *queue;
    ErrWord *err;
    unsigned long long spin;
    int blocks, warps_per_block;
};

struct CompactGroup {
    uint32_t u0, nu;
};

struct LeakTile {
    uint32_t unit, k;
};

struct LaunchPost {
    const Unit *units;
    int nunits;
    const BTrace *bts;
    int nbt;
    UnitRes *ures;
    BTraceRes *btres;
    const Rec *recs;
    Cross *cross;
    uint8_t *recl;
    const uint32_t *bits;
    DevTrace *traces;
    LineRow *lines;
    Sample *log;
    uint64_t log_cap;
    uint32_t n_lines;
    int64_t T;
    uint64_t Tc;
    const CompactGroup *groups;
    int ngroups;
    const LeakTile *ltiles;
    int nltiles;
    const CopyTile *ctiles;
    int nctiles;
    uint64_t *ctile_sum;   // per copy tile: sum, then (after the scan) base counter
    ErrWord *err;
};

size_t walk_smem_per_warp();
int walk_occupancy(int warps_per_block, int *blocks_per_sm);
cudaError_t launch_walk(const LaunchWalk &a, cudaStream_t s);
cudaError_t launch_resolve(const Unit *units, int nunits, UnitRes *ures, const Rec *recs, cudaStream_t s);
cudaError_t launch_fallback(const Unit *units, const BTrace *bts, int nbt, UnitRes *ures, Rec *recs, int64_t T,
                            ErrWord *err, unsigned long long spin, cudaStream_t s);

cudaError_t launch_wait_selftest(ErrWord *err, unsigned long long limit, cudaStream_t s);

cudaError_t launch_scan(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_compact(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_scan2(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_leak(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_epi(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_copy_sum(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_copy_scan(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_copy_apply(const LaunchPost &a, cudaStream_t s);
cudaError_t launch_state(const LaunchPost &a, cudaStream_t s);

cudaError_t launch_reset(DevTrace *traces, LineRow *lines, uint32_t trace, uint32_t n_lines, int64_t F0,
                         uint64_t phase, cudaStream_t s);
cudaError_t launch_scores(const LineRow *lines, uint32_t trace, uint32_t n_lines, uint32_t rule, void *out,
                          cudaStream_t s);

}  // namespace scl
