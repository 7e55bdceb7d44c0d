// scl_host.cu -- the C ABI of libscl (include/scl.h): contexts, batch planning,
// launch sequence, queries, checkpoint / resume, profiling.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/scl.h"
#include "scl_internal.cuh"
#include "scl_launch.h"
#include "scl_views.h"

using namespace scl;

namespace {

constexpr uint32_t STATE_MAGIC = 0x53434c33u;   // "SCL3"

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct ProfEntry {
    const char *name;
    cudaEvent_t a, b;
};

}  // namespace

struct scl_ctx {
    scl_config cfg{};
    uint32_t shift = 4;   // record budget in effect (cfg.sample_budget_shift, resolved and grown)
    int device = 0;
    int num_sms = 0;
    std::string err;
    cudaStream_t last_stream = nullptr;
    // resident state
    DevTrace *traces = nullptr;
    LineRow *lines = nullptr;
    unsigned long long *copies = nullptr;   // copy-volume samples [trace][line][flag]
    Sample *log = nullptr;
    ErrWord *errw = nullptr;
    void *scores = nullptr;
    unsigned *queue = nullptr;
    unsigned long long *stats = nullptr;   // device: chain counters of the last batch
    uint64_t last_units = 0;
    uint64_t last_first_events = 0, last_sketch_events = 0;
    std::vector<uint64_t> h_events;   // host mirror of each trace's event count
    // batch scratch
    DevBuf plan, usum, cand, lists, match, uwalk, utrue, umode, uexp, uplan, uout, pref, recs, btres, ctsum, stage, phit, qrows;
    DevBuf rate;   // scratch of scl_rate_samples
    DevBuf report; // rows of scl_leak_report
    DevBuf tline;  // scratch and output of scl_line_timeline
    void *h_plan = nullptr;
    size_t h_plan_cap = 0;
    cudaEvent_t plan_done = nullptr;
    bool plan_pending = false;
    // the replay's kernels run on a high-priority stream forked from the caller's; the
    // copy-volume sampler (Section 3.5), which shares nothing with the event path, runs on a
    // side stream between the fork and a join before the state fold
    cudaStream_t hi = nullptr, side = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_copy = nullptr, ev_fork = nullptr;
    // host-to-device staging of scl_replay_batch_host: pieces spread over several copy
    // streams (several copy engines at once), joined back before the replay
    static constexpr int NCS = 4;
    cudaStream_t cstream[NCS] = {};
    cudaEvent_t cev[NCS + 1] = {};
    // tuning
    scl_tuning tune{};
    // graph replay of repeated identical batches
    bool graph_on = false;
    cudaGraphExec_t gexec = nullptr;
    // the captured batch: its plan (the graph uploads it from this pinned copy, which only a
    // recapture rewrites, so the host never waits for a running graph to reuse h_plan) and
    // the buffers and tuning it was captured with
    void *g_plan = nullptr;
    size_t g_plan_cap = 0, g_blob = 0;
    std::vector<const void *> g_ptrs;
    scl_tuning g_tune{};
    cudaEvent_t g_done = nullptr;   // recorded after each graph launch (before a recapture)
    bool g_pending = false;
    // profiling
    bool prof = false;
    std::vector<ProfEntry> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<const char *, std::pair<double, uint64_t>>> prof_acc;
};

namespace {

int fail(scl_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(scl_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? SCL_ENOMEM : SCL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

int ensure(scl_ctx *c, DevBuf &b, size_t bytes, cudaStream_t s, const char *what) {
    if (bytes <= b.cap) return SCL_OK;
    size_t nb = std::max(bytes, b.cap + b.cap / 2);
    nb = (nb + 4095) & ~size_t(4095);
    if (b.p) {
        CK(cudaStreamSynchronize(s), "sync before regrow");
        CK(cudaFree(b.p), "cudaFree");
        b.p = nullptr;
        b.cap = 0;
    }
    CK(cudaMalloc(&b.p, nb), what);
    b.cap = nb;
    return SCL_OK;
}

cudaEvent_t pool_event(scl_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Prof {
    scl_ctx *c;
    cudaStream_t s;
    const char *name;
    cudaEvent_t a = nullptr;
    Prof(scl_ctx *c_, cudaStream_t s_, const char *n) : c(c_), s(s_), name(n) {
        if (c->prof) { a = pool_event(c); cudaEventRecord(a, s); }
    }
    ~Prof() {
        if (c->prof) {
            cudaEvent_t b = pool_event(c);
            cudaEventRecord(b, s);
            c->prof_pending.push_back({name, a, b});
        }
    }
};

void prof_collect(scl_ctx *c) {
    for (auto &p : c->prof_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        bool found = false;
        for (auto &q : c->prof_acc)
            if (strcmp(q.first, p.name) == 0) { q.second.first += ms; q.second.second += 1; found = true; break; }
        if (!found) c->prof_acc.push_back({p.name, {ms, 1}});
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->prof_pending.clear();
}

int check_device_error(scl_ctx *c) {
    ErrWord w{};
    CK(cudaMemcpy(&w, c->errw, sizeof w, cudaMemcpyDeviceToHost), "read error word");
    if (w.code == 0) return SCL_OK;
    switch (w.code) {
    case E_RANGE:
        return fail(c, SCL_ERANGE, "line id %u >= n_lines (%u) at event %llu", w.detail0, c->cfg.n_lines,
                    (unsigned long long)w.detail1);
    case E_TIMEOUT:
        return fail(c, SCL_ETIMEOUT, "a device wait exceeded spin_limit (site %u, %llu)", w.detail0,
                    (unsigned long long)w.detail1);
    case E_INTERNAL:
        return fail(c, SCL_EINTERNAL, "internal consistency check failed (site %u, %llu)", w.detail0,
                    (unsigned long long)w.detail1);
    case E_OVERFLOW:
        // a unit's records did not fit: give later batches twice the space
        if (w.detail0 == 3 && c->shift > 0) --c->shift;
        return fail(c, SCL_EOVERFLOW,
                    "record space overflow or uint64 copy-count overflow (site %u, unit/tile %llu); "
                    "lower sample_budget_shift", w.detail0, (unsigned long long)w.detail1);
    default:
        return fail(c, w.code, "device error %d (%u, %llu)", w.code, w.detail0, (unsigned long long)w.detail1);
    }
}

int sync_and_check(scl_ctx *c) {
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->last_stream), "stream sync");
    return check_device_error(c);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

struct EnqArgs {
    char *dp;
    const char *hp;
    size_t blob, o_units, o_bts, o_grp, o_ct, o_ord, o_fit;
    uint32_t nbt;
    int nunits, ngroups, nctiles, nitems;
};

// The device work of one replay call, in stream order (captured into a graph when
// graph replay is on).
// plan_done marks when the pinned plan buffer may be rewritten; it is recorded here
// only outside stream capture (an event recorded during capture is not usable after it).
int enqueue_batch(scl_ctx *c, cudaStream_t s, const EnqArgs &q, bool record_plan) {
    const scl_config &cfg = c->cfg;
    char *dp = q.dp;
    CK(cudaMemcpyAsync(dp, q.hp, q.blob, cudaMemcpyHostToDevice, s), "plan upload");
    if (record_plan) {
        CK(cudaEventRecord(c->plan_done, s), "plan event");
        c->plan_pending = true;
    }
    CK(cudaMemsetAsync(c->btres.p, 0, sizeof(BTraceRes) * q.nbt, s), "memset");
    CK(cudaMemsetAsync(c->queue, 0, sizeof(unsigned) * 4, s), "memset");
    CK(cudaMemsetAsync(c->stats, 0, sizeof(unsigned long long) * NSTATS, s), "memset");
    if (q.nctiles) CK(cudaMemsetAsync(c->ctsum.p, 0, copy_status_bytes(q.nctiles), s), "memset");
    // the kernels run on a high-priority stream forked from the caller's (other work on the
    // device yields SMs to the replay) and joined back at the end
    cudaStream_t s_user = s;
    CK(cudaEventRecord(c->ev_in, s_user), "fork event");
    s = c->hi;
    CK(cudaStreamWaitEvent(s, c->ev_in, 0), "fork the replay");

    const Unit *d_units = reinterpret_cast<const Unit *>(dp + q.o_units);
    const BTrace *d_bts = reinterpret_cast<const BTrace *>(dp + q.o_bts);

    const int nunits = q.nunits;
    const uint32_t nbt = q.nbt;
    LaunchPost a;
    a.units = d_units;
    a.nunits = nunits;
    a.bts = d_bts;
    a.nbt = (int)nbt;
    a.usum = static_cast<const UnitSum *>(c->usum.p);
    a.utrue = static_cast<const UnitTrue *>(c->utrue.p);
    a.uplan = static_cast<UnitPlan *>(c->uplan.p);
    a.uout = static_cast<UnitOut *>(c->uout.p);
    a.btres = static_cast<BTraceRes *>(c->btres.p);
    a.recs = static_cast<FRec *>(c->recs.p);
    a.pref = static_cast<int64_t *>(c->pref.p);
    a.traces = c->traces;
    a.lines = c->lines;
    a.log = c->log;
    a.log_cap = cfg.sample_log_capacity;
    a.n_lines = cfg.n_lines;
    a.T = cfg.threshold;
    a.Tc = (uint64_t)cfg.copy_multiple * (uint64_t)cfg.threshold;
    a.groups = reinterpret_cast<const CompactGroup *>(dp + q.o_grp);
    a.ngroups = q.ngroups;
    a.phit = static_cast<const uint32_t *>(c->phit.p);
    a.err = c->errw;
    // ---- the copy-volume sampler, on a side stream forked after phase 1 (before the scan when
    // there are no units): beside the chain, the scans and the bandwidth-bound exact replay
    // rather than the issue-bound phase 1 (its blocks take the room a replay block of up to 10
    // warps leaves)
    auto copy_pass = [&]() -> cudaError_t {
        if (!q.nctiles) return cudaSuccess;
        if (cudaError_t e = cudaEventRecord(c->ev_fork, s)) return e;
        if (cudaError_t e = cudaStreamWaitEvent(c->side, c->ev_fork, 0)) return e;
        LaunchCopy k;
        k.ctiles = reinterpret_cast<const CopyTile *>(dp + q.o_ct);
        k.nctiles = q.nctiles;
        k.cstatus = c->ctsum.p;
        k.traces = c->traces;
        k.btres = static_cast<BTraceRes *>(c->btres.p);
        k.copies = c->copies;
        k.n_lines = cfg.n_lines;
        k.Tc = (uint64_t)cfg.copy_multiple * (uint64_t)cfg.threshold;
        k.queue = c->queue + 3;
        k.err = c->errw;
        k.spin = cfg.spin_limit;
        k.num_sms = c->num_sms;
        {
            Prof p(c, c->side, "copy");
            if (cudaError_t e = launch_copy(k, c->side)) return e;
        }
        return cudaEventRecord(c->ev_copy, c->side);
    };
    if (nunits) {
        LaunchSketch k;
        k.units = d_units;
        k.nunits = nunits;
        k.bts = d_bts;
        k.nbt = (int)nbt;
        k.usum = static_cast<UnitSum *>(c->usum.p);
        k.cand = static_cast<Cand *>(c->cand.p);
        k.lists = static_cast<SRes *>(c->lists.p);
        k.recs = static_cast<FRec *>(c->recs.p);
        k.uout = static_cast<UnitOut *>(c->uout.p);
        k.match = static_cast<uint8_t *>(c->match.p);
        k.uwalk = static_cast<Walk *>(c->uwalk.p);
        k.utrue = static_cast<UnitTrue *>(c->utrue.p);
        k.umode = static_cast<uint32_t *>(c->umode.p);
        k.uexp = static_cast<int64_t *>(c->uexp.p);
        k.traces = c->traces;
        k.T = cfg.threshold;
        k.warmup = c->tune.ext_events ? c->tune.ext_events : 32768;
        k.queue = c->queue;
        k.err = c->errw;
        k.spin = cfg.spin_limit;
        k.stats = c->stats;
        k.num_sms = c->num_sms;
        k.order = reinterpret_cast<const uint32_t *>(dp + q.o_ord);
        k.nitems = nunits;
        // spread the units over all SMs: fewer warps per block when units are few
        k.warps_per_block = std::max(1, std::min(std::min((int)c->tune.warps_per_block, PHASE1_MAX_WARPS),
                                                 (nunits + c->num_sms - 1) / c->num_sms));
        int bps = 0;
        if (phase1_occupancy(k.warps_per_block, &bps) || bps < 1) bps = 1;
        k.blocks = std::max(1, std::min(bps * c->num_sms, (nunits + k.warps_per_block - 1) / k.warps_per_block));
        {
            // the traces' first units replayed exactly and the other units sketched, from one queue
            Prof p(c, s, "phase1");
            CK(launch_phase1(k, s), "launch phase 1");
        }
        CK(copy_pass(), "copy pass");
        {
            Prof p(c, s, "match");
            CK(launch_match(k, s), "launch match");
        }
        {
            Prof p(c, s, "chain");
            CK(launch_chain(k, s), "launch chain");
        }
        {
            Prof p(c, s, "totals");
            CK(launch_totals(k, s), "launch totals");
        }
    } else {
        CK(copy_pass(), "copy pass");
    }
    {
        Prof p(c, s, "scan");
        CK(launch_scan(a, s), "launch scan");
    }
    if (nunits) {
        LaunchFinal f;
        f.units = d_units;
        f.nunits = nunits;
        f.items = reinterpret_cast<const FItem *>(dp + q.o_fit);
        f.nitems = q.nitems;
        f.phit = static_cast<uint32_t *>(c->phit.p);
        f.piece = c->tune.piece_events ? c->tune.piece_events : FINAL_PIECE;
        f.utrue = a.utrue;
        f.uplan = a.uplan;
        f.lists = static_cast<const SRes *>(c->lists.p);
        f.recs = a.recs;
        f.uout = a.uout;
        f.T = cfg.threshold;
        f.queue = c->queue + 2;
        f.err = c->errw;
        f.spin = cfg.spin_limit;
        f.stats = c->stats;
        f.warps_per_block = std::max(1, std::min((int)c->tune.final_warps, (q.nitems + c->num_sms - 1) / c->num_sms));
        int bps = 0;
        // fewer warps per block if the requested block does not fit an SM
        while (f.warps_per_block > 1 && (final_occupancy(f.warps_per_block, &bps) || bps < 1)) --f.warps_per_block;
        if (final_occupancy(f.warps_per_block, &bps) || bps < 1) bps = 1;
        f.blocks = std::max(1, std::min(bps * c->num_sms, (q.nitems + f.warps_per_block - 1) / f.warps_per_block));
        Prof p(c, s, "final");
        CK(launch_final(f, s), "launch final");
    }

    {
        Prof p(c, s, "compact");
        CK(launch_compact(a, s), "launch compact");
    }
    {
        Prof p(c, s, "mark");
        CK(launch_mark(a, s), "launch mark");
    }
    {
        Prof p(c, s, "epi");
        CK(launch_epi(a, s), "launch epi");
    }
    if (q.nctiles) CK(cudaStreamWaitEvent(s, c->ev_copy, 0), "join the copy pass");
    {
        Prof p(c, s, "state");
        CK(launch_state(a, s), "launch state");
    }
    CK(cudaEventRecord(c->ev_out, s), "join event");
    CK(cudaStreamWaitEvent(s_user, c->ev_out, 0), "join the replay");
    return SCL_OK;
}

namespace {

// Stream capture records kernels without the priority of the stream they were launched on:
// give every kernel node the high priority of the replay stream, as plain launches have.
int graph_priorities(scl_ctx *c, cudaGraph_t g) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priority range");
    (void)least;
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn), "graph nodes");
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn), "graph nodes");
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nd, &t), "graph node type");
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeAttrValue v{};
        v.priority = greatest;
        CK(cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v), "kernel node priority");
    }
    return SCL_OK;
}

}  // namespace

// ============================================================================ C ABI

uint32_t scl_ctx_max_traces(const scl_ctx *c) { return c->cfg.max_traces; }
int scl_ctx_device(const scl_ctx *c) { return c->device; }
int scl_ctx_fail(scl_ctx *c, int code, const char *msg) { return fail(c, code, "%s", msg); }
void scl_ctx_forget_stream(scl_ctx *c) { c->last_stream = nullptr; }

extern "C" {

int scl_config_default(scl_config *cfg) {
    if (!cfg) return SCL_EINVAL;
    memset(cfg, 0, sizeof *cfg);
    cfg->threshold = 10485767;
    cfg->copy_multiple = 2;
    cfg->n_lines = 256;
    cfg->copy_phase = 0;
    cfg->initial_footprint = 0;
    cfg->max_traces = 1;
    cfg->leak_rule = 0;
    cfg->spin_limit = 0;
    cfg->sample_log_capacity = 0;
    cfg->sample_budget_shift = SCL_BUDGET_AUTO;
    cfg->unit_events = 0;
    return SCL_OK;
}

const char *scl_last_error(const scl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void scl_replay_free(scl_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &p : c->prof_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (DevBuf *b : {&c->plan, &c->usum, &c->cand, &c->lists, &c->match, &c->uwalk, &c->utrue, &c->umode, &c->uexp, &c->uplan,
                      &c->uout, &c->pref, &c->recs, &c->btres, &c->ctsum, &c->stage, &c->rate, &c->report, &c->tline, &c->phit, &c->qrows})
        if (b->p) cudaFree(b->p);
    cudaFree(c->traces);
    cudaFree(c->lines);
    cudaFree(c->copies);
    if (c->log) cudaFree(c->log);
    cudaFree(c->errw);
    cudaFree(c->scores);
    cudaFree(c->queue);
    cudaFree(c->stats);
    if (c->h_plan) cudaFreeHost(c->h_plan);
    if (c->plan_done) cudaEventDestroy(c->plan_done);
    if (c->hi) cudaStreamDestroy(c->hi);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_copy) cudaEventDestroy(c->ev_copy);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    for (int i = 0; i < scl_ctx::NCS; ++i)
        if (c->cstream[i]) cudaStreamDestroy(c->cstream[i]);
    for (int i = 0; i <= scl_ctx::NCS; ++i)
        if (c->cev[i]) cudaEventDestroy(c->cev[i]);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->g_plan) cudaFreeHost(c->g_plan);
    if (c->g_done) cudaEventDestroy(c->g_done);
    delete c;
}

int scl_replay_init(scl_ctx **out, const scl_config *cfg_in) {
    if (!out || !cfg_in) return SCL_EINVAL;
    *out = nullptr;
    scl_ctx *c = new scl_ctx();
    c->cfg = *cfg_in;
    scl_config &cfg = c->cfg;
    if (cfg.threshold < 1 || cfg.copy_multiple < 1 || cfg.n_lines == 0 || cfg.max_traces == 0 ||
        cfg.leak_rule > 1 || (cfg.sample_budget_shift > 20 && cfg.sample_budget_shift != SCL_BUDGET_AUTO) ||
        (cfg.unit_events % UNIT_ALIGN) != 0) {
        int r = fail(c, SCL_EINVAL, "invalid config (threshold >= 1, copy_multiple >= 1, n_lines >= 1, "
                                    "max_traces >= 1, leak_rule in {0,1}, unit_events multiple of 1024)");
        scl_replay_free(c);
        return r;
    }
    const unsigned __int128 tc = (unsigned __int128)cfg.copy_multiple * (unsigned __int128)cfg.threshold;
    if (tc > (unsigned __int128)INT64_MAX || cfg.copy_phase >= (uint64_t)tc) {
        int r = fail(c, SCL_EINVAL, "copy threshold out of range or copy_phase >= T_c");
        scl_replay_free(c);
        return r;
    }
    if (cfg.spin_limit == 0) cfg.spin_limit = 1ull << 26;
    if (cfg.sample_budget_shift == SCL_BUDGET_AUTO) {
        // a sample needs |A - F| >= T, so the smaller T, the denser the samples can be
        int lg = 0;
        while (lg < 62 && (int64_t(1) << (lg + 1)) <= cfg.threshold) ++lg;
        c->shift = (uint32_t)std::min(4, std::max(0, lg - 16));
    } else {
        c->shift = cfg.sample_budget_shift;
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    const size_t L = cfg.n_lines, NTr = cfg.max_traces;
    if (e == cudaSuccess) e = cudaMalloc(&c->traces, sizeof(DevTrace) * NTr);
    if (e == cudaSuccess) e = cudaMalloc(&c->lines, sizeof(LineRow) * L * NTr);
    if (e == cudaSuccess) e = cudaMalloc(&c->copies, sizeof(unsigned long long) * 2 * L * NTr);
    if (e == cudaSuccess && cfg.sample_log_capacity)
        e = cudaMalloc(&c->log, sizeof(Sample) * cfg.sample_log_capacity * NTr);
    if (e == cudaSuccess) e = cudaMalloc(&c->errw, sizeof(ErrWord));
    if (e == cudaSuccess) e = cudaMalloc(&c->scores, sizeof(scl_leak_score) * L);
    if (e == cudaSuccess) e = cudaMalloc(&c->queue, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->stats, sizeof(unsigned long long) * NSTATS);
    if (e == cudaSuccess) e = cudaMemset(c->stats, 0, sizeof(unsigned long long) * NSTATS);
    if (e == cudaSuccess) e = cudaMemset(c->errw, 0, sizeof(ErrWord));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->plan_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->g_done, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->hi, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, greatest);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < scl_ctx::NCS && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&c->cstream[i], cudaStreamNonBlocking);
    for (int i = 0; i <= scl_ctx::NCS && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&c->cev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int r = cuda_fail(c, e, "context allocation");
        fprintf(stderr, "scl_replay_init: %s\n", c->err.c_str());
        scl_replay_free(c);
        return r;
    }
    if (e == cudaSuccess)
        e = launch_reset(c->traces, c->lines, c->copies, 0, cfg.max_traces, cfg.n_lines, cfg.initial_footprint, cfg.copy_phase,
                         nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int r = cuda_fail(c, e, "context initialisation");
        scl_replay_free(c);
        return r;
    }
    c->h_events.assign(NTr, 0);
    c->tune.unit_events = cfg.unit_events;   // 0: sized per batch
    c->tune.warps_per_block = PHASE1_MAX_WARPS;
    c->tune.ext_events = 0;
    c->tune.final_warps = 14;
    *out = c;
    return SCL_OK;
}

int scl_tuning_get(const scl_ctx *c, scl_tuning *out) {
    if (!c || !out) return SCL_EINVAL;
    *out = c->tune;
    return SCL_OK;
}

int scl_tuning_set(scl_ctx *c, const scl_tuning *t) {
    if (!c || !t) return SCL_EINVAL;
    if (t->unit_events % UNIT_ALIGN || t->first_events % UNIT_ALIGN || t->warps_per_block < 1 ||
        t->warps_per_block > 16 || t->final_warps < 1 || t->final_warps > 14 || (t->ext_events % 256) ||
        t->fixup > 1 || (t->piece_events % 256))
        return fail(c, SCL_EINVAL, "tuning: unit_events and first_events multiples of 1024 (0: default), "
                                   "warps_per_block 1..16, final_warps 1..14, ext_events and piece_events "
                                   "multiples of %d, fixup 0/1",
                    256);
    c->tune = *t;
    return SCL_OK;
}

int scl_replay_batch(scl_ctx *c, const scl_segment *segs, uint32_t nsegs, void *stream) {
    if (!c) return SCL_EINVAL;
    if (nsegs && !segs) return fail(c, SCL_EINVAL, "segs is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const scl_config &cfg = c->cfg;
    CK(cudaSetDevice(c->device), "cudaSetDevice");

    // ---- validate and group by trace (array order kept within a trace)
    std::vector<int> first_seen(cfg.max_traces, -1);
    std::vector<std::vector<uint32_t>> groups;
    std::vector<uint32_t> gtrace;
    for (uint32_t i = 0; i < nsegs; ++i) {
        const scl_segment &g = segs[i];
        if (g.trace_id >= cfg.max_traces)
            return fail(c, SCL_EINVAL, "segment %u: trace_id %u >= max_traces %u", i, g.trace_id, cfg.max_traces);
        if (g.ev.n && (!g.ev.delta || !g.ev.addr || !g.ev.line || !g.ev.is_python))
            return fail(c, SCL_EINVAL, "segment %u: NULL event array", i);
        if (g.ev.n >= UNIT_ALIGN && !(aligned16(g.ev.delta) && aligned16(g.ev.addr) && aligned16(g.ev.line) &&
                                      aligned16(g.ev.is_python)))
            return fail(c, SCL_EINVAL, "segment %u: event arrays must be 16-byte aligned", i);
        if (g.ev.n >= (1ull << 40)) return fail(c, SCL_EINVAL, "segment %u: too many events", i);
        if (g.cp.n && (!g.cp.size || !g.cp.line || !g.cp.is_python))
            return fail(c, SCL_EINVAL, "segment %u: NULL memcpy array", i);
        int &fs = first_seen[g.trace_id];
        if (fs < 0) {
            fs = (int)groups.size();
            groups.emplace_back();
            gtrace.push_back(g.trace_id);
        }
        groups[fs].push_back(i);
    }
    const uint32_t nbt = (uint32_t)groups.size();
    if (nbt == 0) return SCL_OK;

    // longest trace first: its units enter the walker queue first
    std::vector<uint64_t> tev(nbt, 0);
    for (uint32_t b = 0; b < nbt; ++b)
        for (uint32_t i : groups[b]) tev[b] += segs[i].ev.n;
    std::vector<uint32_t> order(nbt);
    for (uint32_t b = 0; b < nbt; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return tev[x] > tev[y]; });

    // ---- plan
    // events per unit: as tuned, or (0) one unit per resident final-replay warp
    uint64_t UE = c->tune.unit_events;
    if (UE == 0) {
        uint64_t total = 0;
        for (uint32_t i = 0; i < nsegs; ++i) total += segs[i].ev.n;
        const uint64_t warps = (uint64_t)c->num_sms * c->tune.final_warps;
        UE = (total + warps - 1) / warps;
        UE = (UE + UNIT_ALIGN - 1) / UNIT_ALIGN * UNIT_ALIGN;
        UE = std::max<uint64_t>(UE, 32768);
        UE = std::min<uint64_t>(UE, 1ull << 22);
    }
    const uint32_t shift = c->shift;
    std::vector<Unit> units;
    std::vector<BTrace> bts(nbt);
    std::vector<CompactGroup> cgroups;
    std::vector<CopyTile> ctiles;
    uint64_t rec_total = 0, lst_total = 0;
    for (uint32_t bi = 0; bi < nbt; ++bi) {
        const uint32_t b = order[bi];
        BTrace &B = bts[bi];
        memset(&B, 0, sizeof B);
        B.trace = gtrace[b];
        B.u0 = (uint32_t)units.size();
        B.c0 = (uint32_t)ctiles.size();
        uint64_t gidx = c->h_events[B.trace];
        // The trace's first unit is replayed exactly by one warp (k_phase1) beside the sketch
        // of the others.  With fewer traces than SMs those warps run nearly alone, so when
        // more units follow the first one is kept to one warm-up's length and its warp is
        // done well before the sketch; with many traces the first units keep full length
        // (one exact pass instead of a sketch pass and an exact one).
        const uint64_t W = c->tune.ext_events ? c->tune.ext_events : 32768;
        const uint64_t first_len = nbt < (uint32_t)c->num_sms && tev[b] > UE
                                       ? std::min<uint64_t>(UE, std::max<uint64_t>(32768, (W + UNIT_ALIGN - 1) / UNIT_ALIGN * UNIT_ALIGN))
                                       : (c->tune.first_events ? c->tune.first_events : UE);
        for (uint32_t i : groups[b]) {
            const scl_segment &g = segs[i];
            for (uint64_t off = 0, len; off < g.ev.n; off += len) {
                len = std::min<uint64_t>(units.size() == B.u0 ? first_len : UE, g.ev.n - off);
                Unit U;
                memset(&U, 0, sizeof U);
                U.len = len;
                U.delta = g.ev.delta + off;
                U.py = g.ev.is_python + off;
                U.addr = g.ev.addr + off;
                U.line = g.ev.line + off;
                U.gidx0 = gidx;
                U.rec0 = rec_total;
                U.rec_cap = (uint32_t)std::min<uint64_t>((U.len >> shift) + 64, 0xffffffffu);
                U.trace = B.trace;
                U.bt = bi;
                // reset lists: one reset per 32 events covers the thresholds worth listing;
                // a run with more resets leaves its unit to the crossing search
                U.lst0 = lst_total;
                // (a first unit is replayed exactly in phase 1 and needs none)
                U.lst_cap = c->tune.fixup || units.size() == B.u0 ? 0u : (uint32_t)((U.len >> 5) + 64);
                units.push_back(U);
                gidx += U.len;
                rec_total += U.rec_cap;
                lst_total += (uint64_t)NL * U.lst_cap;
            }
            for (uint64_t off = 0; off < g.cp.n; off += COPY_PASS_TILE) {
                CopyTile T{};
                T.len = (uint32_t)std::min<uint64_t>(COPY_PASS_TILE, g.cp.n - off);
                T.size = g.cp.size + off;
                T.line = g.cp.line + off;
                T.py = g.cp.is_python + off;
                T.bt = bi;
                T.t = (uint32_t)ctiles.size();
                T.trace = B.trace;
                ctiles.push_back(T);
            }
            B.n_ev += g.ev.n;
            B.n_cp += g.cp.n;
        }
        B.nu = (uint32_t)units.size() - B.u0;
        B.nc = (uint32_t)ctiles.size() - B.c0;
        if (B.nu) {
            units[B.u0].first = 1;
            units[B.u0 + B.nu - 1].last = 1;
        }
        for (uint32_t k = 0; k < B.nu; k += 8) cgroups.push_back({B.u0 + k, std::min<uint32_t>(8, B.nu - k)});
    }
    const int nunits = (int)units.size();
    const size_t nu1 = std::max<size_t>(1, units.size());

    // ---- phase-1 order: longest work first (a first unit's exact replay costs about twice
    // a sketched unit's events; a sketched unit also streams its warm-up)
    // ---- k_final's pieces: every unit but a trace's first, cut every piece_events (at the next
    // listed reset, found on the device)
    std::vector<FItem> fitems;
    const uint64_t piece = c->tune.piece_events ? c->tune.piece_events : FINAL_PIECE;
    for (uint32_t u = 0; u < (uint32_t)units.size(); ++u) {
        Unit &U = units[u];
        U.fi0 = (uint32_t)fitems.size();
        U.fnp = U.first ? 0u : (uint32_t)((U.len + piece - 1) / piece);
        for (uint32_t p = 0; p < U.fnp; ++p) fitems.push_back({u, p});
    }
    std::vector<uint32_t> p1order(units.size());
    {
        const uint64_t W = c->tune.ext_events ? c->tune.ext_events : 32768;
        std::vector<uint64_t> cost(units.size());
        for (size_t u = 0; u < units.size(); ++u)
            cost[u] = units[u].first ? 2 * units[u].len : units[u].len + std::min<uint64_t>(W, units[u - 1].len);
        for (size_t u = 0; u < units.size(); ++u) p1order[u] = (uint32_t)u;
        std::stable_sort(p1order.begin(), p1order.end(), [&](uint32_t x, uint32_t y) { return cost[x] > cost[y]; });
    }
    // ---- copy tiles in rounds over the traces (every trace's first tile, then every second
    // tile, ...): a trace's tiles stay in order for the look-back, a predecessor was taken
    // long before, and the warps at work spread their counter updates over many traces
    std::vector<CopyTile> corder;
    corder.reserve(ctiles.size());
    {
        uint32_t maxnc = 0;
        for (const BTrace &B : bts) maxnc = std::max(maxnc, B.nc);
        for (uint32_t r = 0; r < maxnc; ++r)
            for (const BTrace &B : bts)
                if (r < B.nc) {
                    CopyTile T = ctiles[B.c0 + r];
                    T.c0 = B.c0;
                    T.last = B.c0 + B.nc - 1;
                    corder.push_back(T);
                }
    }
    // ---- plan blob: units | bts | groups | copy tiles (in their order) | phase-1 order
    const size_t o_units = 0;
    const size_t o_bts = al256(o_units + sizeof(Unit) * units.size());
    const size_t o_grp = al256(o_bts + sizeof(BTrace) * bts.size());
    const size_t o_ct = al256(o_grp + sizeof(CompactGroup) * cgroups.size());
    const size_t o_ord = al256(o_ct + sizeof(CopyTile) * ctiles.size());
    const size_t o_fit = al256(o_ord + sizeof(uint32_t) * p1order.size());
    const size_t blob = al256(o_fit + sizeof(FItem) * fitems.size());
    if (c->plan_pending) {
        CK(cudaEventSynchronize(c->plan_done), "wait for previous plan upload");
        c->plan_pending = false;
    }
    if (blob > c->h_plan_cap) {
        if (c->h_plan) cudaFreeHost(c->h_plan);
        c->h_plan = nullptr;
        c->h_plan_cap = 0;
        CK(cudaMallocHost(&c->h_plan, blob * 2), "pinned plan buffer");
        c->h_plan_cap = blob * 2;
    }
    char *hp = static_cast<char *>(c->h_plan);
    memcpy(hp + o_units, units.data(), sizeof(Unit) * units.size());
    memcpy(hp + o_bts, bts.data(), sizeof(BTrace) * bts.size());
    memcpy(hp + o_grp, cgroups.data(), sizeof(CompactGroup) * cgroups.size());
    memcpy(hp + o_ct, corder.data(), sizeof(CopyTile) * corder.size());
    memcpy(hp + o_ord, p1order.data(), sizeof(uint32_t) * p1order.size());
    memcpy(hp + o_fit, fitems.data(), sizeof(FItem) * fitems.size());

    int r;
    if ((r = ensure(c, c->plan, blob, s, "plan buffer"))) return r;
    if ((r = ensure(c, c->usum, sizeof(UnitSum) * nu1, s, "unit sums"))) return r;
    if ((r = ensure(c, c->cand, sizeof(Cand) * K * nu1, s, "candidates"))) return r;
    if ((r = ensure(c, c->lists, sizeof(SRes) * std::max<uint64_t>(1, lst_total), s, "reset lists"))) return r;
    if ((r = ensure(c, c->match, sizeof(uint8_t) * K * nu1, s, "candidate matches"))) return r;
    if ((r = ensure(c, c->uwalk, sizeof(Walk) * nu1, s, "walks"))) return r;
    if ((r = ensure(c, c->utrue, sizeof(UnitTrue) * nu1, s, "true trajectories"))) return r;
    if ((r = ensure(c, c->umode, sizeof(uint32_t) * nu1, s, "unit modes"))) return r;
    if ((r = ensure(c, c->uexp, sizeof(int64_t) * nu1, s, "explicit counters"))) return r;
    if ((r = ensure(c, c->uplan, sizeof(UnitPlan) * nu1, s, "unit plans"))) return r;
    if ((r = ensure(c, c->uout, sizeof(UnitOut) * nu1, s, "unit outputs"))) return r;
    if ((r = ensure(c, c->pref, sizeof(int64_t) * 3 * nu1, s, "window prefixes"))) return r;
    if ((r = ensure(c, c->recs, sizeof(FRec) * std::max<uint64_t>(1, rec_total), s, "sample records"))) return r;
    if ((r = ensure(c, c->btres, sizeof(BTraceRes) * nbt, s, "batch trace results"))) return r;
    if ((r = ensure(c, c->ctsum, copy_status_bytes(std::max<size_t>(1, ctiles.size())), s, "copy tile states")))
        return r;
    if ((r = ensure(c, c->phit, sizeof(uint32_t) * std::max<size_t>(1, fitems.size()), s, "piece reports"))) return r;

    char *dp = static_cast<char *>(c->plan.p);
    c->last_units = units.size();
    {
        // events through the exact replay of first units and the sketch (other units, each with the
        // warm-up over the tail of the unit before it, from a tile boundary)
        const uint64_t W = c->tune.ext_events ? c->tune.ext_events : 32768;
        uint64_t fe = 0, se = 0;
        for (size_t u = 0; u < units.size(); ++u) {
            if (units[u].first) { fe += units[u].len; continue; }
            const uint64_t pl = units[u - 1].len;
            const uint64_t from = pl > W ? (pl - W) / SKETCH_TILE * SKETCH_TILE : 0;
            se += units[u].len + (pl - from);
        }
        c->last_first_events = fe;
        c->last_sketch_events = se;
    }
    c->last_stream = s;
    EnqArgs q{dp,     hp,    blob,  o_units, o_bts,  o_grp, o_ct, o_ord, o_fit, nbt, nunits, (int)cgroups.size(),
              (int)ctiles.size(), (int)fitems.size()};
    if (c->graph_on && !c->prof && s != nullptr) {
        // relaunch when the plan bytes, the buffers and the tuning equal the captured batch's:
        // the graph is then exactly this batch's work
        const std::vector<const void *> ptrs = {c->plan.p, c->usum.p, c->cand.p, c->lists.p, c->match.p,
                                                c->uwalk.p, c->utrue.p, c->umode.p, c->uexp.p, c->uplan.p,
                                                c->uout.p, c->pref.p, c->recs.p, c->btres.p, c->ctsum.p, c->phit.p};
        const bool same = c->gexec && c->g_blob == blob && c->g_ptrs == ptrs &&
                          memcmp(&c->g_tune, &c->tune, sizeof c->tune) == 0 && memcmp(c->g_plan, hp, blob) == 0;
        if (!same) {
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            if (c->g_pending) {   // an earlier launch may still be reading g_plan
                CK(cudaEventSynchronize(c->g_done), "wait for the previous graph");
                c->g_pending = false;
            }
            if (blob > c->g_plan_cap) {
                if (c->g_plan) cudaFreeHost(c->g_plan);
                c->g_plan = nullptr;
                c->g_plan_cap = 0;
                CK(cudaMallocHost(&c->g_plan, blob), "pinned graph plan");
                c->g_plan_cap = blob;
            }
            memcpy(c->g_plan, hp, blob);
            EnqArgs qg = q;
            qg.hp = static_cast<const char *>(c->g_plan);
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
            const int rq = enqueue_batch(c, s, qg, false);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(s, &g);
            if (rq) { if (g) cudaGraphDestroy(g); return rq; }
            CK(ec, "end capture");
            if (const int rp = graph_priorities(c, g)) { cudaGraphDestroy(g); return rp; }
            const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            CK(ei, "instantiate graph");
            c->g_blob = blob;
            c->g_ptrs = ptrs;
            c->g_tune = c->tune;
        }
        CK(cudaGraphLaunch(c->gexec, s), "graph launch");
        CK(cudaEventRecord(c->g_done, s), "graph event");
        c->g_pending = true;
    } else {
        const int rq = enqueue_batch(c, s, q, true);
        if (rq) return rq;
    }
    for (uint32_t bi = 0; bi < nbt; ++bi) c->h_events[bts[bi].trace] += bts[bi].n_ev;
    return SCL_OK;
}

int scl_replay_batch_host(scl_ctx *c, const scl_segment *segs, uint32_t nsegs, void *stream) {
    if (!c) return SCL_EINVAL;
    if (nsegs && !segs) return fail(c, SCL_EINVAL, "segs is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    size_t need = 0;
    for (uint32_t i = 0; i < nsegs; ++i) {
        const scl_segment &g = segs[i];
        need += al256(g.ev.n * 8) * 2 + al256(g.ev.n * 4) + al256(g.ev.n) + al256(g.cp.n * 8) + al256(g.cp.n * 4) +
                al256(g.cp.n);
    }
    int r = ensure(c, c->stage, std::max<size_t>(need, 256), s, "host staging buffer");
    if (r) return r;
    std::vector<scl_segment> dsegs(segs, segs + nsegs);
    char *p = static_cast<char *>(c->stage.p);
    DeviceViews views;
    // the copies start after the stream's earlier work (which may still read the staging
    // buffer); pieces of at most 64 MiB go round-robin over the copy streams
    CK(cudaEventRecord(c->cev[scl_ctx::NCS], s), "staging fork");
    for (int i = 0; i < scl_ctx::NCS; ++i) CK(cudaStreamWaitEvent(c->cstream[i], c->cev[scl_ctx::NCS], 0), "staging fork");
    int next_cs = 0;
    auto put = [&](const void *src, size_t bytes) -> const void * {
        char *dst = p;
        constexpr size_t PIECE = size_t(64) << 20;
        for (size_t o = 0; o < bytes; o += PIECE) {
            const size_t b = bytes - o < PIECE ? bytes - o : PIECE;
            if (cudaMemcpyAsync(dst + o, static_cast<const char *>(src) + o, b, cudaMemcpyHostToDevice,
                                c->cstream[next_cs]) != cudaSuccess)
                return nullptr;
            next_cs = (next_cs + 1) % scl_ctx::NCS;
        }
        p += al256(bytes);
        return dst;
    };
    for (uint32_t i = 0; i < nsegs; ++i) {
        const scl_segment &g = segs[i];
        scl_segment &d = dsegs[i];
        if (g.ev.n && (!g.ev.delta || !g.ev.addr || !g.ev.line || !g.ev.is_python))
            return fail(c, SCL_EINVAL, "segment %u: NULL event array", i);
        if (g.cp.n && (!g.cp.size || !g.cp.line || !g.cp.is_python))
            return fail(c, SCL_EINVAL, "segment %u: NULL memcpy array", i);
        d.ev.delta = static_cast<const int64_t *>(put(g.ev.delta, g.ev.n * 8));
        d.ev.addr = static_cast<const uint64_t *>(put(g.ev.addr, g.ev.n * 8));
        // event line ids are read only at the few events that sample (Section 3.3): a
        // device-accessible (pinned) host column is read in place instead of copied
        if (const void *lv = g.ev.n ? views.view(g.ev.line) : nullptr)
            d.ev.line = static_cast<const uint32_t *>(lv);
        else
            d.ev.line = static_cast<const uint32_t *>(put(g.ev.line, g.ev.n * 4));
        d.ev.is_python = static_cast<const uint8_t *>(put(g.ev.is_python, g.ev.n));
        d.cp.size = static_cast<const uint64_t *>(put(g.cp.size, g.cp.n * 8));
        d.cp.line = static_cast<const uint32_t *>(put(g.cp.line, g.cp.n * 4));
        d.cp.is_python = static_cast<const uint8_t *>(put(g.cp.is_python, g.cp.n));
        if (!d.ev.delta || !d.ev.addr || !d.ev.line || !d.ev.is_python || !d.cp.size || !d.cp.line || !d.cp.is_python)
            return fail(c, SCL_ECUDA, "host to device copy failed");
    }
    for (int i = 0; i < scl_ctx::NCS; ++i) {
        CK(cudaEventRecord(c->cev[i], c->cstream[i]), "staging join");
        CK(cudaStreamWaitEvent(s, c->cev[i], 0), "staging join");
    }
    return scl_replay_batch(c, dsegs.data(), nsegs, stream);
}

int scl_sync(scl_ctx *c) {
    if (!c) return SCL_EINVAL;
    return sync_and_check(c);
}

int scl_samples(scl_ctx *c, uint32_t trace, scl_sample *out, uint64_t cap, uint64_t *n_out) {
    if (!c || !n_out) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    int r = sync_and_check(c);
    if (r) return r;
    DevTrace t;
    CK(cudaMemcpy(&t, c->traces + trace, sizeof t, cudaMemcpyDeviceToHost), "read trace state");
    *n_out = t.n_samples;
    const uint64_t have = std::min<uint64_t>(t.n_samples, c->cfg.sample_log_capacity);
    if (cap < have) return fail(c, SCL_ERANGE, "output holds %llu samples, %llu needed", (unsigned long long)cap,
                                (unsigned long long)have);
    if (have) {
        static_assert(sizeof(Sample) == sizeof(scl_sample), "sample layout");
        CK(cudaMemcpy(out, c->log + (uint64_t)trace * c->cfg.sample_log_capacity, sizeof(Sample) * have,
                      cudaMemcpyDeviceToHost),
           "read samples");
    }
    if (t.n_samples > have)
        return fail(c, SCL_EOVERFLOW, "%llu samples taken, only the first %llu retained (sample_log_capacity)",
                    (unsigned long long)t.n_samples, (unsigned long long)have);
    return SCL_OK;
}

int scl_line_timeline(scl_ctx *c, uint32_t trace, uint32_t line, uint64_t *idx_out, int64_t *fp_out, uint64_t cap,
                      uint64_t *n_out) {
    if (!c || !n_out || (cap && (!idx_out || !fp_out))) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    if (line >= c->cfg.n_lines) return fail(c, SCL_EINVAL, "line %u out of range", line);
    int r = sync_and_check(c);
    if (r) return r;
    DevTrace t;
    CK(cudaMemcpy(&t, c->traces + trace, sizeof t, cudaMemcpyDeviceToHost), "read trace state");
    const uint64_t have = std::min<uint64_t>(t.n_samples, c->cfg.sample_log_capacity);
    const uint64_t nb = (have + 4095) / 4096;
    const uint64_t kcap = std::max<uint64_t>(cap, 1);
    if ((r = ensure(c, c->tline, sizeof(uint64_t) * (nb + 1 + 2 * kcap), c->last_stream, "timeline"))) return r;
    uint64_t *scratch = static_cast<uint64_t *>(c->tline.p);
    uint64_t *d_idx = scratch + nb + 1;
    int64_t *d_fp = reinterpret_cast<int64_t *>(d_idx + kcap);
    CK(launch_timeline(c->log + (uint64_t)trace * c->cfg.sample_log_capacity, have, line, scratch, cap, d_idx, d_fp,
                       c->last_stream),
       "launch timeline");
    uint64_t total = 0;
    CK(cudaMemcpyAsync(&total, scratch + nb, sizeof total, cudaMemcpyDeviceToHost, c->last_stream), "read count");
    CK(cudaStreamSynchronize(c->last_stream), "sync");
    *n_out = total;
    if (total > cap) return fail(c, SCL_ERANGE, "output holds %llu points, %llu needed", (unsigned long long)cap,
                                 (unsigned long long)total);
    if (total) {
        CK(cudaMemcpy(idx_out, d_idx, sizeof(uint64_t) * total, cudaMemcpyDeviceToHost), "read timeline");
        CK(cudaMemcpy(fp_out, d_fp, sizeof(int64_t) * total, cudaMemcpyDeviceToHost), "read timeline");
    }
    if (t.n_samples > have)
        return fail(c, SCL_EOVERFLOW, "only the first %llu samples are retained (sample_log_capacity)",
                    (unsigned long long)have);
    return SCL_OK;
}

int scl_line_stats(scl_ctx *c, uint32_t trace, scl_line_stat *out, uint32_t cap, uint32_t *n_out) {
    if (!c || !n_out) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    int r = sync_and_check(c);
    if (r) return r;
    const uint32_t L = c->cfg.n_lines;
    *n_out = L;
    if (cap < L) return fail(c, SCL_ERANGE, "output holds %u rows, %u needed", cap, L);
    std::vector<LineRow> rows(L);
    std::vector<unsigned long long> cps(2 * (size_t)L);
    CK(cudaMemcpy(rows.data(), c->lines + (uint64_t)trace * L, sizeof(LineRow) * L, cudaMemcpyDeviceToHost),
       "read line stats");
    CK(cudaMemcpy(cps.data(), c->copies + (uint64_t)trace * L * 2, sizeof(unsigned long long) * 2 * L,
                  cudaMemcpyDeviceToHost),
       "read copy samples");
    // copy bytes are samples * T_c (Section 3.5): formed here, not kept on the device
    const uint64_t Tc = (uint64_t)c->cfg.copy_multiple * (uint64_t)c->cfg.threshold;
    for (uint32_t l = 0; l < L; ++l) {
        scl_line_stat &o = out[l];
        const LineRow &x = rows[l];
        o.n_growth = x.n_growth; o.n_shrink = x.n_shrink;
        o.A = x.A; o.F = x.F; o.A_py = x.A_py; o.F_py = x.F_py;
        o.net = (int64_t)((uint64_t)x.A - (uint64_t)x.F);   // the sum of A - F over the samples
        o.copy_samples[0] = cps[2 * l]; o.copy_samples[1] = cps[2 * l + 1];
        o.copy_bytes[0] = cps[2 * l] * Tc; o.copy_bytes[1] = cps[2 * l + 1] * Tc;
    }
    return SCL_OK;
}

int scl_leak_scores(scl_ctx *c, uint32_t trace, scl_leak_score *out, uint32_t cap, uint32_t *n_out) {
    if (!c || !n_out) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    int r = sync_and_check(c);
    if (r) return r;
    const uint32_t L = c->cfg.n_lines;
    *n_out = L;
    if (cap < L) return fail(c, SCL_ERANGE, "output holds %u rows, %u needed", cap, L);
    CK(launch_scores(c->lines, trace, L, c->cfg.leak_rule, c->scores, c->last_stream), "launch scores");
    CK(cudaMemcpyAsync(out, c->scores, sizeof(scl_leak_score) * L, cudaMemcpyDeviceToHost, c->last_stream),
       "read scores");
    CK(cudaStreamSynchronize(c->last_stream), "sync");
    return SCL_OK;
}

// the range queries: rows formed on the device into one buffer, then one copy to the caller
static int range_rows(scl_ctx *c, uint32_t trace0, uint32_t ntr, void *out, uint64_t cap, uint64_t *n_out, bool stats) {
    if (!c || !n_out || (ntr && !out)) return SCL_EINVAL;
    if ((uint64_t)trace0 + ntr > c->cfg.max_traces)
        return fail(c, SCL_EINVAL, "traces %u .. %u out of range", trace0, trace0 + ntr);
    int r = sync_and_check(c);
    if (r) return r;
    const uint32_t L = c->cfg.n_lines;
    const uint64_t nrows = (uint64_t)ntr * L;
    *n_out = nrows;
    if (cap < nrows) return fail(c, SCL_ERANGE, "output holds %llu rows, %llu needed", (unsigned long long)cap,
                                 (unsigned long long)nrows);
    if (!nrows) return SCL_OK;
    const size_t row = stats ? sizeof(scl_line_stat) : sizeof(scl_leak_score);
    if ((r = ensure(c, c->qrows, row * nrows, c->last_stream, "query rows"))) return r;
    if (stats) {
        const uint64_t Tc = (uint64_t)c->cfg.copy_multiple * (uint64_t)c->cfg.threshold;
        CK(launch_stat_rows(c->lines, c->copies, trace0, nrows, L, Tc, c->qrows.p, c->num_sms, c->last_stream),
           "launch line rows");
    } else {
        CK(launch_score_rows(c->lines, trace0, nrows, L, c->cfg.leak_rule, c->qrows.p, c->num_sms, c->last_stream),
           "launch score rows");
    }
    CK(cudaMemcpyAsync(out, c->qrows.p, row * nrows, cudaMemcpyDeviceToHost, c->last_stream), "read rows");
    CK(cudaStreamSynchronize(c->last_stream), "sync");
    return SCL_OK;
}

int scl_line_stats_range(scl_ctx *c, uint32_t trace0, uint32_t ntr, scl_line_stat *out, uint64_t cap,
                         uint64_t *n_out) {
    return range_rows(c, trace0, ntr, out, cap, n_out, true);
}

int scl_leak_scores_range(scl_ctx *c, uint32_t trace0, uint32_t ntr, scl_leak_score *out, uint64_t cap,
                          uint64_t *n_out) {
    return range_rows(c, trace0, ntr, out, cap, n_out, false);
}

int scl_leak_report(scl_ctx *c, uint32_t trace, scl_leak_report_row *out, uint32_t cap, uint32_t *n_out) {
    if (!c || !n_out) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    int r = sync_and_check(c);
    if (r) return r;
    const uint32_t L = c->cfg.n_lines;
    *n_out = L;
    if (cap < L) return fail(c, SCL_ERANGE, "output holds %u rows, %u needed", cap, L);
    if ((r = ensure(c, c->report, sizeof(scl_leak_report_row) * L, c->last_stream, "leak report"))) return r;
    CK(launch_report(c->lines, c->traces, trace, L, c->cfg.leak_rule, c->cfg.initial_footprint, c->report.p,
                     c->last_stream),
       "launch report");
    CK(cudaMemcpyAsync(out, c->report.p, sizeof(scl_leak_report_row) * L, cudaMemcpyDeviceToHost, c->last_stream),
       "read report");
    CK(cudaStreamSynchronize(c->last_stream), "sync");
    return SCL_OK;
}

int scl_trace_state(scl_ctx *c, uint32_t trace, scl_trace_info *out) {
    if (!c || !out) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    int r = sync_and_check(c);
    if (r) return r;
    DevTrace t;
    CK(cudaMemcpy(&t, c->traces + trace, sizeof t, cudaMemcpyDeviceToHost), "read trace state");
    memset(out, 0, sizeof *out);
    out->n_events = t.n_events; out->n_copies = t.n_copies; out->n_samples = t.n_samples;
    out->c = t.c; out->A = t.A; out->F = t.F; out->A_py = t.A_py; out->F_py = t.F_py;
    out->footprint = t.footprint; out->hwm = t.hwm;
    out->tracked_addr = t.tracked_addr; out->tracked_idx = t.tracked_idx; out->tracked_line = t.tracked_line;
    out->tracked_valid = (uint8_t)t.tracked_valid; out->tracked_reclaimed = (uint8_t)t.tracked_reclaimed;
    out->copy_counter = t.copy_counter;
    return SCL_OK;
}

struct StateHeader {
    uint32_t magic, n_lines;
    int64_t threshold;
    uint32_t copy_multiple, leak_rule;
};

int scl_state_export(scl_ctx *c, uint32_t trace, void *buf, uint64_t cap, uint64_t *n_out) {
    if (!c || !n_out) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    const uint64_t L = c->cfg.n_lines;
    const uint64_t need = sizeof(StateHeader) + sizeof(DevTrace) + (sizeof(LineRow) + 16) * L;
    *n_out = need;
    if (!buf) return SCL_OK;
    if (cap < need) return fail(c, SCL_ERANGE, "state needs %llu bytes", (unsigned long long)need);
    int r = sync_and_check(c);
    if (r) return r;
    StateHeader h{STATE_MAGIC, c->cfg.n_lines, c->cfg.threshold, c->cfg.copy_multiple, c->cfg.leak_rule};
    char *p = static_cast<char *>(buf);
    memcpy(p, &h, sizeof h);
    CK(cudaMemcpy(p + sizeof h, c->traces + trace, sizeof(DevTrace), cudaMemcpyDeviceToHost), "export");
    CK(cudaMemcpy(p + sizeof h + sizeof(DevTrace), c->lines + (uint64_t)trace * L, sizeof(LineRow) * L,
                  cudaMemcpyDeviceToHost),
       "export");
    CK(cudaMemcpy(p + sizeof h + sizeof(DevTrace) + sizeof(LineRow) * L, c->copies + (uint64_t)trace * L * 2, 16 * L,
                  cudaMemcpyDeviceToHost),
       "export");
    return SCL_OK;
}

int scl_state_import(scl_ctx *c, uint32_t trace, const void *buf, uint64_t n) {
    if (!c || !buf) return SCL_EINVAL;
    if (trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    const uint64_t L = c->cfg.n_lines;
    const uint64_t need = sizeof(StateHeader) + sizeof(DevTrace) + (sizeof(LineRow) + 16) * L;
    StateHeader h;
    if (n < sizeof h) return fail(c, SCL_EINVAL, "state buffer too short");
    memcpy(&h, buf, sizeof h);
    if (h.magic != STATE_MAGIC || n != need || h.n_lines != c->cfg.n_lines || h.threshold != c->cfg.threshold ||
        h.copy_multiple != c->cfg.copy_multiple || h.leak_rule != c->cfg.leak_rule)
        return fail(c, SCL_EINVAL, "state was exported under another configuration");
    int r = sync_and_check(c);
    if (r) return r;
    const char *p = static_cast<const char *>(buf);
    DevTrace t;
    memcpy(&t, p + sizeof h, sizeof t);
    if (c->cfg.sample_log_capacity == 0) t.n_samples = t.n_samples;  // counts are kept; records are not
    CK(cudaMemcpy(c->traces + trace, &t, sizeof t, cudaMemcpyHostToDevice), "import");
    CK(cudaMemcpy(c->lines + (uint64_t)trace * L, p + sizeof h + sizeof t, sizeof(LineRow) * L,
                  cudaMemcpyHostToDevice),
       "import");
    CK(cudaMemcpy(c->copies + (uint64_t)trace * L * 2, p + sizeof h + sizeof t + sizeof(LineRow) * L, 16 * L,
                  cudaMemcpyHostToDevice),
       "import");
    c->h_events[trace] = t.n_events;
    return SCL_OK;
}

int scl_trace_reset(scl_ctx *c, uint32_t trace, void *stream) {
    if (!c) return SCL_EINVAL;
    const bool all = trace == SCL_ALL_TRACES;
    if (!all && trace >= c->cfg.max_traces) return fail(c, SCL_EINVAL, "trace %u out of range", trace);
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t t0 = all ? 0 : trace, nt = all ? c->cfg.max_traces : 1;
    {
        Prof p(c, s, "reset");
        CK(launch_reset(c->traces, c->lines, c->copies, t0, nt, c->cfg.n_lines, c->cfg.initial_footprint,
                        c->cfg.copy_phase, s),
           "launch reset");
    }
    for (uint32_t t = t0; t < t0 + nt; ++t) c->h_events[t] = 0;
    c->last_stream = s;
    return SCL_OK;
}

int scl_profile_enable(scl_ctx *c, int on) {
    if (!c) return SCL_EINVAL;
    c->prof = on != 0;
    return SCL_OK;
}

int scl_profile_reset(scl_ctx *c) {
    if (!c) return SCL_EINVAL;
    prof_collect(c);
    c->prof_acc.clear();
    return SCL_OK;
}

int scl_kernel_times(scl_ctx *c, const char **names, double *ms, uint64_t *launches, uint32_t cap,
                     uint32_t *n_out) {
    if (!c || !n_out) return SCL_EINVAL;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    prof_collect(c);
    *n_out = (uint32_t)c->prof_acc.size();
    if (cap < c->prof_acc.size()) return fail(c, SCL_ERANGE, "need %u entries", *n_out);
    for (size_t i = 0; i < c->prof_acc.size(); ++i) {
        if (names) names[i] = c->prof_acc[i].first;
        if (ms) ms[i] = c->prof_acc[i].second.first;
        if (launches) launches[i] = c->prof_acc[i].second.second;
    }
    return SCL_OK;
}

int scl_batch_stats(scl_ctx *c, scl_batch_info *out) {
    if (!c || !out) return SCL_EINVAL;
    int r = sync_and_check(c);
    if (r) return r;
    unsigned long long v[NSTATS];
    CK(cudaMemcpy(v, c->stats, sizeof v, cudaMemcpyDeviceToHost), "read batch stats");
    memset(out, 0, sizeof *out);
    out->units = c->last_units;
    out->walked = v[0];
    out->walked_merged = v[1];
    out->explicit_entries = v[2];
    out->transparent = v[3];
    out->unit_events = c->tune.unit_events;
    out->walked_events = v[4];
    out->searched = v[5];
    out->first_events = c->last_first_events;
    out->sketch_events = c->last_sketch_events;
    return SCL_OK;
}

int scl_rate_samples(scl_ctx *c, const int64_t *delta, const uint32_t *line, const uint8_t *is_python, uint64_t n,
                     const uint64_t *gap, uint64_t n_gaps, uint64_t consumed, uint64_t *counts_out,
                     uint64_t *state_out, void *stream) {
    if (!c) return SCL_EINVAL;
    if ((n && (!delta || !line || !is_python)) || (n_gaps && !gap) || !counts_out || !state_out)
        return fail(c, SCL_EINVAL, "rate samples: NULL array");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int r = ensure(c, c->rate, rate_scratch_bytes(n, n_gaps), s, "rate-sampling scratch");
    if (r) return r;
    CK(launch_rate(delta, line, is_python, n, gap, n_gaps, consumed, c->cfg.n_lines, counts_out, state_out, c->rate.p,
                   s),
       "launch rate sampling");
    c->last_stream = s;
    return SCL_OK;
}

int scl_cpu_attribution(scl_ctx *c, const int64_t *vtime, const uint32_t *line, uint64_t n, int64_t quantum,
                        int64_t t_prev, int64_t *python_out, int64_t *native_out, uint64_t *flags_out,
                        void *stream) {
    if (!c) return SCL_EINVAL;
    if ((n && (!vtime || !line)) || !python_out || !native_out || !flags_out || quantum < 0)
        return fail(c, SCL_EINVAL, "cpu attribution: NULL array or negative quantum");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_cpu_attr(vtime, line, n, quantum, t_prev, c->cfg.n_lines, python_out, native_out, flags_out,
                       c->num_sms, s),
       "launch cpu attribution");
    c->last_stream = s;
    return SCL_OK;
}

int scl_selftest_wait(scl_ctx *c, uint64_t limit, void *stream) {
    if (!c) return SCL_EINVAL;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(c->errw, 0, sizeof(ErrWord), s), "clear error word");
    CK(launch_wait_selftest(c->errw, limit, s), "launch wait self test");
    c->last_stream = s;
    const int r = sync_and_check(c);
    CK(cudaMemset(c->errw, 0, sizeof(ErrWord)), "clear error word");
    return r;
}

int scl_graph_enable(scl_ctx *c, int on) {
    if (!c) return SCL_EINVAL;
    c->graph_on = on != 0;
    if (!c->graph_on && c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SCL_OK;
}

int scl_autotune(scl_ctx *c, const scl_segment *segs, uint32_t nsegs, void *stream, scl_tuning *best_out,
                 double *best_ms_out) {
    if (!c) return SCL_EINVAL;
    if (nsegs == 0 || !segs) return fail(c, SCL_EINVAL, "autotune needs at least one segment");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    // save the resident state of every trace the segments touch; restore it after each trial
    // (traces with consecutive ids are copied as one range)
    std::vector<uint32_t> tr;
    for (uint32_t i = 0; i < nsegs; ++i)
        if (segs[i].trace_id < c->cfg.max_traces) tr.push_back(segs[i].trace_id);
    std::sort(tr.begin(), tr.end());
    tr.erase(std::unique(tr.begin(), tr.end()), tr.end());
    std::vector<std::pair<uint32_t, uint32_t>> ranges;   // (first trace, count)
    for (uint32_t t : tr) {
        if (!ranges.empty() && ranges.back().first + ranges.back().second == t) ++ranges.back().second;
        else ranges.push_back({t, 1});
    }
    const size_t L = c->cfg.n_lines;
    void *save = nullptr;
    const size_t nt = std::max<size_t>(1, tr.size());
    CK(cudaMalloc(&save, (sizeof(DevTrace) + (sizeof(LineRow) + 16) * L) * nt), "autotune state copy");
    DevTrace *save_t = static_cast<DevTrace *>(save);
    LineRow *save_l = reinterpret_cast<LineRow *>(save_t + nt);
    unsigned long long *save_c = reinterpret_cast<unsigned long long *>(save_l + nt * L);
    std::vector<uint64_t> h_ev(tr.size());
    auto copy_state = [&](bool to_save) -> cudaError_t {
        size_t k = 0;
        for (const auto &r : ranges) {
            DevTrace *t = c->traces + r.first;
            LineRow *l = c->lines + (size_t)r.first * L;
            const size_t bt = sizeof(DevTrace) * r.second, bl = sizeof(LineRow) * L * r.second;
            cudaError_t e = to_save ? cudaMemcpyAsync(save_t + k, t, bt, cudaMemcpyDeviceToDevice, s)
                                    : cudaMemcpyAsync(t, save_t + k, bt, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = to_save ? cudaMemcpyAsync(save_l + k * L, l, bl, cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpyAsync(l, save_l + k * L, bl, cudaMemcpyDeviceToDevice, s);
            unsigned long long *cc = c->copies + (size_t)r.first * L * 2;
            const size_t bc = 16 * L * r.second;
            if (e == cudaSuccess)
                e = to_save ? cudaMemcpyAsync(save_c + k * L * 2, cc, bc, cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpyAsync(cc, save_c + k * L * 2, bc, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            k += r.second;
        }
        for (size_t i = 0; i < tr.size(); ++i) {
            if (to_save) h_ev[i] = c->h_events[tr[i]];
            else c->h_events[tr[i]] = h_ev[i];
        }
        return cudaSuccess;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const scl_tuning keep = c->tune;
    const bool prof = c->prof, graph = c->graph_on;
    c->prof = false;
    c->graph_on = false;
    scl_tuning best = keep;
    double best_ms = 1e300;
    int rc = copy_state(true) == cudaSuccess ? SCL_OK : SCL_ECUDA;
    // one timed setting: a warm-up call, then three calls back to back (each plans on the host
    // while the previous one runs, as repeated calls do), from the saved state; the figure is
    // the mean of the three.  The state is restored again at the end.
    std::vector<std::pair<scl_tuning, double>> seen;
    auto measure = [&](const scl_tuning &t) -> double {
        for (const auto &p : seen)
            if (memcmp(&p.first, &t, sizeof t) == 0) return p.second;
        c->tune = t;
        if (copy_state(false) != cudaSuccess) rc = SCL_ECUDA;
        if (!rc) rc = scl_replay_batch(c, segs, nsegs, stream);
        if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = SCL_ECUDA;
        if (!rc) rc = check_device_error(c);
        constexpr int REPS = 3;
        if (!rc) cudaEventRecord(e0, s);
        for (int rep = 0; rep < REPS && !rc; ++rep) rc = scl_replay_batch(c, segs, nsegs, stream);
        if (!rc) {
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = SCL_ECUDA;
        }
        if (!rc) rc = check_device_error(c);
        if (rc) return 1e300;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / REPS;
        seen.push_back({t, per});
        if (per < best_ms) { best_ms = per; best = t; }
        return per;
    };
    // coordinate descent, two passes: each setting in turn takes its best value with the
    // others held at the best found so far
    const uint32_t units[] = {32768, 65536, 131072, 262144, 524288, 1048576, 2097152};
    const uint32_t firsts[] = {0, 524288, 786432, 1048576, 1310720, 1572864};
    const uint32_t pwarps[] = {8, 12, (uint32_t)PHASE1_MAX_WARPS};
    const uint32_t fwarps[] = {10, 12, 14};
    const uint32_t warm[] = {16384, 32768};
    const uint32_t fixups[] = {0, 1};
    const uint32_t pieces[] = {32768, 65536, 131072, 1u << 22};   // (the last: no unit is cut)
    scl_tuning start = keep;
    if (start.ext_events == 0) start.ext_events = 32768;
    measure(start);
    for (int pass = 0; pass < 2 && !rc; ++pass) {
        for (uint32_t v : units) { scl_tuning t = best; t.unit_events = v; if (!rc) measure(t); }
        for (uint32_t v : firsts) { scl_tuning t = best; t.first_events = v; if (!rc) measure(t); }
        for (uint32_t v : pwarps) { scl_tuning t = best; t.warps_per_block = v; if (!rc) measure(t); }
        for (uint32_t v : fwarps) { scl_tuning t = best; t.final_warps = v; if (!rc) measure(t); }
        for (uint32_t v : warm) { scl_tuning t = best; t.ext_events = v; if (!rc) measure(t); }
        for (uint32_t v : fixups) { scl_tuning t = best; t.fixup = v; if (!rc) measure(t); }
        for (uint32_t v : pieces) { scl_tuning t = best; t.piece_events = v; if (!rc) measure(t); }
    }
    if (copy_state(false) != cudaSuccess && !rc) rc = SCL_ECUDA;
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save);
    c->prof = prof;
    c->graph_on = graph;
    c->tune = rc ? keep : best;
    if (rc) return rc == SCL_ECUDA ? fail(c, rc, "autotune: a CUDA call failed") : rc;
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    return SCL_OK;
}

}  // extern "C"
