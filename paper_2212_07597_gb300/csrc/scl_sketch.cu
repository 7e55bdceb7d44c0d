// scl_sketch.cu -- the true entry counter of every unit of the threshold sampler
// (Section 3.2: c <- c + delta; if |c| >= T: sample, c <- 0), found in parallel.
//
// The counter's future depends only on its current value: two runs with equal
// counters at one event take the same resets from there on.  Runs collapse onto
// each other when one event pushes both over the threshold, which happens quickly
// for runs whose counters are close and slowly otherwise.
//
// k_phase1  one persistent kernel; each warp takes units from one queue, longest work first:
//           - the first unit of a trace in the batch, whose entry is the trace's resident
//             state, is replayed exactly once (k_final skips it) and recorded as every
//             candidate of the unit;
//           - any other unit is sketched: the 32 lanes start 32 counters spread over
//             (-T, T) a warm-up stretch before the unit (at the end of the previous unit of
//             the trace) and run them to the unit's start, where they have collapsed into a
//             few distinct values that any run through the warm-up has almost surely
//             joined.  Equal counters are merged (followers copy their leader), and the
//             distinct ones are run through the unit, recording the counter at the start
//             and end, the resets, the last reset and the first largest prefix at a growth
//             reset.  All lanes advance together, 256 events per step.
//           Sharing one queue lets the latency-bound counters and the bandwidth-bound exact
//           replays run side by side on every SM.
// k_match   for each unit and each candidate k of the previous unit: the candidate of
//           this unit whose start counter equals k's end counter, if any.
// k_chain   one block per trace: follows the true candidate from unit to unit through
//           the match table in shared memory; where no candidate carries the true
//           counter the block walks the unit itself (helper warps summarise the steps
//           ahead of the warp that runs the counter).
#include <algorithm>
#include <cstddef>

#include "scl_exact.cuh"
#include "scl_launch.h"

namespace scl {

__device__ __forceinline__ int64_t candidate_entry(int k, int64_t T) {
    // K values evenly spread over [-(T-1), T-1]
    const __int128 span = (__int128)(2 * (T - 1));
    return -(T - 1) + (int64_t)(span * k / (K - 1));
}

// Advance this lane's counter c (if `active`) over one step.  Active lanes with equal
// counters form a group led by its lowest lane (`grp`: this lane's leader); one crossing
// search runs per group, and at each of its resets on_reset(leader_k, pos, growth, Qr) is
// called on all lanes (warp-uniform), for every member of group k to record.
// SP / I: the 64-bit step (StepPrefix, int64_t) or its 32-bit form (StepPrefix32, int32_t).
template <class SP, class I, class F>
__device__ __forceinline__ void advance(const SP &sp, const I *xq, I qmax, I qmin, int lane, I T, bool active, int grp,
                                        I &c, F &&on_reset) {
    unsigned m = __ballot_sync(FULL, active && grp == lane && (c + qmax >= T || c + qmin <= -T));
    I cnew = c + sp.tot;
    while (m) {
        const int k = __ffs(m) - 1;
        m &= m - 1;
        I b = __shfl_sync(FULL, c, k);
        int after = -1;
        while (true) {
            I Qr;
            const int r = first_cross(sp, xq, lane, b, T, after, Qr);
            if (r < 0) break;
            on_reset(k, r, b + Qr > 0, (int64_t)Qr);
            b = -Qr;
            after = r;
            // from c = 0 after the reset, the rest of the step can only cross if its
            // prefix moves T away from Q_r
            if (qmax - Qr < T && qmin - Qr > -T) break;
        }
        if (active && grp == k) cnew = b + sp.tot;
    }
    c = cnew;
}

// One step of every lane's counter: the 32-bit form when T and the step's deltas allow it
// (t32: T <= 2^30), else the 64-bit one.  Returns the step total and prefix extremes.
template <class F>
__device__ __forceinline__ void sketch_step(const StepIn<8> &in, int64_t *xq, int lane, int64_t T, bool t32,
                                            bool active, int grp, int64_t &c, int64_t &tot, int64_t &qmax,
                                            int64_t &qmin, F &&on_reset) {
    if (t32 && __all_sync(FULL, step_fits32(in))) {
        StepPrefix32<8> sp;
        int32_t *xq32 = reinterpret_cast<int32_t *>(xq);
        step_prefix32(in, lane, sp, xq32);
        const int32_t mx = __reduce_max_sync(FULL, sp.lmax), mn = __reduce_min_sync(FULL, sp.lmin);
        int32_t c32 = (int32_t)c;
        advance(sp, (const int32_t *)xq32, mx, mn, lane, (int32_t)T, active, grp, c32, on_reset);
        c = c32;
        tot = sp.tot;
        qmax = mx;
        qmin = mn;
    } else {
        StepPrefix<8> sp;
        step_prefix(in, lane, sp, xq);
        qmax = warp_max(sp.lmax);
        qmin = warp_min(sp.lmin);
        advance(sp, (const int64_t *)xq, qmax, qmin, lane, T, active, grp, c, on_reset);
        tot = sp.tot;
    }
}

// Lanes holding the same counter.  With T <= 2^30 every counter lies in (-2^30, 2^30), so
// its low word identifies it and the 32-bit match serves.
__device__ __forceinline__ unsigned match_counter(int64_t c, bool t32) {
    return t32 ? __match_any_sync(FULL, (unsigned)c) : __match_any_sync(FULL, (unsigned long long)c);
}

// ---------------------------------------------------------------- phase 1: sketch and first units
constexpr int SE = 8;                         // events per lane per sketch step (256 per step)
using SketchRing = Ring<false, 2, 512, SE>;   // two steps per tile: the other tile is in flight
using FirstRing = Ring<true, 2, 256, 8>;
static_assert(SketchRing::kTL == SKETCH_TILE, "the host counts warm-up events in these tiles");

// A warp's shared memory holds one ring at a time: the sketch's (deltas only) or the exact
// replay's (deltas, addresses, flags).  Switching invalidates the old ring's barriers first.
union alignas(128) Phase1Smem {
    SketchRing s;
    FirstRing f;
};
constexpr size_t PHASE1_WARP_SMEM = sizeof(Phase1Smem);
static_assert(PHASE1_WARP_SMEM % 128 == 0, "per-warp slices laid end to end stay aligned");
static_assert(PHASE1_WARP_SMEM * PHASE1_MAX_WARPS <= 227 * 1024, "a block's rings fit one SM's shared memory");

// Candidate counters of unit u (not a trace's first unit): 32 counters spread over (-T, T)
// run through a warm-up over the tail of the previous unit of the trace, collapse, and the
// distinct ones run through the unit recording what k_match / k_chain / k_final need.
// Returns false if a wait timed out.
__device__ bool sketch_unit(SketchRing &sm, uint32_t &phase, int u, const Unit *__restrict__ units, UnitSum *usum,
                            Cand *cand, SRes *lists, int64_t T, uint32_t warmup, ErrWord *err,
                            unsigned long long spin, int lane) {
    const bool t32 = T <= FIT32_T;
    const Unit U = units[u];
    bool ok = true;
    int64_t c;
    {
        // warm-up over the tail of the previous unit of the trace; candidates whose
        // counters become equal run on as one (the lowest lane leads)
        c = candidate_entry(lane, T);
        int lead = lane;
        const Unit Up = units[u - 1];
        const uint64_t from = Up.len > warmup ? ((Up.len - warmup) / SketchRing::kTL) * SketchRing::kTL : 0;
        auto wstep = [&](const StepIn<SE> &in, uint32_t) -> bool {
            const bool act = lead == lane;
            int64_t tot, qmax, qmin;
            sketch_step(in, sm.xq, lane, T, t32, act, lane, c, tot, qmax, qmin, [](int, int, bool, int64_t) {});
            const unsigned same = match_counter(c, t32) & __ballot_sync(FULL, act);
            if (act) lead = __ffs(same) - 1;
            return false;
        };
        ok = ring_walk<false>(sm, Up, from, Up.len, phase, spin, err, lane, wstep);
        // followers take their leader's counter (leaders may have joined others later)
#pragma unroll
        for (int r = 0; r < 5; ++r) lead = __shfl_sync(FULL, lead, lead);
        c = __shfl_sync(FULL, c, lead);
    }
    const int64_t c0 = c;
    const unsigned same = match_counter(c, t32);
    const int leader = __ffs(same) - 1;
    const bool active = leader == lane;
    // the first NL distinct runs record every reset (for the exact replay)
    const uint32_t rank = (uint32_t)__popc(__ballot_sync(FULL, active) & ((1u << lane) - 1u));
    const uint32_t myslot = active && rank < (uint32_t)NL && U.lst_cap ? rank : NO_LIST;
    SRes *L = myslot != NO_LIST ? lists + U.lst0 + (uint64_t)myslot * U.lst_cap : nullptr;
    Cand *C = cand + (size_t)u * K + lane;
    uint32_t n = 0;
    int32_t last = -1;
    int64_t gmax = INT64_MIN, tmax = INT64_MIN;
    uint32_t garg = 0, targ = 0;
    int64_t P = 0, umax = INT64_MIN, umin = INT64_MAX;
    // the distinct runs regroup as they meet: runs whose counters become equal (after both
    // reset at one event) take the same resets from there on, so one search serves the group
    // and each member records them in its own lane
    int grp = lane;
    auto step = [&](const StepIn<SE> &in, uint32_t rel0) -> bool {
        int64_t tot, qmax, qmin;
        bool reset = false;
        sketch_step(in, sm.xq, lane, T, t32, active, grp, c, tot, qmax, qmin, [&](int k, int r, bool growth, int64_t Qr) {
            reset = true;
            if (active && grp == k) {
                const uint32_t pos = rel0 + (uint32_t)r;
                const int64_t Pl = P + Qr;
                if (growth && Pl > gmax) { gmax = Pl; garg = pos; }
                if (n < (uint32_t)RM) {
                    C->pos[n] = pos;
                    C->gp[n] = growth ? Pl : INT64_MIN;
                } else if (growth && Pl > tmax) {
                    tmax = Pl;
                    targ = pos;
                }
                if (L && n < U.lst_cap) {
                    SRes q;
                    q.pos = pos;
                    q.pad = 0;
                    q.P = Pl;
                    L[n] = q;
                }
                ++n;
                last = (int32_t)pos;
            }
        });
        if (reset) {
            const unsigned g = match_counter(c, t32) & __ballot_sync(FULL, active);
            if (active) grp = __ffs(g) - 1;
        }
        // the unit's prefix extremes (for the transparency test of k_chain)
        umax = P + qmax > umax ? P + qmax : umax;
        umin = P + qmin < umin ? P + qmin : umin;
        P += tot;
        return false;
    };
    if (ok) ok = ring_walk<false>(sm, U, 0, U.len, phase, spin, err, lane, step);
    __syncwarp();
    // followers take their leader's run
    if (active) {
        for (uint32_t r = n; r < (uint32_t)RM; ++r) { C->pos[r] = 0xffffffffu; C->gp[r] = INT64_MIN; }
    }
    __syncwarp();
    if (!active) {
        const Cand *Lc = cand + (size_t)u * K + leader;
        for (int r = 0; r < RM; ++r) { C->pos[r] = Lc->pos[r]; C->gp[r] = Lc->gp[r]; }
    }
    C->c0 = c0;
    C->c = __shfl_sync(FULL, c, leader);
    C->last = __shfl_sync(FULL, last, leader);
    C->n = __shfl_sync(FULL, n, leader);
    C->gmax = __shfl_sync(FULL, gmax, leader);
    C->garg = __shfl_sync(FULL, garg, leader);
    C->tmax = __shfl_sync(FULL, tmax, leader);
    C->targ = __shfl_sync(FULL, targ, leader);
    {
        const uint32_t ls = __shfl_sync(FULL, myslot, leader);
        const uint32_t nl = __shfl_sync(FULL, n, leader);
        C->list = ls != NO_LIST && nl <= U.lst_cap ? ls : NO_LIST;
        C->pad = 0;
    }
    if (lane == 0) {
        UnitSum S;   // window totals are filled by k_totals, for the units that need them
        S.total = P; S.totA = 0; S.totApy = 0; S.totSpy = 0; S.minQ = umin; S.maxQ = umax;
        usum[u] = S;
    }
    return ok;
}

// The first unit u of a trace in the batch: its entry is the trace's resident state, so it
// is replayed exactly once (k_final skips it) and the run is recorded as every candidate.
// Returns false if a wait timed out.
template <bool DENSE>
__device__ bool first_unit(FirstRing &fr, uint32_t &phase, int u, const Unit *__restrict__ units, UnitSum *usum,
                           Cand *cand, FRec *recs, UnitOut *uout, const DevTrace *traces, int64_t T, ErrWord *err,
                           unsigned long long spin, int lane) {
    const Unit U = units[u];
    const DevTrace st = traces[U.trace];
    ExactIn in0;
    in0.c = st.c;
    in0.wA = lane == 0 ? st.A : 0;
    in0.wApy = lane == 0 ? st.A_py : 0;
    in0.wSpy = lane == 0 ? st.A_py - st.F_py : 0;
    in0.mark = st.hwm;
    in0.fpb = st.footprint;
    in0.tk = st.tracked_valid ? 2u : 0u;   // as k_scan plans a trace's first unit
    in0.taddr = st.tracked_addr;
    in0.tslot = 0;
    in0.list = nullptr;
    in0.nres = 0;
    in0.exit_c = 0;
    in0.from = 0;
    in0.limit = (uint32_t)U.len;
    in0.n0 = 0;
    in0.rend = 0;
    in0.P0 = 0;
    in0.stop = false;
    ExactRun R;
    R.C0 = cand + (size_t)u * K;
    UnitOut O;
    uint32_t n = 0;
    uint32_t prior;   // (a whole unit: no earlier piece)
    const bool ok = exact_unit<true, DENSE>(fr, phase, U, in0, recs + U.rec0, U.rec_cap, T, spin, err, lane, n, O, &R,
                                     prior);
    if (!ok) return false;   // a wait timed out (the ring may not be reusable)
    Cand *C = cand + (size_t)u * K + lane;
    if (lane == 0)
        for (uint32_t r = n; r < (uint32_t)RM; ++r) { C->pos[r] = 0xffffffffu; C->gp[r] = INT64_MIN; }
    __syncwarp();
    if (lane != 0) {
        const Cand *C0 = R.C0;
        for (int r = 0; r < RM; ++r) { C->pos[r] = C0->pos[r]; C->gp[r] = C0->gp[r]; }
    }
    C->c0 = st.c; C->c = O.c; C->last = R.last; C->n = n;
    C->gmax = R.gmax; C->garg = R.garg; C->tmax = R.tmax; C->targ = R.targ;
    C->list = NO_LIST; C->pad = 0;
    if (lane == 0) {
        UnitSum S;   // window totals are filled by k_totals, for the units that need them
        // (a first unit's prefix extremes are never needed: its entry is exact)
        S.total = R.P; S.totA = 0; S.totApy = 0; S.totSpy = 0; S.minQ = INT64_MIN; S.maxQ = INT64_MAX;
        usum[u] = S;
        uout[u] = O;
        if (n > U.rec_cap) set_error(err, E_OVERFLOW, 3, (unsigned long long)u);
    }
    return true;
}

// Phase 1, one persistent kernel: every warp takes units from one queue (`order`, longest
// work first), replaying a trace's first unit exactly and sketching every other unit, so the
// latency-bound candidate counters and the exact replays share the SMs and a long first unit
// starts early.
template <bool DENSE>
__global__ void __launch_bounds__(32 * PHASE1_MAX_WARPS, 1) k_phase1(const LaunchSketch a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Phase1Smem &sm = *reinterpret_cast<Phase1Smem *>(smem_raw + (size_t)warp * PHASE1_WARP_SMEM);
    int cur = -1;   // ring in use: 0 sketch, 1 exact
    uint32_t phase = 0;
    while (true) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.queue, 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it >= a.nitems) break;
        const int u = (int)a.order[it];
        const int want = a.units[u].first ? 1 : 0;
        if (want != cur) {
            if (cur == 0) ring_release(sm.s, lane);
            if (cur == 1) ring_release(sm.f, lane);
            if (want == 0) ring_init(sm.s, lane); else ring_init(sm.f, lane);
            cur = want;
            phase = 0;
        }
        const bool ok = want ? first_unit<DENSE>(sm.f, phase, u, a.units, a.usum, a.cand, a.recs, a.uout, a.traces, a.T,
                                          a.err, a.spin, lane)
                             : sketch_unit(sm.s, phase, u, a.units, a.usum, a.cand, a.lists, a.T, a.warmup, a.err,
                                           a.spin, lane);
        if (!ok) break;   // a wait timed out: leave (the ring may not be reusable)
    }
}

// ---------------------------------------------------------------- k_match
__global__ void k_match(const Unit *__restrict__ units, int nunits, const Cand *__restrict__ cand, uint8_t *match) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int u = t / K, k = t % K;
    if (u >= nunits) return;
    uint8_t j_found = NO_MATCH;
    if (!units[u].first) {
        const int64_t c = cand[(size_t)(u - 1) * K + k].c;
        for (int j = 0; j < K; ++j)
            if (cand[(size_t)u * K + j].c0 == c) { j_found = (uint8_t)j; break; }
    }
    match[(size_t)u * K + k] = j_found;
}

// ---------------------------------------------------------------- k_chain
constexpr int CHAIN_CHUNK = 1024;   // units per shared-memory chunk of the match table
constexpr int CW = 8;               // warps per chain block: warp 0 runs the counter, the rest help
constexpr int WE = 16;              // events per lane per walk step
constexpr int WSTEP = 32 * WE;      // events per walk step
constexpr int NSLOT = 8;            // walk steps summarised ahead of the counter
constexpr int LCAP = 2048;          // reset-list positions staged in shared memory per list

constexpr uint32_t MODE_TRANSPARENT = 0x100u;   // explicit counter entering, no reset in the unit
constexpr uint32_t MODE_WALKED = 0x200u;        // explicit counter entering, walked here (uwalk)

// one walk step, summarised by a helper warp: the step's prefix sums at every event,
// each lane's extremes over its WE prefixes, the step total and the step extremes
struct alignas(16) WalkSlot {   // xq takes 16-byte stores
    alignas(16) int64_t xq[32 * WE];
    int64_t lmax[32], lmin[32];
    int64_t tot, qmax, qmin;
    volatile int32_t ready;   // index of the step held (-1: none)
    int32_t pad;
};

struct ChainSmem {
    alignas(16) uint8_t m[CHAIN_CHUNK][K];   // 16-byte row loads
    uint16_t mode[CHAIN_CHUNK];
    uint8_t endk[CW][K];         // per warp segment: the candidate leaving it, per entering one
    uint32_t segk[CW];           // the true candidate entering each segment
    uint32_t brk, kout;          // first row the matched run leaves the table; candidate then
    WalkSlot slot[NSLOT];
    uint32_t lpos[NL][LCAP];     // the unit's reset lists (positions), for the merge test
    Walk wres;                   // the walk's result, for every warp
    volatile int32_t consumed;   // walk steps the counter has finished
    volatile int32_t stop;       // the counter is done (or a wait gave up)
};

static_assert(offsetof(ChainSmem, slot) % 16 == 0 && sizeof(WalkSlot) % 16 == 0 &&
                  offsetof(WalkSlot, xq) % 16 == 0,
              "walk slots take 16-byte stores");
static_assert(offsetof(ChainSmem, m) % 16 == 0, "match rows take 16-byte copies");
static_assert(sizeof(ChainSmem) <= 227 * 1024, "the chain block's shared memory fits one SM");

// Walk unit U from counter c until one of its resets is also a reset of a candidate of the
// unit -- from there the run is that candidate's -- or to the unit's end.  The whole block
// takes part: warps 1.. load the unit's steps and write their prefix summaries to the slot
// ring; warp 0 runs the counter over the summaries, locating crossings in the stored
// prefixes.  Lane j of warp 0 holds candidate j's first RM resets; lane s < NL also follows
// reset list s (every reset of a candidate run, in order).  Every wait is bounded.
__device__ Walk walk_coop(ChainSmem &sm, const Unit &U, const Cand *cu, const SRes *lists, int64_t c, int64_t T,
                          int warp, int lane, unsigned long long spin, ErrWord *err) {
    const uint32_t nsteps = (uint32_t)((U.len + WSTEP - 1) / WSTEP);
    if (threadIdx.x == 0) { sm.consumed = 0; sm.stop = 0; }
    if (threadIdx.x < NSLOT) sm.slot[threadIdx.x].ready = -1;
    // list q: its owner (a candidate carrying it) and its positions, staged once
    const uint32_t mylist = cu[lane].list;
    int owner = -1;
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        const unsigned o = __ballot_sync(FULL, mylist == (uint32_t)q);
        const int oq = o ? __ffs(o) - 1 : -1;
        if (lane == q) owner = oq;
        if (oq >= 0) {
            const uint32_t nq = cu[oq].n < (uint32_t)LCAP ? cu[oq].n : (uint32_t)LCAP;
            const SRes *Lq = lists + U.lst0 + (uint64_t)q * U.lst_cap;
            for (uint32_t i = threadIdx.x; i < nq; i += 32 * CW) sm.lpos[q][i] = Lq[i].pos;
        }
    }
    __syncthreads();
    if (warp != 0) {
        // ---- helpers: steps warp-1, warp-1 + (CW-1), ...; the next step's deltas load
        // while the current one is summarised
        const bool vec = (reinterpret_cast<uintptr_t>(U.delta) & 15u) == 0;
        auto load = [&](uint32_t s, int64_t (&d)[WE]) {
            const uint64_t e0 = (uint64_t)s * WSTEP + (uint64_t)lane * WE;
            if (vec && e0 + WE <= U.len) {
                const longlong2 *src = reinterpret_cast<const longlong2 *>(U.delta + e0);
#pragma unroll
                for (int q = 0; q < WE / 2; ++q) { const longlong2 v = src[q]; d[2 * q] = v.x; d[2 * q + 1] = v.y; }
            } else {
#pragma unroll
                for (int q = 0; q < WE; ++q) d[q] = e0 + q < U.len ? U.delta[e0 + q] : 0;
            }
        };
        int64_t cur[WE], nxt[WE];
        uint32_t s = (uint32_t)(warp - 1);
        if (s < nsteps) load(s, cur);
        for (; s < nsteps; s += CW - 1) {
            if (s + (CW - 1) < nsteps) load(s + (CW - 1), nxt);
            // the slot is free once the counter has finished step s - NSLOT
            bool go = true;
            for (unsigned long long it = 0;; ++it) {
                if (sm.stop) { go = false; break; }
                if ((int32_t)s < sm.consumed + NSLOT) break;
                if (it > spin) {
                    if (lane == 0) set_error(err, E_TIMEOUT, 13, (unsigned long long)s);
                    go = false;
                    break;
                }
            }
            if (!__all_sync(FULL, go)) break;
            __threadfence_block();
            WalkSlot &sl = sm.slot[s % NSLOT];
            StepIn<WE> in;
#pragma unroll
            for (int q = 0; q < WE; ++q) { in.d[q] = cur[q]; in.a[q] = 0; }
            in.pw[0] = in.pw[1] = 0;
            StepPrefix<WE> sp;
            step_prefix(in, lane, sp, sl.xq);
            sl.lmax[lane] = sp.lmax;
            sl.lmin[lane] = sp.lmin;
            const int64_t qmax = warp_max(sp.lmax), qmin = warp_min(sp.lmin);
            if (lane == 0) { sl.tot = sp.tot; sl.qmax = qmax; sl.qmin = qmin; }
            __syncwarp();
            __threadfence_block();
            if (lane == 0) sl.ready = (int32_t)s;
#pragma unroll
            for (int q = 0; q < WE; ++q) cur[q] = nxt[q];
        }
    } else {
        // ---- the counter
        Walk W;
        W.last = -1; W.n = 0; W.gmax = INT64_MIN; W.garg = 0; W.into = -1;
        W.walked = (uint32_t)U.len;
        uint32_t mypos[RM];
#pragma unroll
        for (int r = 0; r < RM; ++r) mypos[r] = cu[lane].pos[r];
        // the first-RM test is needed only for candidate runs that have no reset list
        const bool rm_needed = __any_sync(FULL, mylist == NO_LIST);
        const SRes *Ls = lists + U.lst0 + (uint64_t)(lane < NL ? lane : 0) * U.lst_cap;
        const uint32_t lcount = owner >= 0 ? cu[owner].n : 0;
        const uint32_t *lsm = sm.lpos[lane < NL ? lane : 0];
        uint32_t lp = 0;
        uint32_t lnext = lcount ? lsm[0] : 0xffffffffu;
        int64_t P = 0;
        int mj = -1;
        uint32_t mi = 0;
        for (uint32_t s = 0; s < nsteps && mj < 0; ++s) {
            WalkSlot &sl = sm.slot[s % NSLOT];
            bool got = false;
            for (unsigned long long it = 0; it <= spin; ++it)
                if (sl.ready == (int32_t)s) { got = true; break; }
            if (!__all_sync(FULL, got)) {
                if (lane == 0) set_error(err, E_TIMEOUT, 14, (unsigned long long)s);
                break;
            }
            __threadfence_block();
            const int64_t tot = sl.tot;
            const uint32_t rel0 = s * WSTEP;
            if (c + sl.qmax >= T || c + sl.qmin <= -T) {
                StepPrefix<WE> sp;
                sp.lmax = sl.lmax[lane];
                sp.lmin = sl.lmin[lane];
                int64_t b = c;
                int after = -1;
                while (true) {
                    int64_t Qr;
                    const int r = first_cross(sp, sl.xq, lane, b, T, after, Qr);
                    if (r < 0) break;
                    const uint32_t pos = rel0 + (uint32_t)r;
                    const int64_t Pl = P + Qr;
                    if (b + Qr > 0 && Pl > W.gmax) { W.gmax = Pl; W.garg = pos; }
                    ++W.n;
                    W.last = (int32_t)pos;
                    int hit = -1;
                    if (rm_needed) {
#pragma unroll
                        for (int q = 0; q < RM; ++q)
                            if (mypos[q] == pos) hit = q;
                    }
                    const unsigned m = __ballot_sync(FULL, hit >= 0);
                    if (m) {
                        mj = __ffs(m) - 1;
                        mi = (uint32_t)__shfl_sync(FULL, hit, mj);
                        W.walked = pos + 1;
                        break;
                    }
                    bool leq = false;
                    if (lane < NL && lcount) {
                        while (lnext < pos)
                            lnext = ++lp < lcount ? (lp < (uint32_t)LCAP ? lsm[lp] : Ls[lp].pos) : 0xffffffffu;
                        leq = lnext == pos;
                    }
                    const unsigned m2 = __ballot_sync(FULL, leq);
                    if (m2) {
                        const int slx = __ffs(m2) - 1;
                        mj = __shfl_sync(FULL, owner, slx);
                        mi = __shfl_sync(FULL, lp, slx);
                        W.walked = pos + 1;
                        break;
                    }
                    b = -Qr;
                    after = r;
                }
                c = b + tot;
            } else {
                c += tot;
            }
            P += tot;
            __syncwarp();
            if (lane == 0) { __threadfence_block(); sm.consumed = (int32_t)(s + 1); }
        }
        if (lane == 0) sm.stop = 1;
        if (mj >= 0) {
            // the rest of the unit follows candidate mj from its reset mi on
            const Cand &Cj = cu[mj];
            W.n += Cj.n - (mi + 1);
            int64_t sg = INT64_MIN;
            uint32_t sa = 0;
            if (mi + 1 < (uint32_t)RM || Cj.list == NO_LIST) {
                sg = Cj.tmax;
                sa = Cj.targ;
                for (int q = RM - 1; q > (int)mi; --q)
                    if (Cj.gp[q] != INT64_MIN && Cj.gp[q] >= sg) { sg = Cj.gp[q]; sa = Cj.pos[q]; }
            } else {
                // the largest prefix at a growth reset after mi, from the list: the counter at
                // reset r > 0 is P_r - P_(r-1)
                const SRes *Lj = lists + U.lst0 + (uint64_t)Cj.list * U.lst_cap;
                for (uint32_t r = mi + 1 + lane; r < Cj.n; r += 32) {
                    const SRes q = Lj[r];
                    if (q.P - Lj[r - 1].P > 0 && (q.P > sg || (q.P == sg && q.pos < sa))) { sg = q.P; sa = q.pos; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int64_t og = __shfl_xor_sync(FULL, sg, o);
                    const uint32_t oa = __shfl_xor_sync(FULL, sa, o);
                    if (og > sg || (og == sg && og != INT64_MIN && oa < sa)) { sg = og; sa = oa; }
                }
            }
            if (sg != INT64_MIN && sg > W.gmax) { W.gmax = sg; W.garg = sa; }
            W.last = Cj.last;
            W.c = Cj.c;
            W.into = mj;
        } else {
            W.c = c;
        }
        if (lane == 0) sm.wres = W;
    }
    __syncthreads();
    return sm.wres;
}

// entering mode per unit: j < K: the true run is candidate j of the unit;
// MODE_TRANSPARENT / MODE_WALKED: an explicit counter (uexp) entered.
// One block per trace; every warp follows the same chain (so all take part in walks),
// warp 0 writes the results.
__global__ void __launch_bounds__(32 * CW) k_chain(const Unit *__restrict__ units, const BTrace *__restrict__ bts,
                                                  int nbt, const UnitSum *__restrict__ usum,
                                                  const Cand *__restrict__ cand, const SRes *__restrict__ lists,
                                                  const uint8_t *__restrict__ match, Walk *uwalk, UnitTrue *utrue,
                                                  uint32_t *umode, int64_t *uexp, int64_t T, ErrWord *err,
                                                  unsigned long long spin, unsigned long long *stats) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ChainSmem &sm = *reinterpret_cast<ChainSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    if (b >= nbt) return;
    const BTrace B = bts[b];
    if (B.nu == 0) return;
    const bool lead = threadIdx.x == 0;
    if (lead) umode[B.u0] = 0;   // the first unit was replayed from the exact counter
    uint32_t k = 0;              // the true run leaves the previous unit on candidate k...
    bool expl = false;           // ...or as the explicit counter ec
    int64_t ec = 0;
    for (uint32_t c0 = 1; c0 < B.nu; c0 += CHAIN_CHUNK) {
        const uint32_t cn = B.nu - c0 < (uint32_t)CHAIN_CHUNK ? B.nu - c0 : (uint32_t)CHAIN_CHUNK;
        uint32_t i = 0;
        while (i < cn) {
            if (!expl) {
                // ---- the matched run from row i on, resolved in parallel: each warp composes
                // the match table over its segment of rows for all 32 entering candidates at
                // once (in place: row r becomes "candidate at r" per entering candidate), then
                // thread 0 chains the segments.
                __syncthreads();
                {   // rows i .. cn of K bytes, contiguous in global memory: 16-byte loads
                    const uint4 *src = reinterpret_cast<const uint4 *>(match + (size_t)(B.u0 + c0 + i) * K);
                    uint4 *dst = reinterpret_cast<uint4 *>(&sm.m[i][0]);
                    const uint32_t nv = (cn - i) * K / 16;
                    for (uint32_t v = threadIdx.x; v < nv; v += 32 * CW) dst[v] = src[v];
                }
                __syncthreads();
                const uint32_t per = (cn - i + CW - 1) / CW;
                {
                    const uint32_t a = i + warp * per, b = a + per < cn ? a + per : cn;
                    uint32_t kk = (uint32_t)lane;
                    for (uint32_t r = a; r < b; ++r) {
                        const uint32_t nx = kk < (uint32_t)K ? sm.m[r][kk] : NO_MATCH;
                        __syncwarp();
                        sm.m[r][lane] = (uint8_t)nx;
                        __syncwarp();
                        kk = nx;
                    }
                    sm.endk[warp][lane] = (uint8_t)kk;
                }
                __syncthreads();
                if (lead) {
                    uint32_t kc = k, bseg = CW;
                    for (int w = 0; w < CW; ++w) {
                        sm.segk[w] = kc;
                        if (i + w * per >= cn) continue;
                        const uint32_t e = sm.endk[w][kc];
                        if (e == NO_MATCH) { bseg = (uint32_t)w; break; }
                        kc = e;
                    }
                    sm.kout = kc;
                    sm.brk = bseg;   // segment of the break (CW: none)
                }
                __syncthreads();
                const uint32_t bseg = sm.brk;
                uint32_t brk = cn;
                if (bseg < (uint32_t)CW) {   // the first row of that segment leaving the table
                    const uint32_t a = i + bseg * per, b = a + per < cn ? a + per : cn;
                    const uint32_t ks = sm.segk[bseg];
                    for (uint32_t r0 = a; r0 < b; r0 += 32) {
                        const unsigned hm = __ballot_sync(FULL, r0 + lane < b && sm.m[r0 + lane][ks] == NO_MATCH);
                        if (hm) { brk = r0 + __ffs(hm) - 1; break; }
                    }
                }
                for (uint32_t r = i + threadIdx.x; r < brk; r += 32 * CW)
                    sm.mode[r] = sm.m[r][sm.segk[(r - i) / per]];
                if (brk == cn) {
                    k = sm.kout;
                    i = cn;
                    break;
                }
                // the run's candidate at row brk-1 matches nothing at row brk
                {
                    const uint32_t sg = (brk - i) / per, ks = sm.segk[sg];
                    k = brk == i + sg * per ? ks : sm.m[brk - 1][ks];
                }
                i = brk;
                ec = cand[(size_t)(B.u0 + c0 + i - 1) * K + k].c;
                expl = true;
            }
            // ---- explicit counter at row i: does a candidate of this unit start with it?
            const uint32_t u = B.u0 + c0 + i;
            const bool eq = cand[(size_t)u * K + lane].c0 == ec;
            const unsigned mm = __ballot_sync(FULL, eq);
            if (lead) uexp[u] = ec;
            if (mm) {
                k = __ffs(mm) - 1;
                expl = false;
                if (lead) sm.mode[i] = (uint16_t)k;
                ++i;
                continue;
            }
            const UnitSum S = usum[u];
            if (lead) atomicAdd(&stats[2], 1ull);
            if (ec + S.maxQ < T && ec + S.minQ > -T) {
                if (lead) { sm.mode[i] = (uint16_t)MODE_TRANSPARENT; atomicAdd(&stats[3], 1ull); }
                ec += S.total;
                ++i;
                continue;
            }
            const Walk W = walk_coop(sm, units[u], cand + (size_t)u * K, lists, ec, T, warp, lane, spin, err);
            if (lead) {
                uwalk[u] = W;
                sm.mode[i] = (uint16_t)MODE_WALKED;
                atomicAdd(&stats[0], 1ull);
                if (W.into >= 0) atomicAdd(&stats[1], 1ull);
                atomicAdd(&stats[4], (unsigned long long)W.walked);
            }
            ec = W.c;
            if (W.into >= 0) { k = (uint32_t)W.into; expl = false; }
            ++i;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cn; i += 32 * CW) umode[B.u0 + c0 + i] = sm.mode[i];
    }
}

// ---------------------------------------------------------------- k_totals
// One warp per unit.  First the unit's true run from its entering mode (k_chain):
// a candidate's, an explicit counter that takes no sample, or k_chain's walk.  Then,
// for a unit whose true run takes no sample, the sum of mallocs, python mallocs and
// python deltas over it: such units lie inside one open window, whose totals k_scan
// assembles from them.  Units that do sample are never needed whole and keep zeros.
__global__ void k_totals(const Unit *__restrict__ units, int nunits, const Cand *__restrict__ cand,
                         const uint32_t *__restrict__ umode, const Walk *__restrict__ uwalk,
                         const int64_t *__restrict__ uexp, UnitTrue *utrue, UnitSum *usum) {
    const int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= nunits) return;
    const Unit U = units[u];
    const uint32_t md = umode[u];
    UnitTrue Tu;
    Tu.entry_last = -1;
    Tu.list = NO_LIST;
    Tu.pad = 0;
    if (md < (uint32_t)K) {
        const Cand &C = cand[(size_t)u * K + md];
        Tu.entry_c = C.c0; Tu.n = C.n; Tu.gmax = C.gmax; Tu.garg = C.garg; Tu.exit_c = C.c;
        Tu.list = C.list;
        Tu.exit_last = C.last >= 0 ? (int64_t)(U.gidx0 + (uint32_t)C.last) : -1;
    } else if (md == MODE_TRANSPARENT) {
        Tu.entry_c = uexp[u]; Tu.n = 0; Tu.gmax = INT64_MIN; Tu.garg = 0;
        Tu.exit_c = uexp[u] + usum[u].total; Tu.exit_last = -1;
    } else {
        const Walk &W = uwalk[u];
        Tu.entry_c = uexp[u]; Tu.n = W.n; Tu.gmax = W.gmax; Tu.garg = W.garg; Tu.exit_c = W.c;
        Tu.exit_last = W.last >= 0 ? (int64_t)(U.gidx0 + (uint32_t)W.last) : -1;
    }
    if (lane == 0) utrue[u] = Tu;
    if (Tu.n != 0) return;
    int64_t a = 0, ap = 0, sp = 0;
    for (uint64_t e = lane; e < U.len; e += 32) {
        const int64_t x = U.delta[e];
        const int64_t ps = x > 0 ? x : 0;
        a += ps;
        if (U.py[e]) { ap += ps; sp += x; }
    }
    a = warp_sum(a);
    ap = warp_sum(ap);
    sp = warp_sum(sp);
    if (lane == 0) { usum[u].totA = a; usum[u].totApy = ap; usum[u].totSpy = sp; }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_totals(const LaunchSketch &a, cudaStream_t s) {
    k_totals<<<(a.nunits + 7) / 8, 256, 0, s>>>(a.units, a.nunits, a.cand, a.umode, a.uwalk, a.uexp, a.utrue, a.usum);
    return cudaGetLastError();
}

cudaError_t launch_phase1(const LaunchSketch &a, cudaStream_t s) {
    if (!a.nitems) return cudaSuccess;
    const size_t smem = PHASE1_WARP_SMEM * a.warps_per_block;
    // the instance with the exact replay's dense-step test only where dense steps can be common
    auto kern = a.T <= DENSE_T_MAX ? k_phase1<true> : k_phase1<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.blocks, 32 * a.warps_per_block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_match(const LaunchSketch &a, cudaStream_t s) {
    const int threads = a.nunits * K;
    k_match<<<(threads + 255) / 256, 256, 0, s>>>(a.units, a.nunits, a.cand, a.match);
    return cudaGetLastError();
}

cudaError_t launch_chain(const LaunchSketch &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    const size_t smem = sizeof(ChainSmem);
    cudaError_t e = cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<<<a.nbt, 32 * CW, smem, s>>>(a.units, a.bts, a.nbt, a.usum, a.cand, a.lists, a.match, a.uwalk, a.utrue,
                                         a.umode, a.uexp, a.T, a.err, a.spin, a.stats);
    return cudaGetLastError();
}

int phase1_occupancy(int warps_per_block, int *blocks_per_sm) {
    const size_t smem = PHASE1_WARP_SMEM * warps_per_block;
    // (both instances have the same register cap and shared memory)
    cudaError_t e = cudaFuncSetAttribute(k_phase1<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_phase1<false>, 32 * warps_per_block, smem);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace scl
