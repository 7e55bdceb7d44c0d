// scl_exact.cuh -- the exact replay of one unit from a known entering state (one warp).
//
// Per event (Sections 3.2-3.4): c <- c + delta and the open window's totals A, F,
// A_py, F_py grow; a free compares its address with the tracked block; when
// |c| >= T a sample closes the window (kind, totals, footprint, line and flag of
// the triggering event), and a growth sample whose footprint beats the high-water
// mark sets a new mark and starts tracking the sampled block.
//
// 256 events per step.  delta, the python flag and the address are staged through the
// copy ring; the line id of a sample is left to k_compact (which reads it for every
// record in parallel, instead of this warp waiting on one load per sample).  When
// the unit's resets are known in advance (a reset list from the sketch) no crossing
// search runs; otherwise each step's prefix sums locate the crossings.
//
// Used by k_final for every unit whose entry k_chain resolved, and by k_phase1 for the
// first unit of each trace in a batch, whose entry is the trace's resident state; that
// caller also wants the facts the sketch records for a candidate run (FIRST = true).
#pragma once
#include <type_traits>

#include "scl_stage.cuh"

namespace scl {

struct ExactIn {                 // the state entering the unit (or the piece of it replayed)
    int64_t c;                   // counter
    int64_t wA, wApy, wSpy;      // this lane's share of the open-window totals so far
    int64_t mark;                // high-water mark
    int64_t fpb;                 // footprint before the unit
    uint32_t tk;                 // tracked block: 0 none, 1/2 entering (see UnitPlan), 3 a sample of the unit
    uint32_t tslot;              // tk = 3: the record of that sample
    uint64_t taddr;
    const SRes *list;            // the unit's resets in order, or nullptr: search
    uint32_t nres;               // resets listed
    int64_t exit_c;              // counter after the unit (with a list)
    // the span replayed: events [from, limit) are staged; with a list, entries [n0, rend) are
    // the resets it closes, and with `stop` it ends at the last of them.  A whole unit has
    // from = 0, limit = len, n0 = 0, rend = nres, stop = false.
    uint32_t from, limit;
    uint32_t n0, rend;
    int64_t P0;                  // unit-local prefix sum before `from`
    bool stop;
};

struct ExactRun {                // FIRST only: the run's facts, as the sketch records them for a candidate
    Cand *C0;                    // lane 0 writes the first RM reset positions and growth
                                 // prefixes here (the unit's candidate 0)
    int64_t gmax, tmax;          // largest prefix at a growth reset (all / index >= RM)
    uint32_t garg, targ;
    int32_t last;                // last reset position (-1: none)
    int64_t P;                   // unit total
};

// Replays unit U (or one piece of it); writes its records to out[n0 .. cap) and returns false
// if a wait timed out.  n (records taken up to the span's end), enter_hit and the state after
// the span are returned; `prior` is 1 + the record of an earlier piece whose block a free of
// this span hit (0: none), which the caller leaves to a later pass: that record may still be
// in flight from the warp replaying its piece.
//
// The open window's totals are kept warp-uniform.  A step whose deltas all lie in
// [-2^22, 2^22) has lane sums and a warp sum below 2^30 in magnitude, so its share of a
// window is formed in 32 bits and summed over the warp with one redux.sync per total; any
// other step uses 64-bit lane sums and a shuffle reduction.  The frees of the step that
// hit the tracked block are found once per step (a bit per event), and re-found only when
// a sample starts tracking another block.
// thresholds at which the exact replay tests each step for the dense form (below); above, a
// step with every event at least 2T - 1 away from zero is too rare to pay for the test
constexpr int64_t DENSE_T_MAX = 4096;

// DENSE: the kernel instance for T <= DENSE_T_MAX, which tests each searched step for the
// dense form; the other instance carries none of that code (its registers and schedule are
// those of the plain replay).
template <bool FIRST, bool DENSE, class RingT>
__device__ bool exact_unit(RingT &sm, uint32_t &phase, const Unit &U, const ExactIn &in0, FRec *out, uint32_t cap,
                           int64_t T, unsigned long long spin, ErrWord *err, int lane, uint32_t &n_out,
                           UnitOut &O, ExactRun *R, uint32_t &prior) {
    constexpr int E = RingT::kE, STEP = 32 * E;
    static_assert(E == 8, "a lane's events fit one byte of bits");
    int64_t accA = warp_sum(in0.wA), accApy = warp_sum(in0.wApy), accSpy = warp_sum(in0.wSpy);
    int64_t c = in0.c;
    int64_t P = 0;
    int64_t mark = in0.mark;
    const int64_t fpb = in0.fpb;
    uint32_t tk = in0.tk;
    uint64_t taddr = in0.taddr;
    uint32_t tslot = in0.tslot;
    uint32_t enter_hit = 0;
    uint32_t n = in0.n0;
    prior = 0;
    // FIRST: the run's facts (lane-uniform)
    int64_t gmax = INT64_MIN, tmax = INT64_MIN;
    uint32_t garg = 0, targ = 0;
    int32_t last = -1;

    auto hit_tracked = [&]() {
        if (tk == 3 && tslot >= in0.n0) {
            if (lane == 0 && tslot < cap) out[tslot].recl = 1;
        } else if (tk == 3) {
            prior = tslot + 1;
        } else {
            enter_hit = 1;
        }
    };
    // this lane's events at step positions (after, upto], as a bit mask over its E events
    auto range = [&](int after, int upto) -> uint32_t {
        const int lo = after + 1 - lane * E, hi = upto - lane * E;   // event offsets k in [lo, hi]
        if (hi < 0 || lo > E - 1) return 0u;
        const uint32_t up = hi >= E - 1 ? 0xffu : (2u << hi) - 1u;
        const uint32_t dn = lo <= 0 ? 0u : (1u << lo) - 1u;
        return up & ~dn;
    };
    // bit k: event k of this lane is a free of the tracked block (screened on the low address
    // word; a step with a candidate is tested on the full address)
    auto free_bits = [&](const StepIn<E> &in) -> uint32_t {
        uint32_t b = 0;
        if (tk) {
            const uint32_t tlo = (uint32_t)taddr;
#pragma unroll
            for (int k = 0; k < E; ++k) b |= ((int32_t)(in.d[k] >> 32) < 0 && (uint32_t)in.a[k] == tlo) ? 1u << k : 0u;
            if (__any_sync(FULL, b != 0)) {
                b = 0;
#pragma unroll
                for (int k = 0; k < E; ++k) b |= (in.d[k] < 0 && in.a[k] == taddr) ? 1u << k : 0u;
            }
        }
        return b;
    };
    // add the warp's events at step positions (after, upto] (lane bits m; ALL: every event)
    // to the window totals
    auto fold = [&](const StepIn<E> &in, bool fits, uint32_t m, auto all) {
        constexpr bool ALL = decltype(all)::value;
        if (fits) {
            int32_t sA = 0, sApy = 0, sSpy = 0;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int32_t x = ALL || ((m >> k) & 1u) ? (int32_t)in.d[k] : 0;
                const int32_t ps = max(x, 0);
                const int32_t py = (int32_t)min(py_of(in, k), 1u);
                sA += ps;
                sApy += ps * py;
                sSpy += x * py;
            }
            accA += __reduce_add_sync(FULL, sA);
            accApy += __reduce_add_sync(FULL, sApy);
            accSpy += __reduce_add_sync(FULL, sSpy);
        } else {
            int64_t sA = 0, sApy = 0, sSpy = 0;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int64_t x = ALL || ((m >> k) & 1u) ? in.d[k] : 0;
                const int64_t ps = x > 0 ? x : 0;
                sA += ps;
                if (py_of(in, k)) { sApy += ps; sSpy += x; }
            }
            accA += warp_sum(sA);
            accApy += warp_sum(sApy);
            accSpy += warp_sum(sSpy);
        }
    };
    // the sample at step position r, closing the window after the events at (after, r] join
    // it (frees up to it already tested): counter cr there, unit-local prefix Pr there.
    // Returns true if the sample started tracking its block.
    auto close = [&](const StepIn<E> &in, bool fits, int after, int r, uint32_t rel0, int64_t cr,
                     int64_t Pr) -> bool {
        fold(in, fits, range(after, r), std::false_type{});
        const int fl = r / E, kf = r % E;
        uint64_t av = in.a[0];
        uint32_t pyv = py_of(in, 0);
#pragma unroll
        for (int k = 1; k < E; ++k)
            if (k == kf) { av = in.a[k]; pyv = py_of(in, k); }
        av = __shfl_sync(FULL, av, fl);
        pyv = __shfl_sync(FULL, pyv, fl);
        const int64_t fp = fpb + Pr;
        const bool growth = cr > 0;
        const bool hwm = growth && fp > mark;
        const uint32_t rel = rel0 + (uint32_t)r;
        if (lane == 0 && n < cap) {
            FRec Rr;
            Rr.rel = rel;
            Rr.line = 0;   // filled in by k_compact
            Rr.kind = growth ? 1 : -1;
            Rr.is_hwm = hwm ? 1 : 0;
            Rr.recl = 0;
            Rr.py = pyv ? 1 : 0;
            Rr.pad = 0;
            Rr.A = accA; Rr.F = accA - cr; Rr.A_py = accApy; Rr.F_py = accApy - accSpy; Rr.P = Pr;
            out[n] = Rr;
        }
        if (FIRST) {
            if (lane == 0 && n < (uint32_t)RM) { R->C0->pos[n] = rel; R->C0->gp[n] = growth ? Pr : INT64_MIN; }
            if (growth && n >= (uint32_t)RM && Pr > tmax) { tmax = Pr; targ = rel; }
            if (growth && Pr > gmax) { gmax = Pr; garg = rel; }
            last = (int32_t)rel;
        }
        if (hwm) { mark = fp; tk = 3; taddr = av; tslot = n; }
        ++n;
        accA = accApy = accSpy = 0;
        return hwm;
    };
    // A dense step: every event moves the counter by 0 or by at least 2T - 1.  From |c| < T each
    // nonzero event then crosses (|c + d| >= |d| - |c| >= T) and leaves the counter at 0, so
    // every nonzero event is a sample whose window holds just itself (the step's first one
    // also closes the open window), and the step's samples are formed side by side instead of
    // one search and close after another.  The marks (a running maximum of the growth
    // footprints), the tracked block at each free (the last mark-setting sample before it)
    // and the frees' hits follow by warp scans.  Returns false if the step is not dense.
    auto dense = [&](const StepIn<E> &in, uint32_t rel0) -> bool {
        const uint64_t lim = 2 * (uint64_t)T - 1;
        bool is_dense = true;
        uint32_t nzm = 0;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int64_t d = in.d[k];
            const uint64_t ad = d < 0 ? 0ull - (uint64_t)d : (uint64_t)d;
            is_dense &= d == 0 || ad >= lim;
            nzm |= d != 0 ? 1u << k : 0u;
        }
        if (!__all_sync(FULL, is_dense)) return false;
        const int cnt = __popc(nzm);
        int rinc = cnt;   // samples up to this lane (inclusive scan)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, rinc, o);
            if (lane >= o) rinc += y;
        }
        const int total = __shfl_sync(FULL, rinc, 31);
        if (total == 0) return true;   // zero deltas only: nothing moves, no free among them
        const uint32_t nb = n + (uint32_t)(rinc - cnt);   // this lane's first record
        // unit-local prefix through each event
        int64_t lp[E];
        lp[0] = in.d[0];
#pragma unroll
        for (int k = 1; k < E; ++k) lp[k] = lp[k - 1] + in.d[k];
        const int64_t lin = warp_incl_scan(lp[E - 1], lane);
        const int64_t stot = __shfl_sync(FULL, lin, 31);
        const int64_t base = P + lin - lp[E - 1];
        // the step's first sample closes the open window from counter c (warp-uniform)
        const int first_lane = __ffs(__ballot_sync(FULL, cnt != 0)) - 1;
        const int first_k = __ffs(__shfl_sync(FULL, (int)nzm, first_lane)) - 1;
        // growth footprints and the mark before each event: running maximum within the lane,
        // then an exclusive maximum over the lanes below
        int64_t lmx = INT64_MIN;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const bool first = lane == first_lane && k == first_k;
            const int64_t cr = first ? c + in.d[k] : in.d[k];
            if (in.d[k] != 0 && cr > 0) lmx = max(lmx, fpb + base + lp[k]);
        }
        int64_t mx = lmx;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, mx, o);
            if (lane >= o && y > mx) mx = y;
        }
        int64_t mrun = __shfl_up_sync(FULL, mx, 1);
        if (lane == 0) mrun = INT64_MIN;
        mrun = max(mrun, mark);
        // the last mark-setting sample in each lane (its record and address), then the one
        // entering each lane from the lanes below (pos: 1 + its step position, 0: none)
        uint32_t hwm_bits = 0;
        int64_t mm = mrun;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const bool first = lane == first_lane && k == first_k;
            const int64_t cr = first ? c + in.d[k] : in.d[k];
            const int64_t fp = fpb + base + lp[k];
            if (in.d[k] != 0 && cr > 0 && fp > mm) { hwm_bits |= 1u << k; mm = fp; }
        }
        uint32_t hpos = 0, hslot = 0;
        uint64_t haddr = 0;
        if (hwm_bits) {
            const int k = 31 - __clz(hwm_bits);
            hpos = (uint32_t)(lane * E + k) + 1;
            hslot = nb + (uint32_t)__popc(nzm & ((1u << k) - 1u));
#pragma unroll
            for (int q = 0; q < E; ++q)
                if (q == k) haddr = in.a[q];
        }
        uint32_t epos = hpos, eslot = hslot;
        uint64_t eaddr = haddr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yp = __shfl_up_sync(FULL, epos, o);
            const uint32_t ys = __shfl_up_sync(FULL, eslot, o);
            const uint64_t ya = __shfl_up_sync(FULL, eaddr, o);
            if (lane >= o && yp > epos) { epos = yp; eslot = ys; eaddr = ya; }
        }
        // exclusive: the last mark-setting sample of the lanes below
        uint32_t cpos = __shfl_up_sync(FULL, epos, 1), cslot = __shfl_up_sync(FULL, eslot, 1);
        uint64_t caddr = __shfl_up_sync(FULL, eaddr, 1);
        if (lane == 0) cpos = 0;
        // records, and each free tested against the block tracked at it
        uint32_t ctk = cpos ? 3u : tk, cs = cpos ? cslot : tslot;
        uint64_t ca = cpos ? caddr : taddr;
        bool own = false;                  // (ctk, cs) is a record this lane wrote in this step
        uint32_t hit_slot = 0xffffffffu;   // a record a lane below wrote in this step, hit here
        int64_t gbest = INT64_MIN, tbest = INT64_MIN;
        uint32_t gpos = 0, tpos = 0;
        uint32_t r = nb;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int64_t d = in.d[k];
            if (ctk && d < 0 && in.a[k] == ca) {
                if (ctk == 3 && own) {
                    if (cs < cap) out[cs].recl = 1;   // (this thread stored the record above)
                } else if (ctk == 3 && cs >= n) {
                    hit_slot = cs;                    // marked once every lane's records are out
                } else if (ctk == 3 && cs >= in0.n0) {
                    if (cs < cap) out[cs].recl = 1;   // an earlier step's record
                } else if (ctk == 3) {
                    prior = cs + 1;
                } else {
                    enter_hit = 1;
                }
            }
            if (d == 0) continue;
            const bool first = lane == first_lane && k == first_k;
            const int64_t cr = first ? c + d : d;
            const int64_t Pr = base + lp[k];
            const int64_t pos_a = d > 0 ? d : 0;
            const uint32_t pyk = py_of(in, k) ? 1u : 0u;
            const int64_t A = (first ? accA : 0) + pos_a;
            const int64_t Apy = (first ? accApy : 0) + (pyk ? pos_a : 0);
            const int64_t Spy = (first ? accSpy : 0) + (pyk ? d : 0);
            const bool growth = cr > 0;
            const bool hwm = ((hwm_bits >> k) & 1u) != 0;
            const uint32_t rel = rel0 + (uint32_t)(lane * E + k);
            if (r < cap) {
                FRec Rr;
                Rr.rel = rel;
                Rr.line = 0;   // filled in by k_compact
                Rr.kind = growth ? 1 : -1;
                Rr.is_hwm = hwm ? 1 : 0;
                Rr.recl = 0;
                Rr.py = (uint8_t)pyk;
                Rr.pad = 0;
                Rr.A = A; Rr.F = A - cr; Rr.A_py = Apy; Rr.F_py = Apy - Spy; Rr.P = Pr;
                out[r] = Rr;
            }
            if (FIRST) {
                if (r < (uint32_t)RM) { R->C0->pos[r] = rel; R->C0->gp[r] = growth ? Pr : INT64_MIN; }
                if (growth && Pr > gbest) { gbest = Pr; gpos = rel; }
                if (growth && r >= (uint32_t)RM && Pr > tbest) { tbest = Pr; tpos = rel; }
            }
            if (hwm) { ctk = 3; cs = r; ca = in.a[k]; own = true; }
            ++r;
        }
        __syncwarp();   // the step's records are written before the hits mark them
        if (hit_slot != 0xffffffffu && hit_slot < cap) out[hit_slot].recl = 1;
        if (FIRST) {
            // the largest growth prefix and its first position (positions rise with the lanes)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t yb = __shfl_xor_sync(FULL, gbest, o), zb = __shfl_xor_sync(FULL, tbest, o);
                const uint32_t yp = __shfl_xor_sync(FULL, gpos, o), zp = __shfl_xor_sync(FULL, tpos, o);
                if (yb > gbest || (yb == gbest && yp < gpos)) { gbest = yb; gpos = yp; }
                if (zb > tbest || (zb == tbest && zp < tpos)) { tbest = zb; tpos = zp; }
            }
            if (gbest > gmax) { gmax = gbest; garg = gpos; }
            if (tbest > tmax) { tmax = tbest; targ = tpos; }
            const int last_lane = 31 - __clz(__ballot_sync(FULL, cnt != 0));
            const int last_k = 31 - __clz(__shfl_sync(FULL, (int)nzm, last_lane));
            last = (int32_t)(rel0 + (uint32_t)(last_lane * E + last_k));
        }
        // the state after the step: the last sample left the counter at 0 and an empty window
        enter_hit = __any_sync(FULL, enter_hit != 0) ? 1u : 0u;
        prior = __reduce_max_sync(FULL, prior);
        const uint32_t any_hwm = __ballot_sync(FULL, hwm_bits != 0);
        if (any_hwm) {
            const int hl = 31 - __clz(any_hwm);
            tk = 3;
            tslot = __shfl_sync(FULL, hslot, hl);
            taddr = __shfl_sync(FULL, haddr, hl);
            mark = warp_max(lmx);   // every mark-setting sample beat the mark before it
        }
        n += (uint32_t)total;
        c = 0;
        accA = accApy = accSpy = 0;
        P += stot;
        return true;
    };
    // every event of the step joins the open window (no sample in it)
    auto whole_step = [&](const StepIn<E> &in, bool fits) {
        fold(in, fits, 0xffu, std::true_type{});
        if (tk && __any_sync(FULL, free_bits(in) != 0)) hit_tracked();
    };

    bool ok;
    if (!FIRST && in0.list) {
        // ---- the resets are known: no crossing search
        // the list is read 32 entries at a time (lane j holds entry base + j), the next
        // 32 loading while the current ones are used
        const SRes *Ls = in0.list;
        const uint32_t rend = in0.rend;
        auto fetch = [&](uint32_t base, uint32_t &bp, int64_t &bP) {
            const uint32_t i = base + (uint32_t)lane;
            if (i < rend) { const SRes q = Ls[i]; bp = q.pos; bP = q.P; } else { bp = 0xffffffffu; bP = 0; }
        };
        // lane j holds entry (ri & ~31) + j, the next 32 loading behind them
        uint32_t ri = in0.n0;
        uint32_t cpos, npos_b;
        int64_t cP, nP_b;
        fetch(ri & ~31u, cpos, cP);
        fetch((ri & ~31u) + 32, npos_b, nP_b);
        uint32_t npos = __shfl_sync(FULL, cpos, (int)(ri & 31u));
        int64_t nP = __shfl_sync(FULL, cP, (int)(ri & 31u));
        if (ri >= rend) npos = 0xffffffffu;
        int64_t cst = c, Pprev = in0.P0;   // counter at the open window's start, prefix there
        bool done = false;
        const uint32_t from = in0.from;
        auto kstep = [&](const StepIn<E> &in, uint32_t rel0) -> bool {
            const bool fits = __all_sync(FULL, step_fits32(in));
            // a piece's first step leaves out the events before it
            const int a0 = rel0 < from ? (int)(from - rel0) - 1 : -1;
            if (a0 < 0 && npos >= rel0 + (uint32_t)STEP) {
                whole_step(in, fits);
                return false;
            }
            uint32_t fb = free_bits(in);
            int after = a0;
            while (npos < rel0 + (uint32_t)STEP) {
                if (npos < rel0 + (uint32_t)(after + 1)) {   // positions must increase
                    if (lane == 0) set_error(err, E_INTERNAL, 12, (unsigned long long)U.gidx0);
                    npos = 0xffffffffu;
                    break;
                }
                const int r = (int)(npos - rel0);
                if (tk && __any_sync(FULL, (fb & range(after, r)) != 0)) hit_tracked();
                if (close(in, fits, after, r, rel0, cst + (nP - Pprev), nP)) fb = free_bits(in);
                cst = 0;
                Pprev = nP;
                after = r;
                if (++ri < rend) {
                    if ((ri & 31u) == 0) {
                        cpos = npos_b;
                        cP = nP_b;
                        fetch(ri + 32, npos_b, nP_b);
                    }
                    npos = __shfl_sync(FULL, cpos, (int)(ri & 31u));
                    nP = __shfl_sync(FULL, cP, (int)(ri & 31u));
                } else {
                    npos = 0xffffffffu;
                    done = in0.stop;
                }
            }
            if (done) return true;   // the piece ends at this reset: the rest is the next piece's
            if (tk && __any_sync(FULL, (fb & range(after, STEP - 1)) != 0)) hit_tracked();
            fold(in, fits, range(after, STEP - 1), std::false_type{});
            return false;
        };
        ok = ring_walk<true>(sm, U, from / STEP * STEP, in0.limit, phase, spin, err, lane, kstep);
        c = in0.exit_c;
    } else {
        // ---- search for the crossings from the entry counter (in the 32-bit form of a
        // step when T and the step's deltas allow it: the same arithmetic without overflow)
        const bool t32 = T <= FIT32_T;
        auto step = [&](const StepIn<E> &in, uint32_t rel0) -> bool {
            if constexpr (DENSE) {
                if (dense(in, rel0)) return false;
            }
            const bool fits = __all_sync(FULL, step_fits32(in));
            if (t32 && fits) {
                StepPrefix32<E> sp;
                int32_t *xq32 = reinterpret_cast<int32_t *>(sm.xq);
                step_prefix32(in, lane, sp, (int32_t *)nullptr);
                const int32_t T32 = (int32_t)T;
                int32_t b = (int32_t)c;
                if (__ballot_sync(FULL, b + sp.lmax >= T32 || b + sp.lmin <= -T32) == 0) {
                    whole_step(in, true);
                    c += sp.tot;
                    P += sp.tot;
                    return false;
                }
                publish_prefix32(sp, lane, xq32);
                uint32_t fb = free_bits(in);
                int after = -1;
                while (true) {
                    int32_t Qr;
                    const int r = first_cross(sp, (const int32_t *)xq32, lane, b, T32, after, Qr);
                    if (tk && __any_sync(FULL, (fb & range(after, r < 0 ? STEP - 1 : r)) != 0)) hit_tracked();
                    if (r < 0) break;
                    if (close(in, true, after, r, rel0, (int64_t)(b + Qr), P + Qr)) fb = free_bits(in);
                    b = -Qr;
                    after = r;
                }
                fold(in, true, range(after, STEP - 1), std::false_type{});
                c = b + sp.tot;
                P += sp.tot;
                return false;
            }
            StepPrefix<E> sp;
            step_prefix(in, lane, sp, sm.xq);
            if (__ballot_sync(FULL, c + sp.lmax >= T || c + sp.lmin <= -T) == 0) {
                whole_step(in, fits);
                c += sp.tot;
                P += sp.tot;
                return false;
            }
            uint32_t fb = free_bits(in);
            int64_t b = c;
            int after = -1;
            while (true) {
                int64_t Qr;
                const int r = first_cross(sp, sm.xq, lane, b, T, after, Qr);
                // frees up to and including the sample's event see the block tracked so far
                if (tk && __any_sync(FULL, (fb & range(after, r < 0 ? STEP - 1 : r)) != 0)) hit_tracked();
                if (r < 0) break;
                if (close(in, fits, after, r, rel0, b + Qr, P + Qr)) fb = free_bits(in);
                b = -Qr;
                after = r;
            }
            fold(in, fits, range(after, STEP - 1), std::false_type{});
            c = b + sp.tot;
            P += sp.tot;
            return false;
        };
        ok = ring_walk<true>(sm, U, 0, U.len, phase, spin, err, lane, step);
    }
    O.count = n;
    O.enter_hit = enter_hit;
    O.c = c; O.A = accA; O.F = accA - c; O.Apy = accApy; O.Fpy = accApy - accSpy;
    n_out = n;
    if (FIRST) {
        R->gmax = gmax; R->garg = garg; R->tmax = tmax; R->targ = targ; R->last = last; R->P = P;
    }
    return ok;
}

}  // namespace scl
