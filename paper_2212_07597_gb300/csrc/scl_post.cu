// scl_post.cu -- everything after the sampler walk:
//   k_scan     per trace, over its units: sample offsets, footprint at each unit
//              start (Section 3.3: the footprint is tracked at every event), the
//              high-water mark and tracked block entering each unit (Section 3.4),
//              and the sampling window open at each unit start.
//   k_compact  writes the final samples (Section 3.3 entries) to the log and to
//              per-line totals through a shared-memory table; crossings count one
//              tracked malloc for their line.
//   k_mark     a block tracked when a unit starts and freed inside it is marked
//              reclaimed (Section 3.4's pointer comparison spans units).
//   k_epi      closes each object's trial at the next crossing: frees += reclaimed.
//   k_state    folds the batch into the trace's resident state.
#include "scl_internal.cuh"
#include <algorithm>
#include <cstddef>

#include "scl_launch.h"

namespace scl {

constexpr int NT = 256;   // threads per block of the post kernels

__device__ __forceinline__ int64_t warp_incl_max(int64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o && t > v) v = t;
    }
    return v;
}

// block-wide exclusive sum over NT threads; *total gets the block total
__device__ int64_t block_excl_sum(int64_t v, int64_t *sh, int64_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t incl = warp_incl_scan(v, lane);
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int64_t x = lane < NT / 32 ? sh[lane] : 0;
        const int64_t xi = warp_incl_scan(x, lane);
        if (lane < NT / 32) sh[lane] = xi - x;
        if (lane == NT / 32 - 1) sh[NT / 32] = xi;
    }
    __syncthreads();
    const int64_t r = incl - v + sh[w];
    *total = sh[NT / 32];
    __syncthreads();
    return r;
}

__device__ int64_t block_excl_max(int64_t v, int64_t *sh, int64_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t incl = warp_incl_max(v, lane);
    int64_t ex = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0) ex = INT64_MIN;
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int64_t x = lane < NT / 32 ? sh[lane] : INT64_MIN;
        const int64_t xi = warp_incl_max(x, lane);
        int64_t xe = __shfl_up_sync(FULL, xi, 1);
        if (lane == 0) xe = INT64_MIN;
        if (lane < NT / 32) sh[lane] = xe;
        if (lane == NT / 32 - 1) sh[NT / 32] = xi;
    }
    __syncthreads();
    const int64_t r = ex > sh[w] ? ex : sh[w];
    *total = sh[NT / 32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- k_scan
// Per trace, over its units in order (Sections 3.3-3.4): footprint before each unit,
// sample offsets, the high-water mark entering each unit and the tracked block then
// (the first event attaining the largest growth-sample footprint so far, if that
// beats the mark the trace entered the batch with), and the open sampling window
// entering each unit (whole-unit totals plus the tail of the unit holding the last
// reset, which k_final reads back).
struct MaxPos {
    int64_t v;
    uint64_t pos;
    int64_t unit;
};

__device__ __forceinline__ MaxPos mp_better(const MaxPos &a, const MaxPos &b) {   // a earlier than b
    return b.v > a.v ? b : a;
}

__device__ __forceinline__ MaxPos mp_shfl_up(const MaxPos &x, int o) {
    MaxPos y;
    y.v = __shfl_up_sync(FULL, x.v, o);
    y.pos = __shfl_up_sync(FULL, x.pos, o);
    y.unit = __shfl_up_sync(FULL, x.unit, o);
    return y;
}

__device__ __forceinline__ MaxPos mp_shfl(const MaxPos &x, int l) {
    MaxPos y;
    y.v = __shfl_sync(FULL, x.v, l);
    y.pos = __shfl_sync(FULL, x.pos, l);
    y.unit = __shfl_sync(FULL, x.unit, l);
    return y;
}

// N sums (and N (max, first position) scans) over a block of BT threads at once: one set of
// barriers for all of them instead of one per scan.  ex = exclusive result, tot = block total.
template <int BT, int N>
__device__ __forceinline__ void block_excl_sums(const int64_t (&v)[N], int64_t (&ex)[N], int64_t (&tot)[N],
                                                int64_t (*sh)[N]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x[N];
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = v[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int64_t t = __shfl_up_sync(FULL, x[k], o);
            if (lane >= o) x[k] += t;
        }
    }
    if (lane == 31)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[w][k] = x[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int64_t y = lane < BT / 32 ? sh[lane][k] : 0;
            int64_t yi = y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(FULL, yi, o);
                if (lane >= o) yi += t;
            }
            if (lane < BT / 32) sh[lane][k] = yi - y;
            if (lane == BT / 32 - 1) sh[BT / 32][k] = yi;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        ex[k] = x[k] - v[k] + sh[w][k];
        tot[k] = sh[BT / 32][k];
    }
    __syncthreads();
}

template <int BT, int N>
__device__ __forceinline__ void block_excl_maxpos_n(const MaxPos (&v)[N], MaxPos (&ex)[N], MaxPos (&tot)[N],
                                                    MaxPos (*sh)[N]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const MaxPos id = {INT64_MIN, 0, -1};
    MaxPos x[N], e[N];
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = v[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const MaxPos t = mp_shfl_up(x[k], o);
            if (lane >= o) x[k] = mp_better(t, x[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
        e[k] = mp_shfl_up(x[k], 1);
        if (lane == 0) e[k] = id;
        if (lane == 31) sh[w][k] = x[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const MaxPos y = lane < BT / 32 ? sh[lane][k] : id;
            MaxPos yi = y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const MaxPos t = mp_shfl_up(yi, o);
                if (lane >= o) yi = mp_better(t, yi);
            }
            MaxPos ye = mp_shfl_up(yi, 1);
            if (lane == 0) ye = id;
            if (lane < BT / 32) sh[lane][k] = ye;
            if (lane == BT / 32 - 1) sh[BT / 32][k] = yi;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        ex[k] = mp_better(sh[w][k], e[k]);
        tot[k] = sh[BT / 32][k];
    }
    __syncthreads();
}

template <int BT>
__global__ void __launch_bounds__(BT) k_scan(LaunchPost a) {
    __shared__ int64_t sh[BT / 32 + 1][5];
    __shared__ MaxPos shm[BT / 32 + 1][2];
    const int b = blockIdx.x;
    const BTrace B = a.bts[b];
    const DevTrace st = a.traces[B.trace];
    const MaxPos none = {INT64_MIN, 0, -1};
    int64_t ccnt = 0, cfp = st.footprint, cA = 0, cApy = 0, cSpy = 0;
    MaxPos cg = none;     // best growth footprint of the batch so far
    MaxPos clast = none;  // latest reset so far (v = trace index)
    for (uint32_t base = 0; base < B.nu; base += BT) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < B.nu;
        const uint32_t u = B.u0 + (valid ? i : 0);
        const Unit &U = a.units[u];
        const UnitTrue Tu = a.utrue[u];
        const UnitSum S = a.usum[u];
        // sample counts, footprint changes and window totals of the units, scanned at once
        int64_t sv[5] = {valid ? (int64_t)Tu.n : 0, valid ? S.total : 0, valid ? S.totA : 0,
                         valid ? S.totApy : 0, valid ? S.totSpy : 0};
        int64_t se[5], st5[5];
        block_excl_sums<BT, 5>(sv, se, st5, sh);
        const int64_t ec = se[0], ncnt = ccnt + st5[0];
        const int64_t fpb = cfp + se[1], nfp = cfp + st5[1];
        const int64_t eA = se[2], nA = cA + st5[2];
        const int64_t eApy = se[3], nApy = cApy + st5[3];
        const int64_t eSpy = se[4], nSpy = cSpy + st5[4];
        // the best growth footprint and the latest reset before each unit
        MaxPos mv[2] = {none, none};
        if (valid && Tu.gmax != INT64_MIN) { mv[0].v = fpb + Tu.gmax; mv[0].pos = U.gidx0 + Tu.garg; mv[0].unit = u; }
        if (valid && Tu.exit_last >= 0) { mv[1].v = Tu.exit_last; mv[1].pos = (uint64_t)Tu.exit_last; mv[1].unit = u; }
        MaxPos me[2], mt[2];
        block_excl_maxpos_n<BT, 2>(mv, me, mt, shm);
        const MaxPos eg = mp_better(cg, me[0]), gt = mt[0];
        const MaxPos el = mp_better(clast, me[1]), lt = mt[1];
        if (valid) {
            UnitPlan Pn;
            Pn.fp_base = fpb;
            Pn.sample_off = (uint64_t)(ccnt + ec);
            Pn.hwm_in = eg.v > st.hwm ? eg.v : st.hwm;
            if (eg.v > st.hwm) {
                const Unit &W = a.units[eg.unit];
                Pn.enter_kind = 1; Pn.enter_idx = eg.pos; Pn.enter_unit = eg.unit;
                Pn.enter_addr = W.addr[eg.pos - W.gidx0];
            } else if (st.tracked_valid) {
                Pn.enter_kind = 2; Pn.enter_idx = st.tracked_idx; Pn.enter_unit = -1; Pn.enter_addr = st.tracked_addr;
            } else {
                Pn.enter_kind = 0; Pn.enter_idx = 0; Pn.enter_unit = -1; Pn.enter_addr = 0;
            }
            if (i == 0 || el.unit < 0) {
                // no reset yet in this batch: the resident window is still open
                Pn.rb_unit = -1; Pn.rb_from = 0;
                Pn.wA = st.A + cA + eA; Pn.wApy = st.A_py + cApy + eApy; Pn.wSpy = (st.A_py - st.F_py) + cSpy + eSpy;
            } else {
                const Unit &W = a.units[el.unit];
                // totals of the units strictly between the reset's unit and this one
                const UnitSum &SW = a.usum[el.unit];
                (void)SW;
                Pn.rb_unit = el.unit;
                Pn.rb_from = (uint32_t)(el.pos - W.gidx0 + 1);
                Pn.wA = 0; Pn.wApy = 0; Pn.wSpy = 0;
            }
            a.uplan[u] = Pn;
        }
        ccnt = ncnt;
        cfp = nfp;
        cA = nA; cApy = nApy; cSpy = nSpy;
        cg = mp_better(cg, gt);
        clast = mp_better(clast, lt);
    }
    if (threadIdx.x == 0) {
        BTraceRes &BR = a.btres[b];
        BR.n_samples = (uint64_t)ccnt;
        BR.fp_end = cfp;
        BR.hwm_end = cg.v > st.hwm ? cg.v : st.hwm;
        BR.last_cross_unit = cg.v > st.hwm ? cg.unit : -1;
        BR.last_cross_idx = cg.v > st.hwm ? cg.pos : 0;
        BR.pending_hit = 0;
    }
}

// window totals of the units strictly between a reset's unit and the unit it opens
// into: a second pass over the units, once every unit's read-back unit is known
template <int BT>
__global__ void __launch_bounds__(BT) k_scan_window(LaunchPost a) {
    __shared__ int64_t sh[BT / 32 + 1][3];
    const BTrace B = a.bts[blockIdx.x];
    // prefix sums of the unit totals, then differences
    int64_t cA = 0, cApy = 0, cSpy = 0;
    for (uint32_t base = 0; base < B.nu; base += BT) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < B.nu;
        const uint32_t u = B.u0 + (valid ? i : 0);
        const UnitSum S = a.usum[u];
        int64_t sv[3] = {valid ? S.totA : 0, valid ? S.totApy : 0, valid ? S.totSpy : 0};
        int64_t se[3], stt[3];
        block_excl_sums<BT, 3>(sv, se, stt, sh);
        const int64_t eA = se[0], nA = cA + stt[0];
        const int64_t eApy = se[1], nApy = cApy + stt[1];
        const int64_t eSpy = se[2], nSpy = cSpy + stt[2];
        if (valid) {
            a.pref[3 * (size_t)u + 0] = cA + eA;
            a.pref[3 * (size_t)u + 1] = cApy + eApy;
            a.pref[3 * (size_t)u + 2] = cSpy + eSpy;
        }
        cA = nA; cApy = nApy; cSpy = nSpy;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < B.nu; i += BT) {
        const uint32_t u = B.u0 + i;
        UnitPlan &Pn = a.uplan[u];
        if (Pn.rb_unit < 0) continue;
        const uint32_t w1 = (uint32_t)Pn.rb_unit + 1;
        Pn.wA = a.pref[3 * (size_t)u + 0] - a.pref[3 * (size_t)w1 + 0];
        Pn.wApy = a.pref[3 * (size_t)u + 1] - a.pref[3 * (size_t)w1 + 1];
        Pn.wSpy = a.pref[3 * (size_t)u + 2] - a.pref[3 * (size_t)w1 + 2];
    }
}

// ---------------------------------------------------------------- k_compact
// Section 3.3: each final sample goes to the sample log and to its line's totals;
// crossings count one tracked malloc for their line (Section 3.4).
constexpr int HCOLS = 7;   // n_growth, n_shrink, A, F, A_py, F_py, mallocs (the LineRow order)

// one sample into a line's totals (row: HCOLS words in LineRow order; zero terms are skipped)
__device__ __forceinline__ void row_add(unsigned long long *row, bool growth, int64_t A, int64_t F, int64_t Apy,
                                        int64_t Fpy, bool hwm) {
    atomicAdd(&row[growth ? 0 : 1], 1ull);
    if (A) atomicAdd(&row[2], (unsigned long long)A);
    if (F) atomicAdd(&row[3], (unsigned long long)F);
    if (Apy) atomicAdd(&row[4], (unsigned long long)Apy);
    if (Fpy) atomicAdd(&row[5], (unsigned long long)Fpy);
    if (hwm) atomicAdd(&row[6], 1ull);
}
static_assert(offsetof(LineRow, mallocs) == 6 * 8, "row_add's columns are the LineRow words");

__global__ void __launch_bounds__(NT) k_compact(LaunchPost a) {
    extern __shared__ __align__(16) unsigned long long hist[];   // [n_lines][HCOLS] when it fits
    const CompactGroup G = a.groups[blockIdx.x];
    const bool use_smem = a.n_lines <= (uint32_t)SMEM_LINES_MAX;
    if (use_smem) {
        for (uint32_t i = threadIdx.x; i < a.n_lines * HCOLS; i += NT) hist[i] = 0;
        __syncthreads();
    }
    // the whole block walks each unit's records in turn (a group often holds a single unit)
    for (uint32_t k = 0; k < G.nu; ++k) {
        const uint32_t u = G.u0 + k;
        const Unit U = a.units[u];
        const UnitOut O = a.uout[u];
        const UnitPlan &Pn = a.uplan[u];
        const DevTrace &st = a.traces[U.trace];
        Sample *log = a.log ? a.log + (uint64_t)U.trace * a.log_cap : nullptr;
        const uint64_t log_base = st.n_samples + Pn.sample_off;
        LineRow *grow = a.lines + (uint64_t)U.trace * a.n_lines;
        FRec *rec = a.recs + U.rec0;
        const uint32_t cnt = O.count < U.rec_cap ? O.count : U.rec_cap;
        for (uint32_t j = threadIdx.x; j < cnt; j += NT) {
            const FRec r = rec[j];
            // the line of the sample's event (the replay leaves it to this pass); kept in the
            // record for the leak epilogue and the state fold
            uint32_t line = U.line[r.rel];
            rec[j].line = line;
            bool line_ok = true;
            if (line >= a.n_lines) {
                set_error(a.err, E_RANGE, line, U.gidx0 + r.rel);
                line_ok = false;
                line = 0;
            }
            const int64_t fp = Pn.fp_base + r.P;
            if (log && log_base + j < a.log_cap) {
                Sample s;
                s.idx = U.gidx0 + r.rel;
                s.A = r.A; s.F = r.F; s.A_py = r.A_py; s.F_py = r.F_py;
                s.footprint = fp;
                s.line = line;
                s.kind = r.kind;
                s.is_python = r.py;
                s.is_hwm = r.is_hwm;
                s.pad = 0;
                log[log_base + j] = s;
            }
            if (!line_ok) continue;
            row_add(use_smem ? &hist[line * HCOLS] : reinterpret_cast<unsigned long long *>(&grow[line]), r.kind > 0,
                    r.A, r.F, r.A_py, r.F_py, r.is_hwm);
        }
    }
    if (use_smem) {
        __syncthreads();
        const uint32_t tr = a.units[G.u0].trace;   // all units of a group belong to one trace
        LineRow *grow = a.lines + (uint64_t)tr * a.n_lines;
        for (uint32_t l = threadIdx.x; l < a.n_lines; l += NT) {
            const unsigned long long *h = &hist[l * HCOLS];
            if ((h[0] | h[1]) == 0) continue;
            atomicAdd(&grow[l].n_growth, h[0]);
            atomicAdd(&grow[l].n_shrink, h[1]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&grow[l].A), h[2]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&grow[l].F), h[3]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&grow[l].A_py), h[4]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&grow[l].F_py), h[5]);
            if (h[6]) atomicAdd(&grow[l].mallocs, h[6]);
        }
    }
}

// index of the record with unit offset `rel` among a unit's sorted records (or count)
__device__ __forceinline__ uint32_t find_record(const FRec *rec, uint32_t count, uint32_t rel) {
    uint32_t lo = 0, hi = count;
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (rec[m].rel < rel) lo = m + 1; else hi = m;
    }
    return lo < count && rec[lo].rel == rel ? lo : count;
}

// ---------------------------------------------------------------- k_mark
// Section 3.4: the block tracked when a unit starts was freed inside the unit ->
// mark its crossing's record (or the trace's pre-batch block) reclaimed.
//
// The pieces of a unit replayed apart by k_final report here what they could not write
// themselves: a free of the block an earlier piece's sample tracks (that record is marked
// now), or of the block tracked entering the unit.
__global__ void k_mark(LaunchPost a) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= a.nunits) return;
    const UnitOut &O = a.uout[u];
    const Unit &U = a.units[u];
    uint32_t enter = O.enter_hit;
    if (U.fnp > 1) {
        const uint32_t cnt = O.count < U.rec_cap ? O.count : U.rec_cap;
        for (uint32_t i = U.fi0; i < U.fi0 + U.fnp; ++i) {
            const uint32_t h = a.phit[i];
            if (h == PHIT_ENTER) enter = 1;
            else if (h && h - 1 < cnt) a.recs[U.rec0 + h - 1].recl = 1;
            else if (h) set_error(a.err, E_INTERNAL, 13, (unsigned long long)u);
        }
    }
    if (!enter) return;
    const UnitPlan &Pn = a.uplan[u];
    if (Pn.enter_kind == 1) {
        const Unit &W = a.units[Pn.enter_unit];
        const uint32_t cnt = a.uout[Pn.enter_unit].count < W.rec_cap ? a.uout[Pn.enter_unit].count : W.rec_cap;
        FRec *rec = a.recs + W.rec0;
        const uint32_t j = find_record(rec, cnt, (uint32_t)(Pn.enter_idx - W.gidx0));
        if (j < cnt) rec[j].recl = 1;
        else set_error(a.err, E_INTERNAL, 11, (unsigned long long)u);
    } else if (Pn.enter_kind == 2) {
        a.btres[a.units[u].bt].pending_hit = 1;
    }
}

// ---------------------------------------------------------------- k_epi
// Section 3.4: at the next crossing of a maximum, frees is incremented if the
// tracked object was reclaimed.  The batch's last crossing stays open.
__global__ void k_epi(LaunchPost a) {
    const int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= a.nunits) return;
    const Unit U = a.units[u];
    const uint32_t cnt = a.uout[u].count < U.rec_cap ? a.uout[u].count : U.rec_cap;
    const BTraceRes &BR = a.btres[U.bt];
    LineRow *grow = a.lines + (uint64_t)U.trace * a.n_lines;
    const FRec *rec = a.recs + U.rec0;
    for (uint32_t j = lane; j < cnt; j += 32) {
        const FRec r = rec[j];
        if (!r.is_hwm || !r.recl || r.line >= a.n_lines) continue;
        if (BR.last_cross_unit == (int64_t)u && U.gidx0 + r.rel == BR.last_cross_idx) continue;
        atomicAdd(&grow[r.line].frees, 1ull);
    }
}

// ---------------------------------------------------------------- k_state
__global__ void k_state(LaunchPost a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nbt) return;
    const BTrace B = a.bts[b];
    const BTraceRes BR = a.btres[b];
    DevTrace &st = a.traces[B.trace];
    LineRow *grow = a.lines + (uint64_t)B.trace * a.n_lines;
    if (B.nu > 0) {
        const UnitOut &O = a.uout[B.u0 + B.nu - 1];
        st.c = O.c; st.A = O.A; st.F = O.F; st.A_py = O.Apy; st.F_py = O.Fpy;
        st.footprint = BR.fp_end;
        st.hwm = BR.hwm_end;
        if (BR.last_cross_unit >= 0) {
            // the block tracked before the batch closes its trial at the batch's first crossing
            if (st.tracked_valid && (st.tracked_reclaimed || BR.pending_hit) && st.tracked_line < a.n_lines)
                atomicAdd(&grow[st.tracked_line].frees, 1ull);
            const Unit &W = a.units[BR.last_cross_unit];
            const uint32_t cnt = a.uout[BR.last_cross_unit].count < W.rec_cap ? a.uout[BR.last_cross_unit].count
                                                                              : W.rec_cap;
            const FRec *rec = a.recs + W.rec0;
            const uint32_t rel = (uint32_t)(BR.last_cross_idx - W.gidx0);
            const uint32_t j = find_record(rec, cnt, rel);
            st.tracked_valid = 1;
            st.tracked_addr = W.addr[rel];
            st.tracked_idx = BR.last_cross_idx;
            st.tracked_line = j < cnt ? rec[j].line : 0;
            st.tracked_reclaimed = j < cnt ? rec[j].recl : 0;
            if (j >= cnt) set_error(a.err, E_INTERNAL, 12, b);
        } else if (st.tracked_valid && BR.pending_hit) {
            st.tracked_reclaimed = 1;
        }
        st.n_events += B.n_ev;
        st.n_samples += BR.n_samples;
    }
    if (B.n_cp) {
        st.copy_counter = BR.copy_end;
        st.n_copies += B.n_cp;
    }
}

// ---------------------------------------------------------------- reset / scores
__global__ void k_reset(DevTrace *traces, LineRow *lines, unsigned long long *copies, uint32_t trace0, uint32_t ntr,
                        uint32_t n_lines, int64_t F0, uint64_t phase) {
    unsigned long long *rows = reinterpret_cast<unsigned long long *>(lines + (uint64_t)trace0 * n_lines);
    const uint64_t nw = (uint64_t)ntr * n_lines * (sizeof(LineRow) / 8);
    const uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = i0; i < nw; i += stride) rows[i] = 0;
    unsigned long long *cc = copies + (uint64_t)trace0 * n_lines * 2;
    for (uint64_t i = i0; i < (uint64_t)ntr * n_lines * 2; i += stride) cc[i] = 0;
    for (uint64_t k = i0; k < ntr; k += stride) {
        DevTrace t;
        t.c = t.A = t.F = t.A_py = t.F_py = 0;
        t.footprint = F0;
        t.hwm = F0;
        t.tracked_addr = t.tracked_idx = 0;
        t.tracked_line = t.tracked_valid = t.tracked_reclaimed = t.pad0 = 0;
        t.n_events = t.n_copies = t.n_samples = 0;
        t.copy_counter = phase;
        traces[trace0 + k] = t;
    }
}

struct ScoreRow {   // layout of scl_leak_score
    uint32_t line, pad;
    uint64_t mallocs, frees;
    int64_t num, den;
};

// Section 3.4: likelihood = 1 - (frees + 1) / (mallocs - frees + 2) as printed
// (rule 0), or Laplace's rule 1 - (frees + 1) / (mallocs + 2) (rule 1), kept as
// the unreduced fraction num / den.
__global__ void k_scores(const LineRow *lines, uint32_t trace, uint32_t n_lines, uint32_t rule, ScoreRow *out) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    const LineRow &r = lines[(uint64_t)trace * n_lines + l];
    const int64_t m = (int64_t)r.mallocs, f = (int64_t)r.frees;
    ScoreRow s;
    s.line = l; s.pad = 0; s.mallocs = r.mallocs; s.frees = r.frees;
    s.den = rule == 0 ? m - f + 2 : m + 2;
    s.num = s.den - (f + 1);
    out[l] = s;
}

struct StatRow {     // layout of scl_line_stat
    uint64_t n_growth, n_shrink;
    int64_t A, F, A_py, F_py, net;
    uint64_t copy_samples[2], copy_bytes[2];
};

// rows of traces trace0 .. trace0 + ntr - 1, trace-major (the range queries)
__global__ void k_stat_rows(const LineRow *lines, const unsigned long long *copies, uint32_t trace0, uint64_t nrows,
                            uint32_t n_lines, uint64_t Tc, StatRow *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nrows; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t g = (uint64_t)trace0 * n_lines + i;
        const LineRow r = lines[g];
        StatRow o;
        o.n_growth = r.n_growth; o.n_shrink = r.n_shrink;
        o.A = r.A; o.F = r.F; o.A_py = r.A_py; o.F_py = r.F_py;
        o.net = (int64_t)((uint64_t)r.A - (uint64_t)r.F);   // the sum of A - F over the samples
        o.copy_samples[0] = copies[2 * g]; o.copy_samples[1] = copies[2 * g + 1];
        o.copy_bytes[0] = o.copy_samples[0] * Tc; o.copy_bytes[1] = o.copy_samples[1] * Tc;   // Section 3.5
        out[i] = o;
    }
}

__global__ void k_score_rows(const LineRow *lines, uint32_t trace0, uint64_t nrows, uint32_t n_lines, uint32_t rule,
                             ScoreRow *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nrows; i += (uint64_t)gridDim.x * blockDim.x) {
        const LineRow &r = lines[(uint64_t)trace0 * n_lines + i];
        const int64_t m = (int64_t)r.mallocs, f = (int64_t)r.frees;
        ScoreRow s;
        s.line = (uint32_t)(i % n_lines); s.pad = 0; s.mallocs = r.mallocs; s.frees = r.frees;
        s.den = rule == 0 ? m - f + 2 : m + 2;
        s.num = s.den - (f + 1);
        out[i] = s;
    }
}

struct ReportRow {   // layout of scl_leak_report_row
    uint32_t line;
    uint8_t reported, likely, growth, pad;
    uint64_t mallocs, frees;
    int64_t num, den, rate_num;
    uint64_t rate_den;
};

// Section 3.4's report filter: likelihood above 95% and overall growth of at least 1%;
// leak rate = bytes allocated in the line's sample windows per event elapsed.
__global__ void k_report(const LineRow *lines, const DevTrace *traces, uint32_t trace, uint32_t n_lines,
                         uint32_t rule, int64_t F0, ReportRow *out) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    const LineRow &r = lines[(uint64_t)trace * n_lines + l];
    const DevTrace &t = traces[trace];
    const int64_t m = (int64_t)r.mallocs, f = (int64_t)r.frees;
    ReportRow o;
    o.line = l;
    o.pad = 0;
    o.mallocs = r.mallocs;
    o.frees = r.frees;
    o.den = rule == 0 ? m - f + 2 : m + 2;
    o.num = o.den - (f + 1);
    o.likely = (__int128)20 * o.num > (__int128)19 * o.den ? 1 : 0;
    o.growth = t.hwm > 0 && (__int128)100 * ((__int128)t.footprint - F0) >= (__int128)t.hwm ? 1 : 0;
    o.reported = o.likely && o.growth;
    o.rate_num = r.A;
    o.rate_den = t.n_events;
    out[l] = o;
}

// ---------------------------------------------------------------- line timeline
// Section 3.3's memory-trend feed for one line: (event index, footprint) of every retained
// sample whose line is `line`, in trace order.  A stream compaction of the sample log:
// per-block counts, one scan, then each block writes its matches at its offset.
constexpr int TLB = 4096;   // log entries per block

__global__ void __launch_bounds__(NT) k_tl_count(const Sample *log, uint64_t n, uint32_t line, uint64_t *cnt) {
    __shared__ int64_t sh[NT / 32 + 1];
    const uint64_t b0 = (uint64_t)blockIdx.x * TLB;
    int64_t c = 0;
    for (uint64_t i = b0 + threadIdx.x; i < n && i < b0 + TLB; i += NT) c += log[i].line == line;
    int64_t tot;
    (void)block_excl_sum(c, sh, &tot);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (uint64_t)tot;
}

__global__ void __launch_bounds__(NT) k_tl_scan(uint64_t *cnt, uint64_t nb, uint64_t *total) {
    __shared__ int64_t sh[NT / 32 + 1];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < nb; base += NT) {
        const uint64_t i = base + threadIdx.x;
        const int64_t x = i < nb ? (int64_t)cnt[i] : 0;
        int64_t tot;
        const int64_t ex = block_excl_sum(x, sh, &tot);
        if (i < nb) cnt[i] = carry + (uint64_t)ex;
        carry += (uint64_t)tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

// each thread takes TLB/NT consecutive entries, so matches keep their order
__global__ void __launch_bounds__(NT) k_tl_write(const Sample *log, uint64_t n, uint32_t line, const uint64_t *off,
                                                uint64_t cap, uint64_t *idx_out, int64_t *fp_out) {
    __shared__ int64_t sh[NT / 32 + 1];
    constexpr int PT = TLB / NT;
    const uint64_t i0 = (uint64_t)blockIdx.x * TLB + (uint64_t)threadIdx.x * PT;
    int64_t c = 0;
    for (int q = 0; q < PT; ++q) c += i0 + q < n && log[i0 + q].line == line;
    int64_t tot;
    uint64_t o = off[blockIdx.x] + (uint64_t)block_excl_sum(c, sh, &tot);
    for (int q = 0; q < PT; ++q) {
        if (i0 + q < n && log[i0 + q].line == line) {
            if (o < cap) { idx_out[o] = log[i0 + q].idx; fp_out[o] = log[i0 + q].footprint; }
            ++o;
        }
    }
}

cudaError_t launch_timeline(const Sample *log, uint64_t n, uint32_t line, void *scratch, uint64_t cap,
                            uint64_t *idx_out, int64_t *fp_out, cudaStream_t s) {
    const uint64_t nb = (n + TLB - 1) / TLB;
    uint64_t *cnt = static_cast<uint64_t *>(scratch);
    uint64_t *total = cnt + nb;
    cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess || !nb) return e;
    k_tl_count<<<(unsigned)nb, NT, 0, s>>>(log, n, line, cnt);
    k_tl_scan<<<1, NT, 0, s>>>(cnt, nb, total);
    k_tl_write<<<(unsigned)nb, NT, 0, s>>>(log, n, line, cnt, cap, idx_out, fp_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_report(const LineRow *lines, const DevTrace *traces, uint32_t trace, uint32_t n_lines,
                          uint32_t rule, int64_t F0, void *out, cudaStream_t s) {
    k_report<<<(n_lines + 255) / 256, 256, 0, s>>>(lines, traces, trace, n_lines, rule, F0,
                                                    static_cast<ReportRow *>(out));
    return cudaGetLastError();
}

cudaError_t launch_scan(const LaunchPost &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    // one block per trace: 1,024 threads when traces average hundreds of units
    const bool wide = a.nunits / a.nbt > NT;
    if (wide) k_scan<1024><<<a.nbt, 1024, 0, s>>>(a);
    else k_scan<NT><<<a.nbt, NT, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (wide) k_scan_window<1024><<<a.nbt, 1024, 0, s>>>(a);
    else k_scan_window<NT><<<a.nbt, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_compact(const LaunchPost &a, cudaStream_t s) {
    if (!a.ngroups) return cudaSuccess;
    const size_t smem = a.n_lines <= (uint32_t)SMEM_LINES_MAX ? (size_t)a.n_lines * HCOLS * 8 : 0;
    cudaError_t e = cudaFuncSetAttribute(k_compact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem ? smem : 1));
    if (e != cudaSuccess) return e;
    k_compact<<<a.ngroups, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mark(const LaunchPost &a, cudaStream_t s) {
    if (!a.nunits) return cudaSuccess;
    k_mark<<<(a.nunits + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_epi(const LaunchPost &a, cudaStream_t s) {
    if (!a.nunits) return cudaSuccess;
    k_epi<<<(a.nunits + 7) / 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_state(const LaunchPost &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    k_state<<<(a.nbt + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reset(DevTrace *traces, LineRow *lines, unsigned long long *copies, uint32_t trace0,
                         uint32_t ntr, uint32_t n_lines, int64_t F0, uint64_t phase, cudaStream_t s) {
    const uint64_t nw = (uint64_t)ntr * n_lines * (sizeof(LineRow) / 8 + 2);
    uint64_t blocks = (std::max<uint64_t>(nw, ntr) + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_reset<<<(int)blocks, 256, 0, s>>>(traces, lines, copies, trace0, ntr, n_lines, F0, phase);
    return cudaGetLastError();
}

cudaError_t launch_stat_rows(const LineRow *lines, const unsigned long long *copies, uint32_t trace0, uint64_t nrows,
                             uint32_t n_lines, uint64_t Tc, void *out, int num_sms, cudaStream_t s) {
    const int blocks = (int)std::min<uint64_t>((nrows + 255) / 256, (uint64_t)num_sms * 8);
    if (nrows) k_stat_rows<<<blocks, 256, 0, s>>>(lines, copies, trace0, nrows, n_lines, Tc, static_cast<StatRow *>(out));
    return cudaGetLastError();
}

cudaError_t launch_score_rows(const LineRow *lines, uint32_t trace0, uint64_t nrows, uint32_t n_lines, uint32_t rule,
                              void *out, int num_sms, cudaStream_t s) {
    const int blocks = (int)std::min<uint64_t>((nrows + 255) / 256, (uint64_t)num_sms * 8);
    if (nrows) k_score_rows<<<blocks, 256, 0, s>>>(lines, trace0, nrows, n_lines, rule, static_cast<ScoreRow *>(out));
    return cudaGetLastError();
}

cudaError_t launch_scores(const LineRow *lines, uint32_t trace, uint32_t n_lines, uint32_t rule, void *out,
                          cudaStream_t s) {
    k_scores<<<(n_lines + 255) / 256, 256, 0, s>>>(lines, trace, n_lines, rule, static_cast<ScoreRow *>(out));
    return cudaGetLastError();
}

}  // namespace scl
