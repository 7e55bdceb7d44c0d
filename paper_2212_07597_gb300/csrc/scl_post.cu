// scl_post.cu -- everything after the sampler walk:
//   k_scan     per trace, over its units: sample offsets, footprint at each unit
//              start (Section 3.3: the footprint is tracked at every event), and
//              the high-water mark entering each unit (Section 3.4).
//   k_compact  writes the final samples (Section 3.3 entries), attributes each to
//              the line of its triggering event, marks high-water crossings and
//              lists the tracked blocks (Section 3.4: "records the sampled
//              allocation"); per-line totals go through a shared-memory table.
//   k_scan2    the crossing tracked when each unit starts.
//   k_leak     the pointer comparison of every free against the block tracked at
//              that moment (Section 3.4), one bit per object.
//   k_epi      closes each object's trial at the next crossing: frees += reclaimed.
//   k_copy_*   the copy-volume sampler of Section 3.5: one sample per T_c bytes
//              copied, counted from the running byte count.
//   k_state    folds the batch into the trace's resident state.
#include "scl_internal.cuh"
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
__global__ void __launch_bounds__(NT) k_scan(LaunchPost a) {
    __shared__ int64_t sh[NT / 32 + 1];
    const int b = blockIdx.x;
    const BTrace B = a.bts[b];
    const DevTrace &st = a.traces[B.trace];
    int64_t ccnt = 0, cfp = st.footprint, chwm = st.hwm;
    for (uint32_t base = 0; base < B.nu; base += NT) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < B.nu;
        UnitRes *R = valid ? &a.ures[B.u0 + i] : nullptr;
        int64_t tc, tt, tm;
        const int64_t cnt = valid ? (int64_t)R->count : 0;
        const int64_t tot = valid ? R->total : 0;
        const int64_t ec = block_excl_sum(cnt, sh, &tc);
        const int64_t et = block_excl_sum(tot, sh, &tt);
        const int64_t fpb = cfp + et;
        const int64_t mg = (valid && R->has_growth) ? fpb + R->max_growth_P : INT64_MIN;
        const int64_t em = block_excl_max(mg, sh, &tm);
        if (valid) {
            R->sample_off = (uint64_t)(ccnt + ec);
            R->fp_base = fpb;
            R->hwm_in = em > chwm ? em : chwm;
        }
        ccnt += tc;
        cfp += tt;
        chwm = tm > chwm ? tm : chwm;
    }
    if (threadIdx.x == 0) {
        BTraceRes &BR = a.btres[b];
        BR.n_samples = (uint64_t)ccnt;
        BR.fp_end = cfp;
        BR.hwm_end = chwm;
        BR.last_cross_unit = -1;
        BR.pending_hit = 0;
    }
}

// ---------------------------------------------------------------- k_compact
constexpr int HCOLS = 8;   // n_growth, n_shrink, A, F, A_py, F_py, net, mallocs

__device__ __forceinline__ void row_add(unsigned long long *row, bool growth, int64_t A, int64_t F, int64_t Apy,
                                        int64_t Fpy, bool hwm) {
    atomicAdd(&row[growth ? 0 : 1], 1ull);
    atomicAdd(&row[2], (unsigned long long)A);
    atomicAdd(&row[3], (unsigned long long)F);
    if (Apy) atomicAdd(&row[4], (unsigned long long)Apy);
    if (Fpy) atomicAdd(&row[5], (unsigned long long)Fpy);
    atomicAdd(&row[6], (unsigned long long)(A - F));
    if (hwm) atomicAdd(&row[7], 1ull);
}

__global__ void __launch_bounds__(NT) k_compact(LaunchPost a) {
    extern __shared__ __align__(16) unsigned long long hist[];   // [n_lines][HCOLS] when it fits
    const CompactGroup G = a.groups[blockIdx.x];
    const bool use_smem = a.n_lines <= (uint32_t)SMEM_LINES_MAX;
    if (use_smem) {
        for (uint32_t i = threadIdx.x; i < a.n_lines * HCOLS; i += NT) hist[i] = 0;
        __syncthreads();
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((uint32_t)w < G.nu) {
        const uint32_t u = G.u0 + w;
        const Unit U = a.units[u];
        UnitRes &R = a.ures[u];
        const DevTrace &st = a.traces[U.trace];
        Sample *log = a.log ? a.log + (uint64_t)U.trace * a.log_cap : nullptr;
        const uint64_t log_base = st.n_samples + R.sample_off;
        LineRow *grow = a.lines + (uint64_t)U.trace * a.n_lines;
        const Rec *src = a.recs + U.rec0;
        const Rec *spec = a.recs + U.rec0 + U.src_cap;
        int64_t run = R.hwm_in;
        uint32_t ncross = 0;
        for (uint32_t j0 = 0; j0 < R.count; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool valid = j < R.count;
            Rec r;
            if (valid) r = j < R.src_used ? src[j] : spec[R.spec_skip + (j - R.src_used)];
            if (valid && r.rel >= U.len) {   // never index past the unit, whatever the records hold
                set_error(a.err, E_OVERFLOW, 8, u);
                valid = false;
            }
            if (!valid) { r.rel = 0; r.kind = 0; r.A = r.F = r.A_py = r.F_py = r.P = 0; }
            uint32_t line = valid ? U.line[r.rel] : 0;
            const uint8_t py = valid ? U.py[r.rel] : 0;
            bool line_ok = valid;
            if (valid && line >= a.n_lines) {
                set_error(a.err, E_RANGE, line, U.gidx0 + r.rel);
                line_ok = false;
                line = 0;
            }
            const int64_t fp = R.fp_base + r.P;
            const int64_t g = (valid && r.kind > 0) ? fp : INT64_MIN;
            const int64_t incl = warp_incl_max(g, lane);
            int64_t ex = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) ex = INT64_MIN;
            const int64_t before = ex > run ? ex : run;
            const bool hwm = valid && r.kind > 0 && fp > before;
            const int64_t wm = __shfl_sync(FULL, incl, 31);
            run = wm > run ? wm : run;
            if (valid && log && log_base + j < a.log_cap) {
                Sample s;
                s.idx = U.gidx0 + r.rel;
                s.A = r.A; s.F = r.F; s.A_py = r.A_py; s.F_py = r.F_py;
                s.footprint = fp;
                s.line = line;
                s.kind = (int8_t)r.kind;
                s.is_python = py ? 1 : 0;
                s.is_hwm = hwm ? 1 : 0;
                s.pad = 0;
                log[log_base + j] = s;
            }
            if (line_ok) {
                unsigned long long *row = use_smem ? &hist[line * HCOLS] : reinterpret_cast<unsigned long long *>(&grow[line]);
                if (use_smem) {
                    row_add(row, r.kind > 0, r.A, r.F, r.A_py, r.F_py, hwm);
                } else {
                    // global row: the first 7 fields of LineRow match the histogram columns; mallocs is field 11
                    atomicAdd(&row[r.kind > 0 ? 0 : 1], 1ull);
                    atomicAdd(&row[2], (unsigned long long)r.A);
                    atomicAdd(&row[3], (unsigned long long)r.F);
                    atomicAdd(&row[4], (unsigned long long)r.A_py);
                    atomicAdd(&row[5], (unsigned long long)r.F_py);
                    atomicAdd(&row[6], (unsigned long long)(r.A - r.F));
                    if (hwm) atomicAdd(&grow[line].mallocs, 1ull);
                }
            }
            const unsigned hm = __ballot_sync(FULL, hwm);
            if (hwm) {
                const uint32_t k = ncross + __popc(hm & ((1u << lane) - 1u));
                Cross c;
                c.rel = r.rel;
                c.line = line;
                c.addr = U.addr[r.rel];
                a.cross[U.rec0 + k] = c;
            }
            ncross += __popc(hm);
        }
        if (lane == 0) R.n_cross = ncross;
    }
    if (use_smem) {
        __syncthreads();
        // all units of a group belong to one trace
        const uint32_t tr = a.units[G.u0].trace;
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
            atomicAdd(reinterpret_cast<unsigned long long *>(&grow[l].net), h[6]);
            if (h[7]) atomicAdd(&grow[l].mallocs, h[7]);
        }
    }
}

// ---------------------------------------------------------------- k_scan2
__global__ void k_scan2(LaunchPost a) {
    const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= a.nbt) return;
    const BTrace B = a.bts[b];
    int64_t last = -1;
    for (uint32_t base = 0; base < B.nu; base += 32) {
        const uint32_t i = base + lane;
        const bool valid = i < B.nu;
        const bool has = valid && a.ures[B.u0 + i].n_cross > 0;
        const unsigned m = __ballot_sync(FULL, has);
        const unsigned below = m & ((1u << lane) - 1u);
        if (valid) a.ures[B.u0 + i].enter_unit = below ? (int64_t)(B.u0 + base + 31 - __clz(below)) : last;
        if (m) last = (int64_t)(B.u0 + base + 31 - __clz(m));
    }
    if (lane == 0) a.btres[b].last_cross_unit = last;
}

// ---------------------------------------------------------------- k_leak
// Section 3.4: "Every call to free then checks to see whether this object is
// ever reclaimed ... a pointer comparison".  The object tracked at event i is
// the crossing with the largest index below i (or, before the batch's first
// crossing, the block the trace was already tracking).
__global__ void __launch_bounds__(NT) k_leak(LaunchPost a) {
    extern __shared__ __align__(16) unsigned char lsm[];
    uint64_t *s_addr = reinterpret_cast<uint64_t *>(lsm);
    uint32_t *s_rel = reinterpret_cast<uint32_t *>(lsm + sizeof(uint64_t) * LEAK_TILE);
    __shared__ uint32_t s_ja, s_n;
    __shared__ uint64_t s_in_addr, s_in_slot;
    __shared__ int s_in_kind;   // 0 none, 1 crossing slot, 2 block tracked before the batch
    const LeakTile LT = a.ltiles[blockIdx.x];
    const Unit U = a.units[LT.unit];
    const UnitRes &R = a.ures[LT.unit];
    const uint64_t t0 = (uint64_t)LT.k * LEAK_TILE;
    const uint64_t t1 = t0 + LEAK_TILE < U.len ? t0 + LEAK_TILE : U.len;
    const Cross *cr = a.cross + U.rec0;
    if (threadIdx.x == 0) {
        const uint32_t n = R.n_cross;
        uint32_t lo = 0, hi = n;
        while (lo < hi) { uint32_t m = (lo + hi) >> 1; if (cr[m].rel < t0) lo = m + 1; else hi = m; }
        const uint32_t ja = lo;
        hi = n;
        while (lo < hi) { uint32_t m = (lo + hi) >> 1; if (cr[m].rel < t1) lo = m + 1; else hi = m; }
        s_ja = ja;
        s_n = lo - ja <= (uint32_t)LEAK_TILE ? lo - ja : (uint32_t)LEAK_TILE;
        if (ja > 0) {
            s_in_kind = 1; s_in_slot = U.rec0 + ja - 1; s_in_addr = cr[ja - 1].addr;
        } else if (R.enter_unit >= 0) {
            const Unit &Ue = a.units[R.enter_unit];
            const uint64_t slot = Ue.rec0 + a.ures[R.enter_unit].n_cross - 1;
            s_in_kind = 1; s_in_slot = slot; s_in_addr = a.cross[slot].addr;
        } else if (a.traces[U.trace].tracked_valid) {
            s_in_kind = 2; s_in_slot = 0; s_in_addr = a.traces[U.trace].tracked_addr;
        } else {
            s_in_kind = 0; s_in_slot = 0; s_in_addr = 0;
        }
    }
    __syncthreads();
    const uint32_t ja = s_ja, nc = s_n;
    for (uint32_t j = threadIdx.x; j < nc; j += NT) {
        s_rel[j] = cr[ja + j].rel;
        s_addr[j] = cr[ja + j].addr;
    }
    __syncthreads();
    const int in_kind = s_in_kind;
    if (in_kind == 0 && nc == 0) return;
    const uint64_t in_addr = s_in_addr, in_slot = s_in_slot;
    const uint32_t *bits = a.bits + U.bit0;
    const bool vec = (reinterpret_cast<uintptr_t>(U.addr) & 15u) == 0;
    constexpr int PAIRS = LEAK_TILE / (2 * NT);
    ulonglong2 ad[PAIRS];
    uint32_t wd[PAIRS];
#pragma unroll
    for (int r = 0; r < PAIRS; ++r) {
        const uint64_t i = t0 + 2ull * (r * NT + threadIdx.x);
        wd[r] = 0;
        if (i < t1) {
            wd[r] = bits[i >> 5];
            if (vec && i + 1 < t1) ad[r] = *reinterpret_cast<const ulonglong2 *>(U.addr + i);
            else { ad[r].x = U.addr[i]; ad[r].y = i + 1 < t1 ? U.addr[i + 1] : 0; }
        }
    }
#pragma unroll
    for (int r = 0; r < PAIRS; ++r) {
        const uint64_t i = t0 + 2ull * (r * NT + threadIdx.x);
        const uint32_t fb = (wd[r] >> (i & 31)) & 3u;
        if (!fb) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!((fb >> h) & 1u)) continue;
            const uint64_t e = i + h;
            const uint64_t av = h ? ad[r].y : ad[r].x;
            // last crossing of this tile strictly before e
            uint32_t lo = 0, hi = nc;
            while (lo < hi) { uint32_t m = (lo + hi) >> 1; if (s_rel[m] < e) lo = m + 1; else hi = m; }
            if (lo > 0) {
                if (s_addr[lo - 1] == av) a.recl[U.rec0 + ja + lo - 1] = 1;
            } else if (in_kind == 1) {
                if (in_addr == av) a.recl[in_slot] = 1;
            } else if (in_kind == 2) {
                if (in_addr == av) a.btres[U.bt].pending_hit = 1;
            }
        }
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
    const uint32_t n = a.ures[u].n_cross;
    const int64_t last_u = a.btres[U.bt].last_cross_unit;
    LineRow *grow = a.lines + (uint64_t)U.trace * a.n_lines;
    for (uint32_t j = lane; j < n; j += 32) {
        if ((int64_t)u == last_u && j == n - 1) continue;
        if (a.recl[U.rec0 + j]) atomicAdd(&grow[a.cross[U.rec0 + j].line].frees, 1ull);
    }
}

// ---------------------------------------------------------------- copy volume (Section 3.5)
__global__ void __launch_bounds__(NT) k_copy_sum(LaunchPost a) {
    __shared__ int64_t sh[NT / 32 + 1];
    const CopyTile C = a.ctiles[blockIdx.x];
    uint64_t s = 0;
    int ovf = 0;
    for (uint32_t j = threadIdx.x; j < C.len; j += NT) {
        const uint64_t x = C.size[j];
        ovf |= (s + x < s);
        s += x;
    }
    // sizes of one tile are summed in 64 bits; overflow is reported
    if (__syncthreads_or(ovf) && threadIdx.x == 0) set_error(a.err, E_OVERFLOW, 7, blockIdx.x);
    int64_t tot;
    (void)block_excl_sum((int64_t)s, sh, &tot);
    if (threadIdx.x == 0) a.ctile_sum[blockIdx.x] = (uint64_t)tot;
}

__global__ void __launch_bounds__(NT) k_copy_scan(LaunchPost a) {
    __shared__ int64_t sh[NT / 32 + 1];
    const BTrace B = a.bts[blockIdx.x];
    const uint64_t start = a.traces[B.trace].copy_counter;
    uint64_t carry = 0;
    for (uint32_t base = 0; base < B.nc; base += NT) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < B.nc;
        int64_t tot;
        const uint64_t v = valid ? a.ctile_sum[B.c0 + i] : 0;
        const int64_t ex = block_excl_sum((int64_t)v, sh, &tot);
        if (valid) a.ctile_sum[B.c0 + i] = start + carry + (uint64_t)ex;
        carry += (uint64_t)tot;
    }
    if (threadIdx.x == 0) a.btres[blockIdx.x].copy_total = carry;
}

constexpr int CPT = COPY_TILE / NT;   // memcpy events per thread

__global__ void __launch_bounds__(NT) k_copy_apply(LaunchPost a) {
    extern __shared__ __align__(16) unsigned long long chist[];   // [n_lines][4]: samples py0, py1, bytes py0, py1
    __shared__ int64_t sh[NT / 32 + 1];
    const CopyTile C = a.ctiles[blockIdx.x];
    const BTrace &B = a.bts[C.bt];
    const bool use_smem = a.n_lines <= (uint32_t)SMEM_LINES_MAX;
    if (use_smem) {
        for (uint32_t i = threadIdx.x; i < a.n_lines * 4; i += NT) chist[i] = 0;
        __syncthreads();
    }
    const uint64_t base = a.ctile_sum[blockIdx.x];   // copy counter before the tile's first event
    const uint64_t Tc = a.Tc;
    const uint32_t j0 = threadIdx.x * CPT;
    uint64_t loc = 0;
    for (int k = 0; k < CPT; ++k)
        if (j0 + k < C.len) loc += C.size[j0 + k];
    int64_t tot;
    const uint64_t ex = (uint64_t)block_excl_sum((int64_t)loc, sh, &tot);
    LineRow *grow = a.lines + (uint64_t)B.trace * a.n_lines;
    uint64_t run = base + ex;   // bytes counted before event j0
    uint64_t qprev = run / Tc;
    for (int k = 0; k < CPT; ++k) {
        const uint32_t j = j0 + k;
        if (j >= C.len) break;
        run += C.size[j];
        const uint64_t qn = run / Tc;
        const uint64_t q = qn - qprev;
        qprev = qn;
        if (!q) continue;
        const uint32_t line = C.line[j];
        if (line >= a.n_lines) { set_error(a.err, E_RANGE, line, j); continue; }
        const int f = C.py[j] ? 1 : 0;
        if (use_smem) {
            atomicAdd(&chist[line * 4 + f], q);
            atomicAdd(&chist[line * 4 + 2 + f], q * Tc);
        } else {
            atomicAdd(&grow[line].copy_samples[f], q);
            atomicAdd(&grow[line].copy_bytes[f], q * Tc);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (uint32_t l = threadIdx.x; l < a.n_lines; l += NT) {
            const unsigned long long *h = &chist[l * 4];
            if (h[0]) { atomicAdd(&grow[l].copy_samples[0], h[0]); atomicAdd(&grow[l].copy_bytes[0], h[2]); }
            if (h[1]) { atomicAdd(&grow[l].copy_samples[1], h[1]); atomicAdd(&grow[l].copy_bytes[1], h[3]); }
        }
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
        const UnitRes &RL = a.ures[B.u0 + B.nu - 1];
        st.c = RL.tx_c; st.A = RL.tx_A; st.F = RL.tx_F; st.A_py = RL.tx_Apy; st.F_py = RL.tx_Fpy;
        st.footprint = BR.fp_end;
        st.hwm = BR.hwm_end;
        if (BR.last_cross_unit >= 0) {
            if (st.tracked_valid && (st.tracked_reclaimed || BR.pending_hit))
                atomicAdd(&grow[st.tracked_line].frees, 1ull);
            const Unit &Ue = a.units[BR.last_cross_unit];
            const uint64_t slot = Ue.rec0 + a.ures[BR.last_cross_unit].n_cross - 1;
            const Cross c = a.cross[slot];
            st.tracked_valid = 1;
            st.tracked_addr = c.addr;
            st.tracked_line = c.line;
            st.tracked_idx = Ue.gidx0 + c.rel;
            st.tracked_reclaimed = a.recl[slot] ? 1 : 0;
        } else if (st.tracked_valid && BR.pending_hit) {
            st.tracked_reclaimed = 1;
        }
        st.n_events += B.n_ev;
        st.n_samples += BR.n_samples;
    }
    if (B.n_cp) {
        st.copy_counter = (st.copy_counter + BR.copy_total) % a.Tc;
        st.n_copies += B.n_cp;
    }
}

// ---------------------------------------------------------------- reset / scores
__global__ void k_reset(DevTrace *traces, LineRow *lines, uint32_t trace, uint32_t n_lines, int64_t F0,
                        uint64_t phase) {
    unsigned long long *rows = reinterpret_cast<unsigned long long *>(lines + (uint64_t)trace * n_lines);
    const uint64_t nw = (uint64_t)n_lines * (sizeof(LineRow) / 8);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nw; i += (uint64_t)gridDim.x * blockDim.x)
        rows[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevTrace t;
        t.c = t.A = t.F = t.A_py = t.F_py = 0;
        t.footprint = F0;
        t.hwm = F0;
        t.tracked_addr = t.tracked_idx = 0;
        t.tracked_line = t.tracked_valid = t.tracked_reclaimed = t.pad0 = 0;
        t.n_events = t.n_copies = t.n_samples = 0;
        t.copy_counter = phase;
        traces[trace] = t;
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

// ---------------------------------------------------------------- launchers
cudaError_t launch_scan(const LaunchPost &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    k_scan<<<a.nbt, NT, 0, s>>>(a);
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

cudaError_t launch_scan2(const LaunchPost &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    k_scan2<<<(a.nbt + 7) / 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_leak(const LaunchPost &a, cudaStream_t s) {
    if (!a.nltiles) return cudaSuccess;
    const size_t smem = (sizeof(uint64_t) + sizeof(uint32_t)) * LEAK_TILE;
    cudaError_t e = cudaFuncSetAttribute(k_leak, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_leak<<<a.nltiles, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_epi(const LaunchPost &a, cudaStream_t s) {
    if (!a.nunits) return cudaSuccess;
    k_epi<<<(a.nunits + 7) / 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_copy_sum(const LaunchPost &a, cudaStream_t s) {
    if (!a.nctiles) return cudaSuccess;
    k_copy_sum<<<a.nctiles, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_copy_scan(const LaunchPost &a, cudaStream_t s) {
    if (!a.nctiles) return cudaSuccess;
    k_copy_scan<<<a.nbt, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_copy_apply(const LaunchPost &a, cudaStream_t s) {
    if (!a.nctiles) return cudaSuccess;
    const size_t smem = a.n_lines <= (uint32_t)SMEM_LINES_MAX ? (size_t)a.n_lines * 4 * 8 : 0;
    cudaError_t e = cudaFuncSetAttribute(k_copy_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem ? smem : 1));
    if (e != cudaSuccess) return e;
    k_copy_apply<<<a.nctiles, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_state(const LaunchPost &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    k_state<<<(a.nbt + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reset(DevTrace *traces, LineRow *lines, uint32_t trace, uint32_t n_lines, int64_t F0,
                         uint64_t phase, cudaStream_t s) {
    const uint64_t nw = (uint64_t)n_lines * (sizeof(LineRow) / 8);
    int blocks = (int)((nw + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_reset<<<blocks, 256, 0, s>>>(traces, lines, trace, n_lines, F0, phase);
    return cudaGetLastError();
}

cudaError_t launch_scores(const LineRow *lines, uint32_t trace, uint32_t n_lines, uint32_t rule, void *out,
                          cudaStream_t s) {
    k_scores<<<(n_lines + 255) / 256, 256, 0, s>>>(lines, trace, n_lines, rule, static_cast<ScoreRow *>(out));
    return cudaGetLastError();
}

}  // namespace scl
