// scl_sketch.cu -- finding the true entry counter of every unit of the threshold
// sampler (Section 3.2: c <- c + delta; if |c| >= T: sample, c <- 0) in parallel.
//
// Two runs of this counter over the same events agree from any event where both
// have just reset.  The phase difference of two runs changes only by the small
// overshoots at their resets, so two arbitrary runs may take a long time to meet;
// but a run started near another one's counter meets it within a few resets.
//
// k_sketch  one warp per unit; lane k runs the counter from candidate entry value
//           c_k (32 values spread over (-T, T); lane 0 of a trace's first unit runs
//           the exact resident counter) through the whole unit, recording its exit
//           counter, its last reset, its first R reset positions and the largest
//           prefix at its growth resets from each of those on.  The warp advances
//           all lanes together, 128 events per step, from the step's prefix extremes.
// k_link    one warp per unit u after a trace's first: lane k runs the counter that
//           leaves candidate k of unit u-1 through unit u until it shares a reset
//           with one of unit u's candidates ("merge"), or never resets (transparent),
//           or reaches the unit's end.
// k_chain   one warp per trace: follows the true trajectory from the exact first
//           candidate through the link tables, walking a unit on demand only when no
//           precomputed link applies.
#include "scl_launch.h"
#include "scl_stage.cuh"

namespace scl {

__device__ __forceinline__ int64_t candidate_entry(int k, int64_t T) {
    // K values evenly spread over [-(T-1), T-1]
    const __int128 span = (__int128)(2 * (T - 1));
    return -(T - 1) + (int64_t)(span * k / (K - 1));
}

// ---------------------------------------------------------------- k_sketch
__global__ void __launch_bounds__(32 * 12) k_sketch(const Unit *__restrict__ units, int nunits, UnitSum *usum,
                                                    Cand *cand, const DevTrace *traces, int64_t T, unsigned *queue,
                                                    ErrWord *err, unsigned long long spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ring<false> &sm = reinterpret_cast<Ring<false> *>(smem_raw)[warp];
    ring_init(sm, lane);
    uint32_t phase = 0;
    while (true) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(queue, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const Unit U = units[u];
        Cand *C = cand + (size_t)u * K + lane;
        int64_t c = (U.first && lane == 0) ? traces[U.trace].c : candidate_entry(lane, T);
        uint32_t n = 0;
        int32_t last = -1;
        int64_t tmax = INT64_MIN;
        uint32_t targ = 0;
        int64_t P = 0, umax = INT64_MIN, umin = INT64_MAX;
        int64_t accA = 0, accApy = 0, accSpy = 0;
        auto step = [&](const StepIn &in, uint32_t rel0) -> bool {
            StepPrefix sp;
            step_prefix(in, lane, sp);
            const int64_t qmax = warp_max(sp.lmax), qmin = warp_min(sp.lmin);
            umax = P + qmax > umax ? P + qmax : umax;
            umin = P + qmin < umin ? P + qmin : umin;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int64_t x = in.d[k];
                const int64_t ps = x > 0 ? x : 0;
                accA += ps;
                if ((in.pw >> (8 * k)) & 0xffu) { accApy += ps; accSpy += x; }
            }
            unsigned m = __ballot_sync(FULL, c + qmax >= T || c + qmin <= -T);
            int64_t cnew = c + sp.tot;
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                int64_t b = __shfl_sync(FULL, c, k);
                int after = -1;
                while (true) {
                    int64_t Qr;
                    const int r = first_cross(sp, lane, b, T, after, Qr);
                    if (r < 0) break;
                    if (lane == k) {
                        const uint32_t pos = rel0 + (uint32_t)r;
                        const int64_t Pl = P + Qr;
                        const bool growth = b + Qr > 0;
                        if (n < (uint32_t)R) {
                            C->pos[n] = pos;
                            C->suf[n] = growth ? Pl : INT64_MIN;   // turned into suffix maxima at the end
                        } else if (growth && Pl > tmax) {
                            tmax = Pl;
                            targ = pos;
                        }
                        ++n;
                        last = (int32_t)pos;
                    }
                    b = -Qr;
                    after = r;
                }
                if (lane == k) cnew = b + sp.tot;
            }
            c = cnew;
            P += sp.tot;
            return false;
        };
        const bool ok = ring_walk<false>(sm, U, 0, U.len, phase, spin, err, lane, step);
        // suffix maxima over this candidate's first R growth resets (earliest position wins ties)
        const uint32_t nr = n < (uint32_t)R ? n : (uint32_t)R;
        int64_t best = tmax;
        uint32_t barg = targ;
        C->suf[nr] = best;
        C->arg[nr] = barg;
        for (int r = (int)nr - 1; r >= 0; --r) {
            const int64_t g = C->suf[r];
            if (g != INT64_MIN && g >= best) { best = g; barg = C->pos[r]; }
            C->suf[r] = best;
            C->arg[r] = barg;
        }
        for (uint32_t r = nr + 1; r <= (uint32_t)R; ++r) { C->suf[r] = INT64_MIN; C->arg[r] = 0; }
        C->c = c;
        C->last = last;
        C->n = n;
        const int64_t a = warp_sum(accA), ap = warp_sum(accApy), spy = warp_sum(accSpy);
        if (lane == 0) {
            UnitSum S;
            S.total = P; S.totA = a; S.totApy = ap; S.totSpy = spy; S.minQ = umin; S.maxQ = umax;
            usum[u] = S;
        }
        if (!ok) break;
    }
}

// ---------------------------------------------------------------- merge test
// Does unit position `pos` appear among the first R resets of some candidate of the
// unit?  Lane j searches candidate j's sorted list (in shared memory); returns the
// lowest such j (or -1) and the reset index there.
__device__ __forceinline__ int find_merge(const uint32_t (*lists)[R], int lane, uint32_t pos, uint32_t &idx) {
    const uint32_t *L = lists[lane];
    uint32_t lo = 0, hi = R;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (L[mid] < pos) lo = mid + 1; else hi = mid;
    }
    const bool hit = lo < (uint32_t)R && L[lo] == pos;
    const unsigned m = __ballot_sync(FULL, hit);
    if (!m) return -1;
    const int j = __ffs(m) - 1;
    idx = __shfl_sync(FULL, lo, j);
    return j;
}

__device__ __forceinline__ void load_lists(uint32_t (*lists)[R], const Cand *cu, int lane) {
    const uint32_t n = cu[lane].n;
    for (int i = 0; i < R; ++i) lists[lane][i] = (uint32_t)i < n ? cu[lane].pos[i] : 0xffffffffu;
    __syncwarp();
}

struct LinkSmem {
    Ring<false> ring;
    uint32_t lists[K][R];
};

// ---------------------------------------------------------------- k_link
__global__ void __launch_bounds__(32 * 8) k_link(const Unit *__restrict__ units, int nunits,
                                                 const UnitSum *__restrict__ usum, const Cand *__restrict__ cand,
                                                 Link *link, int64_t T, uint32_t cap, unsigned *queue, ErrWord *err,
                                                 unsigned long long spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    LinkSmem &sm = reinterpret_cast<LinkSmem *>(smem_raw)[warp];
    ring_init(sm.ring, lane);
    uint32_t phase = 0;
    while (true) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(queue, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const Unit U = units[u];
        if (U.first) continue;
        const UnitSum S = usum[u];
        load_lists(sm.lists, cand + (size_t)u * K, lane);
        Link Lk;
        Lk.kind = LINK_OPEN; Lk.j = 0; Lk.i = 0; Lk.n = 0; Lk.last = -1; Lk.garg = 0; Lk.gmax = INT64_MIN;
        int64_t c = cand[(size_t)(u - 1) * K + lane].c;
        Lk.c = c;
        bool active = true;
        if (c + S.maxQ < T && c + S.minQ > -T) { Lk.kind = LINK_TRANSPARENT; active = false; }
        int64_t P = 0;
        const uint64_t lim = (cap && cap < U.len) ? cap : U.len;
        auto step = [&](const StepIn &in, uint32_t rel0) -> bool {
            StepPrefix sp;
            step_prefix(in, lane, sp);
            const int64_t qmax = warp_max(sp.lmax), qmin = warp_min(sp.lmin);
            unsigned m = __ballot_sync(FULL, active && (c + qmax >= T || c + qmin <= -T));
            int64_t cnew = c + sp.tot;
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                int64_t b = __shfl_sync(FULL, c, k);
                int after = -1;
                bool merged = false;
                while (true) {
                    int64_t Qr;
                    const int r = first_cross(sp, lane, b, T, after, Qr);
                    if (r < 0) break;
                    const uint32_t pos = rel0 + (uint32_t)r;
                    uint32_t idx = 0;
                    const int j = find_merge(sm.lists, lane, pos, idx);
                    if (lane == k) {
                        const int64_t Pl = P + Qr;
                        if (b + Qr > 0 && Pl > Lk.gmax) { Lk.gmax = Pl; Lk.garg = pos; }
                        ++Lk.n;
                        Lk.last = (int32_t)pos;
                        if (j >= 0) { Lk.kind = LINK_MERGED; Lk.j = (uint32_t)j; Lk.i = idx; active = false; }
                    }
                    if (j >= 0) { merged = true; break; }
                    b = -Qr;
                    after = r;
                }
                if (lane == k && !merged) cnew = b + sp.tot;
            }
            c = cnew;
            P += sp.tot;
            return __ballot_sync(FULL, active) == 0;
        };
        const bool ok = ring_walk<false>(sm.ring, U, 0, lim, phase, spin, err, lane, step);
        if (active) {
            if (lim == U.len) { Lk.kind = LINK_END; Lk.c = c; }
            else Lk.kind = LINK_OPEN;
        }
        link[(size_t)u * K + lane] = Lk;
        if (!ok) break;
    }
}

// ---------------------------------------------------------------- k_chain
// One warp per trace of the batch.  Phase A follows the true state through the
// units -- "candidate k" (the true trajectory ends the previous unit on candidate
// k's) or "explicit c" (the exact counter, when no candidate carries it) -- reading
// the link tables from shared memory; it walks a unit itself only when no
// precomputed link applies.  Phase B then fills UnitTrue for all units in parallel.
constexpr int CHAIN_CHUNK = 1024;   // units per shared-memory chunk

// entering mode of a unit, as recorded by phase A
constexpr uint32_t MODE_WALKED = 0x100u;     // | k: candidate k entering, walked here (uwalk)
constexpr uint32_t MODE_EXPLICIT = 0x200u;   // explicit counter entering, no reset in the unit
constexpr uint32_t MODE_EXPLICIT_WALKED = 0x300u;   // explicit counter entering, walked here (uwalk)

struct ChainSmem {
    uint16_t lk[CHAIN_CHUNK][K];    // link kind << 8 | j
    uint32_t lists[K][R];
};

// Walk unit U from counter c until a reset shared with one of its candidates
// (LINK_MERGED) or the unit's end (LINK_END).  Plain coalesced loads; one warp.
__device__ Link walk_on_demand(const Unit &U, const uint32_t (*lists)[R], int64_t c, int64_t T, int lane) {
    Link Lw;
    Lw.kind = LINK_END; Lw.j = 0; Lw.i = 0; Lw.n = 0; Lw.last = -1; Lw.garg = 0; Lw.gmax = INT64_MIN;
    int64_t P = 0;
    for (uint64_t s0 = 0; s0 < U.len; s0 += STEP) {
        StepIn in;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const uint64_t e = s0 + lane * E + k;
            in.d[k] = e < U.len ? U.delta[e] : 0;
            in.a[k] = 0;
        }
        in.pw = 0;
        StepPrefix sp;
        step_prefix(in, lane, sp);
        int64_t bb = c;
        int after = -1;
        while (true) {
            int64_t Qr;
            const int r = first_cross(sp, lane, bb, T, after, Qr);
            if (r < 0) break;
            const uint32_t pos = (uint32_t)(s0 + r);
            const int64_t Pl = P + Qr;
            if (bb + Qr > 0 && Pl > Lw.gmax) { Lw.gmax = Pl; Lw.garg = pos; }
            ++Lw.n;
            Lw.last = (int32_t)pos;
            uint32_t idx = 0;
            const int jj = find_merge(lists, lane, pos, idx);
            if (jj >= 0) {
                Lw.kind = LINK_MERGED; Lw.j = (uint32_t)jj; Lw.i = idx; Lw.c = 0;
                return Lw;
            }
            bb = -Qr;
            after = r;
        }
        c = bb + sp.tot;
        P += sp.tot;
    }
    Lw.c = c;
    return Lw;
}

__global__ void __launch_bounds__(32) k_chain(const Unit *__restrict__ units, const BTrace *__restrict__ bts, int nbt,
                                             const UnitSum *__restrict__ usum, const Cand *__restrict__ cand,
                                             const Link *__restrict__ link, Link *uwalk, UnitTrue *utrue,
                                             uint32_t *umode, int64_t *uexp, const DevTrace *traces, int64_t T) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ChainSmem &sm = *reinterpret_cast<ChainSmem *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    if (b >= nbt) return;
    const BTrace B = bts[b];
    if (B.nu == 0) return;
    // ---- phase A
    uint32_t mode = 0;   // entering state: candidate `mode` of the previous unit, or 0xff = explicit
    int64_t ec = 0;      // the exact counter when explicit
    for (uint32_t c0 = 1; c0 < B.nu; c0 += CHAIN_CHUNK) {
        const uint32_t cn = B.nu - c0 < (uint32_t)CHAIN_CHUNK ? B.nu - c0 : (uint32_t)CHAIN_CHUNK;
        for (uint32_t i = 0; i < cn; ++i) {
            const Link &L = link[(size_t)(B.u0 + c0 + i) * K + lane];
            sm.lk[i][lane] = (uint16_t)((L.kind << 8) | (L.j & 0xff));
        }
        __syncwarp();
        for (uint32_t i = 0; i < cn; ++i) {
            const uint32_t u = B.u0 + c0 + i;
            if (mode != 0xffu) {
                const uint16_t e = sm.lk[i][mode];
                const uint32_t kind = e >> 8;
                if (kind == LINK_MERGED) {
                    if (lane == 0) umode[u] = mode;
                    mode = e & 0xff;
                    continue;
                }
                const int64_t cin = cand[(size_t)(u - 1) * K + mode].c;
                if (kind == LINK_TRANSPARENT) {
                    if (lane == 0) umode[u] = mode;
                    ec = cin + usum[u].total;
                    mode = 0xffu;
                    continue;
                }
                if (kind == LINK_END) {
                    if (lane == 0) umode[u] = mode;
                    ec = link[(size_t)u * K + mode].c;
                    mode = 0xffu;
                    continue;
                }
                // LINK_OPEN: walk from the exact entering counter
                load_lists(sm.lists, cand + (size_t)u * K, lane);
                const Link Lw = walk_on_demand(units[u], sm.lists, cin, T, lane);
                if (lane == 0) { uwalk[u] = Lw; umode[u] = MODE_WALKED | mode; }
                if (Lw.kind == LINK_MERGED) mode = Lw.j;
                else { ec = Lw.c; mode = 0xffu; }
                __syncwarp();
                continue;
            }
            // explicit entering counter
            const UnitSum S = usum[u];
            if (lane == 0) uexp[u] = ec;
            if (ec + S.maxQ < T && ec + S.minQ > -T) {
                if (lane == 0) umode[u] = MODE_EXPLICIT;
                ec += S.total;
                continue;
            }
            load_lists(sm.lists, cand + (size_t)u * K, lane);
            const Link Lw = walk_on_demand(units[u], sm.lists, ec, T, lane);
            if (lane == 0) { uwalk[u] = Lw; umode[u] = MODE_EXPLICIT_WALKED; }
            if (Lw.kind == LINK_MERGED) mode = Lw.j;
            else ec = Lw.c;
            __syncwarp();
        }
        __syncwarp();
    }
    __syncwarp();
    // ---- phase B
    const int64_t c_first = traces[B.trace].c;
    for (uint32_t i = lane; i < B.nu; i += 32) {
        const uint32_t u = B.u0 + i;
        const Unit U = units[u];
        UnitTrue Tu;
        Tu.entry_last = -1;
        if (i == 0) {   // lane 0 of the first unit ran the exact resident counter
            const Cand &C0 = cand[(size_t)u * K];
            Tu.entry_c = c_first;
            Tu.gmax = C0.suf[0]; Tu.garg = C0.arg[0]; Tu.n = C0.n;
            Tu.exit_c = C0.c;
            Tu.exit_last = C0.last >= 0 ? (int64_t)(U.gidx0 + (uint32_t)C0.last) : -1;
            utrue[u] = Tu;
            continue;
        }
        const uint32_t md = umode[u];
        Link L;
        if (md < (uint32_t)K) {
            L = link[(size_t)u * K + md];
            Tu.entry_c = cand[(size_t)(u - 1) * K + md].c;
            if (L.kind == LINK_TRANSPARENT) L.c = Tu.entry_c + usum[u].total;
        } else if ((md & 0xf00u) == MODE_WALKED) {
            L = uwalk[u];
            Tu.entry_c = cand[(size_t)(u - 1) * K + (md & 0xffu)].c;
        } else if (md == MODE_EXPLICIT) {
            Tu.entry_c = uexp[u];
            L.kind = LINK_TRANSPARENT; L.n = 0; L.last = -1; L.gmax = INT64_MIN; L.garg = 0;
            L.c = uexp[u] + usum[u].total;
        } else {
            L = uwalk[u];
            Tu.entry_c = uexp[u];
        }
        if (L.kind == LINK_TRANSPARENT) {
            Tu.n = 0; Tu.gmax = INT64_MIN; Tu.garg = 0; Tu.exit_c = L.c; Tu.exit_last = -1;
        } else if (L.kind == LINK_MERGED) {
            const Cand &Cj = cand[(size_t)u * K + L.j];
            Tu.n = L.n + (Cj.n - (L.i + 1));
            const int64_t sg = Cj.suf[L.i + 1];
            if (L.gmax != INT64_MIN && L.gmax >= sg) { Tu.gmax = L.gmax; Tu.garg = L.garg; }
            else { Tu.gmax = sg; Tu.garg = Cj.arg[L.i + 1]; }
            Tu.exit_c = Cj.c;
            Tu.exit_last = (int64_t)(U.gidx0 + (uint32_t)Cj.last);
        } else {   // LINK_END: this trajectory shared no reset with a candidate
            Tu.n = L.n; Tu.gmax = L.gmax; Tu.garg = L.garg; Tu.exit_c = L.c;
            Tu.exit_last = L.last >= 0 ? (int64_t)(U.gidx0 + (uint32_t)L.last) : -1;
        }
        utrue[u] = Tu;
    }
}

// ---------------------------------------------------------------- launchers
size_t sketch_smem_per_warp() { return sizeof(Ring<false>); }
size_t link_smem_per_warp() { return sizeof(LinkSmem); }

cudaError_t launch_sketch(const LaunchSketch &a, cudaStream_t s) {
    const size_t smem = sizeof(Ring<false>) * a.warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sketch<<<a.blocks, 32 * a.warps_per_block, smem, s>>>(a.units, a.nunits, a.usum, a.cand, a.traces, a.T,
                                                            a.queue, a.err, a.spin);
    return cudaGetLastError();
}

cudaError_t launch_link(const LaunchSketch &a, cudaStream_t s) {
    const int wpb = 4;
    const size_t smem = sizeof(LinkSmem) * wpb;
    cudaError_t e = cudaFuncSetAttribute(k_link, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_link, 32 * wpb, smem);
    int blocks = bps * a.num_sms;
    const int need = (a.nunits + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k_link<<<blocks, 32 * wpb, smem, s>>>(a.units, a.nunits, a.usum, a.cand, a.link, a.T, a.link_cap,
                                          a.queue + 1, a.err, a.spin);
    return cudaGetLastError();
}

cudaError_t launch_chain(const LaunchSketch &a, cudaStream_t s) {
    if (!a.nbt) return cudaSuccess;
    const size_t smem = sizeof(ChainSmem);
    cudaError_t e = cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<<<a.nbt, 32, smem, s>>>(a.units, a.bts, a.nbt, a.usum, a.cand, a.link, a.uwalk, a.utrue, a.umode,
                                    a.uexp, a.traces, a.T);
    return cudaGetLastError();
}

int sketch_occupancy(int warps_per_block, int *blocks_per_sm) {
    const size_t smem = sizeof(Ring<false>) * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sketch, 32 * warps_per_block, smem);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace scl
