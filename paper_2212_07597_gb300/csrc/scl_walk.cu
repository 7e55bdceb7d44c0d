// scl_walk.cu -- the threshold sampler of Section 3.2 as a chunked speculative scan.
//
// Section 3.2: counters A (bytes allocated) and F (bytes freed) are kept; once
// |A - F| >= T a sample is taken and the counters are reset.  Per event this is
// c <- c + delta; if |c| >= T: sample, c <- 0.  The window totals A, F and their
// Python parts (Section 3.3) ride along and are reported with each sample.
//
// One warp walks one unit.  A step covers STEP = 32*E consecutive events, E per
// lane.  The step's block-relative prefix sums Q_j are formed with one warp scan;
// the step holds no sample iff c + max Q < T and c + min Q > -T, a test that needs
// only each lane's own extremes and one ballot, so the serial dependency per step
// is a few instructions.  Steps that do hold a sample locate it with a ballot,
// close the window with three warp sums, and continue from c = 0 after it.
//
// Event columns reach shared memory through cp.async.bulk copies (16-byte aligned
// tiles, NST-deep ring per warp, mbarrier completion with a bounded wait).
#include "scl_internal.cuh"
#include "scl_launch.h"

namespace scl {

struct WalkSmem {
    int64_t d[NST][TILE];
    uint8_t p[NST][TILE];
    uint64_t bar[NST];
};

struct Walker {
    int lane;
    int64_t T;
    int64_t c;                    // counter A - F of the open window (warp-uniform)
    int64_t P;                    // unit-local prefix sum up to the last walked event
    int64_t accA, accApy, accSpy; // this lane's share of the open window: sum of mallocs,
                                  // python mallocs, python deltas (F follows as A - c)
    Rec *out;
    uint32_t cap, n;
    uint32_t *pub;                // progress counter published for lookahead walkers (may be null)
    // merge detection against a unit's own records
    const Rec *mspec;
    const uint32_t *mpub;
    uint32_t mknown, mq;
    int mmode;                    // 0 none, 1 records still being published, 2 complete
    int merged;
    uint32_t merge_src, merge_spec;

    __device__ __forceinline__ void init(int lane_, int64_t T_) {
        lane = lane_; T = T_; c = 0; P = 0; accA = accApy = accSpy = 0;
        out = nullptr; cap = 0; n = 0; pub = nullptr;
        mspec = nullptr; mpub = nullptr; mknown = 0; mq = 0; mmode = 0;
        merged = 0; merge_src = merge_spec = 0;
    }

    __device__ __forceinline__ void emit(uint32_t rel, int64_t cr, int64_t A, int64_t Apy, int64_t Spy,
                                         int64_t Plocal) {
        if (lane == 0 && n < cap) {
            Rec r;
            r.rel = rel;
            r.kind = cr > 0 ? 1 : -1;
            r.A = A;
            r.F = A - cr;
            r.A_py = Apy;
            r.F_py = Apy - Spy;
            r.P = Plocal;
            out[n] = r;
            if (pub) st_release(pub, n + 1);
        }
        ++n;
        if (mmode) {
            int hit = 0;
            if (lane == 0) {
                uint32_t known = mmode == 1 ? ld_acquire(mpub) : mknown;
                while (mq < known && *(volatile const uint32_t *)&mspec[mq].rel < rel) ++mq;
                if (mq < known && *(volatile const uint32_t *)&mspec[mq].rel == rel) hit = 1;
            }
            hit = __shfl_sync(FULL, hit, 0);
            mq = __shfl_sync(FULL, mq, 0);
            if (hit) { merged = 1; merge_src = n - 1; merge_spec = mq; }
        }
    }

    __device__ __forceinline__ void accumulate(const int64_t (&d)[E], uint32_t pw, int after) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if (lane * E + k > after) {
                int64_t x = d[k];
                int64_t pos = x > 0 ? x : 0;
                accA += pos;
                if ((pw >> (8 * k)) & 0xffu) { accApy += pos; accSpy += x; }
            }
        }
    }

    // one step of STEP events whose first event is at unit offset rel0; returns true to stop
    __device__ __forceinline__ bool step(const int64_t (&d)[E], uint32_t pw, uint32_t rel0) {
        int64_t lp[E];
        lp[0] = d[0];
#pragma unroll
        for (int k = 1; k < E; ++k) lp[k] = lp[k - 1] + d[k];
        int64_t lmax = lp[0], lmin = lp[0];
#pragma unroll
        for (int k = 1; k < E; ++k) { lmax = lp[k] > lmax ? lp[k] : lmax; lmin = lp[k] < lmin ? lp[k] : lmin; }
        const int64_t incl = warp_incl_scan(lp[E - 1], lane);
        const int64_t ex = incl - lp[E - 1];
        const int64_t tot = __shfl_sync(FULL, incl, 31);
        const int64_t hi = c + ex + lmax, lo = c + ex + lmin;
        if (__ballot_sync(FULL, hi >= T || lo <= -T) == 0) {
            accumulate(d, pw, -1);
            c += tot;
            P += tot;
            return false;
        }
        // at least one sample in this step: take them in order
        int64_t b = c;   // counter at event j of the step is b + Q_j until the next sample
        int last = -1;   // step position of the last sample taken
        while (true) {
            int fk = E;
#pragma unroll
            for (int k = E - 1; k >= 0; --k) {
                int64_t v = b + ex + lp[k];
                if (lane * E + k > last && (v >= T || v <= -T)) fk = k;
            }
            unsigned m = __ballot_sync(FULL, fk < E);
            if (!m) break;
            int fl = __ffs(m) - 1;
            int64_t myQ = ex;
#pragma unroll
            for (int k = 0; k < E; ++k) if (k == fk) myQ = ex + lp[k];
            const int kf = __shfl_sync(FULL, fk, fl);
            const int64_t Qr = __shfl_sync(FULL, myQ, fl);
            const int r = fl * E + kf;
            const int64_t cr = b + Qr;
            int64_t sA = accA, sApy = accApy, sSpy = accSpy;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                int pos = lane * E + k;
                if (pos > last && pos <= r) {
                    int64_t x = d[k];
                    int64_t ps = x > 0 ? x : 0;
                    sA += ps;
                    if ((pw >> (8 * k)) & 0xffu) { sApy += ps; sSpy += x; }
                }
            }
            const int64_t wA = warp_sum(sA), wApy = warp_sum(sApy), wSpy = warp_sum(sSpy);
            emit(rel0 + (uint32_t)r, cr, wA, wApy, wSpy, P + Qr);
            accA = accApy = accSpy = 0;
            b = -Qr;
            last = r;
            if (merged) return true;
        }
        accumulate(d, pw, last);
        c = b + tot;
        P += tot;
        return false;
    }
};

// Walk events [0, limit) of unit U.  bits != null: also record which events are
// frees (one bit per event, for the leak pass).  Returns false if a wait timed out.
__device__ bool walk(const Unit &U, uint64_t limit, Walker &w, WalkSmem &sm, uint32_t &phase, uint32_t *bits,
                     unsigned long long spin, ErrWord *err) {
    const int lane = w.lane;
    if (limit == 0) return true;
    const uint64_t ntiles = (limit + TILE - 1) / TILE;
    const bool bulk = ((reinterpret_cast<uintptr_t>(U.delta) | reinterpret_cast<uintptr_t>(U.py)) & 15u) == 0;
    uint32_t pending = 0;

    auto issue = [&](uint64_t t) {
        const int s = (int)(t % NST);
        const uint64_t t0 = t * TILE;
        const uint64_t cnt = limit - t0 < (uint64_t)TILE ? limit - t0 : (uint64_t)TILE;
        if (bulk && cnt == (uint64_t)TILE) {
            if (lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(&sm.bar[s], TILE * 9);
                bulk_g2s(sm.d[s], U.delta + t0, TILE * 8, &sm.bar[s]);
                bulk_g2s(sm.p[s], U.py + t0, TILE, &sm.bar[s]);
            }
            pending |= 1u << s;
        } else {
            for (uint32_t j = lane; j < (uint32_t)cnt; j += 32) {
                sm.d[s][j] = U.delta[t0 + j];
                sm.p[s][j] = U.py[t0 + j];
            }
        }
    };

    for (uint64_t t = 0; t < ntiles && t < (uint64_t)NST; ++t) issue(t);
    bool ok = true;
    for (uint64_t t = 0; t < ntiles; ++t) {
        const int s = (int)(t % NST);
        if (pending & (1u << s)) {
            if (!mbar_wait(&sm.bar[s], (phase >> s) & 1u, spin)) {
                // leave the stage pending: the drain below still waits for its copy
                if (lane == 0) set_error(err, E_TIMEOUT, 1, (unsigned long long)t);
                ok = false;
                break;
            }
            phase ^= 1u << s;
            pending &= ~(1u << s);
        }
        __syncwarp();
        const uint64_t t0 = t * TILE;
        const uint32_t cnt = (uint32_t)(limit - t0 < (uint64_t)TILE ? limit - t0 : (uint64_t)TILE);
        bool stop = false;
        for (uint32_t b = 0; b < cnt; b += STEP) {
            const uint32_t e0 = b + lane * E;
            const int rot = (lane >> 2) & 1;   // alternate 16-byte halves: conflict-free shared loads
            const longlong2 *src = reinterpret_cast<const longlong2 *>(&sm.d[s][e0]);
            const longlong2 h0 = src[rot], h1 = src[rot ^ 1];
            const longlong2 x0 = rot ? h1 : h0, x1 = rot ? h0 : h1;
            int64_t d[E] = {x0.x, x0.y, x1.x, x1.y};
            uint32_t pw = *reinterpret_cast<const uint32_t *>(&sm.p[s][e0]);
            if (e0 + E > cnt) {
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (e0 + k >= cnt) { d[k] = 0; pw &= ~(0xffu << (8 * k)); }
            }
            if (bits) {
                uint32_t nib = 0;
#pragma unroll
                for (int k = 0; k < E; ++k) nib |= (d[k] < 0 ? 1u : 0u) << k;
                uint32_t word = nib << (4 * (lane & 7));
                word |= __shfl_xor_sync(FULL, word, 1);
                word |= __shfl_xor_sync(FULL, word, 2);
                word |= __shfl_xor_sync(FULL, word, 4);
                const uint64_t widx = (t0 + b) / 32 + (lane >> 3);
                if ((lane & 7) == 0 && widx * 32 < limit) bits[widx] = word;
            }
            if (w.step(d, pw, (uint32_t)(t0 + b))) { stop = true; break; }
        }
        if (stop) break;
        __syncwarp();
        if (t + NST < ntiles) issue(t + NST);
    }
    // never leave a bulk copy in flight: a copy of one tile lands within microseconds,
    // so the drain uses its own generous bound whatever the caller's spin limit
    const unsigned long long drain = spin > (1ull << 24) ? spin : (1ull << 24);
    for (int s = 0; s < NST; ++s) {
        if (pending & (1u << s)) {
            const bool got = mbar_wait(&sm.bar[s], (phase >> s) & 1u, drain);
            phase ^= 1u << s;
            if (!got) {
                if (lane == 0) set_error(err, E_TIMEOUT, 2, 0);
                ok = false;
            }
        }
    }
    __syncwarp();
    return ok;
}

__device__ __forceinline__ void load_entry(Walker &w, int64_t c, int64_t A, int64_t F, int64_t Apy, int64_t Fpy) {
    (void)F;
    w.c = c;
    if (w.lane == 0) { w.accA = A; w.accApy = Apy; w.accSpy = Apy - Fpy; }
}

__device__ __forceinline__ void exit_state(Walker &w, int64_t &c, int64_t &A, int64_t &F, int64_t &Apy,
                                           int64_t &Fpy) {
    const int64_t a = warp_sum(w.accA), ap = warp_sum(w.accApy), sp = warp_sum(w.accSpy);
    c = w.c; A = a; F = a - w.c; Apy = ap; Fpy = ap - sp;
}

__global__ void __launch_bounds__(32 * 16) k_walk(const Unit *__restrict__ units, int nunits, UnitRes *ures,
                                                  Rec *recs, uint32_t *pub, uint32_t *bits,
                                                  const DevTrace *traces, int64_t T, uint32_t ext_cap,
                                                  unsigned *queue, ErrWord *err, unsigned long long spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkSmem &sm = reinterpret_cast<WalkSmem *>(smem_raw)[warp];
    if (lane == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    while (true) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(queue, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const Unit U = units[u];
        Walker w;
        w.init(lane, T);
        if (U.first) {
            const DevTrace &st = traces[U.trace];
            load_entry(w, st.c, st.A, st.F, st.A_py, st.F_py);
        }
        w.out = recs + U.rec0 + U.src_cap;
        w.cap = U.spec_cap;
        w.pub = pub + u;
        bool ok = walk(U, U.len, w, sm, phase, bits + U.bit0, spin, err);
        int64_t c, A, F, Apy, Fpy;
        exit_state(w, c, A, F, Apy, Fpy);
        if (lane == 0) {
            UnitRes &R = ures[u];
            R.total = w.P;
            R.ex_c = c; R.ex_A = A; R.ex_F = F; R.ex_Apy = Apy; R.ex_Fpy = Fpy;
            R.n_spec = w.n;
            if (w.n > U.spec_cap) set_error(err, E_OVERFLOW, 3, (unsigned long long)u);
        }
        if (!ok) break;
        if (!U.last) {
            // lookahead: continue into the next unit of the trace from this unit's exit state
            const Unit V = units[u + 1];
            Walker x;
            x.init(lane, T);
            load_entry(x, c, A, F, Apy, Fpy);
            x.out = recs + V.rec0;
            x.cap = V.src_cap;
            x.mspec = recs + V.rec0 + V.src_cap;
            x.mpub = pub + u + 1;
            x.mmode = 1;
            const uint64_t lim = (ext_cap && ext_cap < V.len) ? ext_cap : V.len;
            ok = walk(V, lim, x, sm, phase, nullptr, spin, err);
            if (lane == 0) {
                ures[u + 1].n_src = x.n < V.src_cap ? x.n : V.src_cap;
                if (x.n > V.src_cap) set_error(err, E_OVERFLOW, 4, (unsigned long long)(u + 1));
            }
            if (!ok) break;
        }
    }
}

// ---------------------------------------------------------------- resolution

// count / largest growth prefix of a unit's final records: src[0, src_used) then spec[spec_skip, n_spec)
__device__ void finalize_unit(const Unit &U, UnitRes &R, const Rec *recs, int lane) {
    const Rec *src = recs + U.rec0;
    const Rec *spec = recs + U.rec0 + U.src_cap;
    const uint32_t n_spec = R.n_spec < U.spec_cap ? R.n_spec : U.spec_cap;
    const uint32_t count = R.src_used + (n_spec - R.spec_skip);
    int64_t best = INT64_MIN;
    int has = 0;
    for (uint32_t j = lane; j < count; j += 32) {
        const Rec &r = j < R.src_used ? src[j] : spec[R.spec_skip + (j - R.src_used)];
        if (r.kind > 0) { has = 1; best = r.P > best ? r.P : best; }
    }
    best = warp_max(best);
    has = __any_sync(FULL, has);
    if (lane == 0) { R.count = count; R.has_growth = has; R.max_growth_P = best; }
}

__device__ __forceinline__ bool find_rel(const Rec *spec, uint32_t n, uint32_t rel, uint32_t &pos) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (spec[mid].rel < rel) lo = mid + 1; else hi = mid;
    }
    pos = lo;
    return lo < n && spec[lo].rel == rel;
}

__global__ void k_resolve(const Unit *__restrict__ units, int nunits, UnitRes *ures, const Rec *recs) {
    const int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= nunits) return;
    const Unit U = units[u];
    UnitRes &R = ures[u];
    const uint32_t n_spec = R.n_spec < U.spec_cap ? R.n_spec : U.spec_cap;
    if (U.first) {
        if (lane == 0) {
            R.src_used = 0; R.spec_skip = 0; R.broken = 0;
            R.tx_c = R.ex_c; R.tx_A = R.ex_A; R.tx_F = R.ex_F; R.tx_Apy = R.ex_Apy; R.tx_Fpy = R.ex_Fpy;
        }
        __syncwarp();
        finalize_unit(U, R, recs, lane);
        return;
    }
    const Rec *src = recs + U.rec0;
    const Rec *spec = recs + U.rec0 + U.src_cap;
    const uint32_t n_src = R.n_src;
    int found = 0;
    uint32_t js = 0, qs = 0;
    for (uint32_t base = 0; base < n_src && !found; base += 32) {
        const uint32_t j = base + lane;
        uint32_t q = 0;
        const bool f = j < n_src && find_rel(spec, n_spec, src[j].rel, q);
        const unsigned m = __ballot_sync(FULL, f);
        if (m) {
            const int l = __ffs(m) - 1;
            found = 1;
            js = base + l;
            qs = __shfl_sync(FULL, q, l);
        }
    }
    if (lane == 0) {
        if (found) {
            R.src_used = js + 1; R.spec_skip = qs + 1; R.broken = 0;
            R.tx_c = R.ex_c; R.tx_A = R.ex_A; R.tx_F = R.ex_F; R.tx_Apy = R.ex_Apy; R.tx_Fpy = R.ex_Fpy;
        } else {
            R.broken = 1;
        }
    }
    __syncwarp();
    if (found) finalize_unit(U, R, recs, lane);
}

// One warp per trace of the batch: re-walk, in order, every unit whose lookahead
// never met its own walk, carrying the true counter until it meets one.
__global__ void __launch_bounds__(32) k_fallback(const Unit *__restrict__ units, const BTrace *__restrict__ bts,
                                                 int nbt, UnitRes *ures, Rec *recs, int64_t T, ErrWord *err,
                                                 unsigned long long spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WalkSmem &sm = *reinterpret_cast<WalkSmem *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    if (b >= nbt) return;
    const BTrace B = bts[b];
    if (lane == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    const uint32_t uend = B.u0 + B.nu;
    uint32_t u = B.u0;
    while (true) {
        // next broken unit at or after u
        uint32_t nb = uend;
        for (uint32_t base = u; base < uend; base += 32) {
            const uint32_t v = base + lane;
            const unsigned m = __ballot_sync(FULL, v < uend && ures[v].broken);
            if (m) { nb = base + __ffs(m) - 1; break; }
        }
        if (nb >= uend) break;
        // the unit before nb ends on its own walk's trajectory, so its exit is the true entry of nb
        Walker w;
        w.init(lane, T);
        {
            const UnitRes &Rp = ures[nb - 1];
            load_entry(w, Rp.tx_c, Rp.tx_A, Rp.tx_F, Rp.tx_Apy, Rp.tx_Fpy);
        }
        uint32_t v = nb;
        bool ok = true;
        for (; v < uend; ++v) {
            const Unit V = units[v];
            UnitRes &R = ures[v];
            w.P = 0;
            w.n = 0;
            w.out = recs + V.rec0;
            w.cap = V.src_cap;
            w.mspec = recs + V.rec0 + V.src_cap;
            w.mknown = R.n_spec < V.spec_cap ? R.n_spec : V.spec_cap;
            w.mq = 0;
            w.mmode = 2;
            w.merged = 0;
            ok = walk(V, V.len, w, sm, phase, nullptr, spin, err);
            if (!ok) break;
            if (w.n > V.src_cap && lane == 0) set_error(err, E_OVERFLOW, 5, v);
            if (w.merged) {
                if (lane == 0) {
                    const uint32_t nn = w.n < V.src_cap ? w.n : V.src_cap;
                    R.n_src = nn;
                    R.src_used = w.merge_src + 1 < nn ? w.merge_src + 1 : nn;
                    R.spec_skip = w.merge_spec + 1;
                    R.broken = 0;
                    R.tx_c = R.ex_c; R.tx_A = R.ex_A; R.tx_F = R.ex_F; R.tx_Apy = R.ex_Apy; R.tx_Fpy = R.ex_Fpy;
                }
                __syncwarp();
                finalize_unit(V, R, recs, lane);
                break;
            }
            int64_t c, A, F, Apy, Fpy;
            exit_state(w, c, A, F, Apy, Fpy);
            if (lane == 0) {
                const uint32_t nn = w.n < V.src_cap ? w.n : V.src_cap;
                R.n_src = nn; R.src_used = nn; R.spec_skip = R.n_spec < V.spec_cap ? R.n_spec : V.spec_cap;
                R.broken = 0;
                R.tx_c = c; R.tx_A = A; R.tx_F = F; R.tx_Apy = Apy; R.tx_Fpy = Fpy;
            }
            __syncwarp();
            finalize_unit(V, R, recs, lane);
            // continue into the next unit with the carried counter; accumulators stay in the lanes
        }
        if (!ok) break;
        u = v + 1;
        if (u >= uend) break;
    }
}

// ---------------------------------------------------------------- self test of the bounded wait
// Waits on an mbarrier that nothing arrives at: the wait must give up after
// `limit` polls and report E_TIMEOUT through the error word, leaving the context usable.
__global__ void k_wait_selftest(ErrWord *err, unsigned long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (!mbar_wait(&bar, 0, limit) && threadIdx.x == 0) set_error(err, E_TIMEOUT, 9, limit);
}

cudaError_t launch_wait_selftest(ErrWord *err, unsigned long long limit, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(err, limit);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- launchers

size_t walk_smem_per_warp() { return sizeof(WalkSmem); }

cudaError_t launch_walk(const LaunchWalk &a, cudaStream_t s) {
    const size_t smem = sizeof(WalkSmem) * a.warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_walk<<<a.blocks, 32 * a.warps_per_block, smem, s>>>(a.units, a.nunits, a.ures, a.recs, a.pub, a.bits,
                                                          a.traces, a.T, a.ext_cap, a.queue, a.err, a.spin);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const Unit *units, int nunits, UnitRes *ures, const Rec *recs, cudaStream_t s) {
    if (nunits == 0) return cudaSuccess;
    const int wpb = 8;
    k_resolve<<<(nunits + wpb - 1) / wpb, 32 * wpb, 0, s>>>(units, nunits, ures, recs);
    return cudaGetLastError();
}

cudaError_t launch_fallback(const Unit *units, const BTrace *bts, int nbt, UnitRes *ures, Rec *recs, int64_t T,
                            ErrWord *err, unsigned long long spin, cudaStream_t s) {
    if (nbt == 0) return cudaSuccess;
    const size_t smem = sizeof(WalkSmem);
    cudaError_t e = cudaFuncSetAttribute(k_fallback, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fallback<<<nbt, 32, smem, s>>>(units, bts, nbt, ures, recs, T, err, spin);
    return cudaGetLastError();
}

int walk_occupancy(int warps_per_block, int *blocks_per_sm) {
    const size_t smem = sizeof(WalkSmem) * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk, 32 * warps_per_block, smem);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace scl
