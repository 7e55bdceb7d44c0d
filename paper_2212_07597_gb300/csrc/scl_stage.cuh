// scl_stage.cuh -- per-warp shared-memory ring fed by cp.async.bulk, and the warp
// walk loop over one unit's events built on it.
//
// A unit's columns are read in tiles of TILE events; NST tiles are in flight per
// warp.  Full tiles of 16-byte aligned columns go through one bulk copy per column
// completing on the stage's mbarrier; partial or unaligned tiles are copied by the
// lanes.  Every wait is bounded; whatever happens, no bulk copy is left in flight
// when the walk returns.
#pragma once
#include "scl_internal.cuh"

namespace scl {

template <bool ADDR>
struct Ring;

template <>
struct Ring<false> {
    int64_t d[NST][TILE];
    uint8_t p[NST][TILE];
    uint64_t bar[NST];
    __device__ __forceinline__ uint64_t *a(int) { return nullptr; }
};

template <>
struct Ring<true> {
    int64_t d[NST][TILE];
    uint64_t addr[NST][TILE];
    uint8_t p[NST][TILE];
    uint64_t bar[NST];
    __device__ __forceinline__ uint64_t *a(int s) { return addr[s]; }
};

template <bool ADDR>
__device__ __forceinline__ void ring_init(Ring<ADDR> &sm, int lane) {
    if (lane == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
}

// One step's events for this lane: E consecutive events at tile offset e0.
struct StepIn {
    int64_t d[E];
    uint64_t a[E];
    uint32_t pw;   // python flags, one byte per event
};

// Walk events [from, limit) of unit U (from and limit multiples of STEP, except
// limit may be the unit length).  step(in, rel0) is called per step of STEP events
// starting at unit offset rel0, events past `limit` read as delta 0 / flag 0 /
// address 0; it returns true to stop early.  Returns false if a wait timed out.
template <bool ADDR, class F>
__device__ bool ring_walk(Ring<ADDR> &sm, const Unit &U, uint64_t from, uint64_t limit, uint32_t &phase,
                          unsigned long long spin, ErrWord *err, int lane, F &&step) {
    if (limit <= from) return true;
    const uint64_t t_first = from / TILE;
    const uint64_t ntiles = (limit + TILE - 1) / TILE;
    const bool bulk = ((reinterpret_cast<uintptr_t>(U.delta) | reinterpret_cast<uintptr_t>(U.py) |
                        (ADDR ? reinterpret_cast<uintptr_t>(U.addr) : 0)) & 15u) == 0;
    uint32_t pending = 0;

    auto issue = [&](uint64_t t) {
        const int s = (int)(t % NST);
        const uint64_t t0 = t * TILE;
        const uint64_t cnt = limit - t0 < (uint64_t)TILE ? limit - t0 : (uint64_t)TILE;
        if (bulk && cnt == (uint64_t)TILE) {
            if (lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(&sm.bar[s], TILE * (ADDR ? 17 : 9));
                bulk_g2s(sm.d[s], U.delta + t0, TILE * 8, &sm.bar[s]);
                bulk_g2s(sm.p[s], U.py + t0, TILE, &sm.bar[s]);
                if (ADDR) bulk_g2s(sm.a(s), U.addr + t0, TILE * 8, &sm.bar[s]);
            }
            pending |= 1u << s;
        } else {
            for (uint32_t j = lane; j < (uint32_t)cnt; j += 32) {
                sm.d[s][j] = U.delta[t0 + j];
                sm.p[s][j] = U.py[t0 + j];
                if (ADDR) sm.a(s)[j] = U.addr[t0 + j];
            }
        }
    };

    for (uint64_t t = t_first; t < ntiles && t < t_first + NST; ++t) issue(t);
    bool ok = true;
    for (uint64_t t = t_first; t < ntiles; ++t) {
        const int s = (int)(t % NST);
        if (pending & (1u << s)) {
            if (!mbar_wait(&sm.bar[s], (phase >> s) & 1u, spin)) {
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
        const uint32_t b0 = (t == t_first) ? (uint32_t)(from - t0) : 0u;
        bool stop = false;
        for (uint32_t b = b0; b < cnt; b += STEP) {
            const uint32_t e0 = b + lane * E;
            StepIn in;
            const int rot = (lane >> 2) & 1;   // alternate 16-byte halves: conflict-free shared loads
            {
                const longlong2 *src = reinterpret_cast<const longlong2 *>(&sm.d[s][e0]);
                const longlong2 h0 = src[rot], h1 = src[rot ^ 1];
                const longlong2 x0 = rot ? h1 : h0, x1 = rot ? h0 : h1;
                in.d[0] = x0.x; in.d[1] = x0.y; in.d[2] = x1.x; in.d[3] = x1.y;
            }
            if (ADDR) {
                const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(&sm.a(s)[e0]);
                const ulonglong2 h0 = src[rot], h1 = src[rot ^ 1];
                const ulonglong2 x0 = rot ? h1 : h0, x1 = rot ? h0 : h1;
                in.a[0] = x0.x; in.a[1] = x0.y; in.a[2] = x1.x; in.a[3] = x1.y;
            } else {
                in.a[0] = in.a[1] = in.a[2] = in.a[3] = 0;
            }
            in.pw = *reinterpret_cast<const uint32_t *>(&sm.p[s][e0]);
            if (e0 + E > cnt) {
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (e0 + k >= cnt) { in.d[k] = 0; in.a[k] = 0; in.pw &= ~(0xffu << (8 * k)); }
            }
            if (step(in, (uint32_t)(t0 + b))) { stop = true; break; }
        }
        if (stop) break;
        __syncwarp();
        if (t + NST < ntiles) issue(t + NST);
    }
    // never leave a bulk copy in flight: one tile lands within microseconds, so the
    // drain has its own generous bound whatever the caller's spin limit
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

// Block-relative prefix sums of one step: lane-local inclusive prefixes lp, the
// exclusive prefix ex of this lane's first event, the step total, and the step's
// prefix extremes (all lanes).
struct StepPrefix {
    int64_t lp[E];
    int64_t ex, tot, qmax, qmin, lmax, lmin;
};

__device__ __forceinline__ void step_prefix(const StepIn &in, int lane, StepPrefix &sp) {
    sp.lp[0] = in.d[0];
#pragma unroll
    for (int k = 1; k < E; ++k) sp.lp[k] = sp.lp[k - 1] + in.d[k];
    sp.lmax = sp.lp[0];
    sp.lmin = sp.lp[0];
#pragma unroll
    for (int k = 1; k < E; ++k) {
        sp.lmax = sp.lp[k] > sp.lmax ? sp.lp[k] : sp.lmax;
        sp.lmin = sp.lp[k] < sp.lmin ? sp.lp[k] : sp.lmin;
    }
    const int64_t incl = warp_incl_scan(sp.lp[E - 1], lane);
    sp.ex = incl - sp.lp[E - 1];
    sp.tot = __shfl_sync(FULL, incl, 31);
    sp.lmax += sp.ex;
    sp.lmin += sp.ex;
}

__device__ __forceinline__ int64_t warp_min(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t t = __shfl_xor_sync(FULL, v, o);
        v = t < v ? t : v;
    }
    return v;
}

// First step position after `after` where counter base b + Q crosses +-T; -1 if none.
// Returns the position (lane*E + k) and the prefix Q there (warp-uniform).
__device__ __forceinline__ int first_cross(const StepPrefix &sp, int lane, int64_t b, int64_t T, int after,
                                           int64_t &Qr) {
    int fk = E;
#pragma unroll
    for (int k = E - 1; k >= 0; --k) {
        const int64_t v = b + sp.ex + sp.lp[k];
        if (lane * E + k > after && (v >= T || v <= -T)) fk = k;
    }
    const unsigned m = __ballot_sync(FULL, fk < E);
    if (!m) return -1;
    const int fl = __ffs(m) - 1;
    int64_t myQ = sp.ex;
#pragma unroll
    for (int k = 0; k < E; ++k)
        if (k == fk) myQ = sp.ex + sp.lp[k];
    const int kf = __shfl_sync(FULL, fk, fl);
    Qr = __shfl_sync(FULL, myQ, fl);
    return fl * E + kf;
}

}  // namespace scl
