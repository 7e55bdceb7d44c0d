// scl_stage.cuh -- per-warp shared-memory ring fed by asynchronous copies, and the
// warp walk loop over one unit's events built on it.
//
// A unit's columns are read in tiles of TILE events; NST tiles are in flight per
// warp.  Full tiles of 16-byte aligned columns arrive as 16-byte cp.async copies issued
// by all lanes (each lane's copies then arrive on the stage's mbarrier); the 8-byte
// columns are written in the chunk-permuted layout of swz_el, so the lanes' 16-byte loads
// of their own EL events are free of bank conflicts.  Partial or unaligned tiles are
// copied by the lanes with plain loads into the same layout.  Every wait is bounded;
// whatever happens, no copy is left in flight when the walk returns.
#pragma once
#include "scl_internal.cuh"

namespace scl {

// Ring<ADDR, NS, TL, EL>: NS stages of TL events; EL events per lane per step.
template <bool ADDR, int NS = NST, int TL = TILE, int EL = E>
struct Ring;

// Every array starts on a 16-byte boundary (bulk-copy destinations and 16-byte shared
// loads and stores need it) and the struct size is a multiple of 128, so per-warp rings
// laid end to end stay aligned.
template <int NS, int TL, int EL>
struct alignas(128) Ring<false, NS, TL, EL> {   // deltas only
    static constexpr int kNS = NS, kTL = TL, kE = EL;
    alignas(16) int64_t d[NS][TL];
    alignas(16) int64_t xq[32 * EL];   // every lane's step prefixes, for the crossing search
    alignas(16) uint64_t bar[NS];
    __device__ __forceinline__ uint8_t *p(int) { return nullptr; }
    __device__ __forceinline__ uint64_t *a(int) { return nullptr; }
};

template <int NS, int TL, int EL>
struct alignas(128) Ring<true, NS, TL, EL> {    // deltas, addresses, python flags
    static constexpr int kNS = NS, kTL = TL, kE = EL;
    alignas(16) int64_t d[NS][TL];
    alignas(16) uint64_t addr[NS][TL];
    alignas(16) int64_t xq[32 * EL];
    alignas(16) uint8_t py[NS][TL];
    alignas(16) uint64_t bar[NS];
    __device__ __forceinline__ uint8_t *p(int s) { return py[s]; }
    __device__ __forceinline__ uint64_t *a(int s) { return addr[s]; }
};

template <class RingT>
__device__ __forceinline__ void ring_init(RingT &sm, int lane) {
    static_assert(sizeof(RingT) % 128 == 0, "rings laid end to end must stay aligned");
    static_assert(RingT::kTL % 16 == 0 && (RingT::kTL * 8) % 16 == 0, "bulk copies move 16-byte multiples");
    static_assert(RingT::kE == 8 || RingT::kE == 16, "the staged layout holds 8 or 16 events per lane");
    static_assert(RingT::kTL % (32 * RingT::kE) == 0, "a tile holds whole steps");
    if (lane == 0) {
        for (int s = 0; s < RingT::kNS; ++s) mbar_init(&sm.bar[s], 32);   // one arrival per lane
        fence_mbar_init();
    }
    __syncwarp();
}

// Invalidate a ring's barriers before its shared memory is used as another ring (the
// walk that used it has drained every copy).
template <class RingT>
__device__ __forceinline__ void ring_release(RingT &sm, int lane) {
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < RingT::kNS; ++s) mbar_inval(&sm.bar[s]);
    __syncwarp();
}

// One step's events for this lane: EL consecutive events at tile offset e0.
template <int EL>
struct StepIn {
    int64_t d[EL];
    uint64_t a[EL];
    uint64_t pw[(EL + 7) / 8];   // python flags, one byte per event
};

template <int EL>
__device__ __forceinline__ uint32_t py_of(const StepIn<EL> &in, int k) {
    return (uint32_t)(in.pw[k >> 3] >> (8 * (k & 7))) & 0xffu;
}

// The EL consecutive 64-bit values of tile element e0 (a multiple of EL: one row of the
// staged layout), as EL / 2 16-byte shared loads.
template <int EL, class V>
__device__ __forceinline__ void load_lane(const V *tile, uint32_t e0, V (&out)[EL]) {
    const int r = (int)(e0 / EL);
    const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(tile + EL * r);
#pragma unroll
    for (int q = 0; q < EL / 2; ++q) {
        const ulonglong2 v = src[swz_chunk_el<EL>(r, q)];
        out[2 * q] = (V)v.x;
        out[2 * q + 1] = (V)v.y;
    }
}

// Walk events [from, limit) of unit U (from and limit multiples of STEP, except
// limit may be the unit length).  step(in, rel0) is called per step of STEP events
// starting at unit offset rel0, events past `limit` read as delta 0 / flag 0 /
// address 0; it returns true to stop early.  Returns false if a wait timed out.
template <bool ADDR, class RingT, class F>
__device__ bool ring_walk(RingT &sm, const Unit &U, uint64_t from, uint64_t limit, uint32_t &phase,
                          unsigned long long spin, ErrWord *err, int lane, F &&step) {
    constexpr int NST = RingT::kNS, TILE = RingT::kTL, E = RingT::kE, STEP = 32 * E;
    if (limit <= from) return true;
    const uint64_t t_first = from / TILE;
    const uint64_t ntiles = (limit + TILE - 1) / TILE;
    const bool bulk = ((reinterpret_cast<uintptr_t>(U.delta) |
                        (ADDR ? reinterpret_cast<uintptr_t>(U.py) | reinterpret_cast<uintptr_t>(U.addr) : 0)) & 15u) == 0;
    uint32_t pending = 0;

    auto issue = [&](uint64_t t) {
        const int s = (int)(t % NST);
        const uint64_t t0 = t * TILE;
        const uint64_t cnt = limit - t0 < (uint64_t)TILE ? limit - t0 : (uint64_t)TILE;
        if (bulk && cnt == (uint64_t)TILE) {
            // 16-byte chunk j = lane + 32 i of an 8-byte column (elements 2j, 2j + 1) lands
            // at its permuted place swz_el(2j); eight consecutive lanes fill one 128-byte
            // line of shared memory
            const int64_t *gd = U.delta + t0 + 2 * lane;
#pragma unroll
            for (int i = 0; i < TILE / 64; ++i) cp_async16(&sm.d[s][swz_el<E>(2 * lane + 64 * i)], gd + 64 * i);
            if (ADDR) {
                const uint64_t *ga = U.addr + t0 + 2 * lane;
                uint64_t *sa = sm.a(s);
#pragma unroll
                for (int i = 0; i < TILE / 64; ++i) cp_async16(sa + swz_el<E>(2 * lane + 64 * i), ga + 64 * i);
            }
            if (ADDR)
                for (int j = lane; j < TILE / 16; j += 32) cp_async16(sm.p(s) + 16 * j, U.py + t0 + 16 * j);
            cp_async_arrive(&sm.bar[s]);
            pending |= 1u << s;
        } else {
            for (uint32_t j = lane; j < (uint32_t)cnt; j += 32) {
                const int js = swz_el<E>((int)j);
                sm.d[s][js] = U.delta[t0 + j];
                if (ADDR) {
                    sm.p(s)[j] = U.py[t0 + j];
                    sm.a(s)[js] = U.addr[t0 + j];
                }
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
            StepIn<E> in;
            load_lane<E>(sm.d[s], e0, in.d);
            if (ADDR) {
                load_lane<E>(sm.a(s), e0, in.a);
#pragma unroll
                for (int w = 0; w < (E + 7) / 8; ++w)
                    in.pw[w] = *reinterpret_cast<const unsigned long long *>(sm.p(s) + e0 + 8 * w);
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) in.a[k] = 0;
#pragma unroll
                for (int w = 0; w < (E + 7) / 8; ++w) in.pw[w] = 0;
            }
            if (e0 + E > cnt) {
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (e0 + k >= cnt) { in.d[k] = 0; in.a[k] = 0; in.pw[k >> 3] &= ~(0xffull << (8 * (k & 7))); }
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
// exclusive prefix ex of this lane's first event, the step total, and this lane's
// extremes lmax / lmin of the step prefix over its E events (ex included).  The
// lane's E step prefixes are also stored to xq[lane*E ..] for first_cross.
template <int EL>
struct StepPrefix {
    int64_t lp[EL];
    int64_t ex, tot, lmax, lmin;
};

template <int EL>
__device__ __forceinline__ void step_prefix(const StepIn<EL> &in, int lane, StepPrefix<EL> &sp, int64_t *xq) {
    sp.lp[0] = in.d[0];
#pragma unroll
    for (int k = 1; k < EL; ++k) sp.lp[k] = sp.lp[k - 1] + in.d[k];
    int64_t mx = sp.lp[0], mn = sp.lp[0];
#pragma unroll
    for (int k = 1; k < EL; ++k) {
        mx = sp.lp[k] > mx ? sp.lp[k] : mx;
        mn = sp.lp[k] < mn ? sp.lp[k] : mn;
    }
    const int64_t lt = sp.lp[EL - 1];
    const int64_t incl = warp_incl_scan(lt, lane);
    sp.ex = incl - lt;
    sp.tot = __shfl_sync(FULL, incl, 31);
    sp.lmax = mx + sp.ex;
    sp.lmin = mn + sp.ex;
    if (xq) {   // the staged layout (lane = row)
        longlong2 *dst = reinterpret_cast<longlong2 *>(xq + lane * EL);
#pragma unroll
        for (int q = 0; q < EL / 2; ++q)
            dst[swz_chunk_el<EL>(lane, q)] = make_longlong2(sp.ex + sp.lp[2 * q], sp.ex + sp.lp[2 * q + 1]);
        __syncwarp();
    }
}

// Warp-wide signed 64-bit min, as warp_max.
__device__ __forceinline__ int64_t warp_min(int64_t v) {
    const int hi = (int)(v >> 32);
    const int mh = __reduce_min_sync(FULL, hi);
    const unsigned ml = __reduce_min_sync(FULL, hi == mh ? (unsigned)v : 0xffffffffu);
    return (int64_t)(((uint64_t)(uint32_t)mh << 32) | ml);
}

// First step position after `after` where counter base b + Q crosses +-T; -1 if none.
// Returns the position (lane*EL + k) and the prefix Q there (warp-uniform).  Lanes are
// screened with their extremes; the first candidate lane's EL prefixes (published to xq
// by step_prefix) are then tested by EL lanes at once.
template <int EL>
__device__ __forceinline__ int first_cross(const StepPrefix<EL> &sp, const int64_t *xq, int lane, int64_t b,
                                           int64_t T, int after, int64_t &Qr) {
    const int64_t hi = T - b, lo = -T - b;   // cross iff Q >= hi or Q <= lo
    unsigned m = __ballot_sync(FULL, lane * EL + EL - 1 > after && (sp.lmax >= hi || sp.lmin <= lo));
    while (m) {
        const int fl = __ffs(m) - 1;
        m &= m - 1;
        const int64_t q = lane < EL ? xq[swz_el<EL>(fl * EL + lane)] : 0;
        const unsigned h = __ballot_sync(FULL, lane < EL && fl * EL + lane > after && (q >= hi || q <= lo));
        if (h) {
            const int kf = __ffs(h) - 1;
            Qr = __shfl_sync(FULL, q, kf);
            return fl * EL + kf;
        }
    }
    return -1;
}

// ---- the 32-bit form of a step, for the candidate counters of the sketch.
// When every delta of the step lies in [-2^22, 2^22) the step's prefixes lie in
// (-2^30, 2^30); with T <= 2^30 a counter lies in (-2^30, 2^30) as well, so a counter plus
// a prefix, T minus a counter and every other quantity of the crossing search fit in
// int32.  The result is the same as the 64-bit form's: it is the same arithmetic without
// overflow, in fewer integer instructions.
constexpr int64_t FIT32_T = 1ll << 30;   // largest T for the 32-bit form
constexpr int FIT32_SHIFT = 22;          // deltas in [-2^22, 2^22)

// This lane's deltas all lie in [-2^SHIFT, 2^SHIFT) (SHIFT < 31): each high word is the
// sign extension of its low word (the delta is an int32) and low + 2^SHIFT < 2^(SHIFT+1)
// as unsigned.
template <int SHIFT, int EL>
__device__ __forceinline__ bool deltas_within(const StepIn<EL> &in) {
    static_assert(SHIFT > 0 && SHIFT < 31, "a 32-bit range");
    uint32_t hx = 0, lv = 0;
#pragma unroll
    for (int k = 0; k < EL; ++k) {
        const uint32_t lo = (uint32_t)(uint64_t)in.d[k];
        const uint32_t hi = (uint32_t)((uint64_t)in.d[k] >> 32);
        hx |= hi ^ (uint32_t)((int32_t)lo >> 31);
        lv |= lo + (1u << SHIFT);
    }
    return hx == 0 && (lv >> (SHIFT + 1)) == 0;
}

template <int EL>
__device__ __forceinline__ bool step_fits32(const StepIn<EL> &in) {
    return deltas_within<FIT32_SHIFT>(in);
}

template <int EL>
struct StepPrefix32 {
    int32_t lp[EL];
    int32_t ex, tot, lmax, lmin;
};

// 32-bit rows of EL = 8 prefixes (32 bytes, two 16-byte chunks); chunk c of row r sits at
// chunk c ^ ((r >> 2) & 1), so a quarter warp's 16-byte stores touch eight bank groups.
__device__ __forceinline__ int swz32(int i) {
    const int r = i >> 3, k = i & 7;
    return (r << 3) | ((((k >> 2) ^ (r >> 2)) & 1) << 2) | (k & 3);
}

// Publish this lane's EL step prefixes (ex + lp) to xq for first_cross (staged layout).
template <int EL>
__device__ __forceinline__ void publish_prefix32(const StepPrefix32<EL> &sp, int lane, int32_t *xq) {
    static_assert(EL == 8, "32-bit rows hold 8 prefixes");
    int4 *dst = reinterpret_cast<int4 *>(xq + lane * EL);
    const int s = (lane >> 2) & 1;
    dst[s] = make_int4(sp.ex + sp.lp[0], sp.ex + sp.lp[1], sp.ex + sp.lp[2], sp.ex + sp.lp[3]);
    dst[s ^ 1] = make_int4(sp.ex + sp.lp[4], sp.ex + sp.lp[5], sp.ex + sp.lp[6], sp.ex + sp.lp[7]);
    __syncwarp();
}

// The 32-bit step prefixes; with xq != nullptr they are also published for first_cross
// (a caller that first tests whether the step crosses at all may publish them itself).
template <int EL>
__device__ __forceinline__ void step_prefix32(const StepIn<EL> &in, int lane, StepPrefix32<EL> &sp, int32_t *xq) {
    static_assert(EL == 8, "32-bit rows hold 8 prefixes");
    sp.lp[0] = (int32_t)in.d[0];
#pragma unroll
    for (int k = 1; k < EL; ++k) sp.lp[k] = sp.lp[k - 1] + (int32_t)in.d[k];
    int32_t mx = sp.lp[0], mn = sp.lp[0];
#pragma unroll
    for (int k = 1; k < EL; ++k) {
        mx = max(mx, sp.lp[k]);
        mn = min(mn, sp.lp[k]);
    }
    const int32_t lt = sp.lp[EL - 1];
    int32_t incl = lt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    sp.ex = incl - lt;
    sp.tot = __shfl_sync(FULL, incl, 31);
    sp.lmax = mx + sp.ex;
    sp.lmin = mn + sp.ex;
    if (xq) publish_prefix32(sp, lane, xq);
}

// first_cross on the 32-bit form (same contract)
template <int EL>
__device__ __forceinline__ int first_cross(const StepPrefix32<EL> &sp, const int32_t *xq, int lane, int32_t b,
                                           int32_t T, int after, int32_t &Qr) {
    const int32_t hi = T - b, lo = -T - b;
    unsigned m = __ballot_sync(FULL, lane * EL + EL - 1 > after && (sp.lmax >= hi || sp.lmin <= lo));
    while (m) {
        const int fl = __ffs(m) - 1;
        m &= m - 1;
        const int32_t q = lane < EL ? xq[swz32(fl * EL + lane)] : 0;
        const unsigned h = __ballot_sync(FULL, lane < EL && fl * EL + lane > after && (q >= hi || q <= lo));
        if (h) {
            const int kf = __ffs(h) - 1;
            Qr = __shfl_sync(FULL, q, kf);
            return fl * EL + kf;
        }
    }
    return -1;
}

}  // namespace scl
