// scl_copy.cuh -- the copy-volume sampler of Section 3.5, one warp per tile of memcpys.
//
// Per trace, the memcpy byte counts are summed into a running counter that starts at the
// trace's resident copy counter C0 (< T_c); memcpy j takes
//     q_j = floor((C0 + S_j) / T_c) - floor((C0 + S_(j-1)) / T_c)
// samples (S the inclusive prefix sum of the sizes), each worth T_c copied bytes, counted
// for its line and flag.  The trace's memcpys are cut into tiles of COPY_WTILE; a warp
// stages its tile's three columns in shared memory with one batch of asynchronous copies
// (13 bytes per memcpy, read once), sums it, publishes the sum, finds the counter entering
// its tile from its predecessors' published sums and prefixes (a decoupled look-back: a
// predecessor publishes its sum before it waits on anything, and it was taken from the work
// queue earlier, so every wait ends), publishes its own prefix, and applies the samples.
#pragma once
#include "scl_stage.cuh"

namespace scl {

constexpr uint32_t CS_AGG = 1u, CS_INCL = 2u;

struct CopyStatus {               // one per warp tile, cleared before each batch
    unsigned long long agg;       // bytes copied in the tile (valid from CS_AGG on)
    unsigned long long incl;      // counter after the tile: C0 + bytes up to its end (CS_INCL)
    unsigned int flag;
    unsigned int pad;
};

__device__ __forceinline__ unsigned long long add_carry(unsigned long long a, unsigned long long b, int &ovf) {
    const unsigned long long r = a + b;
    ovf |= r < a;
    return r;
}

// the value, then the flag with release semantics: a reader that acquires the flag sees it
__device__ __forceinline__ void cs_publish(CopyStatus *st, unsigned long long v, bool inclusive) {
    if (inclusive) st->incl = v; else st->agg = v;
    st_release(&st->flag, inclusive ? CS_INCL : CS_AGG);
}

// A warp's staging area for one tile: the sizes in rows of 32 (lane j reads row j) with the
// 16-byte chunks of row r XOR-permuted by r, so the lanes' reads spread over the banks;
// then the lines and flags, and the tile's counts of the COPY_HOT hottest-numbered lines
// (gathered here and added to the trace's rows once per tile).
constexpr int COPY_HOT = 64;
struct alignas(128) CopySmem {
    alignas(16) unsigned long long size[COPY_WTILE];
    alignas(16) uint32_t line[COPY_WTILE];
    alignas(16) uint8_t py[COPY_WTILE];
    alignas(16) unsigned long long hot[2 * COPY_HOT];   // [line][flag]
    alignas(16) uint64_t bar;
};

__device__ __forceinline__ void copy_smem_init(CopySmem &sm, int lane) {
    if (lane == 0) {
        mbar_init(&sm.bar, 32);   // one arrival per lane
        fence_mbar_init();
    }
    __syncwarp();
}

__device__ __forceinline__ void copy_smem_release(CopySmem &sm, int lane) {
    __syncwarp();
    if (lane == 0) mbar_inval(&sm.bar);
    __syncwarp();
}

// staged position of size i: row i / 32, its 16-byte chunk (i % 32) / 2 XOR (row % 16)
__device__ __forceinline__ unsigned long long &staged_size(CopySmem &sm, uint32_t i) {
    const uint32_t r = i >> 5, c = ((i & 31) >> 1) ^ (r & 15);
    return sm.size[(r << 5) | (c << 1) | (i & 1)];
}

// Tile `t` (CopyTile ct) of a trace whose tiles are t0 .. t0 + nc - 1, staged through sm
// (phase: the parity of sm.bar's next completion).  Returns false if a wait gave up.
// All 32 lanes call it.
__device__ bool copy_tile(CopySmem &sm, uint32_t &phase, const CopyTile &ct, uint32_t t, uint32_t t0,
                          CopyStatus *status, unsigned long long C0, unsigned long long Tc, uint32_t n_lines,
                          LineRow *grow, BTraceRes *bres, ErrWord *err, unsigned long long spin, int lane) {
    const uint32_t len = ct.len;
    // ---- stage the tile: a full tile of 16-byte aligned columns by 16-byte asynchronous
    // copies (all in flight at once), anything else by plain loads
    const bool vec = len == (uint32_t)COPY_WTILE &&
                     ((reinterpret_cast<uintptr_t>(ct.size) | reinterpret_cast<uintptr_t>(ct.line) |
                       reinterpret_cast<uintptr_t>(ct.py)) & 15u) == 0;
    if (vec) {
#pragma unroll
        for (int i = 0; i < COPY_WTILE / 64; ++i) {   // sizes: chunk c holds elements 2c, 2c + 1
            const uint32_t c = (uint32_t)lane + 32u * i;
            cp_async16(&staged_size(sm, 2 * c), ct.size + 2 * c);
        }
#pragma unroll
        for (int i = 0; i < COPY_WTILE / 128; ++i) {  // lines: chunk c holds elements 4c .. 4c + 3
            const uint32_t c = (uint32_t)lane + 32u * i;
            cp_async16(&sm.line[4 * c], ct.line + 4 * c);
        }
#pragma unroll
        for (int i = 0; i < COPY_WTILE / 512; ++i) {  // flags: chunk c holds elements 16c .. 16c + 15
            const uint32_t c = (uint32_t)lane + 32u * i;
            cp_async16(&sm.py[16 * c], ct.py + 16 * c);
        }
        for (int i = lane; i < 2 * COPY_HOT; i += 32) sm.hot[i] = 0ull;
        cp_async_arrive(&sm.bar);
        if (!mbar_wait(&sm.bar, phase, spin)) {
            // a 14 KB copy that never lands: report, and leave once it has (bounded)
            if (lane == 0) set_error(err, E_TIMEOUT, 21, t);
            const unsigned long long drain = spin > (1ull << 24) ? spin : (1ull << 24);
            mbar_wait(&sm.bar, phase, drain);
            phase ^= 1u;
            return false;
        }
        phase ^= 1u;
    } else {
        for (uint32_t i = lane; i < (uint32_t)COPY_WTILE; i += 32) {
            staged_size(sm, i) = i < len ? ct.size[i] : 0ull;
            sm.line[i] = i < len ? ct.line[i] : 0u;
            sm.py[i] = i < len ? ct.py[i] : (uint8_t)0;
        }
        for (int i = lane; i < 2 * COPY_HOT; i += 32) sm.hot[i] = 0ull;
        __syncwarp();
    }
    // ---- this lane's 32 consecutive memcpys: their byte count, and the tile's
    int ovf = 0;
    unsigned long long ls = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) ls = add_carry(ls, staged_size(sm, 32 * lane + k), ovf);
    unsigned long long x = ls;   // inclusive prefix over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x = add_carry(x, y, ovf);
    }
    const unsigned long long s = __shfl_sync(FULL, x, 31);
    // ---- the counter entering the tile
    unsigned long long base = 0;
    bool ok = true;
    if (t == t0) {
        base = C0;
        if (lane == 0) cs_publish(&status[t], add_carry(C0, s, ovf), true);
    } else {
        if (lane == 0) cs_publish(&status[t], s, false);
        unsigned long long acc = 0;
        int64_t p = (int64_t)t - 1;   // newest predecessor not yet accounted for
        while (true) {
            // lane j looks at tile p - j (tiles before the trace's first count as its start)
            const int64_t q = p - lane;
            unsigned int f = CS_INCL;
            unsigned long long v = 0;
            if (q >= (int64_t)t0) {
                unsigned long long it = 0;
                while ((f = ld_acquire(&status[q].flag)) == 0 && it < spin) ++it;
                if (f == CS_INCL) v = status[q].incl;
                else if (f == CS_AGG) v = status[q].agg;
            } else if (q == (int64_t)t0 - 1) {
                v = C0;
            }
            if (!__all_sync(FULL, f != 0)) {
                if (lane == 0) set_error(err, E_TIMEOUT, 20, t);
                ok = false;
                break;
            }
            // the nearest predecessor with a prefix ends the look-back; beyond the trace's
            // first tile the start counter stands in for one
            const unsigned done = __ballot_sync(FULL, f == CS_INCL);
            const int stop = done ? __ffs(done) - 1 : 32;
            unsigned long long w = lane <= stop ? v : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = add_carry(w, __shfl_xor_sync(FULL, w, o), ovf);
            acc = add_carry(acc, w, ovf);
            if (done) break;
            p -= 32;
        }
        base = acc;
        if (ok && lane == 0) cs_publish(&status[t], add_carry(base, s, ovf), true);
    }
    if (!ok) return false;
    // ---- samples at each of this lane's memcpys, from the counter before the first
    unsigned long long rem = add_carry(base, x - ls, ovf) % Tc;
    const bool small = Tc <= (1ull << 60);
    for (int k = 0; k < 32; ++k) {
        const uint32_t i = 32 * (uint32_t)lane + (uint32_t)k;
        const unsigned long long sz = staged_size(sm, i);
        unsigned long long qn;
        if (sz / 8 >= Tc || !small) {
            // a division; rem + (sz mod T_c) < 2 T_c fits, as T_c < 2^63
            qn = sz / Tc;
            const unsigned long long r2 = rem + sz % Tc;
            qn += r2 >= Tc;
            rem = r2 >= Tc ? r2 - Tc : r2;
        } else {
            // at most eight subtractions; rem + sz < 9 T_c <= 9 * 2^60 fits
            rem += sz;
            qn = 0;
            while (rem >= Tc) { rem -= Tc; ++qn; }
        }
        if (!qn) continue;
        const uint32_t l = sm.line[i];
        if (l >= n_lines) {
            set_error(err, E_RANGE, l, (unsigned long long)i);
            continue;
        }
        const int f = sm.py[i] ? 1 : 0;
        if (l < (uint32_t)COPY_HOT) atomicAdd(&sm.hot[2 * l + f], qn);
        else atomicAdd(&grow[l].copy_samples[f], qn);
    }
    __syncwarp();
    for (int i = lane; i < 2 * COPY_HOT; i += 32) {
        const unsigned long long v = sm.hot[i];
        if (v) atomicAdd(&grow[i >> 1].copy_samples[i & 1], v);
    }
    __syncwarp();   // the staging area is rewritten by the next tile
    // a carry means the trace's byte count passed 2^64: reported, the counts are invalid
    if (__any_sync(FULL, ovf) && lane == 0) set_error(err, E_OVERFLOW, 7, t);
    // the trace's last tile reports the bytes copied in the batch (for the state fold)
    if (lane == 0 && bres) bres->copy_total = add_carry(base, s, ovf) - C0;
    return true;
}

}  // namespace scl
