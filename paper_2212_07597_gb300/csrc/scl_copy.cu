// scl_copy.cu -- the copy-volume sampler of Section 3.5, one thread block per tile of memcpys.
//
// Per trace, the memcpy byte counts are summed into a running counter that starts at the
// trace's resident copy counter C0 (< T_c); memcpy j takes
//     q_j = floor((C0 + S_j) / T_c) - floor((C0 + S_(j-1)) / T_c)
// samples (S the inclusive prefix sum of the sizes), each worth T_c copied bytes, counted
// for its line and flag.  Only the counter modulo T_c matters for q_j: with r_j the counter
// before memcpy j (below T_c), q_j = floor((r_j + size_j) / T_c), and r_(j+1) is the
// remainder.  So every sum here is kept modulo T_c (two residues add to less than 2^64, as
// T_c < 2^63) and no division is needed unless a size is at least 8 T_c.
//
// A trace's memcpys are cut into tiles of COPY_PASS_TILE, taken by blocks in rounds over the
// traces (every trace's first tile, then every second one, ...).  A block loads its tile
// into registers (each thread CB_PER consecutive memcpys; 13 bytes per memcpy, read once),
// sums it, publishes the sum, finds the counter entering the tile from its predecessors'
// published sums and prefixes (a decoupled look-back: a predecessor publishes its sum
// before it waits on anything, and it took its ticket earlier, so every wait ends; waits
// are bounded), publishes its own prefix, and applies the samples; counts of lines below
// CB_HOT gather in shared memory and reach the trace's counts when the block moves to
// another trace's tile (a long trace's consecutive tiles share one flush).
#include <algorithm>
#include <cstddef>

#include "scl_launch.h"
#include "scl_stage.cuh"

namespace scl {

constexpr int CB_THREADS = 256;
constexpr int CB_BLOCKS = 3;                     // resident blocks per SM (the register budget)
static_assert(COPY_PASS_TILE <= 4096 && COPY_PASS_TILE % (4 * CB_THREADS) == 0, "tile shape");
constexpr int CB_PER = COPY_PASS_TILE / CB_THREADS;   // memcpys per thread (16)
constexpr uint32_t CB_HOT = 1024;                // lines counted in shared memory per tile
constexpr uint32_t CB_FLUSH = 1024;              // tiles of one trace a block counts before a flush

// The look-back state of a tile is one 64-bit word, cleared before each batch, so a reader
// gets flag and value in one load: 0 = nothing yet; 1 .. 2^63 - 1 = the tile's bytes modulo
// T_c, plus one (its aggregate); 2^63 | v = the counter after the tile, modulo T_c (its
// inclusive prefix).  Every residue is below T_c < 2^63, so both forms fit.
constexpr unsigned long long CS_INCL = 1ull << 63;

struct alignas(16) CopyTask {     // the tile a block works on, written by thread 0 (16-byte stores)
    CopyTile ct;
    int valid;
};

struct alignas(16) CopyBlockSmem {
    uint32_t hot[2 * CB_HOT];     // [line][flag] sample counts of the trace's tiles since the last flush
    unsigned long long wsum[CB_THREADS / 32];
    unsigned long long base;
    CopyTask task[2];             // the current tile and the next
    int ok;
};

// A warp's 512 memcpys of a tile, staged by coalesced 16-byte asynchronous copies (each
// lane's own 16 memcpys then read from shared memory).  Sizes sit in the chunk-permuted
// rows of swz_el<16> (128-byte rows, one per lane); lines in 64-byte rows with chunk c of
// row r at c ^ ((r >> 1) & 3); flags in 16-byte rows.  A quarter warp reading one chunk per
// lane then touches eight distinct bank groups in every column.
struct alignas(16) CopyStage {
    unsigned long long size[32 * CB_PER];
    uint32_t line[32 * CB_PER];
    uint8_t py[32 * CB_PER];
};
constexpr size_t COPY_STAGE_BYTES = sizeof(CopyStage) * (CB_THREADS / 32);

__device__ __forceinline__ int line_chunk(int r, int c) { return 4 * r + (c ^ ((r >> 1) & 3)); }

static_assert(offsetof(CopyBlockSmem, task) % 16 == 0 && sizeof(CopyTask) % 16 == 0 && offsetof(CopyTask, ct) == 0,
              "the tile records are copied with 16-byte stores");

// (a + b) mod T_c for a, b < T_c <= 2^63
__device__ __forceinline__ unsigned long long madd(unsigned long long a, unsigned long long b, unsigned long long Tc) {
    const unsigned long long s = a + b;
    return s >= Tc ? s - Tc : s;
}

// a tile's aggregate or inclusive prefix (the word carries everything a reader needs, so
// relaxed ordering suffices)
__device__ __forceinline__ void cs_publish(unsigned long long *st, unsigned long long v, bool inclusive) {
    const unsigned long long w = inclusive ? (CS_INCL | v) : v + 1;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(st), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long cs_load(const unsigned long long *st) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(st) : "memory");
    return w;
}

// the tile of ticket `it` (its description is one 48-byte record of the plan)
__device__ __forceinline__ void copy_job(const LaunchCopy &a, unsigned it, CopyTask &k) {
    k.valid = it < (unsigned)a.nctiles;
    if (!k.valid) return;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.ctiles + it);
    uint4 *dst = reinterpret_cast<uint4 *>(&k.ct);
    const uint4 x = __ldg(src), y = __ldg(src + 1), z = __ldg(src + 2);
    dst[0] = x; dst[1] = y; dst[2] = z;
}

__global__ void __launch_bounds__(CB_THREADS, CB_BLOCKS) k_copy(const LaunchCopy a) {
    __shared__ CopyBlockSmem sm;
    extern __shared__ __align__(128) unsigned char stage_raw[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    CopyStage &stg = reinterpret_cast<CopyStage *>(stage_raw)[w];
    unsigned long long *status = static_cast<unsigned long long *>(a.cstatus);
    const unsigned long long Tc = a.Tc;
    const bool small = Tc <= (1ull << 60);
    const unsigned long long Tc2 = 2 * Tc, Tc4 = 4 * Tc, Tc8 = 8 * Tc;   // (small: no overflow)
    const uint32_t hot = a.n_lines < CB_HOT ? a.n_lines : CB_HOT;
    for (uint32_t i = tid; i < 2 * hot; i += CB_THREADS) sm.hot[i] = 0u;
    // the table holds counts of trace `held` from `nheld` tiles (block-uniform)
    uint32_t held = 0xffffffffu, nheld = 0;
    auto flush = [&]() {
        unsigned long long *gc = a.copies + (uint64_t)held * a.n_lines * 2;
        for (uint32_t i = tid; i < 2 * hot; i += CB_THREADS) {
            const uint32_t c = sm.hot[i];
            if (c) {
                atomicAdd(&gc[i], (unsigned long long)c);
                sm.hot[i] = 0u;
            }
        }
    };
    // A block takes its next ticket once its current tile has found its entering counter,
    // so the fetch overlaps the tile's samples.  A ticket taken earlier would sit unstarted
    // while other tiles wait on its sum (in a long trace, consecutive tickets are consecutive
    // tiles).  A tile waits only on tiles of lower tickets, all of them started, so the
    // lowest unfinished ticket can always proceed.
    if (tid == 0) copy_job(a, atomicAdd(a.queue, 1u), sm.task[0]);
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const CopyTask &K = sm.task[cur];
        if (!K.valid) break;
        const CopyTile ct = K.ct;
        if (ct.trace != held || nheld == CB_FLUSH) {
            // another trace's counts (or enough tiles that the next could near 2^32) leave the
            // table first; the barrier at the end of the tile orders the clearing before its use
            if (held != 0xffffffffu) flush();
            held = ct.trace;
            nheld = 0;
            __syncthreads();
        }
        ++nheld;
        const uint32_t len = ct.len, t = ct.t;
        // ---- this thread's CB_PER consecutive memcpys, loaded into registers
        const uint32_t e0 = (uint32_t)tid * CB_PER;
        unsigned long long v[CB_PER];
        uint32_t ln[CB_PER];
        uint32_t pw[CB_PER / 4];
        // the warp's slice is staged whole when it lies inside the tile and the columns are
        // 16-byte aligned (warp-uniform); otherwise each lane loads its own memcpys
        const uint32_t w0 = (uint32_t)w * 32 * CB_PER;
        const bool staged = w0 + 32 * CB_PER <= len &&
                            ((reinterpret_cast<uintptr_t>(ct.size) | reinterpret_cast<uintptr_t>(ct.line) |
                              reinterpret_cast<uintptr_t>(ct.py)) & 15u) == 0;
        if (staged) {
            const uint64_t *gs = ct.size + w0;
#pragma unroll
            for (int i = 0; i < CB_PER / 2; ++i) {   // chunk j = lane + 32 i: sizes 2j, 2j + 1
                const int j = lane + 32 * i;
                cp_async16(&stg.size[swz_el<CB_PER>(2 * j)], gs + 2 * j);
            }
            const uint32_t *gl = ct.line + w0;
#pragma unroll
            for (int i = 0; i < CB_PER / 4; ++i) {   // chunk j: lines 4j .. 4j + 3 (row j / 4)
                const int j = lane + 32 * i;
                cp_async16(&stg.line[4 * line_chunk(j >> 2, j & 3)], gl + 4 * j);
            }
            cp_async16(&stg.py[CB_PER * lane], ct.py + w0 + CB_PER * lane);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            load_lane<CB_PER>(stg.size, (uint32_t)(CB_PER * lane), v);
            const uint4 *sl = reinterpret_cast<const uint4 *>(stg.line);
#pragma unroll
            for (int q = 0; q < CB_PER / 4; ++q) {
                const uint4 x = sl[line_chunk(lane, q)];
                ln[4 * q] = x.x; ln[4 * q + 1] = x.y; ln[4 * q + 2] = x.z; ln[4 * q + 3] = x.w;
            }
            const uint4 y = reinterpret_cast<const uint4 *>(stg.py)[lane];
            pw[0] = y.x; pw[1] = y.y; pw[2] = y.z; pw[3] = y.w;
            __syncwarp();   // the warp's stage is rewritten by its next tile only after this
        } else {
#pragma unroll
            for (int k = 0; k < CB_PER; ++k) {
                const bool in = e0 + k < len;
                v[k] = in ? ct.size[e0 + k] : 0ull;
                ln[k] = in ? ct.line[e0 + k] : 0u;
            }
#pragma unroll
            for (int q = 0; q < CB_PER / 4; ++q) {
                uint32_t x = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) x |= (e0 + 4 * q + b < len ? (uint32_t)ct.py[e0 + 4 * q + b] : 0u) << (8 * b);
                pw[q] = x;
            }
        }
        // ---- this thread's bytes, modulo T_c.  When 8 T_c < 2^31 and every size of the thread
        // is below 8 T_c, each residue, sum and remainder below fits 32 bits (the same
        // arithmetic in half the instructions)
        bool n32 = Tc8 < (1ull << 31);
#pragma unroll
        for (int k = 0; k < CB_PER; ++k) n32 &= v[k] < Tc8;
        unsigned long long ls = 0;
        if (n32) {
            const uint32_t t1 = (uint32_t)Tc, t2 = (uint32_t)Tc2, t4 = (uint32_t)Tc4;
            uint32_t s32 = 0;
#pragma unroll
            for (int k = 0; k < CB_PER; ++k) {
                uint32_t r = (uint32_t)v[k];
                if (r >= t4) r -= t4;
                if (r >= t2) r -= t2;
                if (r >= t1) r -= t1;
                s32 += r;
                if (s32 >= t1) s32 -= t1;
            }
            ls = s32;
        } else {
#pragma unroll
            for (int k = 0; k < CB_PER; ++k) {
                unsigned long long r = v[k];
                if (r >= Tc8 || !small) {
                    r %= Tc;
                } else {
                    if (r >= Tc4) r -= Tc4;
                    if (r >= Tc2) r -= Tc2;
                    if (r >= Tc) r -= Tc;
                }
                ls = madd(ls, r, Tc);
            }
        }
        // block exclusive scan of the threads' residues
        unsigned long long x = ls;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x = madd(x, y, Tc);
        }
        if (lane == 31) sm.wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            const unsigned long long y = lane < CB_THREADS / 32 ? sm.wsum[lane] : 0ull;
            unsigned long long yi = y;
#pragma unroll
            for (int o = 1; o < CB_THREADS / 32; o <<= 1) {
                const unsigned long long z = __shfl_up_sync(FULL, yi, o);
                if (lane >= o) yi = madd(yi, z, Tc);
            }
            const unsigned long long s = __shfl_sync(FULL, yi, CB_THREADS / 32 - 1);   // the tile's bytes mod T_c
            if (lane < CB_THREADS / 32) sm.wsum[lane] = yi >= y ? yi - y : yi + (Tc - y);   // exclusive
            // ---- the counter entering the tile (warp 0)
            bool ok = true;
            unsigned long long base = 0;
            if (t == ct.c0) {
                // the trace's first tile: the resident counter enters it
                base = a.traces[ct.trace].copy_counter;
                if (lane == 0) cs_publish(&status[t], madd(base, s, Tc), true);
            } else {
                if (lane == 0) cs_publish(&status[t], s, false);
                unsigned long long acc = 0;
                int64_t p = (int64_t)t - 1;   // newest predecessor not yet accounted for
                while (true) {
                    // lane j looks at tile p - j (tiles before the trace's first count as its start)
                    const int64_t q = p - lane;
                    unsigned long long wd = CS_INCL;   // (before the trace: its start)
                    if (q >= (int64_t)ct.c0) {
                        unsigned long long n = 0;
                        // a predecessor publishes its aggregate a few microseconds after it
                        // starts: poll with a short pause, so the waiting lanes leave the L2
                        // to the stores they wait for
                        while ((wd = cs_load(&status[q])) == 0 && n < a.spin) {
                            ++n;
                            __nanosleep(64);
                        }
                    } else if (q == (int64_t)ct.c0 - 1) {
                        wd = CS_INCL | a.traces[ct.trace].copy_counter;
                    }
                    if (!__all_sync(FULL, wd != 0)) {
                        if (lane == 0) set_error(a.err, E_TIMEOUT, 20, t);
                        ok = false;
                        break;
                    }
                    const bool incl = (wd & CS_INCL) != 0;
                    const unsigned long long val = incl ? wd & ~CS_INCL : wd - 1;
                    // the nearest predecessor with a prefix ends the look-back
                    const unsigned done = __ballot_sync(FULL, incl);
                    const int stop = done ? __ffs(done) - 1 : 32;
                    unsigned long long wv = lane <= stop ? val : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) wv = madd(wv, __shfl_xor_sync(FULL, wv, o), Tc);
                    acc = madd(acc, wv, Tc);
                    if (done) break;
                    p -= 32;
                }
                base = acc;
                if (ok && lane == 0) cs_publish(&status[t], madd(base, s, Tc), true);
            }
            if (lane == 0) {
                sm.base = base;
                sm.ok = ok;
                // the trace's last tile gives its counter after the batch (for the state fold)
                if (ok && t == ct.last) a.btres[ct.bt].copy_end = madd(base, s, Tc);
            }
        }
        __syncthreads();
        if (!sm.ok) break;   // a wait gave up (uniform over the block)
        if (tid == 0) copy_job(a, atomicAdd(a.queue, 1u), sm.task[cur ^ 1]);
        // ---- samples at each of this thread's memcpys, from the counter before the first
        unsigned long long rem = madd(madd(sm.base, sm.wsum[w], Tc), x >= ls ? x - ls : x + (Tc - ls), Tc);
        unsigned long long *gc = a.copies + (uint64_t)ct.trace * a.n_lines * 2;
        int ovf = 0;
        auto count = [&](int k, uint32_t qn) {
            const uint32_t l = ln[k];
            if (l >= a.n_lines) {
                set_error(a.err, E_RANGE, l, (unsigned long long)(e0 + k));
                return;
            }
            const int f = ((pw[k >> 2] >> (8 * (k & 3))) & 0xffu) ? 1 : 0;
            // the shared table takes counts of at most 8 per memcpy, so CB_FLUSH tiles add at most
            // 1,024 x 4,096 x 8 = 2^25 per entry (tiles of at most 4,096) and the 32-bit counts
            // cannot wrap; larger
            // counts go to global memory
            if (l < hot && qn <= 8) atomicAdd(&sm.hot[2 * l + f], qn);
            else atomicAdd(&gc[2 * l + f], (unsigned long long)qn);
        };
        if (n32) {
            const uint32_t t1 = (uint32_t)Tc, t2 = (uint32_t)Tc2, t4 = (uint32_t)Tc4, t8 = (uint32_t)Tc8;
            uint32_t r32 = (uint32_t)rem;
#pragma unroll
            for (int k = 0; k < CB_PER; ++k) {
                // r32 + size < T_c + 8 T_c < 2^32: the quotient (at most 8) bit by bit
                r32 += (uint32_t)v[k];
                uint32_t qn = 0;
                if (r32 >= t8) { r32 -= t8; qn = 8; }
                if (r32 >= t4) { r32 -= t4; qn += 4; }
                if (r32 >= t2) { r32 -= t2; qn += 2; }
                if (r32 >= t1) { r32 -= t1; qn += 1; }
                if (qn) count(k, qn);
            }
        }
#pragma unroll
        for (int k = 0; k < CB_PER && !n32; ++k) {
            const unsigned long long sz = v[k];
            ovf |= rem + sz < rem;   // the sequential count would pass 2^64 here
            unsigned long long qn;
            if (sz >= Tc8 || !small) {
                qn = sz / Tc;
                const unsigned long long r2 = rem + sz % Tc;   // < 2 T_c: fits
                qn += r2 >= Tc;
                rem = r2 >= Tc ? r2 - Tc : r2;
            } else {
                // rem + sz < 9 T_c <= 9 * 2^60 fits: the quotient (at most 8) bit by bit
                rem += sz;
                qn = 0;
                if (rem >= Tc8) { rem -= Tc8; qn = 8; }
                if (rem >= Tc4) { rem -= Tc4; qn += 4; }
                if (rem >= Tc2) { rem -= Tc2; qn += 2; }
                if (rem >= Tc) { rem -= Tc; qn += 1; }
            }
            if (!qn) continue;
            if (qn <= 8) {
                count(k, (uint32_t)qn);
            } else {
                const uint32_t l = ln[k];
                if (l >= a.n_lines) {
                    set_error(a.err, E_RANGE, l, (unsigned long long)(e0 + k));
                    continue;
                }
                atomicAdd(&gc[2 * l + (((pw[k >> 2] >> (8 * (k & 3))) & 0xffu) ? 1 : 0)], qn);
            }
        }
        // (this barrier also ends every use of the tile's shared words before the next tile)
        if (__syncthreads_or(ovf) && tid == 0) set_error(a.err, E_OVERFLOW, 7, t);
    }
    if (held != 0xffffffffu) flush();
}

size_t copy_status_bytes(size_t ntiles) { return sizeof(unsigned long long) * ntiles; }

cudaError_t launch_copy(const LaunchCopy &a, cudaStream_t s) {
    if (!a.nctiles) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_copy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COPY_STAGE_BYTES);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_copy, CB_THREADS, COPY_STAGE_BYTES);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(a.nctiles, std::max(1, bps) * a.num_sms));
    k_copy<<<blocks, CB_THREADS, COPY_STAGE_BYTES, s>>>(a);
    return cudaGetLastError();
}

}  // namespace scl
