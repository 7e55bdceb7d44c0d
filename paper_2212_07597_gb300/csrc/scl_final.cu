// scl_final.cu -- the exact replay of each unit, once its entering state is known.
//
// One warp per unit (scl_exact.cuh).  The entering counter, window totals, footprint,
// mark and tracked block come from k_chain / k_scan, so no speculation is left here.
// The first unit of each trace in the batch was already replayed by k_phase1 (its
// entering state is the trace's resident state) and is skipped.
#include "scl_exact.cuh"
#include "scl_launch.h"

namespace scl {

using FinalRing = Ring<true, 3, 256, 8>;

// first index i of a unit's reset list with L[i].pos >= x (n if none), by one warp: each round
// probes 32 entries, so a list of up to 32^k entries takes k rounds
__device__ uint32_t list_lower(const SRes *L, uint32_t n, uint32_t x, int lane) {
    uint32_t lo = 0, hi = n;   // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const uint32_t st = (hi - lo + 31) / 32;
        const uint32_t idx = lo + (uint32_t)lane * st;
        const bool ge = idx >= hi || L[idx].pos >= x;
        const unsigned b = __ballot_sync(FULL, ge);
        if (!b) {
            lo = lo + 31 * st + 1;
        } else {
            const uint32_t k = (uint32_t)(__ffs(b) - 1);
            if (k == 0) return lo;
            const uint32_t nlo = lo + (k - 1) * st + 1, nhi = lo + k * st;
            lo = nlo;
            hi = nhi < hi ? nhi : hi;
        }
    }
    const uint32_t idx = lo + (uint32_t)lane;
    const bool ge = idx >= hi || L[idx].pos >= x;
    const unsigned b = __ballot_sync(FULL, ge);
    return b ? lo + (uint32_t)(__ffs(b) - 1) : hi;
}

// 14 warps per block at most (128 registers: a cap of 136 registers left blocks of only 12
// warps on an SM, and the replay ran 40% longer)
template <bool DENSE>
__global__ void __launch_bounds__(32 * 14) k_final(const LaunchFinal a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FinalRing &sm = reinterpret_cast<FinalRing *>(smem_raw)[warp];
    const Unit *__restrict__ units = a.units;
    const int64_t T = a.T;
    ErrWord *err = a.err;
    const unsigned long long spin = a.spin;
    constexpr uint32_t STEP = FinalRing::kE * 32;
    ring_init(sm, lane);
    uint32_t phase = 0;
    while (true) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.queue, 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it >= a.nitems) break;
        const FItem I = a.items[it];
        const int u = (int)I.u;
        const Unit U = units[u];
        const UnitTrue Tu = a.utrue[u];
        const UnitPlan Pl = a.uplan[u];
        const uint32_t len = (uint32_t)U.len;
        const SRes *L = Tu.list != NO_LIST ? a.lists + U.lst0 + (uint64_t)Tu.list * U.lst_cap : nullptr;
        ExactIn in0;
        in0.fpb = Pl.fp_base;
        in0.list = L;
        in0.nres = Tu.n;
        in0.exit_c = Tu.exit_c;
        in0.tslot = 0;
        in0.limit = len;
        in0.n0 = 0;
        in0.rend = Tu.n;
        in0.P0 = 0;
        in0.stop = false;
        // ---- the piece's span: (start bound, end] at listed resets
        uint32_t from = 0, to = len - 1;
        if (L && U.fnp > 1) {
            const uint64_t PL = a.piece;
            if (I.p + 1 < U.fnp) {
                const uint32_t j = list_lower(L, Tu.n, (uint32_t)((I.p + 1) * PL), lane);
                if (j < Tu.n) {
                    to = L[j].pos;
                    in0.rend = j + 1;
                    in0.stop = true;
                }
            }
            if (I.p > 0) {
                const uint32_t i = list_lower(L, Tu.n, (uint32_t)(I.p * PL), lane);
                const SRes Ri = i < Tu.n ? L[i] : SRes{};
                from = i < Tu.n ? Ri.pos + 1 : len;
                in0.n0 = i + 1;
                in0.P0 = Ri.P;
            }
        } else if (I.p > 0) {
            from = len;   // a unit without a list is replayed whole by its piece 0
        }
        if (from > to) {   // empty piece
            if (lane == 0) a.phit[it] = 0;
            continue;
        }
        if (I.p == 0 || !L) {
            // ---- the open window entering the unit: totals of whole units (from k_scan) plus
            // the tail of the unit that holds the last reset before this one
            int64_t accA = 0, accApy = 0, accSpy = 0;
            if (Pl.rb_unit >= 0) {
                const Unit W = units[Pl.rb_unit];
                for (uint64_t e = Pl.rb_from + lane; e < W.len; e += 32) {
                    const int64_t x = W.delta[e];
                    const int64_t ps = x > 0 ? x : 0;
                    accA += ps;
                    if (W.py[e]) { accApy += ps; accSpy += x; }
                }
            }
            if (lane == 0) { accA += Pl.wA; accApy += Pl.wApy; accSpy += Pl.wSpy; }
            in0.c = Tu.entry_c;
            in0.wA = accA; in0.wApy = accApy; in0.wSpy = accSpy;
            in0.mark = Pl.hwm_in;
            in0.tk = Pl.enter_kind;
            in0.taddr = Pl.enter_addr;
        } else {
            // ---- a piece that starts after listed reset n0 - 1: counter 0, window empty; the
            // mark is the unit's entering one raised by the growth samples before the piece, and
            // the tracked block that of the first sample attaining the highest of them
            in0.c = 0;
            in0.wA = in0.wApy = in0.wSpy = 0;
            int64_t best = INT64_MIN;
            uint32_t barg = 0xffffffffu;
            for (uint32_t j = (uint32_t)lane; j < in0.n0; j += 32) {
                const int64_t Pj = L[j].P;
                const int64_t cr = j ? Pj - L[j - 1].P : Tu.entry_c + Pj;   // the counter at the reset
                if (cr > 0 && Pj > best) { best = Pj; barg = j; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t ob = __shfl_xor_sync(FULL, best, o);
                const uint32_t oa = __shfl_xor_sync(FULL, barg, o);
                if (ob > best || (ob == best && oa < barg)) { best = ob; barg = oa; }
            }
            const int64_t fp = best == INT64_MIN ? INT64_MIN : Pl.fp_base + best;
            if (best != INT64_MIN && fp > Pl.hwm_in) {
                in0.mark = fp;
                in0.tk = 3;
                in0.tslot = barg;
                in0.taddr = U.addr[L[barg].pos];
            } else {
                in0.mark = Pl.hwm_in;
                in0.tk = Pl.enter_kind;
                in0.taddr = Pl.enter_addr;
            }
        }
        in0.from = from;
        in0.limit = to + 1 >= len ? len : (to + STEP) / STEP * STEP < len ? (to + STEP) / STEP * STEP : len;
        if (!L && lane == 0) atomicAdd(&a.stats[5], 1ull);
        UnitOut O;
        uint32_t n = 0, prior = 0;
        const bool ok = exact_unit<false, DENSE>(sm, phase, U, in0, a.recs + U.rec0, U.rec_cap, T, spin, err, lane, n, O,
                                          (ExactRun *)nullptr, prior);
        if (lane == 0) {
            // a hit on the entering block of a piece other than the one that ends the unit, and
            // any hit on an earlier piece's record, are applied by k_mark
            const bool ends = to == len - 1;
            a.phit[it] = prior ? prior : (O.enter_hit && !ends ? PHIT_ENTER : 0u);
            if (ends) {
                a.uout[u] = O;
                if (n > U.rec_cap) set_error(err, E_OVERFLOW, 3, (unsigned long long)u);
            }
            if (ok && n != (L ? in0.rend : Tu.n)) set_error(err, E_INTERNAL, 10, (unsigned long long)u);
        }
        if (!ok) break;
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

cudaError_t launch_final(const LaunchFinal &a, cudaStream_t s) {
    if (!a.nitems) return cudaSuccess;
    const size_t smem = sizeof(FinalRing) * a.warps_per_block;
    // the instance with the dense-step test only where a dense step can occur often
    auto kern = a.T <= DENSE_T_MAX ? k_final<true> : k_final<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.blocks, 32 * a.warps_per_block, smem, s>>>(a);
    return cudaGetLastError();
}

int final_occupancy(int warps_per_block, int *blocks_per_sm) {
    const size_t smem = sizeof(FinalRing) * warps_per_block;
    // (both instances have the same register cap and shared memory)
    cudaError_t e = cudaFuncSetAttribute(k_final<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_final<false>, 32 * warps_per_block, smem);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace scl
