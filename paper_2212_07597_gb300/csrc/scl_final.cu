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

// 14 warps per block at most (128 registers: a cap of 136 registers left blocks of only 12
// warps on an SM, and the replay ran 40% longer)
__global__ void __launch_bounds__(32 * 14) k_final(const LaunchFinal a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FinalRing &sm = reinterpret_cast<FinalRing *>(smem_raw)[warp];
    const Unit *__restrict__ units = a.units;
    const int nunits = a.nunits;
    const int64_t T = a.T;
    ErrWord *err = a.err;
    const unsigned long long spin = a.spin;
    ring_init(sm, lane);
    uint32_t phase = 0;
    while (true) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(a.queue, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const Unit U = units[u];
        if (U.first) continue;   // replayed by k_phase1
        const UnitTrue Tu = a.utrue[u];
        const UnitPlan Pl = a.uplan[u];
        ExactIn in0;
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
        in0.fpb = Pl.fp_base;
        in0.tk = Pl.enter_kind;
        in0.taddr = Pl.enter_addr;
        in0.list = Tu.list != NO_LIST ? a.lists + U.lst0 + (uint64_t)Tu.list * U.lst_cap : nullptr;
        in0.nres = Tu.n;
        in0.exit_c = Tu.exit_c;
        if (!in0.list && lane == 0) atomicAdd(&a.stats[5], 1ull);
        UnitOut O;
        uint32_t n = 0;
        const bool ok = exact_unit<false>(sm, phase, U, in0, a.recs + U.rec0, U.rec_cap, T, spin, err, lane, n, O,
                                          (ExactRun *)nullptr);
        if (lane == 0) {
            a.uout[u] = O;
            if (n > U.rec_cap) set_error(err, E_OVERFLOW, 3, (unsigned long long)u);
            if (ok && n != Tu.n) set_error(err, E_INTERNAL, 10, (unsigned long long)u);
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
    if (!a.nunits) return cudaSuccess;
    const size_t smem = sizeof(FinalRing) * a.warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_final<<<a.blocks, 32 * a.warps_per_block, smem, s>>>(a);
    return cudaGetLastError();
}

int final_occupancy(int warps_per_block, int *blocks_per_sm) {
    const size_t smem = sizeof(FinalRing) * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_final, 32 * warps_per_block, smem);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace scl
