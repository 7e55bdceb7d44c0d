// scl_final.cu -- the exact replay of each unit, once its entering state is known.
//
// Per event (Sections 3.2-3.4): c <- c + delta and the open window's totals A, F,
// A_py, F_py grow; a free compares its address with the tracked block; when
// |c| >= T a sample closes the window (kind, totals, footprint, line and flag of
// the triggering event), and a growth sample whose footprint beats the high-water
// mark sets a new mark and starts tracking the sampled block.
//
// One warp per unit, 128 events per step.  The entering counter, window totals,
// footprint, mark and tracked block come from k_chain / k_scan, so no speculation
// is left here.  delta, the python flag and the address are staged through the
// bulk-copy ring; the line id is read only at the events that trigger a sample.
#include "scl_launch.h"
#include "scl_stage.cuh"

namespace scl {

using FinalRing = Ring<true, 3, 256, 8>;

__global__ void __launch_bounds__(32 * 14) k_final(const Unit *__restrict__ units, int nunits,
                                                  const UnitTrue *__restrict__ utrue,
                                                  const UnitPlan *__restrict__ uplan, const SRes *__restrict__ lists,
                                                  FRec *recs, UnitOut *uout, int64_t T, unsigned *queue, ErrWord *err,
                                                  unsigned long long spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FinalRing &sm = reinterpret_cast<FinalRing *>(smem_raw)[warp];
    ring_init(sm, lane);
    uint32_t phase = 0;
    while (true) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(queue, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const Unit U = units[u];
        const UnitTrue Tu = utrue[u];
        const UnitPlan Pl = uplan[u];
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
        int64_t c = Tu.entry_c;
        int64_t P = 0;
        int64_t mark = Pl.hwm_in;
        const int64_t fpb = Pl.fp_base;
        uint32_t tk = Pl.enter_kind;   // tracked block: 0 none, 1/2 entering (from k_scan), 3 own sample
        uint64_t taddr = Pl.enter_addr;
        uint32_t tslot = 0;
        uint32_t enter_hit = 0;
        uint32_t n = 0;
        FRec *out = recs + U.rec0;
        const uint32_t cap = U.rec_cap;

        // mark the tracked block reclaimed
        auto hit_tracked = [&]() {
            if (tk == 3) {
                if (lane == 0 && tslot < cap) out[tslot].recl = 1;
            } else {
                enter_hit = 1;
            }
        };
        auto add_events = [&](const StepIn<E> &in, int after, int upto, int64_t &sA, int64_t &sApy, int64_t &sSpy) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int pos = lane * E + k;
                if (pos > after && pos <= upto) {
                    const int64_t x = in.d[k];
                    const int64_t ps = x > 0 ? x : 0;
                    sA += ps;
                    if (py_of(in, k)) { sApy += ps; sSpy += x; }
                }
            }
        };
        auto frees_hit = [&](const StepIn<E> &in, int after, int upto) -> bool {
            bool h = false;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int pos = lane * E + k;
                h |= pos > after && pos <= upto && in.d[k] < 0 && in.a[k] == taddr;
            }
            return __any_sync(FULL, h);
        };
        // every event of the step joins the open window (no sample in it)
        auto whole_step = [&](const StepIn<E> &in) {
            bool h = false;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int64_t x = in.d[k];
                h |= x < 0 && in.a[k] == taddr;
                const int64_t ps = x > 0 ? x : 0;
                accA += ps;
                if (py_of(in, k)) { accApy += ps; accSpy += x; }
            }
            if (tk && __any_sync(FULL, h)) hit_tracked();
        };
        // the sample at step position r (frees up to it already tested): counter cr there,
        // unit-local prefix Pr there
        auto close = [&](const StepIn<E> &in, int after, int r, uint32_t rel0, int64_t cr, int64_t Pr) {
            int64_t sA = accA, sApy = accApy, sSpy = accSpy;
            add_events(in, after, r, sA, sApy, sSpy);
            const int64_t wA = warp_sum(sA), wApy = warp_sum(sApy), wSpy = warp_sum(sSpy);
            const int fl = r / E, kf = r % E;
            uint64_t av = in.a[0];
            uint32_t pyv = py_of(in, 0);
#pragma unroll
            for (int k = 1; k < E; ++k)
                if (k == kf) { av = in.a[k]; pyv = py_of(in, k); }
            av = __shfl_sync(FULL, av, fl);
            pyv = __shfl_sync(FULL, pyv, fl);
            const int64_t fp = fpb + Pr;
            const bool growth = cr > 0;
            const bool hwm = growth && fp > mark;
            const uint32_t rel = rel0 + (uint32_t)r;
            if (lane == 0 && n < cap) {
                FRec R;
                R.rel = rel;
                R.line = U.line[rel];
                R.kind = growth ? 1 : -1;
                R.is_hwm = hwm ? 1 : 0;
                R.recl = 0;
                R.py = pyv ? 1 : 0;
                R.pad = 0;
                R.A = wA; R.F = wA - cr; R.A_py = wApy; R.F_py = wApy - wSpy; R.P = Pr;
                out[n] = R;
            }
            if (hwm) { mark = fp; tk = 3; taddr = av; tslot = n; }
            ++n;
            accA = accApy = accSpy = 0;
        };

        bool ok;
        if (Tu.list != NO_LIST) {
            // ---- the true run's resets are known (k_sketch listed them): no crossing search
            const SRes *Ls = lists + U.lst0 + (uint64_t)Tu.list * U.lst_cap;
            const uint32_t nres = Tu.n;
            uint32_t ri = 0;
            uint32_t npos = 0xffffffffu;
            int64_t nP = 0;
            if (nres) { const SRes q = Ls[0]; npos = q.pos; nP = q.P; }
            int64_t cst = c, Pprev = 0;   // counter at the open window's start, prefix there
            auto kstep = [&](const StepIn<E> &in, uint32_t rel0) -> bool {
                if (npos >= rel0 + (uint32_t)STEP) {
                    whole_step(in);
                    return false;
                }
                int after = -1;
                while (npos < rel0 + (uint32_t)STEP) {
                    if (npos < rel0 + (uint32_t)(after + 1)) {   // positions must increase
                        if (lane == 0) set_error(err, E_INTERNAL, 12, (unsigned long long)u);
                        npos = 0xffffffffu;
                        break;
                    }
                    const int r = (int)(npos - rel0);
                    if (tk && frees_hit(in, after, r)) hit_tracked();
                    close(in, after, r, rel0, cst + (nP - Pprev), nP);
                    cst = 0;
                    Pprev = nP;
                    after = r;
                    if (++ri < nres) {
                        const SRes q = Ls[ri];
                        npos = q.pos;
                        nP = q.P;
                    } else {
                        npos = 0xffffffffu;
                    }
                }
                if (tk && frees_hit(in, after, STEP)) hit_tracked();
                add_events(in, after, STEP, accA, accApy, accSpy);
                return false;
            };
            ok = ring_walk<true>(sm, U, 0, U.len, phase, spin, err, lane, kstep);
            c = Tu.exit_c;
        } else {
            // ---- search for the crossings from the true entry counter
            auto step = [&](const StepIn<E> &in, uint32_t rel0) -> bool {
                StepPrefix<E> sp;
                step_prefix(in, lane, sp, sm.xq);
                if (__ballot_sync(FULL, c + sp.lmax >= T || c + sp.lmin <= -T) == 0) {
                    whole_step(in);
                    c += sp.tot;
                    P += sp.tot;
                    return false;
                }
                int64_t b = c;
                int after = -1;
                while (true) {
                    int64_t Qr;
                    const int r = first_cross(sp, sm.xq, lane, b, T, after, Qr);
                    // frees up to and including the sample's event see the block tracked so far
                    if (tk && frees_hit(in, after, r < 0 ? STEP : r)) hit_tracked();
                    if (r < 0) break;
                    close(in, after, r, rel0, b + Qr, P + Qr);
                    b = -Qr;
                    after = r;
                }
                add_events(in, after, STEP, accA, accApy, accSpy);
                c = b + sp.tot;
                P += sp.tot;
                return false;
            };
            ok = ring_walk<true>(sm, U, 0, U.len, phase, spin, err, lane, step);
        }
        const int64_t a = warp_sum(accA), ap = warp_sum(accApy), spy = warp_sum(accSpy);
        if (lane == 0) {
            UnitOut O;
            O.count = n; O.enter_hit = enter_hit;
            O.c = c; O.A = a; O.F = a - c; O.Apy = ap; O.Fpy = ap - spy;
            uout[u] = O;
            if (n > cap) set_error(err, E_OVERFLOW, 3, (unsigned long long)u);
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
    const size_t smem = sizeof(FinalRing) * a.warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(k_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_final<<<a.blocks, 32 * a.warps_per_block, smem, s>>>(a.units, a.nunits, a.utrue, a.uplan, a.lists, a.recs,
                                                           a.uout, a.T, a.queue, a.err, a.spin);
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
