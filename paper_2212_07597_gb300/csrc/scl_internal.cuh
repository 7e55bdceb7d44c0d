// scl_internal.cuh -- device-side layouts and warp primitives of libscl.
//
// Work decomposition.  A batch of segments is cut into *units*: contiguous runs of
// one trace's events, at most `unit_events` long, starting at multiples of 1024
// events.  The threshold sampler of Section 3.2 is a sequential counter; its state
// at each unit start is found in parallel (scl_sketch.cu: candidate counters per
// unit, links between neighbouring units, a per-trace chain), after which every
// unit is replayed exactly and independently (scl_final.cu), and the per-trace
// bookkeeping of Sections 3.3-3.5 follows (scl_post.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace scl {

constexpr unsigned FULL = 0xffffffffu;
constexpr int E = 8;               // events per lane per walker step
constexpr int STEP = 32 * E;       // events per walker step
constexpr int TILE = 256;          // events per shared-memory stage
constexpr int NST = 4;             // stages per walker warp
constexpr int UNIT_ALIGN = 1024;   // unit starts are multiples of this within a segment
constexpr uint64_t FINAL_PIECE = 65536;   // k_final cuts units into pieces of about this many events
constexpr int COPY_TILE = 4096;    // memcpy events per block of the allocation-free copy sampler
constexpr int COPY_PASS_TILE = 4096;   // memcpy events per tile of the batch's copy pass (k_copy)
constexpr int SMEM_LINES_MAX = 1024;  // per-line tables kept in shared memory up to this L

// error codes mirrored from scl.h
constexpr int E_INVAL = -1, E_NOMEM = -2, E_CUDA = -3, E_TIMEOUT = -4, E_OVERFLOW = -5, E_RANGE = -6,
              E_INTERNAL = -7;

// ---------------------------------------------------------------- resident state
struct DevTrace {                   // one per trace slot
    int64_t c, A, F, A_py, F_py;    // counter and open-window totals (Section 3.2)
    int64_t footprint, hwm;         // Section 3.3 footprint, Section 3.4 high-water mark
    uint64_t tracked_addr, tracked_idx;
    uint32_t tracked_line, tracked_valid, tracked_reclaimed, pad0;
    uint64_t n_events, n_copies, n_samples, copy_counter;
};

struct LineRow {                    // one per (trace, line): sample totals (scl_line_stat order) + leak pair
    unsigned long long n_growth, n_shrink;
    long long A, F, A_py, F_py;     // (a line's net total, the sum of A - F, is A - F: formed on query)
    unsigned long long mallocs, frees;
};
static_assert(sizeof(LineRow) == 64, "half a 128-byte line per (trace, line)");
// the copy-volume samples of a (trace, line) live in their own array, [trace][line][flag]
// (16 bytes per line): the copy sampler's updates then touch a compact per-trace block

struct Sample {                     // layout of scl_sample (56 bytes)
    uint64_t idx;
    int64_t A, F, A_py, F_py, footprint;
    uint32_t line;
    int8_t kind;
    uint8_t is_python, is_hwm, pad;
};

// ---------------------------------------------------------------- batch plan
struct Unit {
    const int64_t *delta;
    const uint8_t *py;
    const uint64_t *addr;
    const uint32_t *line;
    uint64_t len;
    uint64_t gidx0;       // trace event index of the unit's first event
    uint64_t rec0;        // first final-record slot of the unit
    uint32_t rec_cap;     // final-record slots of the unit
    uint32_t trace;       // resident trace slot
    uint32_t bt;          // index of the trace within the batch
    uint32_t first, last; // first / last unit of its trace in this batch
    uint32_t lst_cap;     // reset-list slots per candidate run of the unit
    uint64_t lst0;        // first reset-list slot of the unit (NL lists of lst_cap)
    uint32_t fi0, fnp;    // the unit's pieces in k_final: items fi0 .. fi0 + fnp - 1 (none for a first unit)
};

// A piece of a unit for k_final.  Piece p of a unit whose true run has a reset list covers the
// events after the first listed reset at or past p * piece_events (the unit start for p = 0)
// up to and including the first listed reset at or past (p + 1) * piece_events (the unit end
// if there is none).  After a reset the counter is 0 and the window empty, so a piece's entry
// state follows from the list alone.  A unit without a list is replayed whole by its piece 0.
struct FItem {
    uint32_t u, p;
};
constexpr uint32_t PHIT_ENTER = 0xffffffffu;   // a piece freed the block tracked entering its unit

struct BTrace {           // one per trace present in the batch
    uint32_t trace, u0, nu, pad;   // slot, first unit, unit count
    uint64_t n_ev;                 // events of this trace in the batch
    uint64_t n_cp;                 // memcpy events of this trace in the batch
    uint32_t c0, nc;               // copy tiles
};

struct CopyTile {          // a tile of one trace's memcpys; the plan lists them in the order blocks take them
    const uint64_t *size;
    const uint32_t *line;
    const uint8_t *py;
    uint32_t len, bt;
    uint32_t t;            // look-back slot: the tile's index among all tiles in trace order
    uint32_t c0, last;     // slots of the trace's first and last tiles
    uint32_t trace;        // trace slot
};
static_assert(sizeof(CopyTile) == 48, "three 16-byte loads per tile");

// ---- sketch: K candidate counters per unit (one per lane)
constexpr int K = 32;     // candidates per unit
constexpr uint8_t NO_MATCH = 0xff;

struct UnitSum {          // lane-independent facts of a unit
    int64_t total;                 // sum of deltas
    int64_t totA, totApy, totSpy;  // sum of mallocs, python mallocs, python deltas
    int64_t minQ, maxQ;            // extremes of the unit-local inclusive prefix sum
};

constexpr int RM = 32;    // leading resets kept per candidate, to let a walk merge into it

// ---- reset lists: every reset of up to NL distinct candidate runs per unit, so the
// exact replay of a unit whose true run has a complete list needs no crossing search
constexpr int NL = 8;
constexpr uint32_t NO_LIST = 0xffffffffu;
struct SRes {
    uint32_t pos;         // unit offset of the reset
    uint32_t pad;
    int64_t P;            // unit-local prefix sum of deltas up to and including pos
};

struct Cand {             // candidate k of unit u
    int64_t c0;           // its counter at the unit's first event
    int64_t c;            // its counter after the unit
    int32_t last;         // position of its last reset in the unit (-1: none)
    uint32_t n;           // resets in the unit
    int64_t gmax;         // largest unit-local prefix at a growth reset (INT64_MIN: none)
    uint32_t garg, targ;  // first position attaining gmax; same for tmax
    int64_t tmax;         // largest prefix at a growth reset of index >= RM (INT64_MIN: none)
    uint32_t pos[RM];     // positions of its first RM resets
    int64_t gp[RM];       // their prefixes if growth resets, else INT64_MIN
    uint32_t list;        // reset list holding all n resets (< NL), or NO_LIST
    uint32_t pad;
};

struct Walk {             // one unit walked by k_chain from an exact counter
    int64_t c;            // counter after the unit
    int32_t last;
    uint32_t n;
    int64_t gmax;
    uint32_t garg;
    int32_t into;         // candidate of the unit the walk merged into (-1: none)
    uint32_t walked;      // events walked (to the merge, or the whole unit)
};

struct UnitTrue {         // the true trajectory through a unit (k_chain)
    int64_t entry_c;      // counter before the unit's first event
    int64_t entry_last;   // trace index of the last reset before the unit (-1: none in this batch)
    int64_t gmax;         // largest unit-local prefix at a growth sample (INT64_MIN: none)
    uint32_t garg;        // its first position
    uint32_t n;           // samples in the unit
    int64_t exit_c;       // counter after the unit
    int64_t exit_last;    // trace index of the last reset up to the unit's end (-1: none)
    uint32_t list;        // reset list of the true run (NO_LIST: the exact replay searches)
    uint32_t pad;
};

struct UnitPlan {         // per unit, from k_scan
    int64_t fp_base;      // footprint before the unit
    int64_t hwm_in;       // high-water mark entering the unit
    int64_t wA, wApy, wSpy;   // open-window totals entering the unit, except the read-back part
    int64_t rb_unit;      // unit whose tail (rb_from .. end) still belongs to the open window (-1: none)
    uint32_t rb_from, enter_kind;   // enter_kind: 0 none, 1 a crossing of this batch, 2 the block tracked before the batch
    uint64_t enter_idx;   // trace index of the entering tracked block's crossing
    uint64_t enter_addr;
    int64_t enter_unit;   // unit holding that crossing
    uint64_t sample_off;  // first sample of the unit within the trace's batch samples
};

// final sample record (k_final), 56 bytes
struct FRec {
    uint32_t rel;         // event offset within the unit
    uint32_t line;
    int8_t kind;
    uint8_t is_hwm, recl, py;
    uint32_t pad;
    int64_t A, F, A_py, F_py;
    int64_t P;            // unit-local prefix sum at rel
};

struct UnitOut {          // per unit, from k_final
    uint32_t count;       // records written
    uint32_t enter_hit;   // the entering tracked block was freed inside the unit
    int64_t c, A, F, Apy, Fpy;   // state after the unit
};

struct BTraceRes {
    uint64_t n_samples;                         // samples of this trace in the batch
    int64_t fp_end, hwm_end;
    int64_t last_cross_unit;                    // unit of the batch's last crossing (-1: none)
    uint64_t last_cross_idx;                    // its trace index
    uint32_t pending_hit, pad;                  // the block tracked before the batch was freed before the first crossing
    uint64_t copy_end;                          // copy counter after the batch (< T_c)
};

struct ErrWord {
    int code;
    unsigned detail0;
    unsigned long long detail1;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void set_error(ErrWord *e, int code, unsigned d0, unsigned long long d1) {
    if (atomicCAS(&e->code, 0, code) == 0) {
        e->detail0 = d0;
        e->detail1 = d1;
    }
}

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Warp-wide signed 64-bit max: the high words (signed) by one warp reduction, then the low
// words (unsigned) of the lanes holding that high word by a second one.
__device__ __forceinline__ int64_t warp_max(int64_t v) {
    const int hi = (int)(v >> 32);
    const int mh = __reduce_max_sync(FULL, hi);
    const unsigned ml = __reduce_max_sync(FULL, hi == mh ? (unsigned)v : 0u);
    return (int64_t)(((uint64_t)(uint32_t)mh << 32) | ml);
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// -------- mbarrier and asynchronous copies (global -> shared)
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// an mbarrier whose memory is about to hold something else (no operation may be pending)
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 16-byte asynchronous global -> shared copy (cp.async, L2 only), and an arrival on an
// mbarrier that fires when all of this thread's earlier cp.async copies have landed
// (.noinc: the barrier counts these arrivals among its expected ones).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Staged 8-byte columns hold each lane's EL events (one "row" of EL * 8 bytes) with the
// row's 16-byte chunks permuted, so that a quarter warp loading one chunk per lane (eight
// consecutive rows) touches eight distinct bank groups:
//   EL = 8  (64-byte rows, 4 chunks):  chunk c of row r sits at chunk c ^ ((r >> 1) & 3)
//   EL = 16 (128-byte rows, 8 chunks): chunk c of row r sits at chunk c ^ (r & 7)
template <int EL>
__device__ __forceinline__ int swz_chunk_el(int r, int c) {
    static_assert(EL == 8 || EL == 16, "staged rows hold 8 or 16 events");
    return EL == 8 ? c ^ ((r >> 1) & 3) : c ^ (r & 7);
}
template <int EL>
__device__ __forceinline__ int swz_el(int i) {   // element i of a tile -> its staged position
    const int r = i / EL, k = i % EL;
    return r * EL + (swz_chunk_el<EL>(r, k >> 1) << 1) + (k & 1);
}

// Bounded wait for phase `parity` of the barrier, called by all 32 lanes of a warp.
// Every lane polls (so each observes the phase completion); the answer is agreed by
// vote, so all lanes return the same value.  False if `limit` polls passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit) {
    uint32_t a = smem_addr(bar);
    for (unsigned long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (__all_sync(0xffffffffu, ok != 0)) return true;
    }
    return false;
}

}  // namespace scl
