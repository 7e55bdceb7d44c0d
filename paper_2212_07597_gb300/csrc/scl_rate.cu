// scl_rate.cu -- rate-based sampling (Section 3.2), the sampler the paper compares
// threshold sampling against: every byte allocated or freed is a Bernoulli trial; the
// sampled bytes are where the running byte count passes the cumulative gaps (the caller's
// geometric draws, passed in so the draws are the same everywhere).
//
// The sequential countdown becomes two monotone sequences: S_i, the bytes moved up to and
// including event i, and B_k, the position of the k-th sampled byte.  Event i takes one
// sample per B_k in (S_{i-1}, S_i].  Tiles of 4,096 events get their byte range from a scan
// of tile sums; each tile finds its B_k by binary search and places each one at its event
// by a binary search in the tile's prefix, staged in shared memory.
//
// Also here: the Python / native split of CPU-timer interrupts (Section 2.2), the other
// per-line attribution the profiler makes from an event stream.
#include "scl_launch.h"

namespace scl {

namespace {

constexpr int RT = 256;               // threads per block
constexpr int RTILE = 4096;           // events per tile
constexpr int RPT = RTILE / RT;       // events per thread
constexpr int GTILE = 4096;           // gaps per scan block

__device__ __forceinline__ uint64_t absu(int64_t d) { return d < 0 ? (uint64_t)0 - (uint64_t)d : (uint64_t)d; }

__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) { return a + b < a ? ~0ull : a + b; }

// block-wide exclusive sum of uint64 values (saturating); *total = block total
__device__ uint64_t block_excl_sum_sat(uint64_t v, uint64_t *sh, uint64_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl = sat_add(incl, t);
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint64_t x = lane < RT / 32 ? sh[lane] : 0;
        uint64_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi = sat_add(xi, t);
        }
        if (lane < RT / 32) sh[lane] = xi - x;
        if (lane == RT / 32 - 1) sh[RT / 32] = xi;
    }
    __syncthreads();
    const uint64_t r = sat_add(incl - v, sh[w]);
    *total = sh[RT / 32];
    __syncthreads();
    return r;
}

// first index in [lo, hi) with a[idx] > key (hi if none); a non-decreasing
__device__ __forceinline__ uint64_t upper(const uint64_t *a, uint64_t lo, uint64_t hi, uint64_t key) {
    while (lo < hi) {
        const uint64_t m = lo + (hi - lo) / 2;
        if (a[m] <= key) lo = m + 1; else hi = m;
    }
    return lo;
}

// bytes moved by each tile of events; flags |= 4 on a sum past 2^64
__global__ void __launch_bounds__(RT) k_rate_tsum(const int64_t *delta, uint64_t n, uint64_t *tsum, uint64_t *flags) {
    __shared__ uint64_t sh[RT / 32 + 1];
    const uint64_t t0 = (uint64_t)blockIdx.x * RTILE;
    uint64_t s = 0;
    int ovf = 0;
    for (uint64_t j = t0 + threadIdx.x; j < n && j < t0 + RTILE; j += RT) {
        const uint64_t b = absu(delta[j]);
        ovf |= s + b < s;
        s += b;
    }
    uint64_t tot;
    (void)block_excl_sum_sat(s, sh, &tot);
    if (__syncthreads_or(ovf) && threadIdx.x == 0) atomicOr(reinterpret_cast<unsigned long long *>(flags), 4ull);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// exclusive scan of m values in place (one block), *total = their sum (saturating)
__global__ void __launch_bounds__(RT) k_rate_scan(uint64_t *v, uint64_t m, uint64_t *total) {
    __shared__ uint64_t sh[RT / 32 + 1];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < m; base += RT) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t x = i < m ? v[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_sum_sat(x, sh, &tot);
        if (i < m) v[i] = sat_add(carry, ex);
        carry = sat_add(carry, tot);
    }
    if (threadIdx.x == 0) *total = carry;
}

// sums of blocks of gaps; gap[0] counts as gap[0] - consumed
__global__ void __launch_bounds__(RT) k_rate_gsum(const uint64_t *gap, uint64_t ng, uint64_t consumed, uint64_t *gsum) {
    __shared__ uint64_t sh[RT / 32 + 1];
    const uint64_t g0 = (uint64_t)blockIdx.x * GTILE;
    uint64_t s = 0;
    for (uint64_t k = g0 + threadIdx.x; k < ng && k < g0 + GTILE; k += RT) s = sat_add(s, k == 0 ? gap[0] - consumed : gap[k]);
    uint64_t tot;
    (void)block_excl_sum_sat(s, sh, &tot);
    if (threadIdx.x == 0) gsum[blockIdx.x] = tot;
}

// positions of the sampled bytes: pos[k] = gap[0] - consumed + gap[1] + ... + gap[k]
__global__ void __launch_bounds__(RT) k_rate_gpos(const uint64_t *gap, uint64_t ng, uint64_t consumed,
                                                 const uint64_t *goff, uint64_t *pos) {
    __shared__ uint64_t sh[RT / 32 + 1];
    constexpr int GPT = GTILE / RT;
    const uint64_t g0 = (uint64_t)blockIdx.x * GTILE + (uint64_t)threadIdx.x * GPT;
    uint64_t v[GPT];
    uint64_t loc = 0;
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        const uint64_t k = g0 + q;
        v[q] = k < ng ? (k == 0 ? gap[0] - consumed : gap[k]) : 0;
        loc = sat_add(loc, v[q]);
    }
    uint64_t tot;
    uint64_t run = sat_add(goff[blockIdx.x], block_excl_sum_sat(loc, sh, &tot));
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        run = sat_add(run, v[q]);
        if (g0 + q < ng) pos[g0 + q] = run;
    }
}

// each tile: its sampled bytes, each placed at its event; counts per (line, flag)
__global__ void __launch_bounds__(RT) k_rate_apply(const int64_t *delta, const uint32_t *line, const uint8_t *py,
                                                  uint64_t n, const uint64_t *tstart, const uint64_t *pos,
                                                  uint64_t ng, uint32_t n_lines, uint64_t *counts, uint64_t *flags) {
    __shared__ uint64_t pre[RTILE];        // tile-local inclusive prefix of bytes moved
    __shared__ uint64_t sh[RT / 32 + 1];
    __shared__ uint64_t krange[2];
    const uint64_t t0 = (uint64_t)blockIdx.x * RTILE;
    const uint32_t len = (uint32_t)(n - t0 < (uint64_t)RTILE ? n - t0 : (uint64_t)RTILE);
    // each thread: RPT consecutive events
    const uint32_t j0 = threadIdx.x * RPT;
    uint64_t b[RPT];
    uint64_t loc = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        b[q] = j0 + q < len ? absu(delta[t0 + j0 + q]) : 0;
        loc = sat_add(loc, b[q]);
    }
    uint64_t tot;
    uint64_t run = block_excl_sum_sat(loc, sh, &tot);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        run = sat_add(run, b[q]);
        pre[j0 + q] = run;
    }
    const uint64_t lo = tstart[blockIdx.x], hi = sat_add(lo, tot);
    if (threadIdx.x == 0) {
        krange[0] = upper(pos, 0, ng, lo);
        krange[1] = upper(pos, krange[0], ng, hi);
    }
    __syncthreads();
    const uint64_t kl = krange[0], kh = krange[1];
    for (uint64_t k = kl + threadIdx.x; k < kh; k += RT) {
        const uint64_t rel = pos[k] - lo;   // in (0, tot]
        // the event holding byte `rel` of the tile: first j with pre[j] >= rel
        uint32_t a = 0, z = len;
        while (a < z) {
            const uint32_t m = (a + z) >> 1;
            if (pre[m] < rel) a = m + 1; else z = m;
        }
        const uint32_t l = line[t0 + a];
        if (l >= n_lines) {
            atomicOr(reinterpret_cast<unsigned long long *>(flags), 2ull);
            continue;
        }
        atomicAdd(reinterpret_cast<unsigned long long *>(&counts[2 * (uint64_t)l + (py[t0 + a] ? 1 : 0)]), 1ull);
    }
}

// the call's totals: samples, gaps used up, bytes of the next gap consumed, flags
__global__ void k_rate_state(const uint64_t *pos, uint64_t ng, uint64_t consumed, const uint64_t *total,
                             uint64_t *state) {
    if (threadIdx.x != 0) return;
    const uint64_t S = *total;
    const uint64_t K = upper(pos, 0, ng, S);
    state[0] = K;
    state[1] = K;
    if (K < ng) state[2] = K == 0 ? consumed + S : S - pos[K - 1];
    else state[2] = 0;
    if (K == ng && S > (ng ? pos[ng - 1] : 0)) atomicOr(reinterpret_cast<unsigned long long *>(&state[3]), 1ull);
}

}  // namespace

// Section 2.2 (Python vs native time): at each CPU-timer interrupt the elapsed virtual time
// T since the previous one is split between the interrupted line's Python counter (the
// quantum q) and its native counter (the delay T - q).  Reading: T < q (a timer that fired
// early) gives Python T and native 0, so every interval is attributed exactly once.
__global__ void k_cpu_attr(const int64_t *vt, const uint32_t *line, uint64_t n, int64_t q, int64_t t_prev,
                           uint32_t n_lines, int64_t *py, int64_t *nat, uint64_t *flags) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t T = vt[k] - (k ? vt[k - 1] : t_prev);
        const uint32_t l = line[k];
        if (T < 0 || l >= n_lines) {
            atomicOr(reinterpret_cast<unsigned long long *>(flags), T < 0 ? 1ull : 2ull);
            continue;
        }
        const int64_t p = T < q ? T : q;
        atomicAdd(reinterpret_cast<unsigned long long *>(&py[l]), (unsigned long long)p);
        atomicAdd(reinterpret_cast<unsigned long long *>(&nat[l]), (unsigned long long)(T - p));
    }
}

cudaError_t launch_cpu_attr(const int64_t *vt, const uint32_t *line, uint64_t n, int64_t q, int64_t t_prev,
                            uint32_t n_lines, int64_t *py, int64_t *nat, uint64_t *flags, int sms, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(py, 0, sizeof(int64_t) * n_lines, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(nat, 0, sizeof(int64_t) * n_lines, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(flags, 0, sizeof(uint64_t), s)) != cudaSuccess) return e;
    if (!n) return cudaSuccess;
    const uint64_t want = (n + RT - 1) / RT;
    const unsigned grid = (unsigned)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
    k_cpu_attr<<<grid, RT, 0, s>>>(vt, line, n, q, t_prev, n_lines, py, nat, flags);
    return cudaGetLastError();
}

size_t rate_scratch_bytes(uint64_t n, uint64_t ng) {
    const uint64_t nt = (n + RTILE - 1) / RTILE, nb = (ng + GTILE - 1) / GTILE;
    return sizeof(uint64_t) * (2 * (nt + 1) + 2 * (nb + 1) + ng + 8);
}

cudaError_t launch_rate(const int64_t *delta, const uint32_t *line, const uint8_t *py, uint64_t n,
                        const uint64_t *gap, uint64_t ng, uint64_t consumed, uint32_t n_lines, uint64_t *counts,
                        uint64_t *state, void *scratch, cudaStream_t s) {
    const uint64_t nt = (n + RTILE - 1) / RTILE, nb = (ng + GTILE - 1) / GTILE;
    uint64_t *tsum = static_cast<uint64_t *>(scratch);   // becomes the tile starts
    uint64_t *total = tsum + nt;
    uint64_t *gsum = total + 1;                          // becomes the block offsets
    uint64_t *gtot = gsum + nb;
    uint64_t *pos = gtot + 1;
    cudaError_t e;
    if ((e = cudaMemsetAsync(counts, 0, sizeof(uint64_t) * 2 * (size_t)n_lines, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(state, 0, sizeof(uint64_t) * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s)) != cudaSuccess) return e;
    if (nt) {
        k_rate_tsum<<<(unsigned)nt, RT, 0, s>>>(delta, n, tsum, state + 3);
        k_rate_scan<<<1, RT, 0, s>>>(tsum, nt, total);
    }
    if (nb) {
        k_rate_gsum<<<(unsigned)nb, RT, 0, s>>>(gap, ng, consumed, gsum);
        k_rate_scan<<<1, RT, 0, s>>>(gsum, nb, gtot);
        k_rate_gpos<<<(unsigned)nb, RT, 0, s>>>(gap, ng, consumed, gsum, pos);
    }
    if (nt && ng) k_rate_apply<<<(unsigned)nt, RT, 0, s>>>(delta, line, py, n, tsum, pos, ng, n_lines, counts, state + 3);
    k_rate_state<<<1, 32, 0, s>>>(pos, ng, consumed, total, state);
    return cudaGetLastError();
}

}  // namespace scl
