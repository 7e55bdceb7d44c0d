// scl_noalloc.cu -- the copy-volume sampler (Section 3.5) as one entry point that
// allocates no memory, for callers that cannot allocate.
//
// Who cannot allocate: code that runs inside an allocation hook (a profiler's own
// interposition layer must not call the allocator it intercepts), processes whose
// device memory is owned by a caching allocator or capped by a quota (cudaMalloc
// then fails even though the work itself needs only a few MB), and latency-bound
// callers (cudaMalloc / cudaFree synchronise the device).
//
// The only scratch the copy sampler needs -- one 64-bit sum per tile of 4,096
// memcpy events -- lives in the file-scope array below, which every GPU that loads
// this library keeps until the process exits.  All other memory is the caller's.
#include <mutex>

#include "../../include/scl.h"
#include "scl_internal.cuh"

namespace scl {

constexpr uint32_t NA_MAX_TILES = 16384;   // 16,384 tiles x 4,096 events = 67,108,864 memcpy events
constexpr int NA_NT = 256;

// per-tile byte sums, then (after the scan) the copy counter before each tile: 128 KiB
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_MAX_TILES];

// per-device address of g_noalloc_scratch, looked up once per device
static std::mutex g_na_mu;
static unsigned long long *g_na_ptr[64];

__device__ unsigned long long na_block_excl(unsigned long long v, unsigned long long *sh, unsigned long long *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long y = lane < nw ? sh[lane] : 0ull, yi = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(FULL, yi, o);
            if (lane >= o) yi += t;
        }
        if (lane < nw) sh[lane] = yi - y;
        if (lane == nw - 1) sh[32] = yi;
    }
    __syncthreads();
    const unsigned long long r = x - v + sh[w];
    *total = sh[32];
    __syncthreads();
    return r;
}

// per tile: sum of the bytes copied (state[2] |= 1 on uint64 overflow)
__global__ void __launch_bounds__(NA_NT) k_na_sum(const uint64_t *size, uint64_t m, unsigned long long *scratch,
                                                   unsigned long long *state) {
    __shared__ unsigned long long sh[33];
    const uint64_t t0 = (uint64_t)blockIdx.x * COPY_TILE;
    const uint64_t t1 = t0 + COPY_TILE < m ? t0 + COPY_TILE : m;
    unsigned long long s = 0;
    int ovf = 0;
    for (uint64_t j = t0 + threadIdx.x; j < t1; j += NA_NT) {
        const unsigned long long x = size[j];
        ovf |= (s + x < s);
        s += x;
    }
    unsigned long long tot;
    (void)na_block_excl(s, sh, &tot);
    // the block total can wrap even when no thread's partial did
    if (__syncthreads_or(ovf) && threadIdx.x == 0) atomicOr(&state[2], 1ull);
    if (threadIdx.x == 0) scratch[blockIdx.x] = tot;
}

// one block: copy counter before each tile; state[0] = counter after the stream (mod T_c)
__global__ void __launch_bounds__(1024) k_na_scan(unsigned long long *scratch, uint32_t ntiles,
                                                  unsigned long long counter_in, unsigned long long Tc,
                                                  unsigned long long *state) {
    __shared__ unsigned long long sh[33];
    unsigned long long carry = counter_in;
    int ovf = 0;
    for (uint32_t base = 0; base < ntiles; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long v = i < ntiles ? scratch[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = na_block_excl(v, sh, &tot);
        if (i < ntiles) scratch[i] = carry + ex;
        ovf |= (carry + tot < carry);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        state[0] = carry % Tc;
        if (ovf) atomicOr(&state[2], 1ull);
    }
}

// per tile: samples at each memcpy = multiples of T_c passed by the running count
__global__ void __launch_bounds__(NA_NT) k_na_apply(const uint64_t *size, const uint32_t *line, const uint8_t *py,
                                                     uint64_t m, unsigned long long Tc, uint32_t n_lines,
                                                     const unsigned long long *scratch, unsigned long long *samples,
                                                     unsigned long long *bytes, unsigned long long *state) {
    __shared__ unsigned long long sh[33];
    constexpr int CPT = COPY_TILE / NA_NT;
    const uint64_t t0 = (uint64_t)blockIdx.x * COPY_TILE;
    const uint64_t len = m - t0 < (uint64_t)COPY_TILE ? m - t0 : (uint64_t)COPY_TILE;
    const uint32_t j0 = threadIdx.x * CPT;
    unsigned long long loc = 0;
    for (int k = 0; k < CPT; ++k)
        if (j0 + k < len) loc += size[t0 + j0 + k];
    unsigned long long tot;
    const unsigned long long ex = na_block_excl(loc, sh, &tot);
    unsigned long long run = scratch[blockIdx.x] + ex;
    unsigned long long qprev = run / Tc;
    unsigned long long skipped = 0;
    for (int k = 0; k < CPT; ++k) {
        const uint64_t j = t0 + j0 + k;
        if (j0 + k >= len) break;
        run += size[j];
        const unsigned long long qn = run / Tc;
        const unsigned long long q = qn - qprev;
        qprev = qn;
        if (!q) continue;
        const uint32_t l = line[j];
        if (l >= n_lines) { ++skipped; continue; }
        const int f = py[j] ? 1 : 0;
        atomicAdd(&samples[2ull * l + f], q);
        atomicAdd(&bytes[2ull * l + f], q * Tc);
    }
    if (skipped) atomicAdd(&state[1], skipped);
}

}  // namespace scl

using namespace scl;

extern "C" int scl_copy_volume_noalloc(const uint64_t *size, const uint32_t *line, const uint8_t *is_python,
                                       uint64_t m, uint64_t copy_threshold, uint64_t counter_in, uint32_t n_lines,
                                       uint64_t *samples_out, uint64_t *bytes_out, uint64_t *state_out,
                                       void *stream) {
    if (copy_threshold == 0 || counter_in >= copy_threshold || n_lines == 0 || !samples_out || !bytes_out ||
        !state_out)
        return SCL_EINVAL;
    if (m > (uint64_t)NA_MAX_TILES * COPY_TILE) return SCL_EINVAL;   // beyond the static scratch
    if (m && (!size || !line || !is_python)) return SCL_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCL_ECUDA;
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SCL_ECUDA;
            g_na_ptr[dev] = static_cast<unsigned long long *>(p);
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t rows = (size_t)n_lines * 2 * sizeof(uint64_t);
    if (cudaMemsetAsync(samples_out, 0, rows, s) != cudaSuccess) return SCL_ECUDA;
    if (cudaMemsetAsync(bytes_out, 0, rows, s) != cudaSuccess) return SCL_ECUDA;
    if (cudaMemsetAsync(state_out, 0, 3 * sizeof(uint64_t), s) != cudaSuccess) return SCL_ECUDA;
    unsigned long long *st = reinterpret_cast<unsigned long long *>(state_out);
    const uint32_t ntiles = (uint32_t)((m + COPY_TILE - 1) / COPY_TILE);
    if (ntiles) k_na_sum<<<ntiles, NA_NT, 0, s>>>(size, m, scratch, st);
    k_na_scan<<<1, 1024, 0, s>>>(scratch, ntiles, counter_in, copy_threshold, st);
    if (ntiles)
        k_na_apply<<<ntiles, NA_NT, 0, s>>>(size, line, is_python, m, copy_threshold, n_lines, scratch,
                                            reinterpret_cast<unsigned long long *>(samples_out),
                                            reinterpret_cast<unsigned long long *>(bytes_out), st);
    return cudaGetLastError() == cudaSuccess ? SCL_OK : SCL_ECUDA;
}
