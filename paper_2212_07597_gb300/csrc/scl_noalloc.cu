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

// per-device address of g_noalloc_scratch and the id of the CUDA context it was looked up
// in: a context created after a reset of the device may load the module elsewhere, so a
// change of context repeats the lookup
struct NaAddr {
    unsigned long long ctx_id;
    unsigned long long *ptr;
};
static std::mutex g_na_mu;
static NaAddr g_na_addr[64];

// 64-bit add that records a carry out.  Every sum this file forms -- partial, block and
// running -- is a sum of a subset of the memcpy sizes (plus the starting counter), so a
// carry anywhere means the whole byte count passed 2^64, and no carry anywhere means every
// sum is exact.
__device__ __forceinline__ unsigned long long add_c(unsigned long long a, unsigned long long b, int &ovf) {
    const unsigned long long r = a + b;
    ovf |= r < a;
    return r;
}

// block-wide exclusive sum; *total = the block's sum; carries are ORed into ovf
__device__ unsigned long long na_block_excl(unsigned long long v, unsigned long long *sh, unsigned long long *total,
                                            int &ovf) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x = add_c(x, t, ovf);
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const unsigned long long y = lane < nw ? sh[lane] : 0ull;
        unsigned long long yi = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(FULL, yi, o);
            if (lane >= o) yi = add_c(yi, t, ovf);
        }
        if (lane < nw) sh[lane] = yi - y;
        if (lane == nw - 1) sh[32] = yi;
    }
    __syncthreads();
    const unsigned long long r = add_c(x - v, sh[w], ovf);
    *total = sh[32];
    __syncthreads();
    return r;
}

// per tile: sum of the bytes copied (state[2] = 1 when a sum carried past 2^64)
__global__ void __launch_bounds__(NA_NT) k_na_sum(const uint64_t *size, uint64_t m, unsigned long long *scratch,
                                                   unsigned long long *state) {
    __shared__ unsigned long long sh[33];
    const uint64_t t0 = (uint64_t)blockIdx.x * COPY_TILE;
    const uint64_t t1 = t0 + COPY_TILE < m ? t0 + COPY_TILE : m;
    unsigned long long s = 0;
    int ovf = 0;
    for (uint64_t j = t0 + threadIdx.x; j < t1; j += NA_NT) s = add_c(s, size[j], ovf);
    unsigned long long tot;
    (void)na_block_excl(s, sh, &tot, ovf);
    if (__syncthreads_or(ovf) && threadIdx.x == 0) state[2] = 1ull;
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
        const unsigned long long ex = na_block_excl(v, sh, &tot, ovf);
        if (i < ntiles) scratch[i] = add_c(carry, ex, ovf);
        carry = add_c(carry, tot, ovf);
    }
    ovf = __syncthreads_or(ovf);
    if (threadIdx.x == 0) {
        state[0] = carry % Tc;
        if (ovf) state[2] = 1ull;
    }
}

// per tile: samples at each memcpy = multiples of T_c passed by the running count.  When
// the count passed 2^64 (state[2], set by the kernels before this one) nothing is written,
// so the outputs stay cleared.
__global__ void __launch_bounds__(NA_NT) k_na_apply(const uint64_t *size, const uint32_t *line, const uint8_t *py,
                                                     uint64_t m, unsigned long long Tc, uint32_t n_lines,
                                                     const unsigned long long *scratch, unsigned long long *samples,
                                                     unsigned long long *bytes, unsigned long long *state) {
    __shared__ unsigned long long sh[33];
    __shared__ int wrapped;
    constexpr int CPT = COPY_TILE / NA_NT;
    if (threadIdx.x == 0) wrapped = *(volatile unsigned long long *)&state[2] != 0;
    __syncthreads();
    if (wrapped) return;   // the whole block leaves together
    const uint64_t t0 = (uint64_t)blockIdx.x * COPY_TILE;
    const uint64_t len = m - t0 < (uint64_t)COPY_TILE ? m - t0 : (uint64_t)COPY_TILE;
    const uint32_t j0 = threadIdx.x * CPT;
    int ovf = 0;
    unsigned long long loc = 0;
    for (int k = 0; k < CPT; ++k)
        if (j0 + k < len) loc = add_c(loc, size[t0 + j0 + k], ovf);
    unsigned long long tot;
    const unsigned long long ex = na_block_excl(loc, sh, &tot, ovf);
    unsigned long long run = add_c(scratch[blockIdx.x], ex, ovf);
    unsigned long long qprev = run / Tc;
    unsigned long long skipped = 0;
    for (int k = 0; k < CPT && !ovf; ++k) {
        const uint64_t j = t0 + j0 + k;
        if (j0 + k >= len) break;
        run = add_c(run, size[j], ovf);
        const unsigned long long qn = run / Tc;
        const unsigned long long q = qn - qprev;
        qprev = qn;
        if (!q || ovf) continue;
        const uint32_t l = line[j];
        if (l >= n_lines) { ++skipped; continue; }
        const int f = py[j] ? 1 : 0;
        atomicAdd(&samples[2ull * l + f], q);
        atomicAdd(&bytes[2ull * l + f], q * Tc);
    }
    // (the kernels before this one already found any carry; this is a second guard)
    if (ovf) state[2] = 1ull;
    if (skipped) atomicAdd(&state[1], skipped);
}

}  // namespace scl

using namespace scl;

namespace {

// cuCtxGetId of the driver API, reached through the runtime (no link against libcuda):
// the id of the current context, unique for the life of the process
using CtxGetIdFn = int (*)(void *ctx, unsigned long long *id);

CtxGetIdFn ctx_get_id() {
    static CtxGetIdFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetIdFn>(f);
    }();
    return fn;
}

// Device address of g_noalloc_scratch in the current context of device `dev` (current),
// looked up at the first call in each context and cached; nullptr on failure.
unsigned long long *na_scratch_address(int dev) {
    std::lock_guard<std::mutex> g(g_na_mu);
    NaAddr &a = g_na_addr[dev];
    unsigned long long id = 0;
    const CtxGetIdFn get = ctx_get_id();
    const bool have_id = get && a.ptr && get(nullptr, &id) == 0;
    if (have_id && id == a.ctx_id) return a.ptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
    // the lookup made the device's primary context current if it was not yet
    id = 0;
    if (!get || get(nullptr, &id) != 0) {
        a.ptr = nullptr;   // no context id to key on: look the address up at every call
        return static_cast<unsigned long long *>(p);
    }
    a.ctx_id = id;
    a.ptr = static_cast<unsigned long long *>(p);
    return a.ptr;
}

}  // namespace

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
    unsigned long long *scratch = na_scratch_address(dev);
    if (!scratch) return SCL_ECUDA;
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
