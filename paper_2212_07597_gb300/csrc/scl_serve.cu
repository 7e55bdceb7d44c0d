// scl_serve.cu -- serving loop: many profiled processes push trace segments; each
// process keeps its sampler, high-water and leak state resident on the device.
//
// Requests are host-side segments with an offered arrival time.  The loop runs on the
// calling thread with two CUDA streams:
//   - admission: a request joins the batch being filled once it has arrived and the
//     batch's device staging slot (sized from free HBM at start) has room for it;
//   - the filled slot's host->device copies go on the copy stream, and the replay of
//     the batch (scl_replay_batch) waits for them on the compute stream, so the next
//     batch's copies overlap the current batch's kernels (continuous batching: whatever
//     arrived while the device was busy forms the next batch).  Arrays in pinned (or
//     device) memory are gathered into the slot by one kernel per batch that reads them
//     through their device addresses, instead of one copy call per array; pageable
//     arrays are copied with cudaMemcpyAsync; a pinned event line column is not moved
//     at all (the kernels read line ids in place, only at the events that sample);
//   - a slot is reused only after the event recorded behind its replay has completed,
//     which is also when its requests' completion times are taken.
// Segments of one process keep their arrival order: they are replayed in that order
// across batches and, within a batch, in array order.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/scl.h"
#include "scl_launch.h"
#include "scl_views.h"

namespace {

constexpr int NSLOT = 3;
constexpr int NCOL = 7;   // event delta, addr, line, flag; memcpy size, line, flag

struct GatherJob {
    const void *src;   // device-accessible address
    void *dst;
    uint64_t bytes;
};

// one block per job at a time; 16-byte vectors (four in flight per thread) when both
// ends and the size allow, else the widest element that does
__global__ void __launch_bounds__(256) k_gather(const GatherJob *__restrict__ jobs, int njobs) {
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
        const GatherJob J = jobs[j];
        const uintptr_t al = reinterpret_cast<uintptr_t>(J.src) | reinterpret_cast<uintptr_t>(J.dst) | J.bytes;
        const uint64_t nt = blockDim.x;
        if ((al & 15) == 0) {
            const uint4 *src = static_cast<const uint4 *>(J.src);
            uint4 *dst = static_cast<uint4 *>(J.dst);
            const uint64_t nv = J.bytes / 16;
            uint64_t i = threadIdx.x;
            for (; i + 3 * nt < nv; i += 4 * nt) {
                const uint4 r0 = src[i], r1 = src[i + nt], r2 = src[i + 2 * nt], r3 = src[i + 3 * nt];
                dst[i] = r0;
                dst[i + nt] = r1;
                dst[i + 2 * nt] = r2;
                dst[i + 3 * nt] = r3;
            }
            for (; i < nv; i += nt) dst[i] = src[i];
        } else if ((al & 7) == 0) {
            const uint64_t *src = static_cast<const uint64_t *>(J.src);
            uint64_t *dst = static_cast<uint64_t *>(J.dst);
            for (uint64_t i = threadIdx.x; i < J.bytes / 8; i += nt) dst[i] = src[i];
        } else if ((al & 3) == 0) {
            const uint32_t *src = static_cast<const uint32_t *>(J.src);
            uint32_t *dst = static_cast<uint32_t *>(J.dst);
            for (uint64_t i = threadIdx.x; i < J.bytes / 4; i += nt) dst[i] = src[i];
        } else {
            const uint8_t *src = static_cast<const uint8_t *>(J.src);
            uint8_t *dst = static_cast<uint8_t *>(J.dst);
            for (uint64_t i = threadIdx.x; i < J.bytes; i += nt) dst[i] = src[i];
        }
    }
}


size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

size_t request_bytes(const scl_request &r) {
    return al256(r.ev.n * 8) * 2 + al256(r.ev.n * 4) + al256(r.ev.n) + al256(r.cp.n * 8) + al256(r.cp.n * 4) +
           al256(r.cp.n);
}

struct Slot {
    void *dev = nullptr;
    size_t cap = 0, used = 0;
    GatherJob *hjobs = nullptr, *djobs = nullptr;   // pinned table and its device copy
    std::vector<uint32_t> reqs;
    std::vector<scl_segment> segs;
    cudaEvent_t copied = nullptr, done = nullptr;
    bool busy = false;
    uint32_t batch = 0;
};

uint64_t now_ns(std::chrono::steady_clock::time_point t0) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
        .count();
}

}  // namespace

extern "C" int scl_serve(scl_ctx *ctx, const scl_request *reqs, uint32_t n, const scl_serve_opts *opts_in,
                         scl_request_result *out, scl_serve_summary *sum) {
    if (!ctx) return SCL_EINVAL;
    if (n && (!reqs || !out)) return scl_ctx_fail(ctx, SCL_EINVAL, "serve: reqs or out is NULL");
    if (cudaSetDevice(scl_ctx_device(ctx)) != cudaSuccess) return scl_ctx_fail(ctx, SCL_ECUDA, "serve: cudaSetDevice");
    scl_serve_opts opts;
    memset(&opts, 0, sizeof opts);
    if (opts_in) opts = *opts_in;
    const uint32_t max_batch = opts.max_batch ? opts.max_batch : 256;
    size_t largest = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const scl_request &r = reqs[i];
        if (r.trace_id >= scl_ctx_max_traces(ctx))
            return scl_ctx_fail(ctx, SCL_EINVAL, "serve: request trace_id >= max_traces");
        if ((r.ev.n && (!r.ev.delta || !r.ev.addr || !r.ev.line || !r.ev.is_python)) ||
            (r.cp.n && (!r.cp.size || !r.cp.line || !r.cp.is_python)))
            return scl_ctx_fail(ctx, SCL_EINVAL, "serve: NULL request array");
        if (i && r.arrival_ns < reqs[i - 1].arrival_ns)   // admission follows array order
            return scl_ctx_fail(ctx, SCL_EINVAL, "serve: arrival times must not decrease along the array");
        largest = std::max(largest, request_bytes(r));
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return scl_ctx_fail(ctx, SCL_ECUDA, "serve: cudaMemGetInfo");
    // admission budget: the caller's, else half of the free HBM, at most 8 GiB
    size_t budget = opts.hbm_budget ? opts.hbm_budget : std::min<size_t>(free_b / 2, 8ull << 30);
    if (budget > free_b) budget = free_b;
    size_t slot_cap = budget / NSLOT;
    if (slot_cap < largest)   // one request must fit a slot
        return scl_ctx_fail(ctx, SCL_ENOMEM, "serve: a staging slot cannot hold the largest request");
    slot_cap = std::min(slot_cap, largest * (size_t)max_batch);

    cudaStream_t cs = nullptr, ks = nullptr;
    Slot slots[NSLOT];
    int rc = SCL_OK;
    auto cleanup = [&]() {
        for (auto &sl : slots) {
            if (sl.dev) cudaFree(sl.dev);
            if (sl.djobs) cudaFree(sl.djobs);
            if (sl.hjobs) cudaFreeHost(sl.hjobs);
            if (sl.copied) cudaEventDestroy(sl.copied);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        if (cs) cudaStreamDestroy(cs);
        if (ks) cudaStreamDestroy(ks);
    };
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking) != cudaSuccess) {
        cleanup();
        return SCL_ECUDA;
    }
    for (auto &sl : slots) {
        if (cudaMalloc(&sl.dev, slot_cap) != cudaSuccess ||
            cudaMalloc(&sl.djobs, sizeof(GatherJob) * NCOL * max_batch) != cudaSuccess ||
            cudaMallocHost(&sl.hjobs, sizeof(GatherJob) * NCOL * max_batch) != cudaSuccess) {
            cleanup();
            return scl_ctx_fail(ctx, SCL_ENOMEM, "serve: staging slots");
        }
        sl.cap = slot_cap;
        cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }

    const auto t0 = std::chrono::steady_clock::now();
    uint32_t next = 0;          // next request to admit (arrival order = array order)
    uint32_t completed = 0, batches = 0;
    uint64_t events = 0;
    int fill = 0;               // slot being filled
    for (uint32_t i = 0; i < n; ++i) memset(&out[i], 0, sizeof out[i]);

    auto retire = [&](Slot &sl) {
        const uint64_t t = now_ns(t0);
        for (uint32_t r : sl.reqs) {
            out[r].done_ns = t;
            const uint64_t arr = opts.realtime ? reqs[r].arrival_ns : 0;
            out[r].latency_ns = t > arr ? t - arr : 0;
            out[r].batch = sl.batch;
        }
        completed += (uint32_t)sl.reqs.size();
        sl.reqs.clear();
        sl.segs.clear();
        sl.used = 0;
        sl.busy = false;
    };
    auto poll = [&](bool block) {
        for (auto &sl : slots) {
            if (!sl.busy) continue;
            cudaError_t q = block ? cudaEventSynchronize(sl.done) : cudaEventQuery(sl.done);
            if (q == cudaSuccess) retire(sl);
            else if (q != cudaErrorNotReady) rc = SCL_ECUDA;
        }
    };
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, scl_ctx_device(ctx)) != cudaSuccess) sms = 1;
    scl::DeviceViews views;
    auto dispatch = [&](Slot &sl) -> int {
        // pinned or device arrays: one gather kernel on the copy stream; pageable: copy calls
        char *p = static_cast<char *>(sl.dev);
        int nj = 0;
        for (size_t k = 0; k < sl.reqs.size(); ++k) {
            const scl_request &r = reqs[sl.reqs[k]];
            scl_segment g;
            memset(&g, 0, sizeof g);
            g.trace_id = r.trace_id;
            bool bad = false;
            auto put = [&](const void *src, size_t bytes) -> void * {
                char *dst = p;
                p += al256(bytes);
                if (!bytes) return dst;
                if (const void *dv = views.view(src)) {
                    sl.hjobs[nj++] = GatherJob{dv, dst, bytes};
                } else if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs) != cudaSuccess) {
                    bad = true;
                }
                return dst;
            };
            g.ev.n = r.ev.n;
            g.ev.delta = static_cast<const int64_t *>(put(r.ev.delta, r.ev.n * 8));
            g.ev.addr = static_cast<const uint64_t *>(put(r.ev.addr, r.ev.n * 8));
            // event line ids are read only where a sample fires: a pinned column is read in place
            if (const void *lv = r.ev.n ? views.view(r.ev.line) : nullptr) {
                g.ev.line = static_cast<const uint32_t *>(lv);
                p += al256(r.ev.n * 4);
            } else {
                g.ev.line = static_cast<const uint32_t *>(put(r.ev.line, r.ev.n * 4));
            }
            g.ev.is_python = static_cast<const uint8_t *>(put(r.ev.is_python, r.ev.n));
            g.cp.n = r.cp.n;
            g.cp.size = static_cast<const uint64_t *>(put(r.cp.size, r.cp.n * 8));
            g.cp.line = static_cast<const uint32_t *>(put(r.cp.line, r.cp.n * 4));
            g.cp.is_python = static_cast<const uint8_t *>(put(r.cp.is_python, r.cp.n));
            if (bad) return scl_ctx_fail(ctx, SCL_ECUDA, "serve: host-to-device copy");
            sl.segs.push_back(g);
            events += r.ev.n;
        }
        if (nj) {
            if (cudaMemcpyAsync(sl.djobs, sl.hjobs, sizeof(GatherJob) * nj, cudaMemcpyHostToDevice, cs) != cudaSuccess)
                return scl_ctx_fail(ctx, SCL_ECUDA, "serve: gather table upload");
            k_gather<<<std::min(nj, sms * 8), 256, 0, cs>>>(sl.djobs, nj);
            if (cudaGetLastError() != cudaSuccess) return scl_ctx_fail(ctx, SCL_ECUDA, "serve: gather launch");
        }
        if (cudaEventRecord(sl.copied, cs) != cudaSuccess) return SCL_ECUDA;
        if (cudaStreamWaitEvent(ks, sl.copied, 0) != cudaSuccess) return SCL_ECUDA;
        const int r = scl_replay_batch(ctx, sl.segs.data(), (uint32_t)sl.segs.size(), ks);
        if (r) return r;
        if (cudaEventRecord(sl.done, ks) != cudaSuccess) return SCL_ECUDA;
        sl.busy = true;
        sl.batch = batches++;
        return SCL_OK;
    };

    while (completed < n && rc == SCL_OK) {
        poll(false);
        Slot &sl = slots[fill];
        if (sl.busy) {   // every slot is in flight: wait for the oldest (slots fill in turn)
            const cudaError_t q = cudaEventSynchronize(sl.done);
            if (q != cudaSuccess) { rc = SCL_ECUDA; break; }
            retire(sl);
            continue;
        }
        // admit every arrived request that fits
        const uint64_t t = now_ns(t0);
        while (next < n && sl.reqs.size() < max_batch &&
               (!opts.realtime || reqs[next].arrival_ns <= t) && sl.used + request_bytes(reqs[next]) <= sl.cap) {
            sl.used += request_bytes(reqs[next]);
            sl.reqs.push_back(next++);
        }
        if (!sl.reqs.empty()) {
            rc = dispatch(sl);
            fill = (fill + 1) % NSLOT;
            continue;
        }
        if (next < n && opts.realtime) {
            // nothing arrived yet: wait a little (or until a batch completes)
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else if (next >= n) {
            poll(true);
        }
    }
    poll(true);
    const uint64_t wall = now_ns(t0);
    if (sum) {
        memset(sum, 0, sizeof *sum);
        sum->requests = n;
        sum->batches = batches;
        sum->events = events;
        uint64_t first = n ? (opts.realtime ? reqs[0].arrival_ns : 0) : 0;
        sum->wall_s = (double)(wall - std::min(first, wall)) * 1e-9;
        sum->staging_bytes = (uint64_t)slot_cap * NSLOT;
    }
    // the first error a kernel recorded, read while the compute stream still exists
    if (cudaStreamSynchronize(ks) != cudaSuccess && rc == SCL_OK) rc = scl_ctx_fail(ctx, SCL_ECUDA, "serve: stream");
    if (rc == SCL_OK && batches) rc = scl_sync(ctx);
    if (batches) scl_ctx_forget_stream(ctx);
    cleanup();
    return rc;
}
