// scl_views.h -- device addresses of host arrays (internal, host code only).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace scl {

// Device addresses of host arrays, cached per allocation.  cuPointerGetAttributes (found
// through the runtime's driver entry point) gives a pinned allocation's range and device
// address once; later arrays inside a cached range cost a lookup.  Pageable (or unknown)
// memory has no device address: nullptr, and the copy engine moves it.
class DeviceViews {
  public:
    DeviceViews() {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttributes", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ = reinterpret_cast<PFN_cuPointerGetAttributes_v7000>(fn);
    }
    const void *view(const void *p) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        for (const Range &r : ranges_)
            if (a >= r.lo && a < r.hi) return reinterpret_cast<const void *>(a + r.delta);
        if (!get_) return fallback(p);
        unsigned int type = 0;
        CUdeviceptr dptr = 0, start = 0;
        size_t size = 0;
        CUpointer_attribute attrs[] = {CU_POINTER_ATTRIBUTE_MEMORY_TYPE, CU_POINTER_ATTRIBUTE_DEVICE_POINTER,
                                       CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, CU_POINTER_ATTRIBUTE_RANGE_SIZE};
        void *data[] = {&type, &dptr, &start, &size};
        if (get_(4, attrs, data, (CUdeviceptr)a) != CUDA_SUCCESS || !size || !start) return fallback(p);
        if (type != CU_MEMORYTYPE_HOST && type != CU_MEMORYTYPE_DEVICE && type != CU_MEMORYTYPE_UNIFIED)
            return nullptr;
        if (!dptr) return nullptr;
        // dptr is the device address of p itself
        const intptr_t delta = (intptr_t)dptr - (intptr_t)a;
        if (ranges_.size() < 256) ranges_.push_back({(uintptr_t)start, (uintptr_t)start + size, delta});
        return reinterpret_cast<const void *>(dptr);
    }

  private:
    struct Range {
        uintptr_t lo, hi;
        intptr_t delta;
    };
    static const void *fallback(const void *p) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        if (at.type == cudaMemoryTypeHost && at.devicePointer) return at.devicePointer;
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
        return nullptr;
    }
    PFN_cuPointerGetAttributes_v7000 get_ = nullptr;
    std::vector<Range> ranges_;
};

}  // namespace scl
