// lingam_static.cu -- lingam_fit_static: lingam_fit for callers that cannot
// allocate device memory.
//
// Some callers have no way to hand the library a device workspace: a plain C
// or Fortran host program that links this library but has no device
// allocator of its own, a plug-in that runs inside a host application whose
// memory pool owns the whole GPU, or code on a path where calling the CUDA
// allocator is not allowed (a latency-critical loop, or a callback invoked
// while another component holds the allocator).  For them this entry point
// runs the same fit in a fixed scratch area that lives in the library itself:
// a statically sized device array, reserved on every GPU the library is
// loaded on and held until the process exits.
#include <mutex>

#include "common.cuh"
#include "lingam.h"

namespace {

// The scratch area.  Host code must not use this name as a device address;
// the address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[LINGAM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this; it should come before
// any stream capture on that device).
int scratch_on_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LINGAM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return LINGAM_ECUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return LINGAM_OK;
}

}  // namespace

extern "C" int lingam_fit_static(const void* X, long long p, long long n, int* order, double* B,
                                 const lingam_opts* opts, lingam_report* report) {
    const size_t need = lingam_workspace_size(p, n, opts);
    if (need == 0 || need > size_t(LINGAM_STATIC_SCRATCH_BYTES)) return LINGAM_EINVAL;
    void* scratch = nullptr;
    const int st = scratch_on_current_device(&scratch);
    if (st != LINGAM_OK) return st;
    // lingam_fit initialises every part of its workspace it reads, so what the
    // previous call left in the scratch array does not matter.
    return lingam_fit(X, p, n, order, B, scratch, opts, report);
}
