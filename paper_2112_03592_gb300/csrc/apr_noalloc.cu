// apr_convolve_backward_noalloc: the backward pass with its scratch in a fixed device array that
// the library owns, for callers that cannot allocate device memory themselves.
//
// Who needs this: code that runs where cudaMalloc is unavailable or forbidden at call time, e.g.
// inside a host callback or a framework hook that must not allocate, in a process whose memory
// pool is fully reserved by another allocator, or in an embedded pipeline that budgets all device
// memory up front. Such callers still own their inputs and outputs; only the scratch moves here.
#include <cuda_runtime.h>

#include <mutex>

#include "apr_internal.h"

extern "C" size_t apr_backward_workspace_bytes(apr_handle_t h, int32_t k);

namespace {

// 16 MiB of scratch, 256-byte aligned. Every GPU that loads this library keeps this array until the
// process exits. All calls share it and it keeps the previous call's contents.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code the array's name is only
// a host-side stand-in, so the address is looked up once per device with that device current.
apr_status_t scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return APR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return APR_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return APR_OK;
}

}  // namespace

extern "C" {

apr_status_t apr_convolve_backward_noalloc(apr_handle_t h, const float *particles, const float *tree,
                                           const float *stencils, int32_t k, int32_t bc, const float *grad_out,
                                           float *grad_particles, float *grad_stencils, apr_stream_t stream) {
    if (!h) return APR_ERR_INVALID_ARG;
    if (k != 3 && k != 5) return APR_ERR_UNSUPPORTED;
    const size_t need = apr_backward_workspace_bytes(h, k);
    if (need > kNoAllocScratchBytes) {  // APR too large for the fixed scratch
        aprk::set_last_message("apr_convolve_backward_noalloc: this APR needs more scratch than the 16 MiB "
                               "library array; use apr_convolve_backward with a caller workspace");
        return APR_ERR_UNSUPPORTED;
    }
    void *scratch = nullptr;
    const apr_status_t st = scratch_for_current_device(&scratch);
    if (st != APR_OK) return st;
    // the three parts in order on the caller's stream (the concurrent form would create a stream)
    return aprk::convolve_backward(h, particles, tree, stencils, k, bc, grad_out, grad_particles, grad_stencils,
                                   scratch, kNoAllocScratchBytes, stream, false);
}

}  // extern "C"
