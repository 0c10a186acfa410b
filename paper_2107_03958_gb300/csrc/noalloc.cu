// noalloc.cu -- conv_apply_noalloc: the convolution with its spectrum workspace in a fixed,
// file-scope device array instead of memory the caller or the plan allocates.
//
// For callers that cannot call cudaMalloc at the point where they run the convolution: code
// running under a memory budget that forbids new device allocations, inside a real-time loop where
// an allocation could block, or in a host framework that owns all device memory and hands this
// library only input and output buffers.  The plan (moment table, twiddles) is still built by
// conv_plan beforehand; this entry point itself allocates nothing.
#include <mutex>

#include "wsconv_internal.h"

namespace wsc {

// 32 MiB of spectrum workspace, resident on every GPU that loads this library until the process exits.
#define WSCONV_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[WSCONV_NOALLOC_SCRATCH_BYTES];

// Device addresses of the array, looked up once per device (host code may not use the symbol
// itself as a device pointer).
static void *g_scratch_ptr[64];
static std::mutex g_scratch_mu;

static conv_status scratch_for_device(int dev, void **out)
{
    if (dev < 0 || dev >= 64) return fail(CONV_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return CONV_OK;
}

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_apply_noalloc(conv_plan_t p, const void *u, const void *mask, void *out,
                                          int batch, void *stream)
{
    if (!p) return fail(CONV_EINVAL, "plan is NULL");
    if (batch < 0) return fail(CONV_EINVAL, "batch must be >= 0");
    if (batch == 0) return CONV_OK;
    if (!u || !out) return fail(CONV_EINVAL, "u and out must be device pointers");
    if (u == out) return fail(CONV_EINVAL, "out must not alias u");
    if (batch > 65535) return fail(CONV_EINVAL, "batch must be <= 65535");
    const size_t need = spectrum_elems(p) * (p->prec == CONV_P_FP64 ? 16 : 8) * (size_t)batch;
    if (need > WSCONV_NOALLOC_SCRATCH_BYTES)
        return fail(CONV_EINVAL, "conv_apply_noalloc: this plan and batch need " + std::to_string(need) +
                                     " bytes of workspace, above the fixed " +
                                     std::to_string(WSCONV_NOALLOC_SCRATCH_BYTES) + "-byte scratch array");
    if (p->timing) return fail(CONV_EINVAL, "conv_apply_noalloc: per-pass timing is on (it creates CUDA events)");
    int dev = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(CONV_EINVAL, "the current device is not the plan's device");
    void *scratch = nullptr;
    conv_status rc = scratch_for_device(dev, &scratch);
    if (rc != CONV_OK) return rc;
    // Every element the column pass reads was written by the row pass of the same call, so the
    // array needs no clearing between calls.
    return launch_pipeline(p, u, mask, out, batch, 1.0, 0.0, 0.0, scratch, reinterpret_cast<cudaStream_t>(stream));
}
