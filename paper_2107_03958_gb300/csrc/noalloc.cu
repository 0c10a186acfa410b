// noalloc.cu -- conv_apply_noalloc: the convolution with its spectrum workspace in a fixed,
// file-scope device array instead of memory the caller or the plan allocates.
//
// For callers that cannot call cudaMalloc at the point where they run the convolution: code
// running under a memory budget that forbids new device allocations, inside a real-time loop where
// an allocation could block, or in a host framework that owns all device memory and hands this
// library only input and output buffers.  The plan (moment table, twiddles) is still built by
// conv_plan beforehand; this entry point itself allocates nothing.
#include "wsconv_internal.h"

namespace wsc {

// 32 MiB of spectrum workspace.  This file's module holds no kernels, so under CUDA's lazy module
// loading the array is placed on a device when noalloc_lookup first runs there (at the first plan
// built on that device) and stays until the process exits.
#define WSCONV_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[WSCONV_NOALLOC_SCRATCH_BYTES];

// Called by the plan constructor with the plan's device current.  In host code the array's name
// stands for a host-side shadow, not a device address, so the address is asked of the runtime
// and kept in the plan: the plan lives in this context, so the address cannot go stale while the
// plan is valid, and conv_apply_noalloc never loads a module or looks anything up.  A failed
// lookup does not fail the plan; it leaves noalloc_scratch NULL and conv_apply_noalloc reports it.
void noalloc_lookup(conv_plan_s *p)
{
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        p->noalloc_scratch = nullptr;
        p->noalloc_error = std::string("cudaGetSymbolAddress(noalloc scratch) at plan creation: ") +
                           cudaGetErrorString(e);
        return;
    }
    p->noalloc_scratch = ptr;
}

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_apply_noalloc(conv_plan_t p, const void *u, const void *mask, void *out,
                                          int batch, void *stream)
{
    if (!p) return fail(CONV_EINVAL, "plan is NULL");
    if (!p->noalloc_scratch) return fail(CONV_ECUDA, p->noalloc_error);
    // conv_apply's own checks (pointers, aliasing, element alignment of u, out and mask), with the
    // array as the caller's workspace: 256-byte aligned, and batch is not held to batch_max
    void *ws = nullptr;
    conv_status rc = check_apply(p, u, mask, out, batch, 0.0, p->noalloc_scratch, &ws);
    if (rc != CONV_OK || batch == 0) return rc;
    const size_t need = workspace_bytes(p, batch);
    if (need > WSCONV_NOALLOC_SCRATCH_BYTES)
        return fail(CONV_EINVAL, "conv_apply_noalloc: this plan and batch need " + std::to_string(need) +
                                     " bytes of workspace, above the fixed " +
                                     std::to_string(WSCONV_NOALLOC_SCRATCH_BYTES) + "-byte scratch array");
    if (p->timing) return fail(CONV_EINVAL, "conv_apply_noalloc: per-pass timing is on (it creates CUDA events)");
    int dev = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(CONV_EINVAL, "the current device is not the plan's device");
    // Every element the column pass reads was written by the row pass of the same call, so the
    // array needs no clearing between calls.
    return launch_pipeline(p, u, mask, out, batch, 1.0, 0.0, 0.0, ws, reinterpret_cast<cudaStream_t>(stream));
}
