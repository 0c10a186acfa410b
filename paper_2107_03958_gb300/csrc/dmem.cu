// dmem.cu -- device memory of plans, solver workspaces and serving buffers, from a stream-ordered
// memory pool (no counterpart in the paper; this is the memory layer of the runtime around the
// Sec. 2.1 convolution and the Sec. 3.3 solver).
//
// cudaMalloc, cudaFree and cudaMallocHost are implicit synchronisation points: kernels that other
// threads have queued on other streams must drain before work issued after the call can start, and
// cudaFree also waits on the host for the whole device.  A server that builds a plan for every new
// wave number, and evicts idle ones, would serialise the device behind whatever is in flight each
// time.  Allocations from a stream-ordered pool (cudaMallocFromPoolAsync / cudaFreeAsync) are not
// synchronisation points, so plans are built and released here:
//   - one pool per device, owned by this library, that keeps freed memory for reuse (release
//     threshold unbounded) until conv_destroy trims it;
//   - allocation and release on one private stream per device; an allocation is complete, and
//     usable from any stream, when dev_alloc returns;
//   - dev_free returns memory to the pool at once: the caller guarantees that no queued or running
//     work still reads or writes it.
// Page-locked result slots (one double per solver workspace) come from one slab per process,
// allocated once, instead of a cudaMallocHost per workspace.
#include <mutex>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

namespace {

struct DevicePool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
};

std::mutex g_pool_mu;
DevicePool g_pools[64];

// The pool and stream of device `dev`, created on first use; nullptr if that fails.
DevicePool *pool_of(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    DevicePool &P = g_pools[dev];
    if (P.pool) return &P;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return nullptr;
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return nullptr;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    bool ok = cudaMemPoolCreate(&P.pool, &props) == cudaSuccess;
    if (ok) {
        unsigned long long keep = ~0ull;
        ok = cudaMemPoolSetAttribute(P.pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess &&
             cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking) == cudaSuccess;
        if (!ok) {
            cudaMemPoolDestroy(P.pool);
            P.pool = nullptr;
            P.stream = nullptr;
        }
    } else {
        P.pool = nullptr;
    }
    if (!ok) cudaGetLastError();
    if (cur != dev) cudaSetDevice(cur);
    return ok ? &P : nullptr;
}

// Page-locked slots of 64 bytes (one cache line each), carved from slabs of 4096.
constexpr size_t SLOT_BYTES = 64, SLAB_SLOTS = 4096;
std::mutex g_slot_mu;
std::vector<void *> g_free_slots;

}  // namespace

cudaError_t dev_alloc(void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    DevicePool *P = pool_of(dev);
    if (!P) return cudaErrorInitializationError;
    e = cudaMallocFromPoolAsync(ptr, bytes, P->pool, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (*ptr) cudaFreeAsync(*ptr, P->stream);
        *ptr = nullptr;
    }
    return e;
}

void dev_free(void *ptr)
{
    if (!ptr) return;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    DevicePool *P = pool_of(at.device);
    if (!P) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != at.device) cudaSetDevice(at.device);
    if (cudaFreeAsync(ptr, P->stream) != cudaSuccess) cudaGetLastError();
    if (cur != at.device) cudaSetDevice(cur);
}

void dev_pool_trim(int dev)
{
    DevicePool *P = pool_of(dev);
    if (!P) return;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess || cudaMemPoolTrimTo(P->pool, 0) != cudaSuccess)
        cudaGetLastError();
}

double *pinned_slot()
{
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (g_free_slots.empty()) {
        void *slab = nullptr;
        if (cudaMallocHost(&slab, SLOT_BYTES * SLAB_SLOTS) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (size_t i = SLAB_SLOTS; i-- > 0;) g_free_slots.push_back(static_cast<char *>(slab) + i * SLOT_BYTES);
    }
    void *s = g_free_slots.back();
    g_free_slots.pop_back();
    return static_cast<double *>(s);
}

void pinned_slot_release(double *slot)
{
    if (!slot) return;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    g_free_slots.push_back(slot);
}

}  // namespace wsc
