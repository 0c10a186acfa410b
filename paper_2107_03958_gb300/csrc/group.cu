// group.cu -- mixed-size batching: a fixed list of applies, on plans that may differ in n, kernel,
// period, precision and io, captured once into one CUDA graph and run with one graph launch.
//
// Each item is out = A_n(u . mask) for its plan (Sec. 2.1, eq. (An)), the same three persistent
// pass kernels conv_apply launches.  Items on different plans become concurrent branches of the
// graph: a small grid's passes (n = 128 gives 64 row pairs, fewer CTAs than the GPU has SMs) fill
// the SMs left idle by the others.  Items on one plan share its workspace, so they stay in list
// order on that plan's branch.
#include <algorithm>
#include <vector>

#include "wsconv_internal.h"

using namespace wsc;

struct conv_group_s {
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    int items = 0;
};

namespace {

struct Item {
    conv_plan_s *plan;
    const void *u, *mask;
    void *out, *ws;
    int batch;
};

// Capture the items' passes on fresh streams: one branch per distinct plan, forked from and
// joined back into the origin stream, in ThreadLocal mode so other threads' CUDA calls go on.
conv_status capture(const std::vector<Item> &items, cudaGraph_t *graph)
{
    std::vector<conv_plan_s *> plans;
    for (const Item &it : items)
        if (std::find(plans.begin(), plans.end(), it.plan) == plans.end()) plans.push_back(it.plan);
    const size_t nb = plans.size();
    std::vector<cudaStream_t> br(nb, nullptr);
    std::vector<cudaEvent_t> join(nb, nullptr);
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    conv_status rc = CONV_OK;
    bool capturing = false;
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && rc == CONV_OK) rc = cuda_fail(e, what);
        return rc == CONV_OK;
    };
    if (cuda(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking), "cudaStreamCreate") &&
        cuda(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "cudaEventCreate")) {
        for (size_t b = 0; b < nb && rc == CONV_OK; ++b)
            cuda(cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking), "cudaStreamCreate") &&
                cuda(cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming), "cudaEventCreate");
    }
    if (rc == CONV_OK && cuda(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
        capturing = true;
        cuda(cudaEventRecord(fork, origin), "cudaEventRecord");
        for (size_t b = 0; b < nb && rc == CONV_OK; ++b) {
            if (!cuda(cudaStreamWaitEvent(br[b], fork, 0), "cudaStreamWaitEvent")) break;
            for (const Item &it : items) {
                if (it.plan != plans[b]) continue;
                rc = launch_pipeline(it.plan, it.u, it.mask, it.out, it.batch, 1.0, 0.0, 0.0, it.ws, br[b]);
                if (rc != CONV_OK) break;
                cuda(cudaGetLastError(), "pass kernel launch");
                if (rc != CONV_OK) break;
            }
            if (rc == CONV_OK) cuda(cudaEventRecord(join[b], br[b]), "cudaEventRecord") &&
                                   cuda(cudaStreamWaitEvent(origin, join[b], 0), "cudaStreamWaitEvent");
        }
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(origin, &g);
        if (rc == CONV_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
        if (rc == CONV_OK) *graph = g;
        else if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    for (size_t b = 0; b < nb; ++b) {
        if (join[b]) cudaEventDestroy(join[b]);
        if (br[b]) cudaStreamDestroy(br[b]);
    }
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
    return rc;
}

}  // namespace

extern "C" {

conv_status conv_group_create(int count, const conv_plan_t *plans, const void *const *u, const void *const *mask,
                              void *const *out, const int *batch, conv_group_t *group)
{
    if (!group) return fail(CONV_EINVAL, "group output pointer is NULL");
    *group = nullptr;
    if (count < 1) return fail(CONV_EINVAL, "a group needs at least one item");
    if (!plans || !u || !out || !batch) return fail(CONV_EINVAL, "plans, u, out and batch must be arrays of count entries");
    int dev = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    std::vector<Item> items;
    for (int i = 0; i < count; ++i) {
        conv_plan_s *p = plans[i];
        const void *mk = mask ? mask[i] : nullptr;
        void *ws = nullptr;
        conv_status rc = check_apply(p, u[i], mk, out[i], batch[i], 0.0, nullptr, &ws);
        if (rc != CONV_OK) return fail(rc, "item " + std::to_string(i) + ": " + conv_last_error());
        if (p->device != dev) return fail(CONV_EINVAL, "item " + std::to_string(i) + ": the plan is on another device");
        if (p->timing) return fail(CONV_EINVAL, "item " + std::to_string(i) + ": per-pass timing is on (a graph records no timing events)");
        if (batch[i] > 0) items.push_back({p, u[i], mk, out[i], ws, batch[i]});
    }
    // items on different plans run concurrently: none may write another's input or output
    for (size_t i = 0; i < items.size(); ++i)
        for (size_t j = 0; j < items.size(); ++j)
            if (i != j && (items[i].out == items[j].u || (i < j && items[i].out == items[j].out)))
                return fail(CONV_EINVAL, "an item's out is another item's u or out");
    auto *g = new conv_group_s;
    g->device = dev;
    g->items = (int)items.size();
    if (!items.empty()) {
        cudaGraph_t graph = nullptr;
        conv_status rc = capture(items, &graph);
        if (rc != CONV_OK) {
            delete g;
            return rc;
        }
        const cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            delete g;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    *group = g;
    return CONV_OK;
}

conv_status conv_group_launch(conv_group_t g, void *stream)
{
    if (!g) return fail(CONV_EINVAL, "group is NULL");
    int dev = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(CONV_EINVAL, "the current device is not the group's device");
    if (!g->exec) return CONV_OK;  // every item had batch 0
    WSC_CUDA(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
    return CONV_OK;
}

void conv_group_destroy(conv_group_t g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
}

}  // extern "C"
