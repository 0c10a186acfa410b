// host_io.cu -- conv_apply_host: the convolution of densities held in host memory, with the
// host<->device copies pipelined against the passes (no counterpart in the paper; the link
// between host and GPU is slower than the passes, so it has to overlap them).
//
// The batch goes through in chunks of c densities: chunk i's upload (stream `in`), passes
// (stream `run`, the plan's workspace) and download (stream `out`) overlap chunk i+1's upload
// and chunk i-1's download.  Two device slots hold the chunks' densities and results; events
// order each slot's reuse.  The whole call is ordered after earlier work on the caller's
// stream, and later work on that stream after it.
//
// conv_apply_host_multi runs several plans on one batch: each chunk is uploaded once, the plans'
// passes run on it in turn (each with its own workspace and result slot), and each plan's result
// chunk downloads while the next plan's passes run.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "wsconv_internal.h"

struct HostPipe {
    int chunk = 0;                  // densities per chunk
    size_t in_b = 0, out_b = 0;     // bytes of one density in and out
    void *din[2] = {nullptr, nullptr}, *dout[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t start = nullptr, end = nullptr, in_done[2], run_done[2], out_done[2];
    bool ok = false;
};

// Slots of the multi-plan pipeline: with two, a plan's passes on chunk i wait for its download of
// chunk i-2, which trails when the downloads take as long as the passes.  Four (a whole batch of
// quarter-batch chunks) leave only the next call's chunks waiting on this call's downloads.
static const int kMultiSlots = 4;

struct HostMulti {
    int chunk = 0, ns = 0;              // densities per chunk, slots
    size_t in_b = 0;
    std::vector<size_t> out_b;          // per plan
    std::vector<void *> din;            // [slot]
    std::vector<void *> dout;           // [ns k + slot]
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    // start, end, in_done[ns], run_all[ns], run_done[ns K], out_done[ns K]
    std::vector<cudaEvent_t> ev;
    int K() const { return (int)out_b.size(); }
    cudaEvent_t &start() { return ev[0]; }
    cudaEvent_t &end() { return ev[1]; }
    cudaEvent_t &in_done(int s) { return ev[2 + s]; }
    cudaEvent_t &run_all(int s) { return ev[2 + ns + s]; }
    cudaEvent_t &run_done(int k, int s) { return ev[2 + 2 * ns + ns * k + s]; }
    cudaEvent_t &out_done(int k, int s) { return ev[2 + 2 * ns + ns * K() + ns * k + s]; }
};

namespace wsc {

static void destroy_hostmulti(conv_plan_s *p)
{
    HostMulti *hm = p->hostmulti;
    if (!hm) return;
    if (hm->s_in) cudaStreamSynchronize(hm->s_in);
    if (hm->s_run) cudaStreamSynchronize(hm->s_run);
    if (hm->s_out) cudaStreamSynchronize(hm->s_out);
    for (void *q : hm->din)
        if (q) cudaFree(q);
    for (void *q : hm->dout)
        if (q) cudaFree(q);
    for (cudaEvent_t e : hm->ev)
        if (e) cudaEventDestroy(e);
    if (hm->s_in) cudaStreamDestroy(hm->s_in);
    if (hm->s_run) cudaStreamDestroy(hm->s_run);
    if (hm->s_out) cudaStreamDestroy(hm->s_out);
    delete hm;
    p->hostmulti = nullptr;
}

// `ns` slots for `count` plans on chunks of `chunk` densities (kept on plans[0]; rebuilt when the
// slots, the chunk or any plan's density sizes differ from the last call's).
static conv_status make_hostmulti(conv_plan_s *const *plans, int count, int chunk, size_t in_b, int ns)
{
    conv_plan_s *p0 = plans[0];
    std::vector<size_t> out_b(count);
    for (int k = 0; k < count; ++k) {
        const size_t rb = plans[k]->prec == CONV_P_FP64 ? 8 : 4;
        out_b[k] = (size_t)plans[k]->n * plans[k]->n * rb * (plans[k]->io == CONV_IO_R2R ? 1 : 2);
    }
    if (p0->hostmulti && p0->hostmulti->chunk == chunk && p0->hostmulti->ns == ns && p0->hostmulti->in_b == in_b &&
        p0->hostmulti->out_b == out_b)
        return CONV_OK;
    destroy_hostmulti(p0);
    HostMulti *hm = new HostMulti();
    p0->hostmulti = hm;
    hm->chunk = chunk;
    hm->ns = ns;
    hm->in_b = in_b;
    hm->out_b = out_b;
    hm->din.assign(ns, nullptr);
    hm->dout.assign(ns * count, nullptr);
    hm->ev.assign(2 + 2 * ns + 2 * ns * count, nullptr);
    bool good = true;
    for (int s = 0; s < ns && good; ++s) {
        good = cudaMalloc(&hm->din[s], in_b * chunk) == cudaSuccess;
        for (int k = 0; k < count && good; ++k) good = cudaMalloc(&hm->dout[ns * k + s], out_b[k] * chunk) == cudaSuccess;
    }
    if (!good) {
        cudaGetLastError();
        destroy_hostmulti(p0);
        return fail(CONV_ENOMEM, "device slots of the multi-plan host pipeline");
    }
    good = cudaStreamCreateWithFlags(&hm->s_in, cudaStreamNonBlocking) == cudaSuccess &&
           cudaStreamCreateWithFlags(&hm->s_run, cudaStreamNonBlocking) == cudaSuccess &&
           cudaStreamCreateWithFlags(&hm->s_out, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &e : hm->ev)
        good = good && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!good) {
        cudaGetLastError();
        destroy_hostmulti(p0);
        return fail(CONV_ECUDA, "streams or events of the multi-plan host pipeline");
    }
    return CONV_OK;
}

void destroy_hostpipe(conv_plan_s *p)
{
    destroy_hostmulti(p);
    HostPipe *hp = p->hostpipe;
    if (!hp) return;
    if (hp->s_in) cudaStreamSynchronize(hp->s_in);
    if (hp->s_run) cudaStreamSynchronize(hp->s_run);
    if (hp->s_out) cudaStreamSynchronize(hp->s_out);
    for (int i = 0; i < 2; ++i) {
        if (hp->din[i]) cudaFree(hp->din[i]);
        if (hp->dout[i]) cudaFree(hp->dout[i]);
    }
    if (hp->ok) {
        for (int i = 0; i < 2; ++i) {
            cudaEventDestroy(hp->in_done[i]);
            cudaEventDestroy(hp->run_done[i]);
            cudaEventDestroy(hp->out_done[i]);
        }
        cudaEventDestroy(hp->start);
        cudaEventDestroy(hp->end);
    }
    if (hp->s_in) cudaStreamDestroy(hp->s_in);
    if (hp->s_run) cudaStreamDestroy(hp->s_run);
    if (hp->s_out) cudaStreamDestroy(hp->s_out);
    delete hp;
    p->hostpipe = nullptr;
}

// Chunks of about a quarter of the plan's batch (at least one density): enough chunks to overlap,
// each still a batched launch.
static conv_status make_hostpipe(conv_plan_s *p)
{
    HostPipe *hp = new HostPipe();
    p->hostpipe = hp;
    const size_t rb = p->prec == CONV_P_FP64 ? 8 : 4, nn = (size_t)p->n * p->n;
    hp->chunk = std::max(1, (p->batch_max + 3) / 4);
    hp->in_b = nn * rb * (p->io == CONV_IO_C2C ? 2 : 1);
    hp->out_b = nn * rb * (p->io == CONV_IO_R2R ? 1 : 2);
    for (int i = 0; i < 2; ++i)
        if (cudaMalloc(&hp->din[i], hp->in_b * hp->chunk) != cudaSuccess ||
            cudaMalloc(&hp->dout[i], hp->out_b * hp->chunk) != cudaSuccess) {
            cudaGetLastError();
            destroy_hostpipe(p);
            return fail(CONV_ENOMEM, "device slots of the host pipeline");
        }
    bool good = cudaStreamCreateWithFlags(&hp->s_in, cudaStreamNonBlocking) == cudaSuccess &&
                cudaStreamCreateWithFlags(&hp->s_run, cudaStreamNonBlocking) == cudaSuccess &&
                cudaStreamCreateWithFlags(&hp->s_out, cudaStreamNonBlocking) == cudaSuccess;
    const unsigned fl = cudaEventDisableTiming;
    good = good && cudaEventCreateWithFlags(&hp->start, fl) == cudaSuccess &&
           cudaEventCreateWithFlags(&hp->end, fl) == cudaSuccess;
    for (int i = 0; i < 2 && good; ++i)
        good = cudaEventCreateWithFlags(&hp->in_done[i], fl) == cudaSuccess &&
               cudaEventCreateWithFlags(&hp->run_done[i], fl) == cudaSuccess &&
               cudaEventCreateWithFlags(&hp->out_done[i], fl) == cudaSuccess;
    if (!good) {
        cudaGetLastError();
        destroy_hostpipe(p);
        return fail(CONV_ECUDA, "streams or events of the host pipeline");
    }
    hp->ok = true;
    return CONV_OK;
}

}  // namespace wsc

using namespace wsc;

extern "C" conv_status conv_apply_host(conv_plan_t p, const void *u_host, const void *mask, void *out_host,
                                       int batch, void *stream)
{
    if (!p) return fail(CONV_EINVAL, "plan is NULL");
    if (batch < 0) return fail(CONV_EINVAL, "batch must be >= 0");
    if (batch == 0) return CONV_OK;
    if (!u_host || !out_host) return fail(CONV_EINVAL, "u_host and out_host must be host pointers");
    if (p->timing) return fail(CONV_EINVAL, "per-pass timing is enabled on the plan");
    if (!p->hostpipe) {
        const conv_status rc = make_hostpipe(p);
        if (rc != CONV_OK) return rc;
    }
    HostPipe *hp = p->hostpipe;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    WSC_CUDA(cudaEventRecord(hp->start, st));
    WSC_CUDA(cudaStreamWaitEvent(hp->s_in, hp->start, 0));
    WSC_CUDA(cudaStreamWaitEvent(hp->s_run, hp->start, 0));
    WSC_CUDA(cudaStreamWaitEvent(hp->s_out, hp->start, 0));
    const char *uh = static_cast<const char *>(u_host);
    char *oh = static_cast<char *>(out_host);
    int slot = 0;
    for (int b0 = 0; b0 < batch; b0 += hp->chunk, slot ^= 1) {
        const int nb = std::min(hp->chunk, batch - b0);
        // slot reuse: chunk i-2's passes have read din[slot] and its download has read dout[slot]
        WSC_CUDA(cudaStreamWaitEvent(hp->s_in, hp->run_done[slot], 0));
        WSC_CUDA(cudaMemcpyAsync(hp->din[slot], uh + (size_t)b0 * hp->in_b, nb * hp->in_b, cudaMemcpyHostToDevice,
                                 hp->s_in));
        WSC_CUDA(cudaEventRecord(hp->in_done[slot], hp->s_in));
        WSC_CUDA(cudaStreamWaitEvent(hp->s_run, hp->in_done[slot], 0));
        WSC_CUDA(cudaStreamWaitEvent(hp->s_run, hp->out_done[slot], 0));
        const conv_status rc =
            launch_pipeline(p, hp->din[slot], mask, hp->dout[slot], nb, 1.0, 0.0, 0.0, p->ws, hp->s_run);
        if (rc != CONV_OK) return rc;
        WSC_CUDA(cudaEventRecord(hp->run_done[slot], hp->s_run));
        WSC_CUDA(cudaStreamWaitEvent(hp->s_out, hp->run_done[slot], 0));
        WSC_CUDA(cudaMemcpyAsync(oh + (size_t)b0 * hp->out_b, hp->dout[slot], nb * hp->out_b, cudaMemcpyDeviceToHost,
                                 hp->s_out));
        WSC_CUDA(cudaEventRecord(hp->out_done[slot], hp->s_out));
    }
    // the caller's stream continues after the last download (which follows every pass and upload)
    WSC_CUDA(cudaEventRecord(hp->end, hp->s_out));
    WSC_CUDA(cudaStreamWaitEvent(st, hp->end, 0));
    return CONV_OK;
}

extern "C" conv_status conv_apply_host_multi(int count, const conv_plan_t *plans, const void *u_host, const void *mask,
                                             void *const *out_host, int batch, void *stream)
{
    if (count < 1 || !plans) return fail(CONV_EINVAL, "count must be >= 1 and plans an array of count plans");
    if (batch < 0) return fail(CONV_EINVAL, "batch must be >= 0");
    if (!u_host || !out_host) return fail(CONV_EINVAL, "u_host and out_host must be host pointers");
    conv_plan_s *p0 = plans[0];
    int min_bmax = 1 << 30;
    for (int k = 0; k < count; ++k) {
        conv_plan_s *p = plans[k];
        if (!p) return fail(CONV_EINVAL, "plan " + std::to_string(k) + " is NULL");
        if (!out_host[k]) return fail(CONV_EINVAL, "out_host[" + std::to_string(k) + "] is NULL");
        if (p->n != p0->n || p->prec != p0->prec || (p->io == CONV_IO_C2C) != (p0->io == CONV_IO_C2C) ||
            p->device != p0->device)
            return fail(CONV_EINVAL, "the plans must share n, precision, input type (real or complex) and device");
        if (p->timing) return fail(CONV_EINVAL, "per-pass timing is enabled on plan " + std::to_string(k));
        for (int j = 0; j < k; ++j)
            if (plans[j] == p) return fail(CONV_EINVAL, "a plan appears twice (its workspace would be shared)");
        min_bmax = std::min(min_bmax, p->batch_max);
    }
    if (batch == 0) return CONV_OK;
    const size_t rb = p0->prec == CONV_P_FP64 ? 8 : 4;
    const size_t in_b = (size_t)p0->n * p0->n * rb * (p0->io == CONV_IO_C2C ? 2 : 1);
    int chunk = std::max(1, (min_bmax + 3) / 4);
    if (const char *env_c = getenv("WSCONV_HOST_CHUNK"))  // experiments: densities per chunk
        chunk = std::max(1, std::min(min_bmax, atoi(env_c)));
    const char *env_ns = getenv("WSCONV_HOST_SLOTS");  // experiments: slots per pipeline
    const int ns = env_ns ? std::max(2, std::min(8, atoi(env_ns))) : kMultiSlots;
    const conv_status rc0 = make_hostmulti(plans, count, chunk, in_b, ns);
    if (rc0 != CONV_OK) return rc0;
    HostMulti *hm = p0->hostmulti;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    WSC_CUDA(cudaEventRecord(hm->start(), st));
    WSC_CUDA(cudaStreamWaitEvent(hm->s_in, hm->start(), 0));
    WSC_CUDA(cudaStreamWaitEvent(hm->s_run, hm->start(), 0));
    WSC_CUDA(cudaStreamWaitEvent(hm->s_out, hm->start(), 0));
    const char *uh = static_cast<const char *>(u_host);
    int slot = 0;
    for (int b0 = 0; b0 < batch; b0 += chunk, slot = (slot + 1) % ns) {
        const int nb = std::min(chunk, batch - b0);
        // din[slot] is free once chunk i-ns's passes of every plan have read it
        WSC_CUDA(cudaStreamWaitEvent(hm->s_in, hm->run_all(slot), 0));
        WSC_CUDA(cudaMemcpyAsync(hm->din[slot], uh + (size_t)b0 * in_b, nb * in_b, cudaMemcpyHostToDevice, hm->s_in));
        WSC_CUDA(cudaEventRecord(hm->in_done(slot), hm->s_in));
        WSC_CUDA(cudaStreamWaitEvent(hm->s_run, hm->in_done(slot), 0));
        for (int k = 0; k < count; ++k) {
            void *dk = hm->dout[ns * k + slot];
            // plan k's result slot is free once chunk i-ns's download of it has finished
            WSC_CUDA(cudaStreamWaitEvent(hm->s_run, hm->out_done(k, slot), 0));
            const conv_status rc =
                launch_pipeline(plans[k], hm->din[slot], mask, dk, nb, 1.0, 0.0, 0.0, plans[k]->ws, hm->s_run);
            if (rc != CONV_OK) return rc;
            WSC_CUDA(cudaEventRecord(hm->run_done(k, slot), hm->s_run));
            WSC_CUDA(cudaStreamWaitEvent(hm->s_out, hm->run_done(k, slot), 0));
            WSC_CUDA(cudaMemcpyAsync(static_cast<char *>(out_host[k]) + (size_t)b0 * hm->out_b[k], dk,
                                     nb * hm->out_b[k], cudaMemcpyDeviceToHost, hm->s_out));
            WSC_CUDA(cudaEventRecord(hm->out_done(k, slot), hm->s_out));
        }
        WSC_CUDA(cudaEventRecord(hm->run_all(slot), hm->s_run));
    }
    WSC_CUDA(cudaEventRecord(hm->end(), hm->s_out));
    WSC_CUDA(cudaStreamWaitEvent(st, hm->end(), 0));
    return CONV_OK;
}
