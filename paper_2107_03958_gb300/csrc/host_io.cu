// host_io.cu -- conv_apply_host: the convolution of densities held in host memory, with the
// host<->device copies pipelined against the passes (no counterpart in the paper; the link
// between host and GPU is slower than the passes, so it has to overlap them).
//
// The batch goes through in chunks of c densities: chunk i's upload (stream `in`), passes
// (stream `run`, the plan's workspace) and download (stream `out`) overlap chunk i+1's upload
// and chunk i-1's download.  Two device slots hold the chunks' densities and results; events
// order each slot's reuse.  The whole call is ordered after earlier work on the caller's
// stream, and later work on that stream after it.
#include <algorithm>

#include "wsconv_internal.h"

struct HostPipe {
    int chunk = 0;                  // densities per chunk
    size_t in_b = 0, out_b = 0;     // bytes of one density in and out
    void *din[2] = {nullptr, nullptr}, *dout[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t start = nullptr, end = nullptr, in_done[2], run_done[2], out_done[2];
    bool ok = false;
};

namespace wsc {

void destroy_hostpipe(conv_plan_s *p)
{
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
