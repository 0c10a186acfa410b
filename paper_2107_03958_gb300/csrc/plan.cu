// plan.cu -- conv_plan / conv_apply and the rest of the C ABI's host side (Sec. 2.1, eq. (io), (An)).
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

static thread_local std::string g_last_error;

// Armed host-side faults (conv_fault_inject), by kind.
static std::atomic<int> g_fault[4];

bool fault_take(int kind)
{
    if (kind < 1 || kind > 3) return false;
    int c = g_fault[kind].load();
    while (c > 0)
        if (g_fault[kind].compare_exchange_weak(c, c - 1)) return true;
    return false;
}

// CONV_FAULT="alloc:N,wait:N,drop:N" arms faults when the library loads.
[[maybe_unused]] static const bool g_fault_env = [] {
    const char *v = getenv("CONV_FAULT");
    if (!v) return false;
    std::string s(v);
    size_t i = 0;
    while (i < s.size()) {
        size_t j = s.find(',', i);
        if (j == std::string::npos) j = s.size();
        const std::string item = s.substr(i, j - i);
        const size_t c = item.find(':');
        const std::string k = item.substr(0, c);
        const int cnt = c == std::string::npos ? 1 : atoi(item.c_str() + c + 1);
        const int kind = k == "alloc" ? CONV_FAULT_ALLOC : k == "wait" ? CONV_FAULT_WAIT : k == "drop" ? CONV_FAULT_DROP : 0;
        if (kind && cnt >= 0) g_fault[kind].store(cnt);
        i = j + 1;
    }
    return true;
}();

void set_error(const std::string &msg) { g_last_error = msg; }

conv_status fail(conv_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

conv_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return CONV_ECUDA;
}

size_t spectrum_elems(const conv_plan_s *p)
{
    // R2C with complex ghat: the split pipeline's W and W2 (3 h n, plus one for W2's alignment),
    // which also holds the C2C layout (M n) that the unfused passes use
    if (p->io == CONV_IO_R2C && p->complex_ghat) return 3 * (size_t)p->h * p->n + 1;
    return (size_t)(p->io == CONV_IO_R2R ? p->h : p->M) * p->n;
}

size_t workspace_bytes(const conv_plan_s *p, int batch)
{
    if (p->long_lines) return batch > 0 ? long_lines_ws_bytes(p) : 0;  // densities run one at a time
    const size_t esz = p->prec == CONV_P_FP64 ? 16 : 8;
    // the split pass 2's scratch lines follow the spectra on an even element
    const size_t scratch = p->split_scratch_elems ? p->split_scratch_elems + 1 : 0;
    return batch > 0 ? (spectrum_elems(p) * (size_t)batch + scratch) * esz : 0;
}

void stage_twiddles(const FFTDesc &d, std::vector<double> &re_im);

// Per-stage twiddle blocks of the plan's radix sequence, in the plan precision.
static conv_status upload_twiddles(conv_plan_s *p)
{
    if (p->long_lines) return CONV_OK;  // the long-line pipeline keeps its own tables
    std::vector<double> h;
    stage_twiddles(p->fft, h);
    const bool f64 = p->prec == CONV_P_FP64;
    const size_t bytes = h.size() * (f64 ? sizeof(double) : sizeof(float));
    if (dev_alloc(&p->tw, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(CONV_ENOMEM, "cudaMalloc of the twiddle table failed");
    }
    if (f64) {
        WSC_CUDA(cudaMemcpyAsync(p->tw, h.data(), bytes, cudaMemcpyHostToDevice, p->setup_stream));
        WSC_CUDA(cudaStreamSynchronize(p->setup_stream));
    } else {
        std::vector<float> f(h.begin(), h.end());
        WSC_CUDA(cudaMemcpyAsync(p->tw, f.data(), bytes, cudaMemcpyHostToDevice, p->setup_stream));
        WSC_CUDA(cudaStreamSynchronize(p->setup_stream));
    }
    return CONV_OK;
}

std::vector<std::vector<Candidate>> transform_families(conv_plan_s *p);
conv_status apply_candidate(conv_plan_s *p, const Candidate &c);

// Re-upload the stage table and twiddles after the launch configuration changed.
static conv_status reupload(conv_plan_s *p)
{
    dev_free(p->tw);
    p->tw = nullptr;
    conv_status rc = upload_twiddles(p);
    if (rc != CONV_OK) return rc;
    WSC_CUDA(cudaMemcpyAsync(p->fft_dev, &p->fft, sizeof(FFTDesc), cudaMemcpyHostToDevice, p->setup_stream));
    WSC_CUDA(cudaStreamSynchronize(p->setup_stream));
    return CONV_OK;
}

// After a change of launch configuration: a plan workspace large enough for the new one (the
// split pass's scratch lines depend on it).
static conv_status fit_workspace(conv_plan_s *p)
{
    const size_t need = workspace_bytes(p, p->batch_max);
    if (need <= p->ws_bytes) return CONV_OK;
    WSC_CUDA(cudaStreamSynchronize(p->setup_stream));
    dev_free(p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    if (dev_alloc(&p->ws, need) != cudaSuccess) return fail(CONV_ENOMEM, "workspace allocation failed");
    p->ws_bytes = need;
    return CONV_OK;
}

// Autotuner: for every family of launch configurations (elements per thread, fused or not) time
// each distinct option set on zero densities at the plan's batch size, pass by pass; keep each
// pass's fastest option (fused passes choose independently; the plain passes share one) and the
// family with the least total.  Choices are cached per (transform length, n, precision, io,
// batch, compact) for the process.
static conv_status autotune(conv_plan_s *p)
{
    static std::mutex mu;
    static std::map<std::array<int, 6>, Candidate> cache;
    const std::array<int, 6> key = {p->M, p->n, (int)p->prec, (int)p->io, p->batch_max, p->compact ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            conv_status rc = apply_candidate(p, it->second);
            if (rc == CONV_OK) rc = reupload(p);
            return rc == CONV_OK ? fit_workspace(p) : rc;
        }
    }
    const auto fams = transform_families(p);
    size_t total = 0;
    for (const auto &f : fams) total += f.size();
    if (total <= 1) return CONV_OK;
    const int B = p->batch_max;
    const size_t rsz = p->prec == CONV_P_FP64 ? 8 : 4;
    const size_t in_b = (size_t)B * p->n * p->n * rsz * (p->io == CONV_IO_C2C ? 2 : 1);
    const size_t out_b = (size_t)B * p->n * p->n * rsz * (p->io == CONV_IO_R2R ? 1 : 2);
    void *u = nullptr, *out = nullptr;
    if (cudaMalloc(&u, in_b) != cudaSuccess || cudaMalloc(&out, out_b) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(u);
        return fail(CONV_ENOMEM, "autotuner buffers");
    }
    cudaMemsetAsync(u, 0, in_b, p->setup_stream);
    const bool was_timing = p->timing;
    double best_total = 1e300;
    Candidate pick = fams[0][0];
    conv_status rc = CONV_OK;
    for (const auto &fam : fams) {
        const bool fused = fam[0][1] != 0;
        double best_ms[3] = {1e300, 1e300, 1e300}, best_sum = 1e300;
        Candidate fpick = fam[0];
        for (const auto &c : fam) {
            rc = apply_candidate(p, c);
            // a configuration whose workspace (the split pass's scratch lines) exceeds the plan's
            if (rc == CONV_OK && workspace_bytes(p, p->batch_max) > p->ws_bytes) continue;
            if (rc == CONV_OK) rc = reupload(p);
            if (rc != CONV_OK) break;
            p->timing = false;
            for (int w = 0; w < 2; ++w) launch_pipeline(p, u, nullptr, out, B, 1.0, 0.0, 0.0, p->ws, p->setup_stream);
            p->timing = true;
            for (int r = 0; r < 3; ++r) launch_pipeline(p, u, nullptr, out, B, 1.0, 0.0, 0.0, p->ws, p->setup_stream);
            p->timing = false;
            double ms[3];
            long long cnt = 0;
            rc = conv_timing_read(p, ms, &cnt);
            if (rc != CONV_OK) break;
            if (fused) {
                for (int k = 0; k < 3; ++k)
                    if (ms[k] < best_ms[k]) {
                        best_ms[k] = ms[k];
                        fpick[2 + k] = c[2 + k];
                    }
            } else if (ms[0] + ms[1] + ms[2] < best_sum) {
                best_sum = ms[0] + ms[1] + ms[2];
                fpick = c;
            }
        }
        if (rc != CONV_OK) break;
        const double tot = fused ? best_ms[0] + best_ms[1] + best_ms[2] : best_sum;
        if (tot < best_total) {
            best_total = tot;
            pick = fpick;
        }
    }
    p->timing = was_timing;
    cudaFree(u);
    cudaFree(out);
    if (rc != CONV_OK) return rc;
    rc = apply_candidate(p, pick);
    if (rc == CONV_OK) rc = reupload(p);
    if (rc == CONV_OK) rc = fit_workspace(p);
    if (rc == CONV_OK) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = pick;
    }
    return rc;
}

cudaEvent_t *timing_slot(conv_plan_s *p)
{
    if (!p->timing) return nullptr;
    if (p->tev_free.empty()) {
        std::array<cudaEvent_t, 4> e;
        for (auto &x : e)
            if (cudaEventCreate(&x) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
        p->tev_free.push_back(e);
    }
    p->tev_used.push_back(p->tev_free.back());
    p->tev_free.pop_back();
    return p->tev_used.back().data();
}

static size_t elem_bytes(const conv_plan_s *p) { return p->prec == CONV_P_FP64 ? 16 : 8; }

// Argument checks shared by every apply entry point; on success *ws is the workspace to use
// (the caller's, or the plan's for batch <= batch_max).
conv_status check_apply(conv_plan_s *p, const void *u, const void *mask, const void *out, int batch,
                        double alpha_im, void *workspace, void **ws)
{
    if (!p) return fail(CONV_EINVAL, "plan is NULL");
    if (batch < 0) return fail(CONV_EINVAL, "batch must be >= 0");
    if (batch == 0) return CONV_OK;
    if (!u || !out) return fail(CONV_EINVAL, "u and out must be device pointers");
    if (u == out) return fail(CONV_EINVAL, "out must not alias u");
    if (p->io == CONV_IO_R2R && alpha_im != 0.0)
        return fail(CONV_EINVAL, "a real-to-real plan needs a real alpha");
    if (batch > 65535) return fail(CONV_EINVAL, "batch must be <= 65535");
    // element alignment of the caller's arrays; 16 bytes for a caller's workspace
    const size_t rb = p->prec == CONV_P_FP64 ? 8 : 4;
    auto al = [](const void *q, size_t m) { return (reinterpret_cast<uintptr_t>(q) % m) == 0; };
    if (!al(u, p->io == CONV_IO_C2C ? 2 * rb : rb) || !al(out, p->io == CONV_IO_R2R ? rb : 2 * rb) ||
        (mask && !al(mask, rb)))
        return fail(CONV_EINVAL, "u, out and mask must be aligned to their element size");
    if (workspace && !al(workspace, 16)) return fail(CONV_EINVAL, "the workspace must be 16-byte aligned");
    *ws = workspace;
    if (!workspace) {
        if (batch > p->batch_max)
            return fail(CONV_EINVAL, "batch exceeds the plan's batch_max; pass a workspace");
        *ws = p->ws;
    }
    return CONV_OK;
}

// The plan's tables and workspace go back to the memory pool at once (dmem.cu), so with
// wait_device = false the caller must know that no queued or running work uses the plan: the
// serving runtime releases only plans whose requests have completed.  conv_destroy waits for the
// device first, as a cudaFree would, and then trims the pool.
void plan_release(conv_plan_s *p, bool wait_device)
{
    if (!p) return;
    int cur = -1;
    if (wait_device) {
        cudaGetDevice(&cur);
        if (cur != p->device) cudaSetDevice(p->device);
        if (cudaDeviceSynchronize() != cudaSuccess) cudaGetLastError();
    }
    destroy_hostpipe(p);
    destroy_ls_cache(p);
    long_lines_destroy(p);
    if (p->ghat64 != p->ghat_paper) dev_free(p->ghat64);
    dev_free(p->ghat_paper);
    dev_free(p->ghat32);
    dev_free(p->tw);
    dev_free(p->fft_dev);
    if (p->setup_stream) cudaStreamDestroy(p->setup_stream);
    dev_free(p->ws);
    if (p->fp64_twin) plan_release(p->fp64_twin, false);
    for (auto &v : {&p->tev_used, &p->tev_free})
        for (auto &e : *v)
            for (auto x : e) cudaEventDestroy(x);
    if (wait_device) {
        dev_pool_trim(p->device);
        if (cur != p->device) cudaSetDevice(cur);
    }
    delete p;
}

}  // namespace wsc

using namespace wsc;

extern "C" {

const char *conv_last_error(void) { return g_last_error.c_str(); }

void conv_destroy(conv_plan_t p) { plan_release(p, true); }

conv_status conv_plan(const conv_kernel *kernel, int period_num, int period_den, int n,
                      double trunc_a, conv_precision precision, conv_io io, int batch_max,
                      conv_plan_t *plan)
{
    return conv_plan_ex(kernel, period_num, period_den, n, trunc_a, precision, io, batch_max, 0, plan);
}

// The plan constructor behind conv_plan_ex.  share: NULL, or a plan with the same kernel, period,
// n, truncation radius and embedding whose FP64 tables (moments, compact multiplier) are copied
// instead of computed again (the FP64 twin of an FP32 plan).
static conv_status plan_create(const conv_kernel *kernel, int period_num, int period_den, int n, double trunc_a,
                               conv_precision precision, conv_io io, int batch_max, int flags,
                               const conv_moments *moments, const conv_plan_s *share, conv_plan_t *plan)
{
    g_last_error.clear();
    if (!plan) return fail(CONV_EINVAL, "plan output pointer is NULL");
    *plan = nullptr;
    if (!kernel) return fail(CONV_EINVAL, "kernel is NULL");
    if (n < 1) return fail(CONV_EINVAL, "n must be >= 1");
    if (period_num < 1 || period_den < 1) return fail(CONV_EINVAL, "period must be positive");
    if ((long long)n * period_num % period_den != 0)
        return fail(CONV_EINVAL, "M = n * b must be an integer");
    long long Mll = (long long)n * period_num / period_den;
    if (Mll <= n) return fail(CONV_EINVAL, "period b must exceed 1");
    if (Mll > (1 << 24)) return fail(CONV_EUNSUPPORTED, "M too large");
    if (precision != CONV_P_FP64 && precision != CONV_P_FP32)
        return fail(CONV_EINVAL, "unknown precision");
    if (io != CONV_IO_R2R && io != CONV_IO_R2C && io != CONV_IO_C2C)
        return fail(CONV_EINVAL, "unknown io mode");
    if (batch_max < 1) return fail(CONV_EINVAL, "batch_max must be >= 1");
    const int fam = kernel->family;
    if (fam != CONV_K_LOG && fam != CONV_K_POW && fam != CONV_K_HELMHOLTZ && fam != CONV_K_YUKAWA &&
        fam != CONV_K_DX1LOG)
        return fail(CONV_EINVAL, "unknown kernel family");
    if (fam == CONV_K_DX1LOG &&
        (io != CONV_IO_R2R || (flags & CONV_PLAN_COMPACT) || (moments && moments->method != CONV_MOMENTS_CLOSED)))
        return fail(CONV_EUNSUPPORTED, "the non-radial kernel runs R2R on the period-b grid with closed-form moments");
    if ((fam == CONV_K_HELMHOLTZ || fam == CONV_K_YUKAWA) && !(kernel->kappa > 0.0))
        return fail(CONV_EINVAL, "Helmholtz and Yukawa kernels need kappa > 0");
    if (fam == CONV_K_HELMHOLTZ && io == CONV_IO_R2R)
        return fail(CONV_EINVAL, "Helmholtz kernel has a complex ghat: use R2C or C2C");
    conv_moments mo{};
    if (moments) mo = *moments;
    if (mo.method != CONV_MOMENTS_CLOSED && mo.method != CONV_MOMENTS_QUADRATURE && mo.method != CONV_MOMENTS_LOCALIZED)
        return fail(CONV_EINVAL, "unknown moment method");
    if (mo.p > 16 || mo.nodes < 0) return fail(CONV_EINVAL, "moment substitution power must be <= 16, nodes >= 0");
    if (fam == CONV_K_POW) {
        if (!(kernel->gamma > -2.0)) return fail(CONV_EINVAL, "|x|^gamma needs gamma > -2");
        double tg = 2.0 * kernel->gamma;
        if (mo.method == CONV_MOMENTS_CLOSED && std::fabs(tg - std::round(tg)) > 1e-12)
            return fail(CONV_EUNSUPPORTED, "closed-form |x|^gamma moments need 2*gamma integer (use quadrature moments)");
    }
    const int M = (int)Mll;
    if (M % 2) return fail(CONV_EUNSUPPORTED, "M = n b must be even");
    const double b = (double)period_num / period_den;
    double a = trunc_a;
    if (!(a > 0.0)) {
        if (b - 1.0 < std::sqrt(2.0))
            return fail(CONV_EINVAL, "period b < 1 + sqrt 2 admits no default truncation radius; pass trunc_a");
        a = 0.5 * (std::sqrt(2.0) + b - 1.0);
    }
    if (flags & ~(CONV_PLAN_COMPACT | CONV_PLAN_AUTOTUNE)) return fail(CONV_EINVAL, "unknown plan flags");
    if (mo.method == CONV_MOMENTS_LOCALIZED && mo.beta > a)
        return fail(CONV_EINVAL, "localization radius beta must not exceed the truncation radius a");
    conv_plan_s *p = new conv_plan_s();
    p->moments = mo;
    p->kern = *kernel;
    p->pnum = period_num;
    p->pden = period_den;
    p->n = n;
    p->Mb = M;
    p->compact = (flags & CONV_PLAN_COMPACT) != 0;
    p->M = p->compact ? 2 * n : M;
    p->h = p->M / 2 + 1;
    p->b = b;
    p->a = a;
    p->prec = precision;
    p->io = io;
    p->batch_max = batch_max;
    p->complex_ghat = fam == CONV_K_HELMHOLTZ;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(CONV_ECUDA, "no CUDA device");
    }
    if (p->M < 4) {
        delete p;
        return fail(CONV_EUNSUPPORTED, "transform length must be at least 4");
    }
    // plan-time device work runs on a private non-blocking stream, so building a plan never waits
    // for (or stalls) work other threads have in flight on the device; at the greatest priority,
    // so its short kernels start ahead of long-running work queued on other streams
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        cudaGetLastError();
        prio_hi = 0;
    }
    if (cudaStreamCreateWithPriority(&p->setup_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(CONV_ECUDA, "stream creation failed");
    }
    conv_status rc = select_transform(p);
    if (rc == CONV_OK) {
        // the stage table, then the device status word on the next 16-byte boundary
        const size_t err_off = (sizeof(FFTDesc) + 15) & ~(size_t)15;
        if (dev_alloc(&p->fft_dev, err_off + 16) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(CONV_ENOMEM, "cudaMalloc of the stage table failed");
        } else {
            p->dev_err = reinterpret_cast<int *>(reinterpret_cast<char *>(p->fft_dev) + err_off);
            if (cudaMemcpyAsync(p->fft_dev, &p->fft, sizeof(FFTDesc), cudaMemcpyHostToDevice, p->setup_stream) !=
                    cudaSuccess ||
                cudaMemsetAsync(p->dev_err, 0, sizeof(int), p->setup_stream) != cudaSuccess)
                rc = cuda_fail(cudaGetLastError(), "stage table upload");
        }
    }
    if (rc == CONV_OK) rc = upload_twiddles(p);
    if (rc == CONV_OK && p->long_lines) rc = long_lines_init(p);
    if (rc == CONV_OK) rc = share ? copy_ghat(p, share) : build_ghat(p);
    if (rc == CONV_OK) {
        p->ws_bytes = workspace_bytes(p, batch_max);
        if (fault_take(CONV_FAULT_ALLOC)) {
            rc = fail(CONV_ENOMEM, "cudaMalloc of the workspace failed (injected fault)");
        } else if (dev_alloc(&p->ws, p->ws_bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(CONV_ENOMEM, "cudaMalloc of the workspace failed");
        }
    }
    if (rc == CONV_OK) {
        cudaError_t e = cudaStreamSynchronize(p->setup_stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "plan setup");
    }
    if (rc == CONV_OK && (flags & CONV_PLAN_AUTOTUNE) && !p->long_lines) rc = autotune(p);
    if (rc == CONV_OK) noalloc_lookup(p);
    if (rc != CONV_OK) {
        conv_destroy(p);
        return rc;
    }
    *plan = p;
    return CONV_OK;
}

conv_status conv_plan_ex(const conv_kernel *kernel, int period_num, int period_den, int n,
                         double trunc_a, conv_precision precision, conv_io io, int batch_max, int flags,
                         conv_plan_t *plan)
{
    return plan_create(kernel, period_num, period_den, n, trunc_a, precision, io, batch_max, flags, nullptr, nullptr,
                       plan);
}

conv_status conv_plan_moments(const conv_kernel *kernel, int period_num, int period_den, int n, double trunc_a,
                              conv_precision precision, conv_io io, int batch_max, int flags,
                              const conv_moments *moments, conv_plan_t *plan)
{
    return plan_create(kernel, period_num, period_den, n, trunc_a, precision, io, batch_max, flags, moments, nullptr,
                       plan);
}

conv_status conv_device_status(conv_plan_t p, void *stream)
{
    if (!p) return fail(CONV_EINVAL, "null plan");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    WSC_CUDA(cudaStreamSynchronize(st));
    int word = 0;
    WSC_CUDA(cudaMemcpyAsync(&word, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    WSC_CUDA(cudaStreamSynchronize(st));
    if (word != 0) {
        WSC_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), st));
        WSC_CUDA(cudaStreamSynchronize(st));
        return fail((conv_status)word, "a pass kernel's bounded wait for an asynchronous copy gave up; the "
                                       "results of the applies since the last check are incomplete");
    }
    if (p->fp64_twin) return conv_device_status(p->fp64_twin, stream);
    return CONV_OK;
}

conv_status conv_fault_inject(int kind, int count)
{
    if (kind < CONV_FAULT_ALLOC || kind > CONV_FAULT_DROP || count < 0)
        return fail(CONV_EINVAL, "unknown fault kind or negative count");
    g_fault[kind].store(count);
    return CONV_OK;
}

conv_status conv_workspace_size(conv_plan_t p, int batch, size_t *bytes)
{
    if (!p || !bytes || batch < 0) return fail(CONV_EINVAL, "bad argument");
    *bytes = workspace_bytes(p, batch);
    return CONV_OK;
}

conv_status conv_apply_axpby(conv_plan_t p, const void *u, const void *mask, void *out, int batch,
                             double alpha_re, double alpha_im, double beta, void *workspace,
                             void *stream)
{
    void *ws = nullptr;
    conv_status rc = check_apply(p, u, mask, out, batch, alpha_im, workspace, &ws);
    if (rc != CONV_OK || batch == 0) return rc;
    return launch_pipeline(p, u, mask, out, batch, alpha_re, alpha_im, beta, ws,
                           reinterpret_cast<cudaStream_t>(stream));
}

conv_status conv_apply(conv_plan_t p, const void *u, const void *mask, void *out, int batch,
                       void *workspace, void *stream)
{
    return conv_apply_axpby(p, u, mask, out, batch, 1.0, 0.0, 0.0, workspace, stream);
}

conv_status conv_apply_kernels(conv_plan_t shape, const conv_plan_t *plans, const void *u, const void *mask,
                               void *out, int batch, void *workspace, void *stream)
{
    void *ws = nullptr;
    conv_status rc = check_apply(shape, u, mask, out, batch, 0.0, workspace, &ws);
    if (rc != CONV_OK || batch == 0) return rc;
    if (!plans) return fail(CONV_EINVAL, "plans is NULL");
    if (batch > WSC_MAX_SEL)
        return fail(CONV_EINVAL, "conv_apply_kernels takes at most " + std::to_string(WSC_MAX_SEL) + " densities");
    if (shape->long_lines) return fail(CONV_EUNSUPPORTED, "conv_apply_kernels: lines beyond one CTA");
    const void *sel[WSC_MAX_SEL];
    for (int b = 0; b < batch; ++b) {
        const conv_plan_s *q = plans[b];
        if (!q) return fail(CONV_EINVAL, "a plan in the list is NULL");
        if (q->n != shape->n || q->Mb != shape->Mb || q->M != shape->M || q->prec != shape->prec ||
            q->io != shape->io || q->compact != shape->compact || q->complex_ghat != shape->complex_ghat ||
            q->device != shape->device || q->long_lines)
            return fail(CONV_EINVAL, "conv_apply_kernels: every plan must share n, period, precision, io, "
                                     "embedding and multiplier type with the shape plan");
        sel[b] = shape->prec == CONV_P_FP64 ? (const void *)q->ghat64 : q->ghat32;
    }
    // the kernel parameters of this launch carry the tables; the plan field lasts only the launch
    shape->nsel = batch;
    for (int b = 0; b < batch; ++b) shape->sel[b] = sel[b];
    rc = launch_pipeline(shape, u, mask, out, batch, 1.0, 0.0, 0.0, ws, reinterpret_cast<cudaStream_t>(stream));
    shape->nsel = 0;
    return rc;
}

}  // extern "C"

namespace wsc {

// The plans of one conv_apply_multi: the same grid, precision, embedding and pass-1 configuration,
// each R2R or split R2C (both start with the R2R row-pair pass into W[k2][j1]).
static conv_status check_multi(const conv_plan_t *plans, int count)
{
    if (!plans || count < 1) return fail(CONV_EINVAL, "conv_apply_multi: plans is NULL or count < 1");
    const conv_plan_s *p0 = plans[0];
    for (int k = 0; k < count; ++k) {
        const conv_plan_s *q = plans[k];
        if (!q) return fail(CONV_EINVAL, "conv_apply_multi: a plan in the list is NULL");
        if (!q->fused || q->long_lines || !(q->io == CONV_IO_R2R || q->r2c_split))
            return fail(CONV_EUNSUPPORTED, "conv_apply_multi: every plan must run the fused R2R or split R2C passes");
        if (q->timing) return fail(CONV_EINVAL, "conv_apply_multi: per-pass timing is on");
        if (q->n != p0->n || q->Mb != p0->Mb || q->M != p0->M || q->prec != p0->prec || q->compact != p0->compact ||
            q->device != p0->device || q->ed != p0->ed || q->elems != p0->elems || q->rows.tpt != p0->rows.tpt ||
            q->rows.groups != p0->rows.groups)
            return fail(CONV_EINVAL, "conv_apply_multi: every plan must share n, period, precision, embedding "
                                     "and row-pass configuration");
        for (int j = 0; j < k; ++j)
            if (plans[j] == q) return fail(CONV_EINVAL, "conv_apply_multi: a plan appears twice");
    }
    return CONV_OK;
}

static size_t multi_w0_bytes(const conv_plan_s *p, int batch)
{
    const size_t esz = p->prec == CONV_P_FP64 ? 16 : 8;
    return ((size_t)batch * p->h * p->n * esz + 255) & ~(size_t)255;
}

static size_t multi_ws_bytes(const conv_plan_t *plans, int count, int batch)
{
    size_t region = 0;
    for (int k = 0; k < count; ++k) region = std::max(region, workspace_bytes(plans[k], batch));
    return multi_w0_bytes(plans[0], batch) + region;
}

}  // namespace wsc

extern "C" {

conv_status conv_multi_workspace_size(const conv_plan_t *plans, int count, int batch, size_t *bytes)
{
    if (!bytes || batch < 0) return fail(CONV_EINVAL, "bad argument");
    conv_status rc = check_multi(plans, count);
    if (rc != CONV_OK) return rc;
    *bytes = batch > 0 ? multi_ws_bytes(plans, count, batch) : 0;
    return CONV_OK;
}

conv_status conv_apply_multi(const conv_plan_t *plans, int count, const void *u, const void *mask,
                             void *const *outs, int batch, void *workspace, void *stream)
{
    conv_status rc = check_multi(plans, count);
    if (rc != CONV_OK) return rc;
    if (!outs) return fail(CONV_EINVAL, "conv_apply_multi: outs is NULL");
    if (batch < 0) return fail(CONV_EINVAL, "batch must be >= 0");
    if (batch == 0) return CONV_OK;
    for (int k = 0; k < count; ++k) {
        void *ignore = nullptr;
        rc = check_apply(plans[k], u, mask, outs[k], batch, 0.0, workspace, &ignore);
        if (rc != CONV_OK) return rc;
        for (int j = 0; j < k; ++j)
            if (outs[j] == outs[k]) return fail(CONV_EINVAL, "conv_apply_multi: two outputs alias");
    }
    int dev = 0;
    WSC_CUDA(cudaGetDevice(&dev));
    if (dev != plans[0]->device) return fail(CONV_EINVAL, "the current device is not the plans' device");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // without a caller's workspace: one from the memory pool, returned to it in stream order
    void *ws = workspace;
    const size_t need = multi_ws_bytes(plans, count, batch);
    if (!ws && dev_alloc(&ws, need) != cudaSuccess) return fail(CONV_ENOMEM, "conv_apply_multi workspace");
    char *W0 = static_cast<char *>(ws);
    void *region = W0 + multi_w0_bytes(plans[0], batch);
    // pass 1 once, into W0; then passes 2 and 3 of each plan from W0, in its own region
    conv_plan_s *p0 = plans[0];
    p0->run_passes = 1;
    rc = launch_pipeline(p0, u, mask, outs[0], batch, 1.0, 0.0, 0.0, W0, st);
    p0->run_passes = 7;
    for (int k = 0; k < count && rc == CONV_OK; ++k) {
        conv_plan_s *q = plans[k];
        q->run_passes = 6;
        q->w_in = W0;
        rc = launch_pipeline(q, u, mask, outs[k], batch, 1.0, 0.0, 0.0, region, st);
        q->run_passes = 7;
        q->w_in = nullptr;
    }
    if (!workspace) {
        if (cudaFreeAsync(ws, st) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(st);
            dev_free(ws);
        }
    }
    return rc;
}

conv_status conv_get_info(conv_plan_t p, conv_plan_info *info)
{
    if (!p || !info) return fail(CONV_EINVAL, "bad argument");
    std::memset(info, 0, sizeof(*info));
    info->n = p->n;
    info->M = p->Mb;
    info->transform_len = p->M;
    info->compact = p->compact ? 1 : 0;
    info->elems = p->elems;
    info->smem_twiddles = p->tws ? 1 : 0;
    info->fused = p->fused ? 1 : 0;
    info->static_log2 = p->fused && p->ed >= 1000 && p->ed < 2000 ? p->ed - 1000 : 0;
    info->static_len = !p->fused ? 0 : (p->ed >= 2000 ? 3 << (p->ed - 2000) : (p->ed >= 1000 ? 1 << (p->ed - 1000) : 0));
    info->r2c_split = p->r2c_split ? 1 : 0;
    info->long_lines = p->long_lines ? 1 : 0;
    info->cols_pingpong = p->cols.pp ? 1 : 0;
    info->period_num = p->pnum;
    info->period_den = p->pden;
    info->b = p->b;
    info->a = p->a;
    info->precision = p->prec;
    info->io = p->io;
    info->family = p->kern.family;
    info->batch_max = p->batch_max;
    info->nstages = p->fft.nst;
    for (int s = 0; s < p->fft.nst && s < 16; ++s) info->radices[s] = p->fft.R[s];
    info->ghat_bytes = p->ghat_bytes + (p->compact ? p->table_bytes : 0);
    info->workspace_bytes = p->ws_bytes;
    info->threads_rows = p->rows.tpt;
    info->groups_rows = p->rows.groups;
    info->threads_cols = p->cols.tpt;
    info->groups_cols = p->cols.groups;
    return CONV_OK;
}

conv_status conv_ghat_to_host(conv_plan_t p, double *host_out)
{
    if (!p || !host_out) return fail(CONV_EINVAL, "bad argument");
    WSC_CUDA(cudaMemcpy(host_out, p->ghat_paper, p->ghat_bytes, cudaMemcpyDeviceToHost));
    return CONV_OK;
}

conv_status conv_timing_enable(conv_plan_t p, int enable)
{
    if (!p) return fail(CONV_EINVAL, "plan is NULL");
    p->timing = enable != 0;
    return CONV_OK;
}

conv_status conv_timing_read(conv_plan_t p, double ms_out[3], long long *applies)
{
    if (!p || !ms_out) return fail(CONV_EINVAL, "bad argument");
    ms_out[0] = ms_out[1] = ms_out[2] = 0.0;
    for (auto &e : p->tev_used) {
        WSC_CUDA(cudaEventSynchronize(e[3]));
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            WSC_CUDA(cudaEventElapsedTime(&ms, e[k], e[k + 1]));
            ms_out[k] += ms;
        }
    }
    if (applies) *applies = (long long)p->tev_used.size();
    for (auto &e : p->tev_used) p->tev_free.push_back(e);
    p->tev_used.clear();
    return CONV_OK;
}

}  // extern "C"

namespace wsc {
// The FP64 C2C operator of an FP32 plan, for refinement residuals: same kernel, period, n, radius
// and embedding, batch 1, its FP64 tables copied from the FP32 plan's.
conv_status conv_plan_twin(const conv_plan_s *p, conv_plan_s **twin)
{
    return plan_create(&p->kern, p->pnum, p->pden, p->n, p->a, CONV_P_FP64, CONV_IO_C2C, 1,
                       p->compact ? CONV_PLAN_COMPACT : 0, &p->moments, p, twin);
}
}  // namespace wsc
