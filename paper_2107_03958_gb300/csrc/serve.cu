// serve.cu -- continuous-batching request loop over conv_apply and ls_solve (no counterpart in the
// paper; this is the serving layer around the Sec. 2.1 convolution and the Sec. 3.3 solver).
//
// Requests arrive at any time (srv_submit).  A dispatcher thread admits them first-fit against a
// device-memory budget (plan tables, workspaces, Krylov bases) and keeps plans resident in a cache.
//   - Plans are built on builder threads, off the dispatcher: a request whose plan is missing waits
//     for its build while every other request keeps flowing.
//   - Convolution requests wait in one ready queue per transform shape (n, period, precision, io):
//     requests on different kernels (log, |x|^gamma, Helmholtz with any kappa) share a shape.  A
//     shape's queue is launched as one batch when nothing of that shape is on the GPU, or when it
//     holds a full batch; requests that arrive while a batch runs gather into the next one.  A
//     batch of several plans is one conv_apply_kernels launch per pass (each density with its own
//     plan's multiplier) on the leading request's plan, its inputs gathered into that plan's
//     staging buffer and its results scattered back.
//   - Lippmann-Schwinger requests run on worker threads, each solve on its own stream,
//     overlapping with everything else.
// A completion thread polls the batches' events; srv_wait blocks on a request's completion.
// Results do not depend on what else is in flight: each density of a batch is transformed by the
// same kernels with the same arithmetic as alone, and GMRES uses fixed-order reductions.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "wsconv_internal.h"

namespace wsc {

static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct PlanKey {
    int family;
    double gamma, kappa, scale;
    int n, pnum, pden, prec, io;
    bool operator<(const PlanKey &o) const
    {
        return std::tie(family, gamma, kappa, scale, n, pnum, pden, prec, io) <
               std::tie(o.family, o.gamma, o.kappa, o.scale, o.n, o.pnum, o.pden, o.prec, o.io);
    }
};

struct ShapeKey {
    int n, pnum, pden, prec, io;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(n, pnum, pden, prec, io) < std::tie(o.n, o.pnum, o.pden, o.prec, o.io);
    }
};

struct CachedPlan {
    conv_plan_t plan = nullptr;
    cudaStream_t stream = nullptr;
    void *stage_in = nullptr, *stage_out = nullptr;  // batching staging buffers (conv plans)
    size_t bytes = 0;
    int users = 0;       // admitted requests currently holding the plan
    double last_use = 0;
    std::mutex run_mu;   // LS plans: one solve at a time per plan (shared workspace)
};

struct Req {
    long long ticket;
    srv_request r;
    srv_result res;
    size_t need = 0;     // bytes reserved while admitted (beyond the plan)
    bool done = false;
    bool admitted = false;  // taken off the pending queue by the dispatcher
    std::shared_ptr<CachedPlan> cp;
};

struct Batch {
    std::vector<std::shared_ptr<Req>> reqs;
    std::shared_ptr<CachedPlan> cp;  // the leading request's plan: stream, staging, workspace
    ShapeKey shape{};
    cudaEvent_t ev = nullptr;
    int pin = -1;  // pinned slot receiving the plan's device status word after the apply
};

// A plan being built: the bytes reserved for it at admission and the requests waiting for it.
struct BuildJob {
    srv_request r;  // the request that asked first (its kernel and shape)
    size_t reserved = 0;
    std::vector<std::shared_ptr<Req>> waiters;
};

}  // namespace wsc

struct srv_s {
    size_t budget = 0, in_use = 0;
    int max_inflight = 64, batch_max = 16, ls_workers = 4, plan_flags = 0;
    int *status_pin = nullptr;  // pinned host slots, one per batch in flight
    std::vector<int> free_pins;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_done, cv_ls;
    std::deque<std::shared_ptr<wsc::Req>> pending;
    std::map<long long, std::shared_ptr<wsc::Req>> all;
    std::map<wsc::PlanKey, std::shared_ptr<wsc::CachedPlan>> plans;
    std::map<wsc::PlanKey, wsc::BuildJob> building;          // plans being built
    std::deque<wsc::PlanKey> build_queue;                     // ... not yet taken by a builder:
                                                              // convolution plans ahead of LS plans
    int prio_hi = 0, prio_lo = 0;                             // stream priorities (greatest, least)
    std::map<wsc::ShapeKey, std::deque<std::shared_ptr<wsc::Req>>> ready;  // conv requests by shape
    std::map<wsc::ShapeKey, int> shape_inflight;              // batches of a shape on the GPU
    std::deque<wsc::Batch> inflight;
    std::deque<std::shared_ptr<wsc::Req>> ls_queue;
    int inflight_reqs = 0;
    long long next_ticket = 1;
    bool stop = false;
    int device = 0;
    std::condition_variable cv_build;
    std::thread dispatcher, completer;
    std::vector<std::thread> workers, builders;
    srv_stats stats{};
};

namespace wsc {

static size_t elem_bytes_of(int prec) { return prec == CONV_P_FP64 ? 8 : 4; }

static PlanKey key_of(const srv_request &r)
{
    PlanKey k;
    k.family = r.kernel.family;
    k.gamma = r.kernel.gamma;
    k.kappa = r.kernel.kappa;
    k.scale = r.kernel.scale;
    k.n = r.n;
    k.pnum = r.period_num;
    k.pden = r.period_den;
    k.prec = r.kind == SRV_LS ? r.precision : r.precision;
    k.io = r.kind == SRV_LS ? CONV_IO_C2C + 100 : r.io;  // LS plans are cached apart from conv plans
    return k;
}

static ShapeKey shape_of(const srv_request &r)
{
    return ShapeKey{r.n, r.period_num, r.period_den, r.precision, r.io};
}

// Bytes of one LS solve's Krylov basis and vectors.
static size_t request_bytes(const srv_request &r)
{
    if (r.kind != SRV_LS) return 0;
    const size_t N = (size_t)r.n * r.n;
    const int restart = r.restart > 0 ? r.restart : 50;
    return N * 16 * (restart + 5) + N * 8 * 4;
}

// What an LS plan keeps after its first solve, for as long as it stays cached: the Krylov
// workspace (ls_solve keeps one with the plan) and, in mixed precision, the FP64 twin (its copies
// of the moment and compact tables and its workspace).
static size_t ls_resident_bytes(const srv_request &r, int flags)
{
    if (r.kind != SRV_LS) return 0;
    const long long n = r.n, Mb = n * r.period_num / r.period_den;
    const long long M = (flags & CONV_PLAN_COMPACT) ? 2 * n : Mb, h = M / 2 + 1, hb = Mb / 2 + 1;
    size_t twin = 0;
    if (r.precision == CONV_P_FP32)
        twin = (size_t)hb * hb * 16 + ((flags & CONV_PLAN_COMPACT) ? (size_t)h * h * 16 : 0) + (size_t)M * n * 16;
    return request_bytes(r) + twin;
}

// Device bytes of a plan (moment table, twiddles, workspace) plus, for conv plans, the staging
// buffers of one batch, and for LS plans what ls_resident_bytes counts; estimated from the sizes
// before the plan exists.
static size_t plan_bytes_estimate(const srv_request &r, int batch_max, int flags)
{
    const long long n = r.n, Mb = n * r.period_num / r.period_den;
    const long long M = (flags & CONV_PLAN_COMPACT) ? 2 * n : Mb, h = M / 2 + 1;
    const size_t cz = 2 * elem_bytes_of(r.precision);
    const bool c2c = r.kind == SRV_LS || r.io != CONV_IO_R2R;
    const long long hb = Mb / 2 + 1;
    size_t ghat = (size_t)hb * hb * 8 * (r.kernel.family == CONV_K_HELMHOLTZ ? 2 : 1);
    if (flags & CONV_PLAN_COMPACT) ghat += (size_t)h * h * 8 * (r.kernel.family == CONV_K_HELMHOLTZ ? 2 : 1);
    if (r.precision == CONV_P_FP32) ghat += ghat / 2;
    const int B = r.kind == SRV_LS ? 1 : batch_max;
    const bool split = r.kind == SRV_CONV && r.io == CONV_IO_R2C && r.kernel.family == CONV_K_HELMHOLTZ;
    size_t ws = (size_t)(split ? 3 * h + 1 : (c2c ? M : h)) * n * cz * B;
    size_t stage = 0;
    if (r.kind == SRV_CONV) {
        const size_t in_b = (size_t)n * n * (r.io == CONV_IO_C2C ? cz : cz / 2);
        const size_t out_b = (size_t)n * n * (r.io == CONV_IO_R2R ? cz / 2 : cz);
        stage = (in_b + out_b) * batch_max;
    }
    return ghat + ws + stage + ls_resident_bytes(r, flags) + (size_t)M * cz * 4;
}

static void finish(srv_t s, const std::shared_ptr<Req> &q, int status, double t_done)
{
    q->res.status = status;
    q->res.t_done = t_done;
    q->done = true;
    s->in_use -= q->need;
    if (q->cp) {
        q->cp->users--;
        q->cp->last_use = t_done;
    }
    s->inflight_reqs--;
    s->stats.completed++;
    if (status != CONV_OK) s->stats.failed++;
}

// Evict idle cached plans (oldest first) until `need` more bytes fit.  Caller holds s->mu.
static bool make_room(srv_t s, size_t need)
{
    while (s->in_use + need > s->budget) {
        auto victim = s->plans.end();
        for (auto it = s->plans.begin(); it != s->plans.end(); ++it)
            if (it->second->users == 0 && (victim == s->plans.end() || it->second->last_use < victim->second->last_use))
                victim = it;
        if (victim == s->plans.end()) return false;
        auto cp = victim->second;
        s->plans.erase(victim);
        s->in_use -= cp->bytes;
        // idle: every request that held it has completed (their batches' events, their solves'
        // stream syncs), so its memory returns to the pool without a device-wide wait
        cudaStreamSynchronize(cp->stream);
        plan_release(cp->plan, false);
        cudaStreamDestroy(cp->stream);
        dev_free(cp->stage_in);
        dev_free(cp->stage_out);
        s->stats.plans_evicted++;
    }
    return true;
}

// Builds the plan of request r (no lock held); nullptr with the status on failure.
static std::shared_ptr<CachedPlan> build_plan(srv_t s, const srv_request &r, int &status)
{
    cudaSetDevice(s->device);
    auto cp = std::make_shared<CachedPlan>();
    const conv_io io = r.kind == SRV_LS ? CONV_IO_C2C : (conv_io)r.io;
    status = conv_plan_ex(&r.kernel, r.period_num, r.period_den, r.n, 0.0, (conv_precision)r.precision, io,
                          r.kind == SRV_LS ? 1 : s->batch_max, s->plan_flags, &cp->plan);
    if (status != CONV_OK) return nullptr;
    // convolution batches at the greatest priority: a batch is short and its requests wait on it,
    // while LS solves (least priority) run for many milliseconds
    cudaStreamCreateWithPriority(&cp->stream, cudaStreamNonBlocking, s->prio_hi);
    conv_plan_info inf;
    conv_get_info(cp->plan, &inf);
    cp->bytes = inf.ghat_bytes + inf.workspace_bytes + (inf.precision == CONV_P_FP32 ? inf.ghat_bytes / 2 : 0) +
                ls_resident_bytes(r, s->plan_flags);
    if (r.kind == SRV_CONV) {
        const size_t cz = 2 * elem_bytes_of(r.precision);
        const size_t in_b = (size_t)r.n * r.n * (io == CONV_IO_C2C ? cz : cz / 2);
        const size_t out_b = (size_t)r.n * r.n * (io == CONV_IO_R2R ? cz / 2 : cz);
        if (dev_alloc(&cp->stage_in, in_b * s->batch_max) != cudaSuccess ||
            dev_alloc(&cp->stage_out, out_b * s->batch_max) != cudaSuccess) {
            cudaGetLastError();
            dev_free(cp->stage_in);
            cudaStreamDestroy(cp->stream);
            plan_release(cp->plan, false);
            status = fail(CONV_ENOMEM, "serving staging buffers");
            return nullptr;
        }
        cp->bytes += (in_b + out_b) * s->batch_max;
    }
    return cp;
}

static size_t in_bytes(const srv_request &r)
{
    const size_t e = elem_bytes_of(r.precision);
    return (size_t)r.n * r.n * (r.io == CONV_IO_C2C ? 2 * e : e);
}
static size_t out_bytes(const srv_request &r)
{
    const size_t e = elem_bytes_of(r.precision);
    return (size_t)r.n * r.n * (r.io == CONV_IO_R2R ? e : 2 * e);
}

// Launch one batch of same-shape convolution requests on the leading plan's stream.  Caller holds
// s->mu.
static void launch_batch(srv_t s, Batch &bt)
{
    auto &cp = bt.cp;
    const srv_request &r0 = bt.reqs[0]->r;
    const double t0 = now_s();
    const int B = (int)bt.reqs.size();
    conv_status st;
    if (B == 1) {
        st = conv_apply(cp->plan, r0.in, r0.mask, r0.out, 1, nullptr, cp->stream);
    } else {
        const size_t ib = in_bytes(r0), ob = out_bytes(r0);
        conv_plan_t plans[WSC_MAX_SEL];
        for (int i = 0; i < B; ++i) {
            plans[i] = bt.reqs[i]->cp->plan;
            cudaMemcpyAsync((char *)cp->stage_in + i * ib, bt.reqs[i]->r.in, ib, cudaMemcpyDeviceToDevice, cp->stream);
        }
        st = conv_apply_kernels(cp->plan, plans, cp->stage_in, r0.mask, cp->stage_out, B, nullptr, cp->stream);
        for (int i = 0; i < B; ++i)
            cudaMemcpyAsync(bt.reqs[i]->r.out, (char *)cp->stage_out + i * ob, ob, cudaMemcpyDeviceToDevice, cp->stream);
    }
    if (st == CONV_OK && !s->free_pins.empty()) {
        bt.pin = s->free_pins.back();
        s->free_pins.pop_back();
        s->status_pin[bt.pin] = 0;
        cudaMemcpyAsync(&s->status_pin[bt.pin], cp->plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost, cp->stream);
    }
    cudaEventCreateWithFlags(&bt.ev, cudaEventDisableTiming);
    cudaEventRecord(bt.ev, cp->stream);
    for (auto &q : bt.reqs) {
        q->res.t_start = t0;
        q->res.batched_with = B;
        q->res.status = st;
    }
    s->shape_inflight[bt.shape]++;
    s->stats.batches++;
    s->stats.batched_requests += B;
}

// An admitted request whose plan is resident: conv requests join their shape's ready queue, LS
// solves the workers' queue.  Caller holds s->mu.
static void route(srv_t s, const std::shared_ptr<Req> &q, const std::shared_ptr<CachedPlan> &cp)
{
    q->cp = cp;
    cp->users++;
    if (q->r.kind == SRV_LS) {
        s->ls_queue.push_back(q);
        s->cv_ls.notify_one();
    } else {
        s->ready[shape_of(q->r)].push_back(q);
    }
}

static void dispatcher_loop(srv_t s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // admission: first fit in arrival order
        for (auto it = s->pending.begin(); it != s->pending.end();) {
            auto q = *it;
            if (s->inflight_reqs >= s->max_inflight) break;
            const PlanKey k = key_of(q->r);
            const auto pit = s->plans.find(k);
            const auto bit = s->building.find(k);
            const bool have = pit != s->plans.end(), queued = bit != s->building.end();
            // an LS solve on an idle plan uses the Krylov workspace the plan keeps (counted in its
            // bytes); one beside another solve on the same plan allocates its own
            const bool shares = (have && pit->second->users > 0) || (queued && !bit->second.waiters.empty());
            const size_t extra = shares ? request_bytes(q->r) : 0;
            const size_t plan_need = (have || queued) ? 0 : plan_bytes_estimate(q->r, s->batch_max, s->plan_flags);
            const size_t need = extra + plan_need;
            if (need > s->budget) {  // can never fit
                it = s->pending.erase(it);
                q->admitted = true;
                s->inflight_reqs++;
                q->need = 0;
                finish(s, q, fail(CONV_ENOMEM, "request exceeds the serving memory budget"), now_s());
                s->cv_done.notify_all();
                continue;
            }
            if (s->in_use + need > s->budget && !make_room(s, need)) {
                ++it;
                continue;
            }
            it = s->pending.erase(it);
            q->admitted = true;
            s->inflight_reqs++;
            q->need = extra;
            s->in_use += need;
            if (have) {
                route(s, q, pit->second);
            } else if (queued) {
                bit->second.waiters.push_back(q);
            } else {
                BuildJob &job = s->building[k];
                job.r = q->r;
                job.reserved = plan_need;
                job.waiters.push_back(q);
                // a convolution waits only for its plan, a solve runs for many times longer:
                // convolution plans are built first
                if (q->r.kind == SRV_CONV) {
                    auto pos = s->build_queue.begin();
                    while (pos != s->build_queue.end() && pos->io < CONV_IO_C2C + 100) ++pos;
                    s->build_queue.insert(pos, k);
                } else {
                    s->build_queue.push_back(k);
                }
                s->cv_build.notify_one();
            }
        }
        // launch: a shape's ready requests go as one batch when nothing of that shape is on the GPU
        // or a full batch is waiting; a batch shares one mask
        for (auto &kv : s->ready) {
            auto &dq = kv.second;
            while (!dq.empty() && (s->shape_inflight[kv.first] == 0 || (int)dq.size() >= s->batch_max)) {
                Batch bt;
                bt.shape = kv.first;
                bt.cp = dq.front()->cp;
                const void *mask = dq.front()->r.mask;
                for (auto qi = dq.begin(); qi != dq.end() && (int)bt.reqs.size() < s->batch_max;) {
                    if ((*qi)->r.mask == mask) {
                        bt.reqs.push_back(*qi);
                        qi = dq.erase(qi);
                    } else {
                        ++qi;
                    }
                }
                launch_batch(s, bt);
                s->inflight.push_back(bt);
            }
        }
        s->cv_dispatch.wait_for(lk, std::chrono::microseconds(200));
    }
}

// Builder: takes a plan key from the queue, builds the plan without the lock, then makes it
// resident and routes the requests that waited for it (or fails them with the build's status).
static void builder_loop(srv_t s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_build.wait(lk, [&] { return s->stop || !s->build_queue.empty(); });
        if (s->build_queue.empty()) break;
        const PlanKey k = s->build_queue.front();
        s->build_queue.pop_front();
        const srv_request r = s->building[k].r;
        lk.unlock();
        int status = CONV_OK;
        auto cp = build_plan(s, r, status);
        lk.lock();
        BuildJob job = std::move(s->building[k]);
        s->building.erase(k);
        if (cp) {
            s->in_use += cp->bytes;
            s->in_use -= job.reserved;
            s->plans[k] = cp;
            s->stats.plans_built++;
            for (auto &q : job.waiters) route(s, q, cp);
        } else {
            s->in_use -= job.reserved;
            const double t = now_s();
            for (auto &q : job.waiters) finish(s, q, status, t);
            s->cv_done.notify_all();
        }
        s->cv_dispatch.notify_one();
    }
}

static void completer_loop(srv_t s)
{
    cudaSetDevice(s->device);
    while (true) {
        std::vector<Batch> done;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop && s->inflight.empty()) break;
            for (auto it = s->inflight.begin(); it != s->inflight.end();) {
                if (cudaEventQuery(it->ev) == cudaSuccess) {
                    done.push_back(*it);
                    it = s->inflight.erase(it);
                } else {
                    ++it;
                }
            }
            const double t = now_s();
            for (auto &bt : done) {
                cudaEventDestroy(bt.ev);
                if (bt.pin >= 0) {
                    // a pass kernel gave up on a bounded wait: the batch's results are incomplete
                    if (s->status_pin[bt.pin] != 0) {
                        for (auto &q : bt.reqs) q->res.status = (conv_status)s->status_pin[bt.pin];
                        cudaMemsetAsync(bt.cp->plan->dev_err, 0, sizeof(int), bt.cp->stream);
                    }
                    s->free_pins.push_back(bt.pin);
                }
                for (auto &q : bt.reqs) finish(s, q, q->res.status, t);
                s->shape_inflight[bt.shape]--;
            }
            if (!done.empty()) {
                s->cv_done.notify_all();
                s->cv_dispatch.notify_one();
            }
        }
        if (done.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

static void ls_worker(srv_t s)
{
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, s->prio_lo);
    while (true) {
        std::shared_ptr<Req> q;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_ls.wait(lk, [&] { return s->stop || !s->ls_queue.empty(); });
            if (s->ls_queue.empty()) break;
            q = s->ls_queue.front();
            s->ls_queue.pop_front();
        }
        ls_opts o = {q->r.restart > 0 ? q->r.restart : 50, q->r.max_iters > 0 ? q->r.max_iters : 2000,
                     q->r.tol > 0 ? q->r.tol : 1e-10, q->r.precision == CONV_P_FP32 ? 1 : 0, 1e-5, 1};
        ls_info info{};
        conv_status rc;
        {
            std::lock_guard<std::mutex> plk(q->cp->run_mu);
            q->res.t_start = now_s();
            rc = ls_solve(q->cp->plan, q->r.m, q->r.in, q->r.out, &o, &info, st);
        }
        std::lock_guard<std::mutex> lk(s->mu);
        q->res.iters = info.iters;
        q->res.rel_residual = info.rel_residual;
        q->res.batched_with = 1;
        finish(s, q, rc, now_s());
        s->cv_done.notify_all();
        s->cv_dispatch.notify_one();
    }
    cudaStreamDestroy(st);
}

}  // namespace wsc

using namespace wsc;

extern "C" {

conv_status srv_create(size_t mem_budget_bytes, int max_inflight, int conv_batch_max, int ls_workers,
                       int plan_flags, srv_t *out)
{
    if (!out || mem_budget_bytes == 0 || max_inflight < 1 || conv_batch_max < 1 || ls_workers < 1)
        return fail(CONV_EINVAL, "bad serving parameters");
    if (plan_flags & ~(CONV_PLAN_COMPACT | CONV_PLAN_AUTOTUNE)) return fail(CONV_EINVAL, "unknown plan flags");
    srv_s *s = new srv_s();
    s->plan_flags = plan_flags;
    s->budget = mem_budget_bytes;
    s->max_inflight = max_inflight;
    s->batch_max = conv_batch_max;
    s->ls_workers = ls_workers;
    cudaGetDevice(&s->device);
    if (cudaDeviceGetStreamPriorityRange(&s->prio_lo, &s->prio_hi) != cudaSuccess) {
        cudaGetLastError();
        s->prio_lo = s->prio_hi = 0;
    }
    if (cudaHostAlloc(&s->status_pin, (size_t)(max_inflight + 1) * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(CONV_ENOMEM, "pinned status slots");
    }
    for (int i = max_inflight; i >= 0; --i) s->free_pins.push_back(i);
    s->dispatcher = std::thread(dispatcher_loop, s);
    s->completer = std::thread(completer_loop, s);
    for (int i = 0; i < ls_workers; ++i) s->workers.emplace_back(ls_worker, s);
    for (int i = 0; i < 4; ++i) s->builders.emplace_back(builder_loop, s);
    *out = s;
    return CONV_OK;
}

conv_status srv_submit(srv_t s, const srv_request *r, long long *ticket)
{
    if (!s || !r || !ticket) return fail(CONV_EINVAL, "bad argument");
    if (r->kind != SRV_CONV && r->kind != SRV_LS) return fail(CONV_EINVAL, "unknown request kind");
    if (!r->in || !r->out || (r->kind == SRV_LS && !r->m)) return fail(CONV_EINVAL, "missing request buffers");
    if (r->kind == SRV_LS && r->kernel.family != CONV_K_HELMHOLTZ)
        return fail(CONV_EINVAL, "Lippmann-Schwinger requests need the Helmholtz kernel");
    auto q = std::make_shared<Req>();
    q->r = *r;
    std::memset(&q->res, 0, sizeof(q->res));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(CONV_EINVAL, "server is shutting down");
        q->ticket = s->next_ticket++;
        q->res.t_submit = now_s();
        // an injected CONV_FAULT_DROP loses the request here: it has a ticket but never queues
        if (!fault_take(CONV_FAULT_DROP)) s->pending.push_back(q);
        s->all[q->ticket] = q;
        s->stats.submitted++;
        *ticket = q->ticket;
    }
    s->cv_dispatch.notify_one();
    return CONV_OK;
}

conv_status srv_wait(srv_t s, long long ticket, double timeout_s, srv_result *res)
{
    if (!s) return fail(CONV_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(CONV_EINVAL, "unknown ticket");
    auto q = it->second;
    auto pred = [&] { return q->done; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
            return fail(CONV_ETIMEOUT, "request not finished within the timeout");
    } else {
        s->cv_done.wait(lk, pred);
    }
    if (res) *res = q->res;
    s->all.erase(ticket);
    return CONV_OK;
}

conv_status srv_cancel(srv_t s, long long ticket)
{
    if (!s) return fail(CONV_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return fail(CONV_EINVAL, "unknown ticket");
        auto q = it->second;
        if (q->done) return CONV_OK;
        if (q->admitted) return fail(CONV_EINVAL, "the request already runs; wait for it");
        for (auto pit = s->pending.begin(); pit != s->pending.end(); ++pit)
            if (pit->get() == q.get()) {
                s->pending.erase(pit);
                break;
            }
        q->admitted = true;
        q->need = 0;
        s->inflight_reqs++;  // finish() counts it out again
        finish(s, q, CONV_ECANCELLED, now_s());
    }
    s->cv_done.notify_all();
    return CONV_OK;
}

conv_status srv_get_stats(srv_t s, srv_stats *out)
{
    if (!s || !out) return fail(CONV_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->bytes_in_use = s->in_use;
    out->plans_cached = (int)s->plans.size();
    return CONV_OK;
}

void srv_destroy(srv_t s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_dispatch.notify_all();
    s->cv_ls.notify_all();
    s->cv_build.notify_all();
    for (auto &b : s->builders) b.join();
    s->dispatcher.join();
    for (auto &w : s->workers) w.join();
    s->completer.join();
    for (auto &kv : s->plans) {
        cudaStreamSynchronize(kv.second->stream);
        plan_release(kv.second->plan, false);
        cudaStreamDestroy(kv.second->stream);
        dev_free(kv.second->stage_in);
        dev_free(kv.second->stage_out);
    }
    dev_pool_trim(s->device);
    cudaFreeHost(s->status_pin);
    delete s;
}

}  // extern "C"
