// api.cpp -- the extern "C" entry points declared in include/smc.h and
// include/smc_kernels.h, and the serving loop.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "../../include/smc.h"
#include "../../include/smc_kernels.h"
#include "engine.h"

using namespace smc;

struct smc_ctx {
    Ctx c;
};

#define CKS(expr)                                          \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_status(_e);     \
    } while (0)

namespace smc {

// ---------------------------------------------------------------------------
// Serving: admission by memory budget, continuous batching of every admitted
// request's jobs in shared launches, retirement as soon as a request's jobs
// are all done.
// ---------------------------------------------------------------------------
// the serving thread, started by the first submission (caller holds c.qmu)
static void start_worker(Ctx &c)
{
    if (c.worker_started) return;
    c.worker_started = true;
    c.worker = std::thread([&c] {
        cudaSetDevice(c.device);
        serve_loop(&c);
    });
}

static void finish_failed(Ctx &c, Request *r, int st)
{
    r->status = st;
    r->t_done = std::chrono::steady_clock::now();
    r->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    r->state.store(2, std::memory_order_release);
    (void)c;
}

void serve_loop(Ctx *cp)
{
    Ctx &c = *cp;
    for (;;) {
        // capacity as the engine sees it (c.used and the free slots change
        // under c.mu only); admission below adds up everything it admits in
        // one pass against this snapshot
        size_t used_now = 0, slots_now = 0;
        {
            std::lock_guard<std::recursive_mutex> g(c.mu);
            used_now = c.used;
            slots_now = c.free_slots.size();
        }
        std::vector<Request *> admitted;
        {
            std::unique_lock<std::mutex> lk(c.qmu);
            if (c.queue.empty() && c.running.empty()) {
                c.qcv.wait(lk, [&] { return c.stop || !c.queue.empty(); });
            }
            if (c.stop && c.queue.empty() && c.running.empty()) return;
            size_t pending = 0, pending_slots = 0;
            while (!c.queue.empty()) {
                Request *r = c.queue.front();
                const size_t need = request_bytes(*r);
                const size_t nK = (size_t)(r->k_max - r->k_min + 1);
                if (need > c.budget || nK > (size_t)MAX_SLOTS) {
                    c.queue.pop_front();
                    finish_failed(c, r, SMC_ENOMEM);
                    c.done_cv.notify_all();
                    continue;
                }
                if (used_now + pending + need > c.budget || pending_slots + nK > slots_now) break;
                c.queue.pop_front();
                admitted.push_back(r);
                pending += need;
                pending_slots += nK;
            }
            if (admitted.empty() && c.running.empty() && !c.queue.empty()) {
                // nothing of this loop holds memory, yet the head request does
                // not fit: memory held outside the serving loop must be
                // released first (smc_release); wait for a new event
                c.qcv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        std::vector<Request *> finished;
        bool requeued = false;
        {
            std::lock_guard<std::recursive_mutex> g(c.mu);
            for (size_t i = 0; i < admitted.size(); ++i) {
                Request *r = admitted[i];
                int st = setup_request(c, *r);
                if (st == ST_NO_ROOM) {
                    // budget or job slots taken meanwhile (by calls outside the
                    // serving loop): this request and the later admitted ones
                    // go back to the head of the queue, in order, and wait
                    free_request_device(c, *r);
                    std::lock_guard<std::mutex> lk(c.qmu);
                    for (size_t k = admitted.size(); k-- > i;) c.queue.push_front(admitted[k]);
                    requeued = true;
                    break;
                }
                if (st != SMC_OK) {
                    free_request_device(c, *r);
                    std::lock_guard<std::mutex> lk(c.qmu);
                    finish_failed(c, r, st);
                    c.done_cv.notify_all();
                    continue;
                }
                r->state = 1;
                if (r->fp64) {
                    // plain path: the request runs alone, to completion
                    std::vector<Request *> one{r};
                    st = run_requests(c, one);
                    if (st != SMC_OK) finish_failed(c, r, st);
                    finished.push_back(r);
                } else {
                    c.running.push_back(r);
                }
            }
            if (!c.running.empty()) {
                int st = run_chunk(c, c.running, 4);
                // which requests have every job done
                std::vector<Request *> still;
                for (Request *r : c.running) {
                    bool all_done = st != SMC_OK;
                    if (!all_done) {
                        all_done = true;
                        for (int sl : r->slots) {
                            int state = 0;
                            cudaMemcpy(&state, &c.d_jobs[sl].state, sizeof(int), cudaMemcpyDeviceToHost);
                            if (state == JOB_ACTIVE) {
                                all_done = false;
                                break;
                            }
                        }
                    }
                    if (all_done) {
                        std::vector<Request *> one{r};
                        int fs = st == SMC_OK ? finalize_requests(c, one) : st;
                        if (fs != SMC_OK) {
                            free_request_device(c, *r);
                            finish_failed(c, r, fs);
                        }
                        finished.push_back(r);
                    } else {
                        still.push_back(r);
                    }
                }
                c.running.swap(still);
            }
        }
        if (!finished.empty()) {
            std::lock_guard<std::mutex> lk(c.qmu);
            c.done_cv.notify_all();
        }
        if (requeued && c.running.empty()) {
            // nothing of this loop runs to free memory: wait for a new event
            std::unique_lock<std::mutex> lk(c.qmu);
            c.qcv.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

}  // namespace smc

extern "C" {

const char *smc_strerror(int s)
{
    switch (s) {
    case SMC_OK: return "ok";
    case SMC_EINVAL: return "invalid argument";
    case SMC_ENOMEM: return "out of memory or over the context's memory budget";
    case SMC_ECUDA: return "CUDA runtime error";
    case SMC_ETIMEOUT: return "timed out";
    case SMC_EMAXSTAGES: return "beta did not reach 1 within max_stages";
    case SMC_ENOTREADY: return "result not ready";
    case SMC_ECANCELLED: return "cancelled";
    case SMC_ENUMERIC: return "every particle energy is non-finite";
    default: return "unknown status";
    }
}

int smc_create(smc_ctx **out, const smc_create_opts *opts)
{
    if (!out) return SMC_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return SMC_ECUDA;
    const int dev = opts ? opts->device : 0;
    if (dev < 0 || dev >= ndev) return SMC_EINVAL;
    if (opts && (opts->graph_mode < SMC_GRAPH_WHILE || opts->graph_mode > SMC_GRAPH_NONE))
        return SMC_EINVAL;
    CKS(cudaSetDevice(dev));
    smc_ctx *ctx = new smc_ctx();
    Ctx &c = ctx->c;
    c.device = dev;
    if (opts && opts->cuda_stream) {
        c.stream = (cudaStream_t)opts->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return SMC_ECUDA;
        }
        c.own_stream = true;
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c.budget = (opts && opts->mem_budget_bytes) ? opts->mem_budget_bytes : (size_t)(0.8 * fr);
    c.graph_mode = opts ? opts->graph_mode : SMC_GRAPH_WHILE;
    // SMC_GRAPH_CHUNKED=1 in the environment: replay four-stage graphs instead of
    // one graph with a conditional while node (kernel profilers cannot replay
    // kernels of the latter)
    if (const char *g = getenv("SMC_GRAPH_CHUNKED"))
        if (g[0] == '1' && c.graph_mode == SMC_GRAPH_WHILE) c.graph_mode = SMC_GRAPH_CHUNKED;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    c.h_jobs.assign(MAX_SLOTS, JobDev{});
    for (int s = MAX_SLOTS - 1; s >= 0; --s) c.free_slots.push_back(s);
    bool ok = cudaMalloc((void **)&c.d_jobs, sizeof(JobDev) * MAX_SLOTS) == cudaSuccess &&
              cudaMemset(c.d_jobs, 0, sizeof(JobDev) * MAX_SLOTS) == cudaSuccess &&
              cudaMalloc((void **)&c.d_lists, sizeof(int) * LIST_AREA) == cudaSuccess &&
              cudaMalloc((void **)&c.d_nactive, 2 * sizeof(int)) == cudaSuccess &&
              cudaHostAlloc((void **)&c.h_nactive, sizeof(int) * NACTIVE_SLOTS, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&c.h_nactive_dev, c.h_nactive, 0) == cudaSuccess;
    if (!ok) {
        smc_destroy(ctx);
        return SMC_ECUDA;
    }
    for (int k = 0; k < NACTIVE_SLOTS; ++k) c.h_nactive[k] = 0;
    *out = ctx;
    return SMC_OK;
}

int smc_destroy(smc_ctx *ctx)
{
    if (!ctx) return SMC_EINVAL;
    Ctx &c = ctx->c;
    bool started = false;
    {
        std::lock_guard<std::mutex> lk(c.qmu);
        started = c.worker_started;
        c.stop = true;
        for (Request *r : c.queue) {
            r->status = SMC_ECANCELLED;
            r->state = 2;
        }
        c.queue.clear();
    }
    if (started) {
        c.qcv.notify_all();
        c.worker.join();
    }
    cudaSetDevice(c.device);
    for (auto &kv : c.reqs) {
        free_request_device(c, *kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(c.stream);
    if (c.d_jobs) cudaFree(c.d_jobs);
    if (c.d_lists) cudaFree(c.d_lists);
    if (c.d_nactive) cudaFree(c.d_nactive);
    if (c.h_nactive) cudaFreeHost(c.h_nactive);
    if (c.own_stream) cudaStreamDestroy(c.stream);
    delete ctx;
    return SMC_OK;
}

int smc_run_batch(smc_ctx *ctx, const smc_request *reqs, int32_t count, int32_t on_device,
                  smc_job *out)
{
    if (!ctx || !reqs || count < 1 || !out) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    std::vector<Request *> rs;
    auto cleanup = [&](int st) {
        for (Request *r : rs) {
            free_request_device(c, *r);
            delete r;
        }
        cudaStreamSynchronize(c.stream);
        return st;
    };
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < count; ++i) {
        Request *r = nullptr;
        int st = make_request(c, reqs[i], on_device != 0, r);
        if (st != SMC_OK) return cleanup(st);
        r->t_submit = t0;
        rs.push_back(r);
        st = setup_request(c, *r);
        if (st != SMC_OK) return cleanup(st == ST_NO_ROOM ? SMC_ENOMEM : st);
        r->state = 1;
    }
    int st = run_requests(c, rs);
    if (st != SMC_OK) return cleanup(st);
    std::lock_guard<std::mutex> lk(c.qmu);
    for (int i = 0; i < count; ++i) {
        rs[i]->id = c.next_id++;
        c.reqs[rs[i]->id] = rs[i];
        out[i] = rs[i]->id;
    }
    return SMC_OK;
}

int smc_run(smc_ctx *ctx, const double *x, const double *y, const double *sigma, int64_t n,
            int32_t k_min, int32_t k_max, int32_t family, int32_t bg, int32_t bg_degree,
            const smc_priors *priors, const smc_options *opts, smc_job *out)
{
    smc_request rq{x, y, sigma, n, k_min, k_max, family, bg, bg_degree, priors, opts};
    return smc_run_batch(ctx, &rq, 1, 0, out);
}

int smc_submit(smc_ctx *ctx, const smc_request *req, smc_job *out)
{
    if (!ctx || !req || !out) return SMC_EINVAL;
    Ctx &c = ctx->c;
    Request *r = nullptr;
    int st = make_request(c, *req, false, r);
    if (st != SMC_OK) return st;
    r->t_submit = std::chrono::steady_clock::now();
    // the queue lock only: the serving thread holds the engine lock (c.mu)
    // while it runs stages, and a submission must not wait for that
    {
        std::lock_guard<std::mutex> lk(c.qmu);
        r->id = c.next_id++;
        c.reqs[r->id] = r;
        c.queue.push_back(r);
        start_worker(c);
    }
    c.qcv.notify_all();
    *out = r->id;
    return SMC_OK;
}

int smc_submit_batch(smc_ctx *ctx, const smc_request *reqs, int32_t count, smc_job *out)
{
    if (!ctx || !reqs || count < 1 || !out) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::vector<Request *> rs;
    for (int i = 0; i < count; ++i) {
        Request *r = nullptr;
        const int st = make_request(c, reqs[i], false, r);
        if (st != SMC_OK) {
            for (Request *q : rs) delete q;
            return st;
        }
        rs.push_back(r);
    }
    const auto t0 = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(c.qmu);
        for (Request *r : rs) {
            r->t_submit = t0;
            r->id = c.next_id++;
            c.reqs[r->id] = r;
            c.queue.push_back(r);
        }
        start_worker(c);
    }
    c.qcv.notify_all();
    for (int i = 0; i < count; ++i) out[i] = rs[i]->id;
    return SMC_OK;
}

int smc_request_bytes(smc_ctx *ctx, const smc_request *req, size_t *bytes)
{
    if (!ctx || !req || !bytes) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);  // the tile table
    Request *r = nullptr;
    const int st = make_request(c, *req, false, r);
    if (st != SMC_OK) return st;
    *bytes = request_bytes(*r);
    delete r;
    return SMC_OK;
}

int smc_poll(smc_ctx *ctx, smc_job job, int32_t *done)
{
    if (!ctx || !done) return SMC_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->c.qmu);
    Request *r = nullptr;
    {
        auto it = ctx->c.reqs.find(job);
        if (it != ctx->c.reqs.end()) r = it->second;
    }
    if (!r) return SMC_EINVAL;
    *done = r->state == 2;
    return SMC_OK;
}

int smc_wait(smc_ctx *ctx, smc_job job, double timeout_s)
{
    if (!ctx) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::unique_lock<std::mutex> lk(c.qmu);
    auto it = c.reqs.find(job);
    if (it == c.reqs.end()) return SMC_EINVAL;
    Request *r = it->second;
    auto pred = [&] { return r->state == 2; };
    if (timeout_s < 0) {
        c.done_cv.wait(lk, pred);
    } else if (!c.done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return SMC_ETIMEOUT;
    }
    return SMC_OK;
}

int smc_result(smc_ctx *ctx, smc_job job, smc_result_view *out)
{
    if (!ctx || !out) return SMC_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->c.qmu);
    auto it = ctx->c.reqs.find(job);
    if (it == ctx->c.reqs.end()) return SMC_EINVAL;
    Request *r = it->second;
    if (r->state != 2) return SMC_ENOTREADY;
    smc_result_view v{};
    v.k_min = r->k_min;
    v.k_max = r->k_max;
    v.dim_max = r->dim_max;
    v.status = r->status;
    v.log_z = r->log_z.empty() ? nullptr : r->log_z.data();
    v.p_k = r->p_k.empty() ? nullptr : r->p_k.data();
    v.n_stages = r->n_stages.empty() ? nullptr : r->n_stages.data();
    v.job_status = r->job_status.empty() ? nullptr : r->job_status.data();
    v.post_mean = r->mean.empty() ? nullptr : r->mean.data();
    v.post_sd = r->sdv.empty() ? nullptr : r->sdv.data();
    v.samples = r->samples.empty() ? nullptr : r->samples.data();
    v.n_samples = r->n_samples;
    v.latency_ms = r->latency_ms;
    v.selected_k = r->selected_k;
    *out = v;
    return SMC_OK;
}

int smc_release(smc_ctx *ctx, smc_job job)
{
    if (!ctx) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(c.qmu);
        auto it = c.reqs.find(job);
        if (it == c.reqs.end()) return SMC_EINVAL;
        r = it->second;
        if (r->state != 2) return SMC_ENOTREADY;
        c.reqs.erase(it);
    }
    free_request_device(c, *r);
    delete r;
    return SMC_OK;
}

// ---------------------------------------------------------------------------
// Step-level entry points (include/smc_kernels.h)
// ---------------------------------------------------------------------------
static double host_xref(const smc_request *spec)
{
    double lo = spec->x[0], hi = spec->x[0];
    for (int64_t i = 1; i < spec->n; ++i) {
        lo = std::min(lo, spec->x[i]);
        hi = std::max(hi, spec->x[i]);
    }
    return 0.5 * (lo + hi);
}

static int single_job(smc_ctx *ctx, const smc_request *spec, int32_t K, int32_t precision,
                      int64_t T, int64_t S, Request *&r)
{
    if (!spec || !spec->opts) return SMC_EINVAL;
    smc_request rq = *spec;
    rq.k_min = rq.k_max = K;
    smc_options o = *spec->opts;
    o.energy_fp64 = precision ? 1 : 0;
    o.keep_samples = 0;
    rq.opts = &o;
    int st = make_request(ctx->c, rq, false, r);
    if (st != SMC_OK) return st;
    st = setup_request(ctx->c, *r, T, S);
    if (st != SMC_OK) {
        free_request_device(ctx->c, *r);
        delete r;
        r = nullptr;
    }
    return st == ST_NO_ROOM ? SMC_ENOMEM : st;
}

// natural value -> sampling coordinate of component j (centres shifted for FP32 jobs)
static double to_sampling(const Request &r, const smc_prior &p, bool centre, double v, double xref)
{
    double u = p.kind == SMC_LOG_UNIFORM ? std::log(v) : v;
    if (centre && !r.fp64) u -= xref;
    return u;
}
static double to_natural(const Request &r, const smc_prior &p, bool centre, double u, double xref)
{
    double v = p.kind == SMC_LOG_UNIFORM ? std::exp(u) : u;
    if (centre && !r.fp64) v += xref;
    return v;
}

static smc_prior prior_of(const Request &r, int K, int j)
{
    if (!r.comp.empty()) return r.comp[j];
    if (j < r.p * K) {
        switch (j % r.p) {
        case 0: return r.pri.amp;
        case 1: return r.pri.centre;
        case 2: return r.pri.width;
        default: return r.pri.eta;
        }
    }
    return r.pri.bg[j - r.p * K];
}

// peak centres are held relative to the grid midpoint in FP32 jobs; the App. D
// phase shift d2theta (component 1 of a phase) is an offset, not a centre
static bool is_centre_comp(const Request &r, int K, int j)
{
    return r.family != SMC_XRD_PHASE && j < r.p * K && j % r.p == 1;
}

static int upload_particles(Ctx &c, const Request &r, int K, const double *nat, int64_t count,
                            double xref, void *dst_th, int64_t stride)
{
    const int d = job_dim(r.family, K, r.bg, r.bg_degree);
    if (r.fp64) {
        std::vector<double> buf((size_t)d * stride, 0.0);
        for (int j = 0; j < d; ++j)
            for (int64_t i = 0; i < count; ++i)
                buf[(size_t)j * stride + i] =
                    to_sampling(r, prior_of(r, K, j), is_centre_comp(r, K, j), nat[i * d + j], xref);
        CKS(cudaMemcpy(dst_th, buf.data(), 8 * buf.size(), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> buf((size_t)d * stride, 0.0f);
        for (int j = 0; j < d; ++j)
            for (int64_t i = 0; i < count; ++i)
                buf[(size_t)j * stride + i] = (float)to_sampling(
                    r, prior_of(r, K, j), is_centre_comp(r, K, j), nat[i * d + j], xref);
        CKS(cudaMemcpy(dst_th, buf.data(), 4 * buf.size(), cudaMemcpyHostToDevice));
    }
    return SMC_OK;
}

static int download_particles(Ctx &c, const Request &r, int K, const void *src_th, int64_t count,
                              double xref, double *nat, int64_t stride)
{
    (void)c;
    const int d = job_dim(r.family, K, r.bg, r.bg_degree);
    std::vector<double> buf((size_t)d * stride);
    if (r.fp64) {
        CKS(cudaMemcpy(buf.data(), src_th, 8 * buf.size(), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> f((size_t)d * stride);
        CKS(cudaMemcpy(f.data(), src_th, 4 * f.size(), cudaMemcpyDeviceToHost));
        for (size_t a = 0; a < f.size(); ++a) buf[a] = f[a];
    }
    for (int j = 0; j < d; ++j)
        for (int64_t i = 0; i < count; ++i)
            nat[i * d + j] = to_natural(r, prior_of(r, K, j), is_centre_comp(r, K, j),
                                        buf[(size_t)j * stride + i], xref);
    return SMC_OK;
}

static void drop(smc_ctx *ctx, Request *r)
{
    free_request_device(ctx->c, *r);
    cudaStreamSynchronize(ctx->c.stream);
    delete r;
}

int smc_k_philox(smc_ctx *ctx, uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n)
{
    if (!ctx || !ctr || !out || n < 0) return SMC_EINVAL;
    if (n == 0) return SMC_OK;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    uint32_t *d = nullptr;
    CKS(cudaMalloc((void **)&d, 32 * n));
    cudaError_t e = cudaMemcpy(d, ctr, 16 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(seed, d, d + 4 * n, n, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 4 * n, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return cuda_status(e);
}

int smc_k_energy(smc_ctx *ctx, const smc_request *spec, int32_t K, const double *nat,
                 int64_t count, int32_t precision, double *E_out)
{
    if (!ctx || !spec || !nat || !E_out || count < 1) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    Request *r = nullptr;
    int st = single_job(ctx, spec, K, precision, count, count, r);
    if (st != SMC_OK) return st;
    const double xref = host_xref(spec);
    const int sl = r->slots[0];
    JobDev jb = c.h_jobs[sl];
    st = upload_particles(c, *r, K, nat, count, xref, r->fp64 ? (void *)jb.th64 : (void *)jb.th, count);
    if (st == SMC_OK) st = cuda_status(cudaMemcpy(c.d_lists, &sl, 4, cudaMemcpyHostToDevice));
    if (st == SMC_OK) st = cuda_status(launch_energy(c.d_jobs, c.d_lists, 1, (int)count, r->fp64, c.stream));
    if (st == SMC_OK) st = cuda_status(cudaStreamSynchronize(c.stream));
    if (st == SMC_OK) {
        if (r->fp64) {
            st = cuda_status(cudaMemcpy(E_out, jb.E64, 8 * count, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(count);
            st = cuda_status(cudaMemcpy(f.data(), jb.E, 4 * count, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < count; ++i) E_out[i] = f[i];
        }
    }
    drop(ctx, r);
    return st;
}

int smc_k_prior(smc_ctx *ctx, const smc_request *spec, int32_t K, int64_t count, int32_t precision,
                double *nat_out, double *E_out)
{
    if (!ctx || !spec || !nat_out || !E_out || count < 1) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    Request *r = nullptr;
    int st = single_job(ctx, spec, K, precision, count, count, r);
    if (st != SMC_OK) return st;
    const double xref = host_xref(spec);
    const JobDev jb = c.h_jobs[r->slots[0]];
    st = download_particles(c, *r, K, r->fp64 ? (const void *)jb.th64 : (const void *)jb.th, count,
                            xref, nat_out, count);
    if (st == SMC_OK) {
        if (r->fp64) {
            st = cuda_status(cudaMemcpy(E_out, jb.E64, 8 * count, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(count);
            st = cuda_status(cudaMemcpy(f.data(), jb.E, 4 * count, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < count; ++i) E_out[i] = f[i];
        }
    }
    drop(ctx, r);
    return st;
}

int smc_k_reweight(smc_ctx *ctx, const double *E, int64_t T, double beta, double rho,
                   int32_t precision, double *delta, double *logz_inc, int32_t *final_step,
                   uint64_t *q_out)
{
    if (!ctx || !E || T < 2 || T > (1 << 24) || !delta || !logz_inc || !final_step) return SMC_EINVAL;
    if (!(beta >= 0.0 && beta < 1.0) || !(rho > 0.0 && rho < 1.0)) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    if (c.free_slots.empty()) return SMC_ENOMEM;
    const size_t e = precision ? 8 : 4;
    char *a = nullptr;
    const size_t bytes = ((T * e + 255) & ~size_t(255)) + 16 * T + 1024 + 8 * RW_SPLIT_MAX;
    CKS(cudaMalloc((void **)&a, bytes));
    JobDev jb{};
    jb.T = jb.S = (int)T;
    jb.fp64 = precision ? 1 : 0;
    if (precision)
        jb.E64 = (double *)a;
    else
        jb.E = (float *)a;
    char *b = a + ((T * e + 255) & ~size_t(255));
    jb.w64 = (double *)b;
    jb.q = (unsigned long long *)(b + 8 * T);
    char *tail = b + 16 * T;
    jb.lam = (double *)tail;
    jb.step = (double *)(tail + 64);
    jb.stepf = (float *)(tail + 128);
    jb.acc = (unsigned long long *)(tail + 192);
    jb.prop = (unsigned long long *)(tail + 256);
    jb.pri = (const PriorDev *)(tail + 320);
    jb.rwpart = (double *)(tail + 1024);
    jb.d = 0;
    jb.beta = beta;
    jb.rho = rho;
    jb.logz = 0.0;
    jb.state = JOB_ACTIVE;
    jb.max_stages = 1 << 30;
    const int sl = c.free_slots.back();
    int st = SMC_OK;
    if (precision) {
        st = cuda_status(cudaMemcpy(jb.E64, E, 8 * T, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(T);
        for (int64_t i = 0; i < T; ++i) f[i] = (float)E[i];
        st = cuda_status(cudaMemcpy(jb.E, f.data(), 4 * T, cudaMemcpyHostToDevice));
    }
    if (st == SMC_OK) st = cuda_status(cudaMemcpy(c.d_jobs + sl, &jb, sizeof(JobDev), cudaMemcpyHostToDevice));
    if (st == SMC_OK) st = cuda_status(cudaMemcpy(c.d_lists, &sl, 4, cudaMemcpyHostToDevice));
    if (st == SMC_OK) st = cuda_status(launch_reweight(c.d_jobs, c.d_lists, 1, precision != 0, T, c.stream));
    if (st == SMC_OK) st = cuda_status(cudaStreamSynchronize(c.stream));
    JobDev o{};
    if (st == SMC_OK) st = cuda_status(cudaMemcpy(&o, c.d_jobs + sl, sizeof(JobDev), cudaMemcpyDeviceToHost));
    if (st == SMC_OK && q_out) st = cuda_status(cudaMemcpy(q_out, jb.q, 8 * T, cudaMemcpyDeviceToHost));
    if (st == SMC_OK) {
        if (o.status != 0) {
            st = o.status;
        } else {
            *delta = o.delta;
            *logz_inc = o.logz;
            *final_step = o.final_step;
        }
    }
    JobDev z{};
    cudaMemcpy(c.d_jobs + sl, &z, sizeof(JobDev), cudaMemcpyHostToDevice);
    cudaFree(a);
    return st;
}

int smc_k_resample(smc_ctx *ctx, const uint64_t *q, int64_t T, int64_t M, uint32_t u32,
                   int32_t *anc)
{
    if (!ctx || !q || !anc || T < 1 || M < 1 || T > (1 << 24) || M > (1 << 24)) return SMC_EINVAL;
    uint64_t tot = 0;
    for (int64_t i = 0; i < T; ++i) {
        if (q[i] > (1ull << 40)) return SMC_EINVAL;
        tot += q[i];
    }
    if (tot == 0) return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    char *a = nullptr;
    CKS(cudaMalloc((void **)&a, 8 * T + 4 * M + 256));
    unsigned long long *dq = (unsigned long long *)a;
    int *da = (int *)(a + ((8 * T + 255) & ~size_t(255)));
    cudaError_t e = cudaMemcpy(dq, q, 8 * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_resample_raw(dq, (int)T, (int)M, u32, da, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaMemcpy(anc, da, 4 * M, cudaMemcpyDeviceToHost);
    cudaFree(a);
    return cuda_status(e);
}

int smc_k_mh_stage(smc_ctx *ctx, const smc_request *spec, int32_t K, const double *nat_start,
                   const double *E_start, int64_t S, const double *step, double beta,
                   uint32_t stage, int32_t precision, double *nat_out, double *E_out,
                   int64_t *acc, int64_t *prop)
{
    if (!ctx || !spec || !spec->opts || !nat_start || !E_start || !step || !nat_out || !E_out ||
        !acc || !prop || S < 1 || stage < 1 || !(beta >= 0.0 && beta <= 1.0))
        return SMC_EINVAL;
    Ctx &c = ctx->c;
    std::lock_guard<std::recursive_mutex> g(c.mu);
    cudaSetDevice(c.device);
    const int64_t n = spec->opts->sweeps;
    const int64_t T = spec->opts->waste_free ? S * n : S;
    if (T > (1 << 24)) return SMC_EINVAL;
    Request *r = nullptr;
    int st = single_job(ctx, spec, K, precision, T, S, r);
    if (st != SMC_OK) return st;
    const double xref = host_xref(spec);
    const int sl = r->slots[0];
    const int d = job_dim(r->family, K, r->bg, r->bg_degree);
    JobDev jb{};
    st = cuda_status(cudaMemcpy(&jb, c.d_jobs + sl, sizeof(JobDev), cudaMemcpyDeviceToHost));
    if (st == SMC_OK)
        st = upload_particles(c, *r, K, nat_start, S, xref, r->fp64 ? (void *)jb.ths64 : (void *)jb.ths, S);
    if (st == SMC_OK) {
        if (r->fp64) {
            st = cuda_status(cudaMemcpy(jb.Es64, E_start, 8 * S, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> f(S);
            for (int64_t i = 0; i < S; ++i) f[i] = (float)E_start[i];
            st = cuda_status(cudaMemcpy(jb.Es, f.data(), 4 * S, cudaMemcpyHostToDevice));
        }
    }
    if (st == SMC_OK && d > 0) {
        std::vector<float> sf(d);
        for (int j = 0; j < d; ++j) sf[j] = (float)step[j];
        st = cuda_status(cudaMemcpy(jb.step, step, 8 * d, cudaMemcpyHostToDevice));
        if (st == SMC_OK) st = cuda_status(cudaMemcpy(jb.stepf, sf.data(), 4 * d, cudaMemcpyHostToDevice));
        if (st == SMC_OK) st = cuda_status(cudaMemset(jb.acc, 0, 8 * d));
        if (st == SMC_OK) st = cuda_status(cudaMemset(jb.prop, 0, 8 * d));
    }
    jb.beta = beta;
    jb.stage = (int)stage - 1;
    jb.state = JOB_ACTIVE;
    jb.status = 0;
    jb.next_chain = 0;
    if (st == SMC_OK) st = cuda_status(cudaMemcpy(c.d_jobs + sl, &jb, sizeof(JobDev), cudaMemcpyHostToDevice));
    if (st == SMC_OK) st = cuda_status(cudaMemcpy(c.d_lists, &sl, 4, cudaMemcpyHostToDevice));
    if (st == SMC_OK) {
        if (r->fp64)
            st = cuda_status(launch_mh_plain(c.d_jobs, c.d_lists, 1, (int)S, c.stream));
        else
            st = cuda_status(launch_mh(c.d_jobs, c.d_lists, 1, kernel_family(r->family) | (r->full ? MH_COUPLED : 0), r->tile.J, r->tile.G, r->tile.R, 0, c.stream, K));
    }
    if (st == SMC_OK) st = cuda_status(cudaStreamSynchronize(c.stream));
    if (st == SMC_OK)
        st = download_particles(c, *r, K, r->fp64 ? (const void *)jb.th64 : (const void *)jb.th, T, xref,
                                nat_out, T);
    if (st == SMC_OK) {
        if (r->fp64) {
            st = cuda_status(cudaMemcpy(E_out, jb.E64, 8 * T, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(T);
            st = cuda_status(cudaMemcpy(f.data(), jb.E, 4 * T, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < T; ++i) E_out[i] = f[i];
        }
    }
    if (st == SMC_OK && d > 0) {
        std::vector<unsigned long long> a(d), p(d);
        st = cuda_status(cudaMemcpy(a.data(), jb.acc, 8 * d, cudaMemcpyDeviceToHost));
        if (st == SMC_OK) st = cuda_status(cudaMemcpy(p.data(), jb.prop, 8 * d, cudaMemcpyDeviceToHost));
        for (int j = 0; j < d; ++j) {
            acc[j] = (int64_t)a[j];
            prop[j] = (int64_t)p[j];
        }
    }
    drop(ctx, r);
    return st;
}

int smc_set_tile(smc_ctx *ctx, int32_t family, int64_t n_max, int32_t J, int32_t G, int32_t regs)
{
    if (!ctx) return SMC_EINVAL;
    std::lock_guard<std::recursive_mutex> g(ctx->c.mu);
    if (J == 0) {
        std::lock_guard<std::mutex> tl(ctx->c.tmu);
        ctx->c.tiles.clear();
        return SMC_OK;
    }
    const int coupled = family & MH_COUPLED;
    family &= ~MH_COUPLED;
    if (family < 0 || family > 4 || (family == SMC_XRD_PHASE && !coupled)) return SMC_EINVAL;
    family = kernel_family(family) | coupled;
    if (n_max < 1 || !mh_tile_supported(family, J, G, regs) || 32L * J * G < 1) return SMC_EINVAL;
    std::lock_guard<std::mutex> tl(ctx->c.tmu);
    ctx->c.tiles.push_back({family, n_max, J, G, regs});
    return SMC_OK;
}

int smc_profile_reset(smc_ctx *ctx, int32_t enable_events)
{
    if (!ctx) return SMC_EINVAL;
    std::lock_guard<std::recursive_mutex> g(ctx->c.mu);
    ctx->c.prof = smc_profile{};
    ctx->c.prof_events = enable_events != 0;
    return SMC_OK;
}

int smc_profile_read(smc_ctx *ctx, smc_profile *out)
{
    if (!ctx || !out) return SMC_EINVAL;
    std::lock_guard<std::recursive_mutex> g(ctx->c.mu);
    *out = ctx->c.prof;
    return SMC_OK;
}

}  // extern "C"
