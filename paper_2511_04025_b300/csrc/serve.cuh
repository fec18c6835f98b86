// serve.cuh -- continuous batching of homogenisation requests inside libshl.
//
// Requests are copied at submit into a FIFO.  A pool of worker slots, each a
// private context (own non-blocking stream, own workspaces), takes the head
// request as soon as a slot is idle and the request's HBM footprint fits the
// budget; work of different requests therefore overlaps on the GPU while
// earlier ones are still iterating.  Admission counts the bytes actually held:
// every slot's workspace (max of what it holds and what its request needs)
// plus the warm-start cache.  Warm starts: the final displacements of each
// session (18 FP64 planes) stay on the device, keyed by session id, LRU-evicted
// with stream-ordered frees so that eviction never synchronises the device.
// Included by shl.cu after the solver.
#pragma once

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <memory>
#include <thread>
#include <unordered_map>

namespace shl {

struct ServeJob {
    uint64_t ticket = 0;
    shl_request req{};
    std::vector<double> pos, q, alpha;  // owned copies of the design arrays
    size_t footprint = 0;
    bool done = false, running = false;
    shl_result res{};
    // batch jobs: the slot's stream waits on `after` before the job's first
    // launch and records `finished` after its last, so that the caller's
    // stream can be ordered around work that ran on the slots' streams
    cudaEvent_t after = nullptr, finished = nullptr;
    std::string err;  // the slot's error text when the job failed
};

struct WarmEntry {
    int r = 0;
    double *x = nullptr;
    size_t bytes = 0;
    uint64_t tick = 0;
};

struct Server {
    shl_ctx *owner = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeJob *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<ServeJob>> jobs;
    std::vector<std::thread> threads;
    std::vector<shl_ctx *> slot_ctx;
    std::vector<size_t> slot_bytes;  // bytes held (or reserved) per slot
    std::unordered_map<int64_t, WarmEntry> warm;
    size_t warm_bytes = 0;
    size_t budget = 0;
    uint64_t next_ticket = 1, completed = 0, tick = 0;
    int running = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    size_t held() const {
        size_t h = warm_bytes;
        for (size_t b : slot_bytes) h += b;
        return h;
    }
};

inline size_t ctx_ws_bytes(shl_ctx *c) {
    size_t b = 0;
    for (auto &kv : c->ws.slots) b += kv.second.second;
    return b;
}

// Evict least-recently used warm entries until `need` more bytes fit (lock held).
inline void warm_evict(Server *sv, size_t need, cudaStream_t s) {
    while (!sv->warm.empty() && sv->held() + need > sv->budget) {
        auto victim = sv->warm.begin();
        for (auto it = sv->warm.begin(); it != sv->warm.end(); ++it)
            if (it->second.tick < victim->second.tick) victim = it;
        cudaFreeAsync(victim->second.x, s);
        sv->warm_bytes -= victim->second.bytes;
        sv->warm.erase(victim);
    }
}

inline void serve_worker(Server *sv, int slot) {
    shl_ctx *w = sv->slot_ctx[slot];
    cudaSetDevice(w->device);
    for (;;) {
        ServeJob *job = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop) return;
                if (!sv->queue.empty()) {
                    ServeJob *head = sv->queue.front();
                    const size_t mine = sv->slot_bytes[slot];
                    const size_t need = head->footprint > mine ? head->footprint - mine : 0;
                    if (need > 0) warm_evict(sv, need, w->stream);
                    if (sv->held() + need <= sv->budget) {
                        job = head;
                        sv->queue.pop_front();
                        sv->slot_bytes[slot] = mine + need;
                        job->running = true;
                        ++sv->running;
                        job->res.t_admit = sv->now();
                        job->res.slot = slot;
                        break;
                    }
                }
                sv->cv_work.wait(lk);
            }
        }
        // run the design on this slot's context and stream
        const int r = job->req.r;
        const size_t NV = (size_t)18 * r * r * r;
        shl_design d = job->req.design;
        d.pos = job->pos.data();
        d.q = job->q.data();
        d.alpha = job->alpha.empty() ? nullptr : job->alpha.data();
        double *x64 = nullptr;
        int rc = ws_get_t(w, "serve_x64", NV, &x64);
        bool warm = false;
        if (rc == SHL_OK && job->req.opts.warm_start && job->req.session >= 0) {
            std::lock_guard<std::mutex> lk(sv->mu);
            auto it = sv->warm.find(job->req.session);
            if (it != sv->warm.end() && it->second.r == r) {
                cudaMemcpyAsync(x64, it->second.x, NV * sizeof(double), cudaMemcpyDeviceToDevice, w->stream);
                cudaStreamSynchronize(w->stream);
                it->second.tick = ++sv->tick;
                warm = true;
            }
        }
        if (rc == SHL_OK && job->after && cudaStreamWaitEvent(w->stream, job->after, 0) != cudaSuccess)
            rc = set_err(w, SHL_ECUDA, "serving: stream wait failed");
        if (rc == SHL_OK) {
            std::lock_guard<std::recursive_mutex> wl(w->mu);
            rc = homogenize_impl(w, &d, r, &job->req.opts, job->res.C, &job->res.stats, w->stream, x64, warm);
        }
        if (job->finished) cudaEventRecord(job->finished, w->stream);
        job->res.warm = warm ? 1 : 0;
        if (job->res.stats.status == SHL_OK && rc != SHL_OK) job->res.stats.status = rc;
        if (rc != SHL_OK) job->err = w->err;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->slot_bytes[slot] = std::max(sv->slot_bytes[slot], ctx_ws_bytes(w));
            // keep the session's displacements for the next warm start
            if (job->req.session >= 0 && (rc == SHL_OK || rc == SHL_ENOCONV)) {
                const size_t bytes = NV * sizeof(double);
                auto it = sv->warm.find(job->req.session);
                if (it != sv->warm.end() && it->second.bytes != bytes) {
                    cudaFreeAsync(it->second.x, w->stream);
                    sv->warm_bytes -= it->second.bytes;
                    sv->warm.erase(it);
                    it = sv->warm.end();
                }
                if (it == sv->warm.end()) {
                    warm_evict(sv, bytes, w->stream);
                    if (sv->held() + bytes <= sv->budget) {
                        WarmEntry e;
                        e.r = r;
                        e.bytes = bytes;
                        if (cudaMallocAsync(reinterpret_cast<void **>(&e.x), bytes, w->stream) == cudaSuccess) {
                            sv->warm_bytes += bytes;
                            it = sv->warm.emplace(job->req.session, e).first;
                        } else {
                            cudaGetLastError();
                        }
                    }
                }
                if (it != sv->warm.end()) {
                    cudaMemcpyAsync(it->second.x, x64, bytes, cudaMemcpyDeviceToDevice, w->stream);
                    cudaStreamSynchronize(w->stream);
                    it->second.r = r;
                    it->second.tick = ++sv->tick;
                }
            }
            job->res.t_done = sv->now();
            job->done = true;
            job->running = false;
            --sv->running;
            ++sv->completed;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

inline int serve_start(shl_ctx *ctx, Server **out) {
    if (ctx->serve) {
        *out = static_cast<Server *>(ctx->serve);
        return SHL_OK;
    }
    auto *sv = new Server();
    sv->owner = ctx;
    sv->t0 = std::chrono::steady_clock::now();
    const int slots = ctx->opts.max_batch > 0 ? ctx->opts.max_batch : 16;
    size_t budget = (size_t)ctx->opts.hbm_budget_bytes;
    if (!budget) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = (size_t)(0.4 * (double)fr);
    }
    sv->budget = budget;
    for (int i = 0; i < slots; ++i) {
        shl_ctx *w = new shl_ctx();
        w->device = ctx->device;
        w->stream_ordered_alloc = true;
        if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete w;
            break;
        }
        sv->slot_ctx.push_back(w);
        sv->slot_bytes.push_back(0);
    }
    if (sv->slot_ctx.empty()) {
        delete sv;
        return set_err(ctx, SHL_ECUDA, "serving: could not create worker streams");
    }
    for (size_t i = 0; i < sv->slot_ctx.size(); ++i) sv->threads.emplace_back(serve_worker, sv, (int)i);
    ctx->serve = sv;
    *out = sv;
    return SHL_OK;
}

inline void serve_stop(shl_ctx *ctx) {
    auto *sv = static_cast<Server *>(ctx->serve);
    if (!sv) return;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv_done.wait(lk, [&] { return sv->running == 0; });
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->threads) t.join();
    for (auto &kv : sv->warm) cudaFreeAsync(kv.second.x, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (auto *w : sv->slot_ctx) {
        cudaStreamSynchronize(w->stream);
        aux_release(w);
        ws_free_all(w);
        cudaStreamDestroy(w->stream);
        delete w;
    }
    delete sv;
    ctx->serve = nullptr;
}

}  // namespace shl

namespace shl {

// Queue one validated request on the context's server (started on first use).
inline int serve_enqueue(shl_ctx *ctx, const shl_request *req, cudaEvent_t after, cudaEvent_t finished,
                         uint64_t *ticket) {
    cudaSetDevice(ctx->device);
    Server *sv = nullptr;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        SHL_TRY(serve_start(ctx, &sv));
    }
    auto job = std::make_unique<ServeJob>();
    job->after = after;
    job->finished = finished;
    job->req = *req;
    const int n = req->design.n, K = req->design.K;
    job->pos.assign(req->design.pos, req->design.pos + 3 * n);
    job->q.assign(req->design.q, req->design.q + n);
    if (req->design.alpha) job->alpha.assign(req->design.alpha, req->design.alpha + (K + 1) * (K + 1) * (K + 1));
    job->footprint = design_footprint(req->r, &req->opts);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (job->footprint > sv->budget)
        return set_err(ctx, SHL_EINVAL, "serving: request footprint %zu bytes exceeds the HBM budget %zu",
                       job->footprint, sv->budget);
    job->ticket = sv->next_ticket++;
    job->res.t_submit = sv->now();
    job->res.slot = -1;
    *ticket = job->ticket;
    sv->queue.push_back(job.get());
    sv->jobs.emplace(job->ticket, std::move(job));
    sv->cv_work.notify_all();
    return SHL_OK;
}

}  // namespace shl

extern "C" {

int shl_serve_submit(shl_ctx *ctx, const shl_request *req, uint64_t *ticket) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    if (!req || !ticket) return set_err(ctx, SHL_EINVAL, "serving: NULL request or ticket");
    SHL_TRY(validate_solve_opts(ctx, &req->opts));
    SHL_TRY(validate_design(ctx, &req->design, req->r));
    return serve_enqueue(ctx, req, nullptr, nullptr, ticket);
}

static int serve_take(shl_ctx *ctx, uint64_t ticket, shl_result *out, bool block) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    auto *sv = static_cast<Server *>(ctx->serve);
    if (!sv) return set_err(ctx, SHL_ENOTFOUND, "serving: unknown ticket %llu", (unsigned long long)ticket);
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return set_err(ctx, SHL_ENOTFOUND, "serving: unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second->done) {
        if (!block) return SHL_EAGAIN;
        ServeJob *j = it->second.get();
        sv->cv_done.wait(lk, [&] { return j->done; });
    }
    if (out) *out = it->second->res;
    if (!it->second->err.empty()) ctx->err = it->second->err;  // why the request failed
    sv->jobs.erase(it);
    return SHL_OK;
}

int shl_serve_poll(shl_ctx *ctx, uint64_t ticket, shl_result *out) { return serve_take(ctx, ticket, out, false); }

int shl_serve_wait(shl_ctx *ctx, uint64_t ticket, shl_result *out) { return serve_take(ctx, ticket, out, true); }

int shl_serve_cancel(shl_ctx *ctx, uint64_t ticket) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    auto *sv = static_cast<Server *>(ctx->serve);
    if (!sv) return set_err(ctx, SHL_ENOTFOUND, "serving: unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return set_err(ctx, SHL_ENOTFOUND, "serving: unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->running || it->second->done) return SHL_EAGAIN;
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
        if (*q == it->second.get()) {
            sv->queue.erase(q);
            break;
        }
    sv->jobs.erase(it);
    sv->cv_work.notify_all();
    return SHL_OK;
}

int shl_serve_drain(shl_ctx *ctx) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    auto *sv = static_cast<Server *>(ctx->serve);
    if (!sv) return SHL_OK;
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&] { return sv->queue.empty() && sv->running == 0; });
    return SHL_OK;
}

int shl_serve_info_get(shl_ctx *ctx, shl_serve_info *out) {
    if (!ctx || !out) return set_err(ctx, SHL_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    auto *sv = static_cast<Server *>(ctx->serve);
    if (!sv) {
        out->slots = ctx->opts.max_batch > 0 ? ctx->opts.max_batch : 16;
        out->budget_bytes = ctx->opts.hbm_budget_bytes;
        return SHL_OK;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    out->slots = (int32_t)sv->slot_ctx.size();
    out->queued = (int32_t)sv->queue.size();
    out->running = sv->running;
    out->completed = sv->completed;
    out->held_bytes = sv->held();
    out->budget_bytes = sv->budget;
    return SHL_OK;
}

}  // extern "C"
