// server.cu -- a continuous-batching request engine on one GPU.
//
// Requests (kind, n) are queued as they are submitted.  Each worker thread
// owns a context and a CUDA stream; whenever it is idle it admits the queued
// requests in arrival order while their estimated device footprint, added to
// the estimates of the batches already running and to the results still held
// by clients, fits the server's HBM budget (a worker with nothing else
// running always admits one), runs them as one batch (exact_batch), and
// publishes every result.  While one worker's batch is on the GPU, requests
// that arrive meanwhile are admitted by the next idle worker, so batches
// overlap on the device.  All workers' contexts draw on one shared byte
// counter capped at the budget, so the budget also bounds what they really
// hold together.  Results stay in device memory until the client fetches or
// releases them; buffers are freed by the worker that allocated them.
#include "cat_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace cat {
void ctx_init(Ctx &c, int device, size_t budget);
void ctx_release(Ctx &c);
void exact_batch(Ctx &c, const cat_request *reqs, size_t count, uint32_t *out, size_t cap,
                 uint64_t *offsets, uint64_t *lengths, cudaStream_t s);
}  // namespace cat

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Device bytes a request may hold while it is computed: a fixed part (sieve
// segments, small tables: measured at most 1.35 MB) and a part per limb of
// the result bound (level arrays, three-prime transforms, leaves: measured at
// most 124 bytes per limb from n = 10^4 to 3 * 10^8, all three kinds), with
// headroom; a batch's estimate is the sum over its requests.
constexpr uint64_t kFootprintFixed = 2u << 20;
constexpr uint64_t kFootprintPerLimb = 256;

struct Worker;

struct ResultBuf {
    Worker *owner = nullptr;
    uint32_t *p = nullptr;
    size_t bytes = 0;
    int refs = 0;  // results still held by clients
};

struct Job {
    cat_request req{};
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    int error = 0;
    uint64_t t_submit = 0, t_start = 0, t_end = 0;
    ResultBuf *buf = nullptr;
    uint64_t off = 0, len = 0, batch = 0;
};

struct Worker {
    std::thread th;
    cat::Ctx ctx;
    cudaStream_t stream = nullptr;
    std::vector<ResultBuf *> to_free;  // released by clients, freed by this worker
};

}  // namespace

struct cat_server {
    int device = 0;
    size_t budget = 0;
    size_t max_batch = 4096;
    std::atomic<size_t> used{0};  // bytes all workers' contexts hold (hard cap)
    std::atomic<size_t> used_peak{0};
    size_t reserved = 0;          // footprint estimates of the running batches
    size_t resident = 0;          // bytes of results still held by clients
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Job> jobs;
    std::vector<std::unique_ptr<Worker>> workers;
    bool stop = false;
    uint64_t next_ticket = 1, next_batch = 1;
    std::string init_error;
};

namespace {

void release_buf(cat_server *sv, ResultBuf *b)
{
    // caller holds sv->mu
    if (--b->refs == 0) {
        sv->resident -= b->bytes;
        b->owner->to_free.push_back(b);
    }
}

uint64_t footprint(const cat_request &r)
{
    return kFootprintFixed + cat::bound_limbs(r.n, r.kind) * kFootprintPerLimb;
}

// Whether f more bytes of estimated footprint may start now (caller holds
// sv->mu): always when nothing is running, else when the running batches'
// estimates, the resident results and f fit the budget.
bool fits(const cat_server *sv, uint64_t f)
{
    return !sv->budget || sv->reserved == 0 || sv->resident + sv->reserved + f <= sv->budget;
}

void worker_loop(cat_server *sv, Worker *w)
{
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<uint64_t> tickets;
        std::vector<cat_request> reqs;
        std::vector<ResultBuf *> frees;
        uint64_t batch_id = 0;
        uint64_t foot = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                return sv->stop || !w->to_free.empty() ||
                       (!sv->queue.empty() && fits(sv, footprint(sv->jobs[sv->queue.front()].req)));
            });
            frees.swap(w->to_free);
            if (sv->stop && sv->queue.empty() && frees.empty()) return;
            while (!sv->queue.empty() && reqs.size() < sv->max_batch) {
                Job &j = sv->jobs[sv->queue.front()];
                const uint64_t f = footprint(j.req);
                if (!fits(sv, foot + f)) break;
                if (!reqs.empty() && sv->budget &&
                    sv->resident + sv->reserved + foot + f > sv->budget)
                    break;
                foot += f;
                j.state = 1;
                j.t_start = now_ns();
                tickets.push_back(sv->queue.front());
                reqs.push_back(j.req);
                sv->queue.pop_front();
            }
            sv->reserved += foot;
            batch_id = sv->next_batch++;
        }
        for (ResultBuf *b : frees) {
            cat::dev_free(w->ctx, b->p, b->bytes, w->stream);
            delete b;
        }
        if (reqs.empty()) continue;
        std::vector<uint64_t> offs(reqs.size()), lens(reqs.size());
        ResultBuf *buf = new ResultBuf;
        buf->owner = w;
        int rc = CAT_OK;
        std::string msg;
        try {
            const size_t cap = [&] {
                size_t t = 0;
                for (auto &r : reqs) t += cat::bound_limbs(r.n, r.kind);
                return t;
            }();
            buf->bytes = 4 * cap;
            buf->p = (uint32_t *)cat::dev_alloc(w->ctx, buf->bytes, w->stream);
            cat::exact_batch(w->ctx, reqs.data(), reqs.size(), buf->p, cap, offs.data(),
                             lens.data(), w->stream);
            cudaStreamSynchronize(w->stream);
        } catch (const cat::Error &e) {
            rc = e.code;
            msg = e.msg;
        } catch (...) {
            rc = CAT_ECUDA;
        }
        const uint64_t t_end = now_ns();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->reserved -= foot;
            for (size_t i = 0; i < tickets.size(); i++) {
                auto it = sv->jobs.find(tickets[i]);
                if (it == sv->jobs.end()) continue;  // released while running
                Job &j = it->second;
                j.t_end = t_end;
                j.batch = batch_id;
                if (rc == CAT_OK) {
                    j.state = 2;
                    j.buf = buf;
                    j.off = offs[i];
                    j.len = lens[i];
                    buf->refs++;
                } else {
                    j.state = 3;
                    j.error = rc;
                }
            }
            if (buf->refs == 0)
                w->to_free.push_back(buf);
            else
                sv->resident += buf->bytes;
        }
        if (rc != CAT_OK && buf->p == nullptr) {
            std::lock_guard<std::mutex> lk(sv->mu);
            auto &tf = w->to_free;
            tf.erase(std::remove(tf.begin(), tf.end(), buf), tf.end());
            delete buf;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

int cat_server_create(int device, size_t hbm_budget_bytes, int workers, size_t max_batch,
                      cat_server **out)
{
    if (!out || workers < 1 || workers > 64) return CAT_EINVAL;
    *out = nullptr;
    auto *sv = new cat_server;
    sv->device = device;
    sv->budget = hbm_budget_bytes;
    if (max_batch) sv->max_batch = max_batch;
    try {
        for (int i = 0; i < workers; i++) {
            auto w = std::make_unique<Worker>();
            cat::ctx_init(w->ctx, device, 0);
            // one hard cap for all workers together
            w->ctx.shared_in_use = &sv->used;
            w->ctx.shared_peak = &sv->used_peak;
            w->ctx.shared_budget = hbm_budget_bytes;
            cat::check_cuda(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking),
                            "cudaStreamCreateWithFlags");
            sv->workers.push_back(std::move(w));
        }
    } catch (const cat::Error &e) {
        for (auto &w : sv->workers) {
            if (w->stream) cudaStreamDestroy(w->stream);
            cat::ctx_release(w->ctx);
        }
        delete sv;
        return e.code;
    }
    for (auto &w : sv->workers) w->th = std::thread(worker_loop, sv, w.get());
    *out = sv;
    return CAT_OK;
}

int cat_server_submit(cat_server *sv, int kind, uint64_t n, uint64_t *ticket)
{
    if (!sv || !ticket || n >= (1ull << 31) || kind < CAT_CATALAN || kind > CAT_FACTORIAL)
        return CAT_EINVAL;
    // admission denial: a request whose estimated footprint alone exceeds the
    // whole budget is never queued
    if (sv->budget && footprint(cat_request{kind, n}) > sv->budget) return CAT_ENOMEM;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return CAT_EINVAL;
        const uint64_t t = sv->next_ticket++;
        Job &j = sv->jobs[t];
        j.req.kind = kind;
        j.req.n = n;
        j.t_submit = now_ns();
        sv->queue.push_back(t);
        *ticket = t;
    }
    sv->cv_work.notify_one();
    return CAT_OK;
}

static int fill_result(const Job &j, cat_server_result *res)
{
    if (res) {
        res->kind = j.req.kind;
        res->n = j.req.n;
        res->limbs = j.state == 2 ? j.buf->p + j.off : nullptr;
        res->length = j.len;
        res->t_submit_ns = j.t_submit;
        res->t_start_ns = j.t_start;
        res->t_end_ns = j.t_end;
        res->batch = j.batch;
    }
    return j.state == 2 ? CAT_OK : (j.state == 3 ? j.error : CAT_EBUSY);
}

int cat_server_poll(cat_server *sv, uint64_t ticket, cat_server_result *res)
{
    if (!sv) return CAT_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return CAT_EINVAL;
    return fill_result(it->second, res);
}

int cat_server_wait(cat_server *sv, uint64_t ticket, uint64_t timeout_ms, cat_server_result *res)
{
    if (!sv) return CAT_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto done = [&] {
        auto it = sv->jobs.find(ticket);
        return it == sv->jobs.end() || it->second.state >= 2;
    };
    if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return CAT_ETIMEOUT;
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return CAT_EINVAL;
    return fill_result(it->second, res);
}

int cat_server_fetch(cat_server *sv, uint64_t ticket, uint32_t *dst, size_t cap, int to_host,
                     size_t *out_len)
{
    if (!sv || !out_len || (cap && !dst)) return CAT_EINVAL;
    const uint32_t *src = nullptr;
    uint64_t len = 0;
    ResultBuf *buf = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(ticket);
        if (it == sv->jobs.end()) return CAT_EINVAL;
        if (it->second.state < 2) return CAT_EBUSY;
        if (it->second.state == 3) return it->second.error;
        src = it->second.buf->p + it->second.off;
        len = it->second.len;
        *out_len = len;
        if (len > cap) return CAT_ERANGE;
        // the buffer stays allocated while the copy reads it, even if another
        // thread releases the ticket meanwhile
        buf = it->second.buf;
        buf->refs++;
    }
    cudaSetDevice(sv->device);
    const bool ok = !len || cudaMemcpy(dst, src, 4 * len,
                                       to_host ? cudaMemcpyDeviceToHost
                                               : cudaMemcpyDeviceToDevice) == cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        release_buf(sv, buf);
    }
    sv->cv_work.notify_all();
    return ok ? CAT_OK : CAT_ECUDA;
}

int cat_server_release(cat_server *sv, uint64_t ticket)
{
    if (!sv) return CAT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(ticket);
        if (it == sv->jobs.end()) return CAT_EINVAL;
        if (it->second.state == 0 || it->second.state == 1) return CAT_EBUSY;
        if (it->second.buf) release_buf(sv, it->second.buf);
        sv->jobs.erase(it);
    }
    sv->cv_work.notify_all();
    return CAT_OK;
}

int cat_batch_footprint(const cat_request *reqs, size_t count, size_t *bytes)
{
    if (!bytes || (count && !reqs)) return CAT_EINVAL;
    uint64_t t = 0;
    for (size_t i = 0; i < count; i++) {
        if (reqs[i].n >= (1ull << 31) || reqs[i].kind < CAT_CATALAN ||
            reqs[i].kind > CAT_FACTORIAL)
            return CAT_EINVAL;
        t += footprint(reqs[i]);
    }
    *bytes = (size_t)t;
    return CAT_OK;
}

int cat_server_memory(cat_server *sv, size_t *in_use, size_t *peak)
{
    if (!sv) return CAT_EINVAL;
    if (in_use) *in_use = sv->used.load();
    if (peak) *peak = sv->used_peak.load();
    return CAT_OK;
}

int cat_server_pending(cat_server *sv, size_t *queued, size_t *total)
{
    if (!sv) return CAT_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (queued) *queued = sv->queue.size();
    if (total) *total = sv->jobs.size();
    return CAT_OK;
}

void cat_server_destroy(cat_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->queue.clear();
        for (auto &kv : sv->jobs)
            if (kv.second.buf) release_buf(sv, kv.second.buf);
        sv->jobs.clear();
    }
    sv->cv_work.notify_all();
    for (auto &w : sv->workers)
        if (w->th.joinable()) w->th.join();
    for (auto &w : sv->workers) {
        cudaSetDevice(sv->device);
        for (ResultBuf *b : w->to_free) {
            cat::dev_free(w->ctx, b->p, b->bytes, w->stream);
            delete b;
        }
        cudaStreamSynchronize(w->stream);
        cudaStreamDestroy(w->stream);
        cat::ctx_release(w->ctx);
    }
    delete sv;
}

}  // extern "C"
