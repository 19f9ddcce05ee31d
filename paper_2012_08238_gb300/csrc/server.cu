// Serving loop: continuous batching of sparse-FFT requests on one device.
//
// A worker thread admits queued requests while they fit in the slot count and
// the device-memory budget (plans are cached and reused; idle plans are
// evicted least-recently-used when a new one must fit), launches whatever it
// admitted as one batch on one of two streams, and goes back to admitting
// while that batch runs.  Completion is signalled in stream order by a host
// callback, which frees the slots and wakes waiters.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "sfft_internal.cuh"

namespace sfft {
size_t plan_device_bytes(int64_t N, int32_t K, int32_t B, int64_t w, int32_t L, int32_t c, int32_t T,
                         const sfft_opts &o);
}

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

using PlanKey =
    std::tuple<int64_t, int64_t, int32_t, int32_t, int32_t, uint64_t, int32_t, int32_t, int32_t, int32_t, int32_t,
               int32_t, int32_t>;

struct Request {
    uint64_t ticket = 0;
    sfft_request req{};
    PlanKey key;
    int64_t t_submit = 0, t_done = 0;
    bool done = false;
    sfft_status status = SFFT_OK;
    int32_t k_out = 0;
    int64_t samples = 0;
    sfft_plan *plan = nullptr;
};

struct CachedPlan {
    sfft_plan *plan;
    PlanKey key;
    size_t bytes;
    bool busy;
    uint64_t last_use;
};

struct Batch;

}  // namespace

struct sfft_server {
    int device = 0;
    size_t budget = 0;
    int32_t max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;       // worker wake-up
    std::condition_variable done_cv;  // waiters
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> tickets;
    std::list<CachedPlan> plans;
    size_t plan_bytes = 0;
    uint64_t next_ticket = 1, use_clock = 0;
    int32_t in_use = 0;  // admitted, unfinished requests
    int inflight = 0;    // batches on the device
    bool region_busy[2] = {false, false};
    bool stop = false, paused = false;
    cudaStream_t streams[2] = {nullptr, nullptr};
    int32_t *kout_dev = nullptr;   // [2][max_slots]
    int32_t *kout_host = nullptr;  // pinned mirror
    std::thread worker;
};

namespace {

struct Batch {
    sfft_server *srv;
    int region;
    std::vector<Request *> reqs;
};

// Host callback, runs in stream order after the batch and its k_out copy.
void CUDART_CB on_batch_done(void *arg) {
    Batch *b = static_cast<Batch *>(arg);
    sfft_server *s = b->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const int64_t t = now_ns();
        for (size_t i = 0; i < b->reqs.size(); ++i) {
            Request *r = b->reqs[i];
            r->k_out = s->kout_host[b->region * s->max_slots + (int32_t)i];
            r->t_done = t;
            r->done = true;
            for (auto &cp : s->plans)
                if (cp.plan == r->plan) cp.busy = false;
        }
        s->in_use -= (int32_t)b->reqs.size();
        s->inflight -= 1;
        s->region_busy[b->region] = false;
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
    delete b;
}

// Find or create a plan for request r; evicts idle plans to stay in budget.
// Returns false when it cannot fit now (caller retries later).
bool acquire_plan(sfft_server *s, Request *r, std::unique_lock<std::mutex> &lk) {
    for (auto &cp : s->plans) {
        if (!cp.busy && cp.key == r->key) {
            cp.busy = true;
            cp.last_use = ++s->use_clock;
            r->plan = cp.plan;
            return true;
        }
    }
    const sfft_request &q = r->req;
    const size_t need = sfft::plan_device_bytes(q.N, q.K, q.B, q.w, q.L, q.opts.c > 0 ? q.opts.c : 2,
                                                q.opts.T > 0 ? q.opts.T : (q.L + 1) / 2, q.opts);
    while (s->plan_bytes + need > s->budget) {
        auto victim = s->plans.end();
        for (auto it = s->plans.begin(); it != s->plans.end(); ++it)
            if (!it->busy && (victim == s->plans.end() || it->last_use < victim->last_use)) victim = it;
        if (victim == s->plans.end()) return false;
        s->plan_bytes -= victim->bytes;
        sfft_plan *old = victim->plan;
        s->plans.erase(victim);
        lk.unlock();
        sfft_plan_destroy(old);
        lk.lock();
    }
    lk.unlock();
    sfft_plan *p = nullptr;
    const sfft_status st = sfft_plan_create_ex(&p, q.N, q.K, q.B, q.w, q.L, q.seed, &q.opts);
    lk.lock();
    if (st != SFFT_OK) {
        r->status = st;
        r->plan = nullptr;
        return true;  // admitted as a failed request
    }
    sfft_plan_info info;
    sfft_plan_get_info(p, &info);
    s->plans.push_back(CachedPlan{p, r->key, info.device_bytes, true, ++s->use_clock});
    s->plan_bytes += info.device_bytes;
    r->plan = p;
    r->samples = info.samples_touched;
    return true;
}

void worker_main(sfft_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] {
            const bool can_launch = !s->queue.empty() && s->inflight < 2 && s->in_use < s->max_slots && !s->paused;
            return can_launch || (s->stop && s->queue.empty());
        });
        if (s->stop && s->queue.empty()) break;
        int region = s->region_busy[0] ? 1 : 0;
        std::vector<Request *> batch, failed;
        while (!s->queue.empty() && s->in_use + (int32_t)batch.size() < s->max_slots) {
            Request *r = s->queue.front();
            // one location method per batch; the next batch takes the other
            if (!batch.empty() && r->req.opts.method != batch[0]->req.opts.method) break;
            if (r->plan == nullptr) {
                if (!acquire_plan(s, r, lk)) break;  // wait for running batches to free plans
            }
            s->queue.pop_front();
            if (r->status != SFFT_OK) failed.push_back(r);
            else batch.push_back(r);
        }
        const int64_t t = now_ns();
        for (Request *r : failed) {
            r->done = true;
            r->t_done = t;
        }
        if (!failed.empty()) s->done_cv.notify_all();
        if (batch.empty()) {
            if (s->inflight == 0 && !s->queue.empty() && failed.empty()) {
                // nothing running can free memory: the head request cannot be served
                Request *r = s->queue.front();
                s->queue.pop_front();
                r->status = SFFT_EBUSY;
                r->done = true;
                r->t_done = now_ns();
                s->done_cv.notify_all();
            } else if (s->inflight > 0) {
                s->cv.wait(lk);  // a completion will wake us
            }
            continue;
        }
        s->in_use += (int32_t)batch.size();
        s->inflight += 1;
        s->region_busy[region] = true;
        lk.unlock();

        std::vector<sfft_plan *> plans;
        std::vector<const float *> xs;
        std::vector<int32_t *> idxs;
        std::vector<float *> vals;
        for (Request *r : batch) {
            plans.push_back(r->plan);
            xs.push_back(r->req.x_dev);
            idxs.push_back(r->req.idx_dev);
            vals.push_back(r->req.val_dev);
            sfft_plan_info info;
            sfft_plan_get_info(r->plan, &info);
            r->samples = info.samples_touched;
        }
        cudaStream_t st = s->streams[region];
        int32_t *kdev = s->kout_dev + region * s->max_slots;
        int32_t *khost = s->kout_host + region * s->max_slots;
        Batch *b = new Batch{s, region, batch};
        sfft_status est = sfft_execute_batch(plans.data(), xs.data(), idxs.data(), vals.data(), kdev,
                                             (int32_t)batch.size(), st);
        cudaError_t ce = cudaSuccess;
        if (est == SFFT_OK) ce = cudaMemcpyAsync(khost, kdev, sizeof(int32_t) * batch.size(), cudaMemcpyDeviceToHost, st);
        if (est == SFFT_OK && ce == cudaSuccess) ce = cudaLaunchHostFunc(st, on_batch_done, b);
        lk.lock();
        if (est != SFFT_OK || ce != cudaSuccess) {
            const sfft_status bad = est != SFFT_OK ? est : SFFT_ECUDA;
            for (Request *r : batch) {
                r->status = bad;
                r->done = true;
                r->t_done = now_ns();
                for (auto &cp : s->plans)
                    if (cp.plan == r->plan) cp.busy = false;
            }
            s->in_use -= (int32_t)batch.size();
            s->inflight -= 1;
            s->region_busy[region] = false;
            delete b;
            s->done_cv.notify_all();
        }
    }
    // drain: wait for batches still on the device
    s->done_cv.wait(lk, [&] { return s->inflight == 0; });
}

bool valid_request(const sfft_request *q) {
    return q && q->x_dev && q->idx_dev && q->val_dev;
}

}  // namespace

extern "C" sfft_status sfft_server_create(sfft_server **srv, size_t hbm_budget_bytes, int32_t max_slots) {
    if (!srv || max_slots < 1 || hbm_budget_bytes == 0) {
        sfft::set_error("server needs a pointer, max_slots >= 1 and a non-zero budget");
        return SFFT_EINVAL;
    }
    *srv = nullptr;
    sfft_server *s = new (std::nothrow) sfft_server();
    if (!s) return SFFT_ENOMEM;
    cudaGetDevice(&s->device);
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->kout_dev, sizeof(int32_t) * 2 * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&s->kout_host, sizeof(int32_t) * 2 * max_slots);
    if (e != cudaSuccess) {
        for (auto st : s->streams)
            if (st) cudaStreamDestroy(st);
        if (s->kout_dev) cudaFree(s->kout_dev);
        delete s;
        return sfft::cuda_fail(e, "server resources");
    }
    s->worker = std::thread(worker_main, s);
    *srv = s;
    return SFFT_OK;
}

extern "C" sfft_status sfft_submit(sfft_server *s, const sfft_request *q, uint64_t *ticket) {
    if (!s || !ticket || !valid_request(q)) {
        sfft::set_error("NULL server, ticket or request buffer");
        return SFFT_EINVAL;
    }
    const int32_t c = q->opts.c > 0 ? q->opts.c : 2;
    const int32_t T = q->opts.T > 0 ? q->opts.T : (q->L + 1) / 2;
    const size_t need = sfft::plan_device_bytes(q->N, q->K, q->B, q->w, q->L, c, T, q->opts);
    if (need == 0) return SFFT_EINVAL;  // sizes rejected, reason already set
    if (need > s->budget) {
        sfft::set_error("request's plan alone exceeds the server's memory budget");
        return SFFT_EBUSY;
    }
    Request *r = new (std::nothrow) Request();
    if (!r) return SFFT_ENOMEM;
    r->req = *q;
    r->key = PlanKey(q->N, q->w, q->K, q->B, q->L, q->seed, c, T, q->opts.method, q->opts.comb, q->opts.estimator,
                     q->opts.refine, q->opts.search_bits);
    r->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            sfft::set_error("server is shutting down");
            return SFFT_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->tickets[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv.notify_all();
    *ticket = r->ticket;
    return SFFT_OK;
}

static sfft_status take_result(sfft_server *s, Request *r, sfft_result *res) {
    if (res) {
        res->k_out = r->k_out;
        res->status = r->status;
        res->samples_touched = r->samples;
        res->latency_ns = r->t_done - r->t_submit;
    }
    const sfft_status st = r->status;
    s->tickets.erase(r->ticket);
    delete r;
    if (st != SFFT_OK) sfft::set_error("request failed");
    return st;
}

extern "C" sfft_status sfft_poll(sfft_server *s, uint64_t ticket, sfft_result *res) {
    if (!s) return SFFT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        sfft::set_error("unknown ticket");
        return SFFT_EINVAL;
    }
    if (!it->second->done) return SFFT_EPENDING;
    return take_result(s, it->second, res);
}

extern "C" sfft_status sfft_wait(sfft_server *s, uint64_t ticket, int64_t timeout_ms, sfft_result *res) {
    if (!s) return SFFT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        sfft::set_error("unknown ticket");
        return SFFT_EINVAL;
    }
    Request *r = it->second;
    if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] { return r->done; })) {
        sfft::set_error("wait timed out");
        return SFFT_ETIMEDOUT;
    }
    return take_result(s, r, res);
}

extern "C" sfft_status sfft_server_set_paused(sfft_server *s, int32_t paused) {
    if (!s) return SFFT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv.notify_all();
    return SFFT_OK;
}

extern "C" void sfft_server_destroy(sfft_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->paused = false;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (auto &cp : s->plans) sfft_plan_destroy(cp.plan);
    for (auto &kv : s->tickets) delete kv.second;
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    cudaFree(s->kout_dev);
    cudaFreeHost(s->kout_host);
    delete s;
}
