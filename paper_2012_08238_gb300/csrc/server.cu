// Serving loop: continuous batching of sparse-FFT requests on one device.
//
// Requests queue up; a worker thread admits them while the slot count and the
// device-memory budget allow, forms a batch of whatever it admitted (one
// location method per batch) and launches it on one of two streams, then goes
// back to admitting while that batch runs (continuous batching: requests that
// arrive while others are on the GPU join the next batch as slots free up).
//
// Plans are cached by shape, not by seed: (N, B, w, L, options and, for the
// voting method, K rounded up to a power of two).  A request takes an idle
// cached plan of its shape and rebinds it to its own K and seed (new sigma,
// tau: a descriptor upload on the batch stream), so a stream of distinct
// seeds reuses a few plans and their shared tables.  A shape with no idle
// plan is built by a separate builder thread while the worker keeps
// admitting the requests it can serve; idle plans are evicted least recently
// used when a new one must fit the budget.  Completion is signalled in
// stream order by a host callback, which frees the slots and wakes waiters.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <set>
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

// shape of a cached plan: N, w, K capacity, B, L, c, T, method, comb, estimator, refine, search bits, residual,
// precision, gather mode
using PlanKey =
    std::tuple<int64_t, int64_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t,
               int32_t, int32_t, int32_t, int32_t>;

struct Request {
    uint64_t ticket = 0;
    sfft_request req{};
    PlanKey key;
    int32_t K_cap = 0;
    int64_t t_submit = 0, t_done = 0;
    bool done = false;
    sfft_status status = SFFT_OK;
    int32_t k_out = 0;
    sfft_plan *plan = nullptr;
};

struct CachedPlan {
    sfft_plan *plan;
    PlanKey key;
    size_t bytes;
    bool busy;
    uint64_t last_use;
};

struct BuildJob {
    PlanKey key;
    sfft_request req;  // sizes, options and a seed to build with
    int32_t K_cap;
};

}  // namespace

struct sfft_server {
    int device = 0;
    size_t budget = 0;
    int32_t max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;        // worker wake-up
    std::condition_variable done_cv;   // waiters
    std::condition_variable build_cv;  // builder wake-up
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> tickets;
    std::list<CachedPlan> plans;
    std::deque<BuildJob> builds;  // shapes waiting for the builder
    std::set<PlanKey> building;   // shapes queued or being built
    std::vector<sfft_plan *> graveyard;  // evicted plans, destroyed outside the lock
    size_t plan_bytes = 0;        // cached plans plus the ones being built
    uint64_t next_ticket = 1, use_clock = 0;
    int32_t in_use = 0;  // admitted, unfinished requests
    int inflight = 0;    // batches on the device
    bool region_busy[2] = {false, false};
    bool stop = false, paused = false;
    cudaStream_t streams[2] = {nullptr, nullptr};
    int32_t *kout_dev = nullptr;   // [2][max_slots]
    int32_t *kout_host = nullptr;  // pinned mirror
    std::thread worker, builder;
};

namespace {

struct Batch {
    sfft_server *srv;
    int region;
    std::vector<Request *> reqs;
};

void release_plan(sfft_server *s, sfft_plan *p) {
    for (auto &cp : s->plans)
        if (cp.plan == p) {
            cp.busy = false;
            cp.last_use = ++s->use_clock;
        }
}

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
            release_plan(s, r->plan);
        }
        s->in_use -= (int32_t)b->reqs.size();
        s->inflight -= 1;
        s->region_busy[b->region] = false;
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
    delete b;
}

size_t key_bytes(const sfft_request &q, int32_t K_cap) {
    return sfft::plan_device_bytes(q.N, K_cap, q.B, q.w, q.L, q.opts.c > 0 ? q.opts.c : 2,
                                   q.opts.T > 0 ? q.opts.T : (q.L + 1) / 2, q.opts);
}

// Evicts idle plans, least recently used first, until `need` more bytes fit
// the budget (the evicted plans are destroyed later, outside the lock: a
// cudaFree may wait for the device, whose completion callbacks take the
// lock).  False when the busy plans alone leave no room.
bool make_room(sfft_server *s, size_t need) {
    while (s->plan_bytes + need > s->budget) {
        auto victim = s->plans.end();
        for (auto it = s->plans.begin(); it != s->plans.end(); ++it)
            if (!it->busy && (victim == s->plans.end() || it->last_use < victim->last_use)) victim = it;
        if (victim == s->plans.end()) return false;
        s->plan_bytes -= victim->bytes;
        s->graveyard.push_back(victim->plan);
        s->plans.erase(victim);
    }
    return true;
}

// Destroys the evicted plans with the lock released.
void bury(sfft_server *s, std::unique_lock<std::mutex> &lk) {
    if (s->graveyard.empty()) return;
    std::vector<sfft_plan *> dead;
    dead.swap(s->graveyard);
    lk.unlock();
    for (sfft_plan *p : dead) sfft_plan_destroy(p);
    lk.lock();
}

// What the worker can do with a queued request now.
enum Take { kTakeReady, kTakeWait, kTakeBuilding, kTakeNoRoom };

Take try_take(sfft_server *s, Request *r) {
    for (auto &cp : s->plans)
        if (!cp.busy && cp.key == r->key) {
            cp.busy = true;
            cp.last_use = ++s->use_clock;
            r->plan = cp.plan;
            return kTakeReady;
        }
    if (s->building.count(r->key)) return kTakeBuilding;
    // every cached plan of this shape is busy (or there is none): build one
    // more if it fits, else wait for a running batch to free one
    bool any = false;
    for (auto &cp : s->plans) any = any || cp.key == r->key;
    const size_t need = key_bytes(r->req, r->K_cap);
    if (!make_room(s, need)) return any ? kTakeWait : kTakeNoRoom;
    s->plan_bytes += need;  // reserved until the builder reports
    s->building.insert(r->key);
    s->builds.push_back(BuildJob{r->key, r->req, r->K_cap});
    s->build_cv.notify_one();
    return kTakeBuilding;
}

void builder_main(sfft_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->build_cv.wait(lk, [&] { return s->stop || !s->builds.empty(); });
        if (s->builds.empty()) break;  // stop requested and nothing left
        BuildJob job = s->builds.front();
        s->builds.pop_front();
        const size_t reserved = key_bytes(job.req, job.K_cap);
        lk.unlock();
        sfft_plan *p = nullptr;
        const sfft_request &q = job.req;
        const sfft_status st = sfft::plan_create(&p, q.N, q.K, job.K_cap, q.B, q.w, q.L, q.seed, &q.opts);
        const size_t bytes = reserved;  // the plan's scratch, as sized at admission
        lk.lock();
        s->building.erase(job.key);
        s->plan_bytes -= reserved;
        if (st == SFFT_OK) {
            s->plans.push_back(CachedPlan{p, job.key, bytes, false, ++s->use_clock});
            s->plan_bytes += bytes;
        } else {
            // fail every queued request of this shape
            const int64_t t = now_ns();
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                if ((*it)->key == job.key) {
                    (*it)->status = st;
                    (*it)->done = true;
                    (*it)->t_done = t;
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
            s->done_cv.notify_all();
        }
        s->cv.notify_all();
    }
}

void fail_batch(sfft_server *s, std::vector<Request *> &batch, sfft_status bad) {
    for (Request *r : batch) {
        r->status = bad;
        r->done = true;
        r->t_done = now_ns();
        release_plan(s, r->plan);
    }
}

constexpr size_t kScanWindow = 4096;  // queued requests looked at per admission round

void worker_main(sfft_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] {
            const bool can_launch = !s->queue.empty() && s->inflight < 2 && s->in_use < s->max_slots && !s->paused;
            return can_launch || (s->stop && s->queue.empty() && s->building.empty());
        });
        if (s->stop && s->queue.empty() && s->building.empty()) break;
        bury(s, lk);
        const int region = s->region_busy[0] ? 1 : 0;
        std::vector<Request *> batch;
        int32_t method = -1;
        bool stuck = false;  // the head request can never be served
        size_t seen = 0;
        for (auto it = s->queue.begin(); it != s->queue.end() && seen < kScanWindow &&
                                         s->in_use + (int32_t)batch.size() < s->max_slots;
             ++seen) {
            Request *r = *it;
            // one location method per batch; the others wait for the next one
            if (method >= 0 && r->req.opts.method != method) {
                ++it;
                continue;
            }
            const Take tk = try_take(s, r);
            if (tk == kTakeReady) {
                method = r->req.opts.method;
                batch.push_back(r);
                it = s->queue.erase(it);
                continue;
            }
            if (tk == kTakeNoRoom && it == s->queue.begin() && s->inflight == 0 && batch.empty() &&
                s->building.empty())
                stuck = true;
            ++it;
        }
        if (batch.empty()) {
            if (stuck) {
                // nothing running or being built can free memory for the head request
                Request *r = s->queue.front();
                s->queue.pop_front();
                r->status = SFFT_EBUSY;
                r->done = true;
                r->t_done = now_ns();
                s->done_cv.notify_all();
            } else {
                s->cv.wait(lk);  // a completion or a finished build will wake us
            }
            continue;
        }
        s->in_use += (int32_t)batch.size();
        s->inflight += 1;
        s->region_busy[region] = true;
        lk.unlock();

        cudaStream_t st = s->streams[region];
        std::vector<sfft_plan *> plans;
        std::vector<const float *> xs;
        std::vector<int32_t *> idxs;
        std::vector<float *> vals;
        sfft_status est = SFFT_OK;
        for (Request *r : batch) {
            // the request's own K and seed, uploaded ahead of the batch on its stream
            if (est == SFFT_OK) est = sfft::plan_rebind(r->plan, r->req.K, r->req.seed, st);
            plans.push_back(r->plan);
            xs.push_back(r->req.x_dev);
            idxs.push_back(r->req.idx_dev);
            vals.push_back(r->req.val_dev);
        }
        int32_t *kdev = s->kout_dev + region * s->max_slots;
        int32_t *khost = s->kout_host + region * s->max_slots;
        Batch *b = new Batch{s, region, batch};
        if (est == SFFT_OK)
            est = sfft_execute_batch(plans.data(), xs.data(), idxs.data(), vals.data(), kdev, (int32_t)batch.size(),
                                     st);
        cudaError_t ce = cudaSuccess;
        if (est == SFFT_OK) ce = cudaMemcpyAsync(khost, kdev, sizeof(int32_t) * batch.size(), cudaMemcpyDeviceToHost, st);
        if (est == SFFT_OK && ce == cudaSuccess) ce = cudaLaunchHostFunc(st, on_batch_done, b);
        lk.lock();
        if (est != SFFT_OK || ce != cudaSuccess) {
            fail_batch(s, batch, est != SFFT_OK ? est : SFFT_ECUDA);
            s->in_use -= (int32_t)batch.size();
            s->inflight -= 1;
            s->region_busy[region] = false;
            delete b;
            s->done_cv.notify_all();
        }
    }
    // drain: wait for batches still on the device
    s->done_cv.wait(lk, [&] { return s->inflight == 0; });
    bury(s, lk);
}

bool valid_request(const sfft_request *q) { return q && q->x_dev && q->idx_dev && q->val_dev; }

int32_t pow2_at_least(int32_t v) {
    int32_t p = 1;
    while (p < v) p <<= 1;
    return p;
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
    s->builder = std::thread(builder_main, s);
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
    // voting plans serve every K up to the next power of two (within the size limits)
    int32_t K_cap = q->K;
    if (q->opts.method == SFFT_METHOD_VOTING && q->K >= 1) {
        K_cap = pow2_at_least(q->K);
        if (K_cap > sfft::kMaxK || (int64_t)K_cap > q->N) K_cap = q->K;
    }
    // validates sizes and options (the reason is set on failure)
    const size_t need = sfft::plan_device_bytes(q->N, K_cap, q->B, q->w, q->L, c, T, q->opts);
    if (need == 0) return SFFT_EINVAL;
    if (need > s->budget) {
        sfft::set_error("request's plan alone exceeds the server's memory budget");
        return SFFT_EBUSY;
    }
    Request *r = new (std::nothrow) Request();
    if (!r) return SFFT_ENOMEM;
    r->req = *q;
    r->K_cap = K_cap;
    r->key = PlanKey(q->N, q->w, K_cap, q->B, q->L, c, T, q->opts.method, q->opts.comb, q->opts.estimator,
                     q->opts.refine, q->opts.search_bits, q->opts.residual, q->opts.precision, q->opts.mode);
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

static sfft_status take_result(sfft_server *s, Request *r, sfft_result *res, std::unique_lock<std::mutex> &lk) {
    const sfft_request q = r->req;
    if (res) {
        res->k_out = r->k_out;
        res->status = r->status;
        res->latency_ns = r->t_done - r->t_submit;
        res->samples_touched = -1;
    }
    const sfft_status st = r->status;
    s->tickets.erase(r->ticket);
    delete r;
    lk.unlock();
    // counted on the caller's thread, from the request's own parameters
    if (res && q.count_samples && st == SFFT_OK)
        res->samples_touched = sfft::samples_touched_of(q.N, q.B, q.w, q.L, q.seed, q.opts);
    if (st != SFFT_OK) sfft::set_error("request failed");
    return st;
}

extern "C" sfft_status sfft_poll(sfft_server *s, uint64_t ticket, sfft_result *res) {
    if (!s) return SFFT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        sfft::set_error("unknown ticket");
        return SFFT_EINVAL;
    }
    if (!it->second->done) return SFFT_EPENDING;
    return take_result(s, it->second, res, lk);
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
    return take_result(s, r, res, lk);
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
    s->build_cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->builds.clear();
    }
    s->build_cv.notify_all();
    if (s->builder.joinable()) s->builder.join();
    for (auto &st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (auto &cp : s->plans) sfft_plan_destroy(cp.plan);
    for (sfft_plan *p : s->graveyard) sfft_plan_destroy(p);
    for (auto &kv : s->tickets) delete kv.second;
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    cudaFree(s->kout_dev);
    cudaFreeHost(s->kout_host);
    delete s;
}
