// serve.cu -- a request loop over the growth and reduction kernels.
//
// Clients submit ensemble requests (model, N, chain count, trials, beta eps,
// seed) from any thread.  A scheduler thread admits them in arrival order as
// soon as a slot and enough of the device-memory budget are free, and enqueues
// the request's growth and FP64 reduction at once on a stream of its own, so
// requests that arrive while others are on the GPU run concurrently with them
// (the block scheduler interleaves the kernels of all active streams).  Output
// memory comes from a stream-ordered pool; the statistics land in pinned host
// memory.  With shortest_first the streams carry priorities by the request's
// work (decades of pair tests): when SMs free up, the blocks of smaller
// requests are dispatched first, so a small request does not wait behind the
// waves of a large one (nothing is preempted).  Completion is detected with event queries on the host -- no kernel
// ever waits -- and waits by clients are bounded condition-variable waits.
// A request's chains are a pure function of its parameters (stateless Philox
// keyed by seed, ensemble, chain and step), so its result does not depend on
// what else is running.
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace {

enum State { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Request {
    uint64_t ticket = 0;
    rosen_request req;
    State state = QUEUED;
    int status = ROSEN_OK;
    char message[256] = "";
    int level = 0;             // stream priority class (0: the least work)
    size_t work_bytes = 0;     // outputs + reduction workspace (freed at completion)
    size_t coord_bytes = 0;    // stored conformations (freed at release)
    void *work = nullptr;
    void *coords = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    rosen_stats *host_stats = nullptr;   // pinned
    rosen_stats stats;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    bool in_queue = false;     // still referenced by the admission queue
    bool released = false;     // the client has let go of the ticket
};

}  // namespace

struct rosen_server {
    rosen_serve_config cfg;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_done;   // a request finished
    std::condition_variable cv_work;   // new submission or shutdown
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<std::vector<cudaStream_t>> streams;   // idle streams per priority class
    int prio_greatest = 0;     // CUDA priority of class 0 (numerically lowest)
    int levels = 1;
    std::vector<cudaEvent_t> events;
    std::vector<rosen_stats *> pinned;
    size_t used = 0;
    std::vector<std::pair<void *, size_t>> to_free;   // released conformations
    cudaStream_t free_stream = nullptr;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    // counters
    uint64_t n_submitted = 0, n_rejected = 0, n_done = 0, n_failed = 0;
};

namespace {

using namespace rosen;

bool valid_model(const rosen_request &r)
{
    return r.model == ROSEN_MODEL_LATTICE || r.model == ROSEN_MODEL_OFFLATTICE;
}

constexpr size_t kLongWorkspaceCap = size_t(1) << 30;

bool long_request(const rosen_request &r)
{
    return r.model == ROSEN_MODEL_LATTICE ? r.N > ROSEN_LATTICE_NMAX : r.N > ROSEN_OFFLATTICE_NMAX;
}

// Workspace of a long-chain request: the default size, at most 1 GiB (fewer
// chains in flight), at least one table or chain slot.
size_t long_workspace_bytes(const rosen_request &r)
{
    if (!long_request(r)) return 0;
    const bool lat = r.model == ROSEN_MODEL_LATTICE;
    const size_t want = lat ? rosen_lattice_long_workspace_size(r.N, r.C)
                            : rosen_offlattice_long_workspace_size(r.N, r.C);
    const size_t one = lat ? rosen_lattice_long_workspace_size(r.N, 1)
                           : rosen_offlattice_long_workspace_size(r.N, 1);
    return align256(std::max(one, std::min(want, kLongWorkspaceCap)));
}

// Device bytes a request holds while it runs, and what stored conformations
// keep after it finishes.
void request_bytes(const rosen_request &r, size_t *work, size_t *coords)
{
    const size_t C = (size_t)r.C, N = (size_t)r.N;
    size_t b = long_workspace_bytes(r);
    if (r.model == ROSEN_MODEL_LATTICE)
        b += align256(16 * C) + align256(4 * C) + align256(4 * C) + align256(8 * C);
    else
        b += 3 * align256(4 * C) + align256(C);
    if (r.max_attempts > 1) b += align256(2 * C);   // attempts per chain (restart mode)
    b += align256(rosen_reduce_workspace_size(r.C)) + align256(sizeof(rosen_stats));
    *work = b;
    *coords = r.store_coords ? align256(12 * N * C) : 0;
}

// Priority class of a request (shortest_first): decades of its pair tests
// (chains x (N-1)(N-2)/2 x trials per step), class 0 -- the highest priority,
// well under a millisecond of GPU time -- below 1e8, up to the last class.
int work_level(const rosen_request &r, int levels)
{
    const double n = (double)r.N;
    const double pairs = (double)r.C * (n - 1.0) * (n - 2.0) * 0.5 *
                         (r.model == ROSEN_MODEL_LATTICE ? 1.0 : (double)r.k);
    int level = pairs < 1.0 ? 0 : (int)floor(log10(pairs)) - 7;
    if (level < 0) level = 0;
    if (level > levels - 1) level = levels - 1;
    return level;
}

int validate_request(const rosen_request &r)
{
    if (!valid_model(r)) return set_error(ROSEN_EINVAL, "rosen_serve_submit: unknown model %d", r.model);
    if (r.C < 1) return set_error(ROSEN_EINVAL, "rosen_serve_submit: C must be >= 1");
    if (r.model == ROSEN_MODEL_LATTICE) {
        rosen_lattice_params p;
        memset(&p, 0, sizeof p);
        p.seed = r.seed;
        p.ensemble = r.ensemble;
        p.N = r.N;
        p.C = r.C;
        p.beta_eps = r.beta_eps;
        p.flags = r.store_coords ? ROSEN_STORE_COORDS : 0;
        p.max_attempts = r.max_attempts;
        rosen_lattice_out o;
        memset(&o, 0, sizeof o);
        o.coords = r.store_coords ? reinterpret_cast<int32_t *>(16) : nullptr;
        return lattice_validate(&p, &o, ROSEN_LATTICE_LONG_NMAX, "rosen_serve_submit");
    }
    rosen_offlattice_params p;
    memset(&p, 0, sizeof p);
    p.seed = r.seed;
    p.ensemble = r.ensemble;
    p.N = r.N;
    p.C = r.C;
    p.k = r.k;
    p.potential = r.potential;
    p.sigma = r.sigma;
    p.cutoff = r.cutoff;
    p.beta_eps = r.beta_eps;
    p.flags = r.store_coords ? ROSEN_STORE_COORDS : 0;
    p.max_attempts = r.max_attempts;
    rosen_offlattice_out o;
    memset(&o, 0, sizeof o);
    o.coords = r.store_coords ? reinterpret_cast<float *>(16) : nullptr;
    return offlattice_validate(&p, &o, ROSEN_OFFLATTICE_LONG_NMAX, "rosen_serve_submit");
}

void fail(Request *q, int status, const char *msg)
{
    q->state = FAILED;
    q->status = status;
    snprintf(q->message, sizeof q->message, "%s", msg);
}

// Return a failed request's scratch to the pool (stream-ordered).
void release_work(Request *q)
{
    if (q->work) cudaFreeAsync(q->work, q->stream);
    q->work = nullptr;
}

// Enqueue a request's whole pass on its stream (scheduler thread, lock held).
void launch(rosen_server *s, Request *q)
{
    const rosen_request &r = q->req;
    const size_t C = (size_t)r.C;
    cudaError_t e = cudaMallocFromPoolAsync(&q->work, q->work_bytes, s->pool, q->stream);
    if (e == cudaSuccess && q->coord_bytes)
        e = cudaMallocFromPoolAsync(&q->coords, q->coord_bytes, s->pool, q->stream);
    if (e != cudaSuccess) {
        fail(q, ROSEN_ENOMEM, cudaGetErrorString(e));
        release_work(q);
        return;
    }
    unsigned char *p = static_cast<unsigned char *>(q->work);
    const size_t long_bytes = long_workspace_bytes(r);
    void *long_ws = long_bytes ? p : nullptr;   // long chains: their workspace first
    p += long_bytes;
    rosen_reduce_in in;
    memset(&in, 0, sizeof in);
    in.N = r.N;
    in.C = r.C;
    int st;
    if (r.model == ROSEN_MODEL_LATTICE) {
        rosen_lattice_out o;
        memset(&o, 0, sizeof o);
        o.counts = reinterpret_cast<uint16_t *>(p);
        p += align256(16 * C);
        o.logw = reinterpret_cast<float *>(p);
        p += align256(4 * C);
        o.r2 = reinterpret_cast<int32_t *>(p);
        p += align256(4 * C);
        o.n2rg2 = reinterpret_cast<int64_t *>(p);
        p += align256(8 * C);
        if (r.max_attempts > 1) {
            o.attempts = reinterpret_cast<uint16_t *>(p);
            p += align256(2 * C);
        }
        o.coords = static_cast<int32_t *>(q->coords);
        rosen_lattice_params lp;
        memset(&lp, 0, sizeof lp);
        lp.seed = r.seed;
        lp.ensemble = r.ensemble;
        lp.N = r.N;
        lp.C = r.C;
        lp.beta_eps = r.beta_eps;
        lp.flags = q->coords ? ROSEN_STORE_COORDS : 0;
        lp.max_attempts = r.max_attempts;
        st = long_ws ? rosen_lattice_grow_long(&lp, &o, long_ws, long_bytes, q->stream)
                     : rosen_lattice_grow(&lp, &o, q->stream);
        in.attempts = o.attempts;
        in.kind = ROSEN_REDUCE_LATTICE;
        in.use_counts = r.beta_eps == 0.0;
        in.logw = o.logw;
        in.counts = o.counts;
        in.r2_i = o.r2;
        in.n2rg2 = o.n2rg2;
    } else {
        rosen_offlattice_out o;
        memset(&o, 0, sizeof o);
        o.logw = reinterpret_cast<float *>(p);
        p += align256(4 * C);
        o.r2 = reinterpret_cast<float *>(p);
        p += align256(4 * C);
        o.rg2 = reinterpret_cast<float *>(p);
        p += align256(4 * C);
        o.alive = p;
        p += align256(C);
        if (r.max_attempts > 1) {
            o.attempts = reinterpret_cast<uint16_t *>(p);
            p += align256(2 * C);
        }
        o.coords = static_cast<float *>(q->coords);
        rosen_offlattice_params op;
        memset(&op, 0, sizeof op);
        op.seed = r.seed;
        op.ensemble = r.ensemble;
        op.N = r.N;
        op.C = r.C;
        op.k = r.k;
        op.potential = r.potential;
        op.sigma = r.sigma;
        op.cutoff = r.cutoff;
        op.beta_eps = r.beta_eps;
        op.flags = q->coords ? ROSEN_STORE_COORDS : 0;
        op.max_attempts = r.max_attempts;
        st = long_ws ? rosen_offlattice_grow_long(&op, &o, long_ws, long_bytes, q->stream)
                     : rosen_offlattice_grow(&op, &o, q->stream);
        in.attempts = o.attempts;
        in.kind = ROSEN_REDUCE_OFFLATTICE;
        in.k = r.k;
        in.logw = o.logw;
        in.r2_f = o.r2;
        in.rg2_f = o.rg2;
    }
    rosen_stats *dstats = reinterpret_cast<rosen_stats *>(p);
    p += align256(sizeof(rosen_stats));
    const size_t ws = rosen_reduce_workspace_size(r.C);
    if (st == ROSEN_OK) st = rosen_reduce(&in, dstats, p, ws, q->stream);
    if (st != ROSEN_OK) {
        fail(q, st, rosen_last_error());
        release_work(q);
        return;
    }
    e = cudaMemcpyAsync(q->host_stats, dstats, sizeof(rosen_stats), cudaMemcpyDeviceToHost,
                        q->stream);
    // The outputs are scratch once the statistics are copied; conformations stay.
    if (e == cudaSuccess) e = cudaFreeAsync(q->work, q->stream);
    q->work = nullptr;
    if (e == cudaSuccess) e = cudaEventRecord(q->done, q->stream);
    if (e != cudaSuccess) fail(q, ROSEN_ECUDA, cudaGetErrorString(e));
}

void scheduler(rosen_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        bool progressed = false;
        // Conformations the clients released.
        for (auto &f : s->to_free) {
            cudaFreeAsync(f.first, s->free_stream);
            s->used -= f.second;
            progressed = true;
        }
        s->to_free.clear();
        // Completions.
        for (size_t i = 0; i < s->running.size();) {
            Request *q = s->running[i];
            const cudaError_t e = (q->state == FAILED) ? cudaSuccess : cudaEventQuery(q->done);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            if (q->state != FAILED) {
                if (e == cudaSuccess) {
                    q->stats = *q->host_stats;
                    q->state = DONE;
                    ++s->n_done;
                } else {
                    fail(q, ROSEN_ECUDA, cudaGetErrorString(e));
                }
            }
            if (q->state == FAILED) ++s->n_failed;
            q->t_done = now_ns();
            s->used -= q->work_bytes;
            if (q->state == FAILED) {
                // A failed request gives back everything it reserved, whether
                // or not its conformations were ever allocated.
                if (q->coords) cudaFreeAsync(q->coords, q->stream);
                q->coords = nullptr;
                s->used -= q->coord_bytes;
            }
            s->streams[q->level].push_back(q->stream);
            s->events.push_back(q->done);
            s->pinned.push_back(q->host_stats);
            q->stream = nullptr;
            q->done = nullptr;
            q->host_stats = nullptr;
            s->running[i] = s->running.back();
            s->running.pop_back();
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // Admissions, in arrival order.
        while (!s->stop && !s->queue.empty() && (int)s->running.size() < s->cfg.max_slots) {
            Request *q = s->queue.front();
            if (q->state == CANCELLED) {
                s->queue.pop_front();
                q->in_queue = false;
                if (q->released) delete q;
                continue;
            }
            const size_t need = q->work_bytes + q->coord_bytes;
            if (s->used + need > s->cfg.mem_budget_bytes) break;
            // A stream of the request's priority class (created on first use;
            // at most max_slots per class are ever in use).
            std::vector<cudaStream_t> &idle = s->streams[q->level];
            if (idle.empty()) {
                cudaStream_t st;
                if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking,
                                                 s->prio_greatest + q->level) != cudaSuccess) {
                    cudaGetLastError();
                    break;   // the request stays queued; retried at the next pass
                }
                idle.push_back(st);
            }
            s->queue.pop_front();
            q->in_queue = false;
            s->used += need;
            q->stream = idle.back();
            idle.pop_back();
            q->done = s->events.back();
            s->events.pop_back();
            q->host_stats = s->pinned.back();
            s->pinned.pop_back();
            q->state = RUNNING;
            q->t_admit = now_ns();
            launch(s, q);
            s->running.push_back(q);
            progressed = true;
        }
        if (s->stop && s->running.empty()) break;
        if (!progressed) {
            // Nothing to do right now: sleep until a submission arrives, or
            // briefly while work is on the GPU.
            if (s->running.empty())
                s->cv_work.wait_for(lock, std::chrono::milliseconds(50));
            else {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
                lock.lock();
            }
        }
    }
}

void fill_result(const Request *q, rosen_result *out)
{
    memset(out, 0, sizeof *out);
    out->ticket = q->ticket;
    out->status = q->state == DONE ? ROSEN_OK : (q->state == CANCELLED ? ROSEN_ECLOSED : q->status);
    out->stats = q->stats;
    out->t_submit_ns = q->t_submit;
    out->t_admit_ns = q->t_admit;
    out->t_done_ns = q->t_done;
    out->coords = q->coords;
    snprintf(out->message, sizeof out->message, "%s", q->message);
}

}  // namespace

extern "C" int rosen_serve_create(const rosen_serve_config *cfg, rosen_server **out)
{
    if (!cfg || !out) return set_error(ROSEN_EINVAL, "rosen_serve_create: NULL argument");
    if (cfg->max_slots < 1 || cfg->max_slots > 1024 || cfg->max_queue < 1 ||
        cfg->mem_budget_bytes == 0 || (cfg->shortest_first != 0 && cfg->shortest_first != 1))
        return set_error(ROSEN_EINVAL, "rosen_serve_create: max_slots in [1, 1024], max_queue >= 1, "
                                       "a non-zero budget and shortest_first 0 or 1 are required");
    rosen_server *s = new rosen_server();
    s->cfg = *cfg;
    s->device = cfg->device;
    cudaError_t e = cudaSetDevice(s->device);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = cfg->mem_budget_bytes;   // keep freed blocks for reuse up to the budget
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->free_stream, cudaStreamNonBlocking);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    // Without shortest_first every stream has the default priority.
    s->prio_greatest = cfg->shortest_first ? greatest : 0;
    s->levels = cfg->shortest_first ? least - greatest + 1 : 1;
    if (s->levels < 1) s->levels = 1;
    s->streams.resize((size_t)s->levels);
    for (int i = 0; e == cudaSuccess && i < cfg->max_slots; ++i) {
        cudaEvent_t ev;
        rosen_stats *h;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h), sizeof(rosen_stats));
        if (e == cudaSuccess) {
            s->events.push_back(ev);
            s->pinned.push_back(h);
        }
    }
    if (e != cudaSuccess) {
        if (s->free_stream) cudaStreamDestroy(s->free_stream);
        for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
        for (rosen_stats *h : s->pinned) cudaFreeHost(h);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return set_error(ROSEN_ECUDA, "rosen_serve_create: %s", cudaGetErrorString(e));
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return ROSEN_OK;
}

extern "C" int rosen_serve_submit(rosen_server *s, const rosen_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket) return set_error(ROSEN_EINVAL, "rosen_serve_submit: NULL argument");
    int st = validate_request(*r);
    if (st != ROSEN_OK) return st;
    Request *q = new Request();
    q->req = *r;
    request_bytes(*r, &q->work_bytes, &q->coord_bytes);
    q->level = work_level(*r, s->levels);
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) {
        delete q;
        return set_error(ROSEN_ECLOSED, "rosen_serve_submit: server is shutting down");
    }
    if (q->work_bytes + q->coord_bytes > s->cfg.mem_budget_bytes) {
        ++s->n_rejected;
        const size_t need = q->work_bytes + q->coord_bytes;
        delete q;
        return set_error(ROSEN_EINVAL, "rosen_serve_submit: request needs %zu bytes, more than "
                                       "the whole budget of %zu", need,
                         (size_t)s->cfg.mem_budget_bytes);
    }
    if ((int64_t)s->queue.size() >= s->cfg.max_queue) {
        ++s->n_rejected;
        delete q;
        return set_error(ROSEN_EBUSY, "rosen_serve_submit: queue full (%d)", s->cfg.max_queue);
    }
    q->ticket = s->next_ticket++;
    q->t_submit = now_ns();
    q->in_queue = true;
    s->queue.push_back(q);
    s->all[q->ticket] = q;
    ++s->n_submitted;
    *ticket = q->ticket;
    s->cv_work.notify_one();
    return ROSEN_OK;
}

extern "C" int rosen_serve_poll(rosen_server *s, uint64_t ticket, rosen_result *out)
{
    if (!s || !out) return set_error(ROSEN_EINVAL, "rosen_serve_poll: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(ROSEN_ENOTFOUND, "rosen_serve_poll: unknown ticket");
    const Request *q = it->second;
    if (q->state == QUEUED || q->state == RUNNING) return ROSEN_EAGAIN;
    fill_result(q, out);
    return ROSEN_OK;
}

extern "C" int rosen_serve_wait(rosen_server *s, uint64_t ticket, int64_t timeout_ns, rosen_result *out)
{
    if (!s || !out) return set_error(ROSEN_EINVAL, "rosen_serve_wait: NULL argument");
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
    for (;;) {
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return set_error(ROSEN_ENOTFOUND, "rosen_serve_wait: unknown ticket");
        const Request *q = it->second;
        if (q->state != QUEUED && q->state != RUNNING) {
            fill_result(q, out);
            return ROSEN_OK;
        }
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
            auto it2 = s->all.find(ticket);
            if (it2 != s->all.end() && it2->second->state != QUEUED && it2->second->state != RUNNING) {
                fill_result(it2->second, out);
                return ROSEN_OK;
            }
            return set_error(ROSEN_ETIMEOUT, "rosen_serve_wait: ticket %llu not done",
                             (unsigned long long)ticket);
        }
    }
}

extern "C" int rosen_serve_cancel(rosen_server *s, uint64_t ticket)
{
    if (!s) return set_error(ROSEN_EINVAL, "rosen_serve_cancel: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(ROSEN_ENOTFOUND, "rosen_serve_cancel: unknown ticket");
    Request *q = it->second;
    if (q->state != QUEUED)
        return set_error(ROSEN_EBUSY, "rosen_serve_cancel: ticket already admitted");
    q->state = CANCELLED;
    s->cv_done.notify_all();
    return ROSEN_OK;
}

extern "C" int rosen_serve_release(rosen_server *s, uint64_t ticket)
{
    if (!s) return set_error(ROSEN_EINVAL, "rosen_serve_release: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(ROSEN_ENOTFOUND, "rosen_serve_release: unknown ticket");
    Request *q = it->second;
    if (q->state == QUEUED || q->state == RUNNING)
        return set_error(ROSEN_EBUSY, "rosen_serve_release: ticket still in flight");
    if (q->coords) {
        // Freed by the scheduler thread, stream-ordered, on its own stream.
        s->to_free.push_back({q->coords, q->coord_bytes});
        q->coords = nullptr;
        s->cv_work.notify_one();
    }
    s->all.erase(it);
    // A cancelled request may still sit in the queue: the scheduler deletes it.
    if (q->in_queue) q->released = true;
    else delete q;
    return ROSEN_OK;
}

extern "C" int rosen_serve_info(rosen_server *s, rosen_serve_counters *out)
{
    if (!s || !out) return set_error(ROSEN_EINVAL, "rosen_serve_info: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->n_submitted;
    out->rejected = s->n_rejected;
    out->completed = s->n_done;
    out->failed = s->n_failed;
    out->queued = s->queue.size();
    out->running = s->running.size();
    out->bytes_in_use = s->used;
    return ROSEN_OK;
}

extern "C" int rosen_serve_destroy(rosen_server *s)
{
    if (!s) return ROSEN_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (Request *q : s->queue)
            if (q->state == QUEUED) q->state = CANCELLED;
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    s->th.join();   // the scheduler drains the running requests first
    cudaSetDevice(s->device);
    std::vector<Request *> owned;
    for (auto &kv : s->all) owned.push_back(kv.second);
    for (Request *q : s->queue)
        if (q->released) owned.push_back(q);
    for (Request *q : owned) {
        if (q->coords) cudaFreeAsync(q->coords, s->free_stream);
        delete q;
    }
    for (auto &f : s->to_free) cudaFreeAsync(f.first, s->free_stream);
    cudaStreamSynchronize(s->free_stream);
    cudaStreamDestroy(s->free_stream);
    for (auto &pool : s->streams)
        for (cudaStream_t st : pool) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    for (rosen_stats *h : s->pinned) cudaFreeHost(h);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return ROSEN_OK;
}
