// serve.cu -- a request loop with continuous admission and time-sliced
// execution over the single-ensemble kernels.
//
// Clients submit ensemble requests (model, N, chain count, trials, beta eps,
// seed) from any thread.  One scheduler thread:
//  - admits waiting requests in arrival order as soon as a slot and enough of
//    the device-memory budget are free; a request that does not fit may be
//    passed by later ones that do, for at most kPassLimitNs, after which
//    nothing behind it is admitted until it fits;
//  - grows every admitted request in slices, chain ranges of about kSliceNs
//    of GPU time but at least twice the chains the GPU grows at once (so a
//    slice fills the GPU), with the single-ensemble kernels
//    (lattice_grow_range / offlattice_grow_range; long chains in one piece
//    through the long-chain entry points).  A request's slices alternate
//    between two streams of its own, so its next slice starts while the
//    last blocks of the previous one finish;
//  - chooses the request of each next slice by policy: arrival order, or
//    (shortest_first) the least estimated remaining GPU time, discounted by
//    the time the request has waited.  Under shortest_first a request that
//    has been admitted for longer than kStarveNs plus kStarveOwn times its
//    own estimated GPU time is overdue: the oldest overdue request gets every
//    other slice, so no request starves and short requests still pass it;
//    while requests wait for admission (the server is saturated, and short
//    requests wait in the queue anyway) it gets every slice;
//  - keeps about kLookaheadNs of slices enqueued so that the GPU does not
//    idle between slices (the next slice's blocks start as the last ones of
//    the running slice finish);
//  - after a request's last slice, enqueues its FP64 reduction, the copy of
//    its statistics to pinned host memory, the release of its scratch and an
//    event that marks it done.
// So a request that arrives while a large one runs starts within about one
// slice, and requests overlap on the GPU at slice boundaries.  No kernel
// waits on anything: completion is found with event queries on the host, and
// every client wait is a bounded condition-variable wait.
//
// Every chain of a request is grown by the same kernel, with the same lanes
// per chain, as rosen_lattice_grow / rosen_offlattice_grow would grow it,
// and its random numbers are a pure function of (seed, ensemble, chain,
// step); the reduction is rosen_reduce's.  A request's result is therefore
// the same, bit for bit, alone, in any mix, and through the single-ensemble
// entry points.
//
// Device memory of a request (outputs, reduction scratch, the real-space
// chain counters and deferral mask, a long-chain workspace, stored
// conformations) comes from one stream-ordered pool and is counted against
// the budget from admission until it is returned.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace {

enum State { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

constexpr int64_t kSliceNs = 4'000'000;        // target GPU time of a slice
constexpr int64_t kLookaheadNs = 8'000'000;    // estimated work kept enqueued
constexpr int kMaxInflight = 16;               // slices enqueued at once
constexpr int64_t kPassLimitNs = 1'000'000'000;   // longest a request may be passed over
constexpr double kAgingNs = 1e9;               // shortest_first: waiting discount scale
constexpr int64_t kStarveNs = 1'000'000'000;   // shortest_first: overdue after this wait
constexpr double kStarveOwn = 2.0;             //   plus this many times its own GPU time

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
    size_t work_bytes = 0;     // outputs + scratch (freed after the reduction)
    size_t coord_bytes = 0;    // stored conformations (freed at release)
    void *work = nullptr;
    void *coords = nullptr;
    // carved from work at admission
    rosen_lattice_params lp;
    rosen_lattice_out lo;
    rosen_offlattice_params op;
    rosen_offlattice_out oo;
    rosen_reduce_in rin;
    void *rws = nullptr;       // reduction workspace
    size_t rws_bytes = 0;
    rosen_stats *dstats = nullptr;
    void *scratch = nullptr;   // real space: two sets of chain counters, the deferral mask
    void *long_ws = nullptr;   // long chains: their workspace
    size_t long_bytes = 0;
    cudaStream_t streams[2] = {nullptr, nullptr};   // slices alternate between them
    cudaEvent_t done = nullptr;
    cudaEvent_t join = nullptr;   // orders the two streams (set-up, end)
    int nslices = 0;
    int64_t resident = 0;      // chains the GPU grows at once for this request
    rosen_stats *host_stats = nullptr;   // pinned
    rosen_stats stats;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int64_t t_passed = 0;      // first time a later request was admitted past it
    int64_t next_chain = 0;    // first chain not yet in a slice
    int inflight = 0;          // slices enqueued and not yet seen complete
    bool finishing = false;    // the reduction (or, after a failure, the end) is enqueued
    double ns_per_chain = 0.0; // estimated GPU time per chain
    bool in_queue = false;     // still referenced by the admission queue
    bool released = false;     // the client has let go of the ticket
};

struct Slice {
    Request *q = nullptr;
    int64_t chains = 0;
    double est_ns = 0.0;
    cudaEvent_t start = nullptr, end = nullptr;
};

}  // namespace

struct rosen_server {
    rosen_serve_config cfg;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_done;   // a request finished
    std::condition_variable cv_work;   // new submission, release or shutdown
    std::deque<Request *> queue;
    std::vector<Request *> active;     // admitted, not yet finished
    std::vector<Slice> slices;         // enqueued slices, oldest first
    std::unordered_map<uint64_t, Request *> all;
    std::vector<cudaStream_t> streams;       // idle streams
    std::vector<cudaEvent_t> done_events;    // idle completion events
    std::vector<cudaEvent_t> timing_events;  // idle slice events
    cudaEvent_t last_end = nullptr;    // end of the last slice seen complete
    std::vector<rosen_stats *> pinned;
    std::map<uint64_t, double> rate;   // GPU ns per chain by request class
    size_t used = 0;
    std::vector<std::pair<void *, size_t>> to_free;   // released conformations
    cudaStream_t free_stream = nullptr;
    uint64_t next_ticket = 1;
    bool overdue_turn = false;         // shortest_first: the next shared slice's turn
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

// Real-space chain counters (one set per stream) and deferral mask
// (shared-memory kernels).
size_t scratch_bytes(const rosen_request &r)
{
    if (r.model != ROSEN_MODEL_OFFLATTICE || long_request(r)) return 0;
    return align256(2 * offlattice_range_counter_bytes() + offlattice_range_mask_bytes(r.C));
}

// Device bytes a request holds while it runs, and what stored conformations
// keep after it finishes.
void request_bytes(const rosen_request &r, size_t *work, size_t *coords)
{
    const size_t C = (size_t)r.C, N = (size_t)r.N;
    size_t b = long_workspace_bytes(r) + scratch_bytes(r);
    if (r.model == ROSEN_MODEL_LATTICE)
        b += align256(16 * C) + align256(4 * C) + align256(4 * C) + align256(8 * C);
    else
        b += 3 * align256(4 * C) + align256(C);
    if (r.max_attempts > 1) b += align256(2 * C);   // attempts per chain (restart mode)
    b += align256(rosen_reduce_workspace_size(r.C)) + align256(sizeof(rosen_stats));
    *work = b;
    *coords = r.store_coords ? align256(12 * N * C) : 0;
}

// Class of a request for the GPU-time estimate: model, potential, trials,
// chain-length bucket of 16.
uint64_t rate_key(const rosen_request &r)
{
    return ((uint64_t)r.model << 56) | ((uint64_t)(r.potential & 0xFF) << 48) |
           ((uint64_t)(r.k & 0xFFFF) << 32) | (uint64_t)(r.N / 16);
}

// First estimate of a class's GPU time per chain (ns), from GB300 timings of
// the single-ensemble kernels at N = 64 (lattice 1.2 ns, hard spheres 0.55 k,
// Lennard-Jones 1.8 k per chain) scaled by N^2; refined by measured slices.
double default_ns_per_chain(const rosen_request &r)
{
    const double f = ((double)r.N / 64.0) * ((double)r.N / 64.0);
    double base;
    if (r.model == ROSEN_MODEL_LATTICE) base = 1.2;
    else base = (r.potential == ROSEN_LJ ? 1.8 : 0.55) * (double)r.k;
    return std::max(0.05, base * f);
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

// Pointers of a request's outputs and scratch inside its work allocation.
void carve(Request *q)
{
    const rosen_request &r = q->req;
    const size_t C = (size_t)r.C;
    unsigned char *p = static_cast<unsigned char *>(q->work);
    q->long_bytes = long_workspace_bytes(r);
    q->long_ws = q->long_bytes ? p : nullptr;   // long chains: their workspace first
    p += q->long_bytes;
    const size_t sb = scratch_bytes(r);
    q->scratch = sb ? p : nullptr;
    p += sb;
    rosen_reduce_in &in = q->rin;
    memset(&in, 0, sizeof in);
    in.N = r.N;
    in.C = r.C;
    if (r.model == ROSEN_MODEL_LATTICE) {
        rosen_lattice_out &o = q->lo;
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
        rosen_lattice_params &lp = q->lp;
        memset(&lp, 0, sizeof lp);
        lp.seed = r.seed;
        lp.ensemble = r.ensemble;
        lp.N = r.N;
        lp.C = r.C;
        lp.beta_eps = r.beta_eps;
        lp.flags = q->coords ? ROSEN_STORE_COORDS : 0;
        lp.max_attempts = r.max_attempts;
        in.attempts = o.attempts;
        in.kind = ROSEN_REDUCE_LATTICE;
        in.use_counts = r.beta_eps == 0.0;
        in.logw = o.logw;
        in.counts = o.counts;
        in.r2_i = o.r2;
        in.n2rg2 = o.n2rg2;
    } else {
        rosen_offlattice_out &o = q->oo;
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
        rosen_offlattice_params &op = q->op;
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
        in.attempts = o.attempts;
        in.kind = ROSEN_REDUCE_OFFLATTICE;
        in.k = r.k;
        in.logw = o.logw;
        in.r2_f = o.r2;
        in.rg2_f = o.rg2;
    }
    q->dstats = reinterpret_cast<rosen_stats *>(p);
    p += align256(sizeof(rosen_stats));
    q->rws = p;
    q->rws_bytes = rosen_reduce_workspace_size(r.C);
}

cudaEvent_t take_event(std::vector<cudaEvent_t> &pool, unsigned flags)
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, flags) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Resources of a request that is no longer on the GPU go back to the pools.
void retire(rosen_server *s, Request *q)
{
    for (cudaStream_t &st : q->streams) {
        if (st) s->streams.push_back(st);
        st = nullptr;
    }
    if (q->done) s->done_events.push_back(q->done);
    if (q->join) s->done_events.push_back(q->join);
    if (q->host_stats) s->pinned.push_back(q->host_stats);
    q->done = nullptr;
    q->join = nullptr;
    q->host_stats = nullptr;
}

// Admit q (lock held): stream, completion event, pinned statistics, device
// memory from the pool, and the set-up of its scratch.  A request whose
// memory cannot be had fails at once and gives its reservation back.
bool admit(rosen_server *s, Request *q)
{
    while (s->streams.size() < 2) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return false;     // stays queued; retried at the next pass
        }
        s->streams.push_back(st);
    }
    cudaEvent_t done = take_event(s->done_events, cudaEventDisableTiming);
    if (!done) return false;
    cudaEvent_t join = take_event(s->done_events, cudaEventDisableTiming);
    if (!join) {
        s->done_events.push_back(done);
        return false;
    }
    if (s->pinned.empty()) {
        rosen_stats *h = nullptr;
        if (cudaMallocHost(reinterpret_cast<void **>(&h), sizeof(rosen_stats)) != cudaSuccess) {
            cudaGetLastError();
            s->done_events.push_back(done);
            s->done_events.push_back(join);
            return false;
        }
        s->pinned.push_back(h);
    }
    for (cudaStream_t &st : q->streams) {
        st = s->streams.back();
        s->streams.pop_back();
    }
    q->done = done;
    q->join = join;
    q->host_stats = s->pinned.back();
    s->pinned.pop_back();
    q->state = RUNNING;
    q->t_admit = now_ns();
    const uint64_t key = rate_key(q->req);
    auto it = s->rate.find(key);
    q->ns_per_chain = it != s->rate.end() ? it->second : default_ns_per_chain(q->req);

    cudaStream_t s0 = q->streams[0];
    cudaError_t e = cudaMallocFromPoolAsync(&q->work, q->work_bytes, s->pool, s0);
    if (e == cudaSuccess && q->coord_bytes)
        e = cudaMallocFromPoolAsync(&q->coords, q->coord_bytes, s->pool, s0);
    if (e == cudaSuccess) {
        carve(q);
        if (q->scratch) e = cudaMemsetAsync(q->scratch, 0, scratch_bytes(q->req), s0);
    }
    // The second stream starts after the allocation and the set-up.
    if (e == cudaSuccess) e = cudaEventRecord(q->join, s0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->streams[1], q->join, 0);
    if (e == cudaSuccess && !q->long_ws) {
        q->resident = q->req.model == ROSEN_MODEL_LATTICE ? lattice_resident_chains(&q->lp)
                                                          : offlattice_resident_chains(&q->op);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(q, ROSEN_ENOMEM, cudaGetErrorString(e));
        if (q->work) cudaFreeAsync(q->work, s0);
        if (q->coords) cudaFreeAsync(q->coords, s0);
        q->work = q->coords = nullptr;
        cudaGetLastError();
        q->t_done = now_ns();
        ++s->n_failed;
        retire(s, q);
        s->cv_done.notify_all();
        return true;          // taken off the queue, finished (failed)
    }
    s->used += q->work_bytes + q->coord_bytes;
    s->active.push_back(q);
    return true;
}

// Enqueue the end of a request on its stream: the reduction, the copy of the
// statistics, the release of its scratch and the completion event.  After a
// failure only the release and the event (so its in-flight slices finish
// before its memory is reused).
void finish(Request *q)
{
    q->finishing = true;
    cudaStream_t s0 = q->streams[0];
    // The end runs on the first stream once the second has drained.
    if (cudaEventRecord(q->join, q->streams[1]) != cudaSuccess ||
        cudaStreamWaitEvent(s0, q->join, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(q->streams[1]);
    }
    int st = ROSEN_OK;
    if (q->state != FAILED) {
        st = rosen_reduce(&q->rin, q->dstats, q->rws, q->rws_bytes, s0);
        if (st == ROSEN_OK &&
            cudaMemcpyAsync(q->host_stats, q->dstats, sizeof(rosen_stats), cudaMemcpyDeviceToHost,
                            s0) != cudaSuccess)
            st = set_error(ROSEN_ECUDA, "copying the statistics: %s",
                           cudaGetErrorString(cudaGetLastError()));
        if (st != ROSEN_OK) fail(q, st, rosen_last_error());
    }
    // The outputs are scratch once the statistics are copied; conformations stay.
    if (q->work) cudaFreeAsync(q->work, s0);
    q->work = nullptr;
    if (cudaEventRecord(q->done, s0) != cudaSuccess) {
        // Without the event the stream is synchronised here instead.
        cudaGetLastError();
        cudaStreamSynchronize(s0);
        cudaEventRecord(q->done, 0);
    }
}

// Enqueue the next slice of q on the stream after the last one's:
// chains [next_chain, next_chain + n), or the whole request for long chains.
// A slice holds about kSliceNs of estimated GPU time but at least twice the
// chains the GPU grows at once, and starts at a multiple of 32 chains (the
// deferral mask's words).
void launch_slice(rosen_server *s, Request *q)
{
    const int64_t C = q->req.C;
    int64_t n = C - q->next_chain;
    if (!q->long_ws) {
        const double per = std::max(q->ns_per_chain, 1e-3);
        int64_t want = std::max<int64_t>((int64_t)((double)kSliceNs / per), 2 * q->resident);
        want = std::max<int64_t>(32, (want + 31) / 32 * 32);
        if (n - want >= want / 2) n = want;   // else: the remainder in one slice
    }
    const int lane = q->nslices & 1;
    cudaStream_t st_q = q->streams[lane];
    ++q->nslices;
    Slice sl;
    sl.q = q;
    sl.chains = n;
    sl.est_ns = (double)n * q->ns_per_chain;
    sl.start = take_event(s->timing_events, cudaEventDefault);
    sl.end = take_event(s->timing_events, cudaEventDefault);
    int st = ROSEN_OK;
    if (sl.start) cudaEventRecord(sl.start, st_q);
    const int64_t c_lo = q->next_chain, c_hi = c_lo + n;
    if (q->long_ws) {
        st = q->req.model == ROSEN_MODEL_LATTICE
                 ? rosen_lattice_grow_long(&q->lp, &q->lo, q->long_ws, q->long_bytes, st_q)
                 : rosen_offlattice_grow_long(&q->op, &q->oo, q->long_ws, q->long_bytes, st_q);
    } else if (q->req.model == ROSEN_MODEL_LATTICE) {
        st = lattice_grow_range(&q->lp, &q->lo, c_lo, c_hi, st_q);
    } else {
        unsigned char *sc = static_cast<unsigned char *>(q->scratch);
        const size_t cb = offlattice_range_counter_bytes();
        st = offlattice_grow_range(&q->op, &q->oo, c_lo, c_hi, sc + lane * cb,
                                   reinterpret_cast<uint32_t *>(sc + 2 * cb), st_q);
    }
    if (sl.end) cudaEventRecord(sl.end, st_q);
    q->next_chain = c_hi;
    if (st != ROSEN_OK) {
        fail(q, st, rosen_last_error());
        q->next_chain = C;
    }
    if (sl.start && sl.end) {
        ++q->inflight;
        s->slices.push_back(sl);
    } else {
        if (sl.start) s->timing_events.push_back(sl.start);
        if (sl.end) s->timing_events.push_back(sl.end);
    }
    if (q->next_chain >= C) finish(q);
}

// The request whose slice goes next: the oldest (arrival order), or
// (shortest_first) the one with the least estimated remaining GPU time
// divided by 1 + its waiting time in seconds, alternating with the oldest
// overdue request while there is one (which goes first outright while
// requests wait for admission).  At most two slices of one request (one per
// stream) are enqueued at once.
Request *pick(rosen_server *s, int64_t now)
{
    Request *overdue = nullptr, *best = nullptr;
    double best_key = 0.0;
    for (Request *q : s->active) {
        if (q->finishing || q->inflight >= 2 || q->next_chain >= q->req.C) continue;
        if (!s->cfg.shortest_first) {
            if (!best || q->t_submit < best->t_submit) best = q;
            continue;
        }
        const double own = (double)q->req.C * q->ns_per_chain;
        if ((double)(now - q->t_admit) > (double)kStarveNs + kStarveOwn * own) {
            if (!overdue || q->t_submit < overdue->t_submit) overdue = q;
            continue;
        }
        const double rem = (double)(q->req.C - q->next_chain) * q->ns_per_chain;
        const double key = rem / (1.0 + (double)(now - q->t_submit) / kAgingNs);
        if (!best || key < best_key) {
            best = q;
            best_key = key;
        }
    }
    if (overdue && best) {
        if (!s->queue.empty()) return overdue;
        s->overdue_turn = !s->overdue_turn;
        return s->overdue_turn ? overdue : best;
    }
    return overdue ? overdue : best;
}

// Completed slices (oldest first): refine the GPU-time estimates.  A slice's
// own time is measured from the later of its start and the end of the slice
// completed before it, so the time it spent queued behind another slice is
// not counted.
bool reap_slices(rosen_server *s)
{
    bool progressed = false;
    for (size_t i = 0; i < s->slices.size();) {
        Slice &sl = s->slices[i];
        const cudaError_t e = cudaEventQuery(sl.end);
        if (e == cudaErrorNotReady) {
            ++i;
            continue;
        }
        Request *q = sl.q;
        if (e == cudaSuccess) {
            float ms = 0.f, since = -1.f;
            if (cudaEventElapsedTime(&ms, sl.start, sl.end) != cudaSuccess) ms = -1.f;
            if (s->last_end && cudaEventElapsedTime(&since, s->last_end, sl.end) != cudaSuccess)
                since = -1.f;
            cudaGetLastError();
            float own = ms;
            if (since >= 0.f && since < own) own = since;
            if (own > 0.f && sl.chains > 0) {
                const double per = (double)own * 1e6 / (double)sl.chains;
                q->ns_per_chain = 0.5 * q->ns_per_chain + 0.5 * per;
                // Only a slice of at least the chains the GPU grows at once
                // measures the class's rate: a smaller one takes about the
                // time of one chain whatever its size (and any wait for the
                // SMs, divided by few chains, would inflate the rate).
                if (sl.chains >= q->resident) {
                    const uint64_t key = rate_key(q->req);
                    auto it = s->rate.find(key);
                    s->rate[key] = it == s->rate.end() ? per : 0.8 * it->second + 0.2 * per;
                }
            }
            if (s->last_end) s->timing_events.push_back(s->last_end);
            s->last_end = sl.end;
            s->timing_events.push_back(sl.start);
        } else {
            cudaGetLastError();
            if (q->state != FAILED) fail(q, ROSEN_ECUDA, cudaGetErrorString(e));
            s->timing_events.push_back(sl.start);
            s->timing_events.push_back(sl.end);
        }
        --q->inflight;
        s->slices.erase(s->slices.begin() + (ptrdiff_t)i);
        progressed = true;
    }
    return progressed;
}

// Requests whose completion event has fired.
bool reap_requests(rosen_server *s)
{
    bool progressed = false;
    for (size_t i = 0; i < s->active.size();) {
        Request *q = s->active[i];
        if (!q->finishing || q->inflight > 0) {
            ++i;
            continue;
        }
        const cudaError_t e = cudaEventQuery(q->done);
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
                cudaGetLastError();
                fail(q, ROSEN_ECUDA, cudaGetErrorString(e));
            }
        }
        if (q->state == FAILED) {
            ++s->n_failed;
            // A failed request gives back everything it reserved.
            if (q->coords) cudaFreeAsync(q->coords, q->streams[0]);
            q->coords = nullptr;
            s->used -= q->coord_bytes;
        }
        s->used -= q->work_bytes;
        q->t_done = now_ns();
        retire(s, q);
        s->active[i] = s->active.back();
        s->active.pop_back();
        progressed = true;
    }
    return progressed;
}

// Admissions in arrival order; a request that does not fit the budget may be
// passed by later ones for at most kPassLimitNs, then nothing behind it is
// admitted until it fits.
bool admit_waiting(rosen_server *s, int64_t now)
{
    bool progressed = false;
    for (auto it = s->queue.begin();
         it != s->queue.end() && !s->stop && (int)s->active.size() < s->cfg.max_slots;) {
        Request *q = *it;
        if (q->state == CANCELLED) {
            it = s->queue.erase(it);
            q->in_queue = false;
            if (q->released) delete q;
            progressed = true;
            continue;
        }
        const size_t need = q->work_bytes + q->coord_bytes;
        if (s->used + need > s->cfg.mem_budget_bytes) {
            if (q->t_passed == 0) q->t_passed = now;
            if (now - q->t_passed > kPassLimitNs) break;
            ++it;
            continue;
        }
        if (!admit(s, q)) break;
        it = s->queue.erase(it);
        q->in_queue = false;
        progressed = true;
    }
    return progressed;
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
        progressed |= reap_slices(s);
        if (reap_requests(s)) {
            progressed = true;
            s->cv_done.notify_all();
        }
        const int64_t now = now_ns();
        if (admit_waiting(s, now)) {
            progressed = true;
            s->cv_done.notify_all();   // requests that failed at admission
        }
        // Slices: keep about kLookaheadNs of estimated work enqueued.
        double queued = 0.0;
        for (const Slice &sl : s->slices) queued += sl.est_ns;
        while ((int)s->slices.size() < kMaxInflight && queued < (double)kLookaheadNs) {
            Request *q = pick(s, now);
            if (!q) break;
            const size_t before = s->slices.size();
            launch_slice(s, q);
            if (s->slices.size() > before) queued += s->slices.back().est_ns;
            progressed = true;
        }
        if (s->stop && s->active.empty()) break;
        if (!progressed) {
            // Nothing to do right now: sleep until a submission arrives, or
            // briefly while work is on the GPU.
            if (s->active.empty())
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

void destroy_resources(rosen_server *s)
{
    if (s->free_stream) cudaStreamDestroy(s->free_stream);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->done_events) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->timing_events) cudaEventDestroy(ev);
    if (s->last_end) cudaEventDestroy(s->last_end);
    for (rosen_stats *h : s->pinned) cudaFreeHost(h);
    if (s->pool) cudaMemPoolDestroy(s->pool);
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
    props.maxSize = (size_t)cfg->pool_max_bytes;   // 0: no cap
    if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = cfg->mem_budget_bytes;   // keep freed blocks for reuse up to the budget
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) {
        // A block freed by a request whose stream still has work queued is not
        // handed to another request with a wait on that stream: the new
        // request would otherwise start only when the old one's queued slices
        // have run.  (Blocks whose frees have completed are still reused.)
        int no = 0;
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->free_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        destroy_resources(s);
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
    out->running = s->active.size();
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
    destroy_resources(s);
    delete s;
    return ROSEN_OK;
}
