// batch.cu -- many ensembles of uneven chain length and model in one graph
// launch.
//
// The ensembles of a batch are split into classes that share a kernel shape:
// lattice ensembles by chain-length bucket, real-space ensembles by potential,
// trial count and chain-length bucket.  Each class runs one persistent kernel
// whose blocks take (ensemble, chain range) items from a queue sorted by
// decreasing cost (N^2 k per chain), so long and short chains, large and small
// ensembles share the GPU without tail effects.  The shape of every class
// (lattice: chains per block; real space: lanes per chain) is picked by timing
// the candidates on a sample of the class.  A member with at least
// kOwnLaunchWaves times the chains its single-ensemble kernel grows at once
// fills the GPU by itself: it runs as that kernel's own launch (a persistent
// grid over its chains) on the class's stream, before the class kernel, and
// the class kernel serves the smaller members.  Growth of all classes (on
// forked streams, so they overlap) and the FP64 reduction of every ensemble
// are captured once into a CUDA graph; each run is one graph launch.
//
// Every chain is grown by the same device code as the single-ensemble entry
// points and every ensemble is reduced by the same tile and merge code as
// rosen_reduce.  Lattice ensembles are therefore identical, bit for bit, to
// growing and reducing them alone; real-space ensembles are identical bit for
// bit when grown alone with the lanes per chain the batch chose (the group
// sums of a few FP32 observables follow the lane layout), and otherwise take
// the same paths with observables within their FP32 rounding bounds.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

struct rosen_batch;

namespace rosen {
namespace {

// A member is grown by its own single-ensemble launch from this many waves of
// resident chains up.
constexpr int64_t kOwnLaunchWaves = 4;

struct ClassPlan {
    bool lattice;
    bool lj;
    std::vector<char> own;      // per member: grown by its own single-ensemble launch
    std::vector<size_t> own_off;   // real space: offset of its counters and mask in d_own
    void *d_own = nullptr;      // real space: scratch of the members with their own launch
    size_t own_bytes = 0;
    bool longc = false; // long chains: members grown one after another by the
                        // hash-table / cell-grid kernels in one class workspace
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    int k;            // real space: trials per step (max over the class)
    int Nmax;
    std::vector<int> members;   // ensemble indices
    // shape (after tuning)
    int B = 0;        // lattice: chains (= threads) per block
    int G = 0, T = 0; // real space: lanes per chain, trials per lane
    int cpb = 0;      // chains per block
    size_t smem = 0;
    int grid = 0;
    int n_items = 0;
    BatchItem *d_items = nullptr;
    void *d_args = nullptr;     // LatticeArgs[] or OffArgs[] of the members
    int *d_head = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    double tuned_ms_per_work = 0.0;
};

// Chain-length bucket of a class: a class's shared memory is sized for its
// longest chain, so buckets are narrow enough (32 monomers up to 256, then
// 128) that shorter members do not lose much occupancy.
int bucket_of(int N)
{
    if (N <= 256) return (N + 31) / 32 * 32;
    return (N + 127) / 128 * 128;
}

}  // namespace
}  // namespace rosen

using namespace rosen;

struct rosen_batch {
    std::vector<rosen_ensemble> ens;
    std::vector<ClassPlan> classes;
    std::vector<size_t> out_off;          // byte offset of each ensemble's outputs
    unsigned char *d_out = nullptr;       // per-chain outputs of every ensemble
    std::vector<rosen_lattice_out> lat_out;
    std::vector<rosen_offlattice_out> off_out;
    unsigned long long *d_counters = nullptr;   // [3], real-space diagnostics
    void *d_rargs = nullptr;              // ReduceArgs[n]
    int64_t *d_tile_off = nullptr;        // [n+1]
    int64_t total_tiles = 0;
    void *d_part = nullptr;
    rosen_stats *d_stats = nullptr;
    cudaStream_t s0 = nullptr;
    cudaEvent_t forked = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool tuned = false;
    int sms = 0;
    int device = -1;
};

namespace {

int cuda_fail(const char *what, cudaError_t e)
{
    return set_error(ROSEN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return cuda_fail(#call, _e);         \
    } while (0)

rosen_lattice_params lat_params(const rosen_ensemble &e)
{
    rosen_lattice_params p;
    memset(&p, 0, sizeof p);
    p.seed = e.seed;
    p.ensemble = e.ensemble;
    p.N = e.N;
    p.C = e.C;
    p.chain0 = 0;
    p.beta_eps = e.beta_eps;
    p.flags = 0;
    p.lanes_per_chain = 0;
    p.max_attempts = e.max_attempts;
    return p;
}

rosen_offlattice_params off_params(const rosen_ensemble &e, int lanes)
{
    rosen_offlattice_params p;
    memset(&p, 0, sizeof p);
    p.seed = e.seed;
    p.ensemble = e.ensemble;
    p.N = e.N;
    p.C = e.C;
    p.chain0 = 0;
    p.k = e.k;
    p.potential = e.potential;
    p.sigma = e.sigma;
    p.cutoff = e.cutoff;
    p.beta_eps = e.beta_eps;
    p.flags = 0;
    p.lanes_per_chain = lanes;
    p.max_attempts = e.max_attempts;
    return p;
}

double chain_cost(const rosen_ensemble &e)
{
    const double n = (double)e.N;
    return e.model == ROSEN_MODEL_LATTICE ? n * n : n * n * (double)e.k;
}

// Items of a class for chains [0, limit_e) of every member; sorted by cost.
std::vector<BatchItem> make_items(const rosen_batch *b, const ClassPlan &c, double fraction)
{
    std::vector<BatchItem> items;
    std::vector<double> cost;
    for (size_t m = 0; m < c.members.size(); ++m) {
        if (!c.own.empty() && c.own[m]) continue;
        const rosen_ensemble &e = b->ens[c.members[m]];
        int64_t limit = e.C;
        if (fraction < 1.0)
            limit = std::min<int64_t>(e.C, std::max<int64_t>(c.cpb, (int64_t)(e.C * fraction)));
        for (int64_t c0 = 0; c0 < limit; c0 += c.cpb) {
            BatchItem it;
            it.ens = (uint32_t)m;
            it.c0 = c0;
            it.n = (uint32_t)std::min<int64_t>(c.cpb, limit - c0);
            items.push_back(it);
            cost.push_back(chain_cost(e) * it.n);
        }
    }
    std::vector<size_t> order(items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<BatchItem> sorted(items.size());
    for (size_t q = 0; q < order.size(); ++q) sorted[q] = items[order[q]];
    return sorted;
}

int upload_args(rosen_batch *b, ClassPlan &c)
{
    const size_t sz = c.lattice ? lattice_args_size() : offlattice_args_size();
    std::vector<unsigned char> host(sz * c.members.size());
    for (size_t m = 0; m < c.members.size(); ++m) {
        const int e = c.members[m];
        if (c.lattice) {
            const rosen_lattice_params p = lat_params(b->ens[e]);
            lattice_make_args(&p, &b->lat_out[e], host.data() + m * sz);
        } else {
            const rosen_offlattice_params p = off_params(b->ens[e], c.G);
            offlattice_make_args(&p, &b->off_out[e], b->d_counters, host.data() + m * sz);
        }
    }
    if (c.d_args) cudaFree(c.d_args);
    CK(cudaMalloc(&c.d_args, host.size()));
    CK(cudaMemcpy(c.d_args, host.data(), host.size(), cudaMemcpyHostToDevice));
    return ROSEN_OK;
}

int shape_class(rosen_batch *b, ClassPlan &c)
{
    if (c.longc) return ROSEN_OK;
    int bps = 0;
    int st;
    if (c.lattice) {
        st = lattice_batch_prepare(c.B, c.Nmax, &c.smem, &bps);
        c.cpb = c.B;
    } else {
        c.T = (c.k + c.G - 1) / c.G;
        c.T = c.T <= 1 ? 1 : (c.T <= 2 ? 2 : 4);
        st = offlattice_batch_prepare(c.G, c.T, c.lj, c.Nmax, &c.cpb, &c.smem, &bps);
    }
    if (st != ROSEN_OK) return st;
    if (bps < 1) return set_error(ROSEN_ENOMEM, "batch class does not fit on an SM");
    c.grid = b->sms * bps;
    return upload_args(b, c);
}

int upload_items(ClassPlan &c, const std::vector<BatchItem> &items)
{
    // Real-space classes hand out chains by a 32-bit ticket counter.
    if (!c.lattice && (uint64_t)items.size() * (uint64_t)c.cpb >= (uint64_t(1) << 31))
        return set_error(ROSEN_EINVAL, "rosen_batch: a real-space class of more than 2^31 chains; "
                                       "split the ensembles over several batches");
    if (c.d_items) cudaFree(c.d_items);
    c.d_items = nullptr;
    c.n_items = (int)items.size();
    if (items.empty()) return ROSEN_OK;
    CK(cudaMalloc(&c.d_items, items.size() * sizeof(BatchItem)));
    CK(cudaMemcpy(c.d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    return ROSEN_OK;
}

// Members with their own launch, largest first, through the single-ensemble
// range launches (default lanes per chain, as rosen_*_grow would grow them).
int launch_own(const rosen_batch *b, const ClassPlan &c, cudaStream_t s)
{
    if (c.d_own && cudaMemsetAsync(c.d_own, 0, c.own_bytes, s) != cudaSuccess)
        return set_error(ROSEN_ECUDA, "batch: clearing the members' scratch");
    for (size_t m = 0; m < c.members.size(); ++m) {
        if (!c.own[m]) continue;
        const int e = c.members[m];
        int st;
        if (c.lattice) {
            const rosen_lattice_params p = lat_params(b->ens[e]);
            st = lattice_grow_range(&p, &b->lat_out[e], 0, p.C, s);
        } else {
            const rosen_offlattice_params p = off_params(b->ens[e], 0);
            unsigned char *sc = static_cast<unsigned char *>(c.d_own) + c.own_off[m];
            st = offlattice_grow_range(&p, &b->off_out[e], 0, p.C, sc,
                                       reinterpret_cast<uint32_t *>(
                                           sc + offlattice_range_counter_bytes()),
                                       s);
        }
        if (st != ROSEN_OK) return st;
    }
    return ROSEN_OK;
}

int launch_class(const rosen_batch *b, const ClassPlan &c, cudaStream_t s, bool shared_only = false)
{
    if (!c.longc && !shared_only) {
        const int st = launch_own(b, c, s);
        if (st != ROSEN_OK) return st;
    }
    if (c.longc) {
        for (int e : c.members) {
            int st;
            if (c.lattice) {
                const rosen_lattice_params p = lat_params(b->ens[e]);
                st = rosen_lattice_grow_long(&p, &b->lat_out[e], c.d_ws, c.ws_bytes, s);
            } else {
                const rosen_offlattice_params p = off_params(b->ens[e], 0);
                st = rosen_offlattice_grow_long(&p, &b->off_out[e], c.d_ws, c.ws_bytes, s);
            }
            if (st != ROSEN_OK) return st;
        }
        return ROSEN_OK;
    }
    if (c.n_items == 0) return ROSEN_OK;
    if (c.lattice)
        lattice_batch_launch(c.d_args, c.d_items, c.n_items, c.d_head, c.B, c.smem, c.grid, s);
    else
        offlattice_batch_launch(c.G, c.T, c.lj, c.d_args, c.d_items, c.n_items, c.d_head, c.cpb,
                                c.Nmax, c.smem, c.grid, s);
    return ROSEN_OK;
}

// Time every candidate shape of a class on a sample of its chains and keep
// the fastest per unit of work.
int tune_class(rosen_batch *b, ClassPlan &c)
{
    if (make_items(b, c, 1.0).empty()) return ROSEN_OK;   // every member has its own launch
    std::vector<int> cands;
    if (c.lattice) {
        for (int B : {64, 128, 256})
            if (lattice_smem_bytes(c.Nmax, B) <= 200 * 1024) cands.push_back(B);
    } else {
        for (int G : {8, 16, 32})
            if ((c.k + G - 1) / G <= 4) cands.push_back(G);
    }
    // The untuned default shape is kept unless another is clearly faster on
    // the sample (which, for small classes, holds few chains per group).
    int def = 0;
    if (c.lattice) {
        def = 128;
        while (def > 32 && lattice_smem_bytes(c.Nmax, def) > 200 * 1024) def /= 2;
    } else {
        def = offlattice_default_lanes(c.k, c.lj, c.Nmax);
    }
    double best = 1e300, def_per = 1e300;
    int best_cand = cands.empty() ? 0 : cands[0];
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double work = 0.0;
    for (int cand : cands) {
        if (c.lattice) c.B = cand;
        else c.G = cand;
        int st = shape_class(b, c);
        if (st != ROSEN_OK) continue;
        const std::vector<BatchItem> items = make_items(b, c, 1.0 / 16.0);
        work = 0.0;
        for (const BatchItem &it : items) work += chain_cost(b->ens[c.members[it.ens]]) * it.n;
        st = upload_items(c, items);
        if (st != ROSEN_OK) return st;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaMemsetAsync(c.d_head, 0, sizeof(int), b->s0));
            CK(cudaEventRecord(e0, b->s0));
            launch_class(b, c, b->s0, true);
            CK(cudaEventRecord(e1, b->s0));
            CK(cudaStreamSynchronize(b->s0));
            CK(cudaGetLastError());
            CK(cudaEventElapsedTime(&ms, e0, e1));
        }
        const double per = ms / std::max(work, 1.0);
        if (cand == def) def_per = per;
        if (per < best) {
            best = per;
            best_cand = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (def_per < 1e300 && best > 0.9 * def_per) {
        best_cand = def;
        best = def_per;
    }
    if (c.lattice) c.B = best_cand;
    else c.G = best_cand;
    c.tuned_ms_per_work = best;
    int st = shape_class(b, c);
    if (st != ROSEN_OK) return st;
    return upload_items(c, make_items(b, c, 1.0));
}

int capture(rosen_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal));
    // The first failure inside the capture is kept to report it by name.
    const char *what = nullptr;
    cudaError_t first = cudaSuccess;
    auto note = [&](cudaError_t r, const char *w) {
        if (r != cudaSuccess && first == cudaSuccess) {
            first = r;
            what = w;
        }
    };
    for (ClassPlan &c : b->classes) note(cudaMemsetAsync(c.d_head, 0, sizeof(int), b->s0), "memset");
    note(cudaEventRecord(b->forked, b->s0), "fork");
    for (ClassPlan &c : b->classes) {
        note(cudaStreamWaitEvent(c.stream, b->forked, 0), "wait fork");
        if (launch_class(b, c, c.stream) != ROSEN_OK && first == cudaSuccess) {
            first = cudaErrorLaunchFailure;
            what = "long-chain class launch";
        }
        note(cudaGetLastError(), c.lattice ? "lattice class launch" : "real-space class launch");
        note(cudaEventRecord(c.done, c.stream), "record join");
        note(cudaStreamWaitEvent(b->s0, c.done, 0), "join");
    }
    reduce_batch_launch(b->d_rargs, b->d_tile_off, (int)b->ens.size(), b->total_tiles, b->d_part,
                        b->d_stats, b->s0);
    note(cudaGetLastError(), "reduction launch");
    cudaError_t e = cudaStreamEndCapture(b->s0, &g);
    if (first != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(what, first);
    }
    if (e != cudaSuccess) return cuda_fail("cudaStreamEndCapture", e);
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail("cudaGraphInstantiate", e);
    return ROSEN_OK;
}

// Members longer than the shared-memory kernels take go to long classes.
bool is_long(const rosen_ensemble &e)
{
    return e.model == ROSEN_MODEL_LATTICE ? e.N > ROSEN_LATTICE_NMAX : e.N > ROSEN_OFFLATTICE_NMAX;
}

int validate_ensemble(const rosen_ensemble &e, int idx)
{
    if (e.model == ROSEN_MODEL_LATTICE) {
        const rosen_lattice_params p = lat_params(e);
        rosen_lattice_out o;
        memset(&o, 0, sizeof o);
        const int st = lattice_validate(&p, &o, ROSEN_LATTICE_LONG_NMAX);
        if (st != ROSEN_OK) return set_error(st, "ensemble %d: %s", idx, rosen_last_error());
    } else if (e.model == ROSEN_MODEL_OFFLATTICE) {
        const rosen_offlattice_params p = off_params(e, 0);
        rosen_offlattice_out o;
        memset(&o, 0, sizeof o);
        const int st = offlattice_validate(&p, &o, ROSEN_OFFLATTICE_LONG_NMAX);
        if (st != ROSEN_OK) return set_error(st, "ensemble %d: %s", idx, rosen_last_error());
    } else {
        return set_error(ROSEN_EINVAL, "ensemble %d: unknown model %d", idx, e.model);
    }
    if (e.C < 1) return set_error(ROSEN_EINVAL, "ensemble %d: C must be >= 1", idx);
    return ROSEN_OK;
}

void free_batch(rosen_batch *b)
{
    for (ClassPlan &c : b->classes) {
        if (c.d_items) cudaFree(c.d_items);
        if (c.d_args) cudaFree(c.d_args);
        if (c.d_head) cudaFree(c.d_head);
        if (c.d_ws) cudaFree(c.d_ws);
        if (c.d_own) cudaFree(c.d_own);
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_out) cudaFree(b->d_out);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->d_rargs) cudaFree(b->d_rargs);
    if (b->d_tile_off) cudaFree(b->d_tile_off);
    if (b->d_part) cudaFree(b->d_part);
    if (b->d_stats) cudaFree(b->d_stats);
    if (b->s0) cudaStreamDestroy(b->s0);
    if (b->forked) cudaEventDestroy(b->forked);
    delete b;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int create(rosen_batch *b, const rosen_ensemble *ens, int n)
{
    b->ens.assign(ens, ens + n);
    CK(cudaGetDevice(&b->device));
    CK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
    CK(cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming));

    // Per-chain outputs, one packed allocation.
    size_t total = 0;
    b->out_off.resize(n);
    for (int e = 0; e < n; ++e) {
        b->out_off[e] = total;
        const size_t C = (size_t)ens[e].C;
        if (ens[e].model == ROSEN_MODEL_LATTICE)
            total += align256(16 * C) + align256(4 * C) + align256(4 * C) + align256(8 * C);
        else
            total += align256(4 * C) * 3 + align256(C);
        if (ens[e].max_attempts > 1) total += align256(2 * C);   // attempts (restart mode)
    }
    CK(cudaMalloc(&b->d_out, std::max<size_t>(total, 256)));
    CK(cudaMalloc(&b->d_counters, 3 * sizeof(unsigned long long)));
    CK(cudaMemset(b->d_counters, 0, 3 * sizeof(unsigned long long)));
    b->lat_out.assign(n, rosen_lattice_out());
    b->off_out.assign(n, rosen_offlattice_out());
    std::vector<unsigned char> rargs(reduce_args_size() * n);
    std::vector<int64_t> tile_off(n + 1, 0);
    for (int e = 0; e < n; ++e) {
        unsigned char *p = b->d_out + b->out_off[e];
        const size_t C = (size_t)ens[e].C;
        rosen_reduce_in in;
        memset(&in, 0, sizeof in);
        in.N = ens[e].N;
        in.C = ens[e].C;
        if (ens[e].model == ROSEN_MODEL_LATTICE) {
            rosen_lattice_out &o = b->lat_out[e];
            memset(&o, 0, sizeof o);
            o.counts = reinterpret_cast<uint16_t *>(p);
            p += align256(16 * C);
            o.logw = reinterpret_cast<float *>(p);
            p += align256(4 * C);
            o.r2 = reinterpret_cast<int32_t *>(p);
            p += align256(4 * C);
            o.n2rg2 = reinterpret_cast<int64_t *>(p);
            p += align256(8 * C);
            if (ens[e].max_attempts > 1) o.attempts = reinterpret_cast<uint16_t *>(p);
            in.attempts = o.attempts;
            in.kind = ROSEN_REDUCE_LATTICE;
            in.use_counts = ens[e].beta_eps == 0.0;
            in.logw = o.logw;
            in.counts = o.counts;
            in.r2_i = o.r2;
            in.n2rg2 = o.n2rg2;
        } else {
            rosen_offlattice_out &o = b->off_out[e];
            memset(&o, 0, sizeof o);
            o.logw = reinterpret_cast<float *>(p);
            p += align256(4 * C);
            o.r2 = reinterpret_cast<float *>(p);
            p += align256(4 * C);
            o.rg2 = reinterpret_cast<float *>(p);
            p += align256(4 * C);
            o.alive = p;
            p += align256(C);
            if (ens[e].max_attempts > 1) o.attempts = reinterpret_cast<uint16_t *>(p);
            in.attempts = o.attempts;
            in.kind = ROSEN_REDUCE_OFFLATTICE;
            in.k = ens[e].k;
            in.logw = o.logw;
            in.r2_f = o.r2;
            in.rg2_f = o.rg2;
        }
        reduce_make_args(&in, rargs.data() + e * reduce_args_size());
        tile_off[e + 1] = tile_off[e] + reduce_tiles(ens[e].C);
    }
    b->total_tiles = tile_off[n];
    CK(cudaMalloc(&b->d_rargs, rargs.size()));
    CK(cudaMemcpy(b->d_rargs, rargs.data(), rargs.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&b->d_tile_off, sizeof(int64_t) * (n + 1)));
    CK(cudaMemcpy(b->d_tile_off, tile_off.data(), sizeof(int64_t) * (n + 1),
                  cudaMemcpyHostToDevice));
    CK(cudaMalloc(&b->d_part, reduce_partial_bytes() * std::max<int64_t>(b->total_tiles, 1)));
    CK(cudaMalloc(&b->d_stats, sizeof(rosen_stats) * n));

    // Classes.
    for (int e = 0; e < n; ++e) {
        const rosen_ensemble &x = ens[e];
        const bool lat = x.model == ROSEN_MODEL_LATTICE;
        const bool lj = !lat && x.potential == ROSEN_LJ;
        const bool lg = is_long(x);
        const int bk = lg ? -1 : bucket_of(x.N);
        ClassPlan *found = nullptr;
        for (ClassPlan &c : b->classes)
            if (c.lattice == lat && c.lj == lj && (lat || c.k == x.k) && c.longc == lg &&
                (lg || bucket_of(c.Nmax) == bk))
                found = &c;
        if (!found) {
            b->classes.push_back(ClassPlan());
            found = &b->classes.back();
            found->lattice = lat;
            found->lj = lj;
            found->longc = lg;
            found->k = lat ? 0 : x.k;
            found->Nmax = 0;
        }
        found->members.push_back(e);
        found->Nmax = std::max(found->Nmax, x.N);
    }
    for (ClassPlan &c : b->classes) {
        CK(cudaMalloc(&c.d_head, sizeof(int)));
        CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
        if (c.longc) {
            // One workspace for the members in turn: the largest default size
            // among them, at most 8 GiB (fewer chains in flight, same results),
            // at least one table or chain slot of the longest member.
            size_t want = 0, least = 0;
            for (int e : c.members) {
                const rosen_ensemble &x = b->ens[e];
                const size_t w = c.lattice ? rosen_lattice_long_workspace_size(x.N, x.C)
                                           : rosen_offlattice_long_workspace_size(x.N, x.C);
                const size_t one = c.lattice ? rosen_lattice_long_workspace_size(x.N, 1)
                                             : rosen_offlattice_long_workspace_size(x.N, 1);
                want = std::max(want, w);
                least = std::max(least, one);
            }
            c.ws_bytes = std::max(least, std::min(want, (size_t)8 << 30));
            CK(cudaMalloc(&c.d_ws, c.ws_bytes));
            continue;
        }
        // Members that fill the GPU by themselves get their own launch
        // (real space: with their own chain counters and deferral mask).
        c.own.assign(c.members.size(), 0);
        c.own_off.assign(c.members.size(), 0);
        for (size_t m = 0; m < c.members.size(); ++m) {
            const rosen_ensemble &x = b->ens[c.members[m]];
            int64_t res;
            if (c.lattice) {
                const rosen_lattice_params p = lat_params(x);
                res = lattice_resident_chains(&p);
            } else {
                const rosen_offlattice_params p = off_params(x, 0);
                res = offlattice_resident_chains(&p);
            }
            if (res > 0 && x.C >= kOwnLaunchWaves * res) {
                c.own[m] = 1;
                if (!c.lattice) {
                    c.own_off[m] = c.own_bytes;
                    c.own_bytes += align256(offlattice_range_counter_bytes() +
                                            offlattice_range_mask_bytes(x.C));
                }
            }
        }
        if (c.own_bytes) CK(cudaMalloc(&c.d_own, c.own_bytes));
        // Untuned default shape: 128 chains per block (fewer if the keys of
        // the longest chain would not fit), or the default lanes per chain.
        if (c.lattice) {
            c.B = 128;
            while (c.B > 32 && lattice_smem_bytes(c.Nmax, c.B) > 200 * 1024) c.B /= 2;
        } else {
            c.G = offlattice_default_lanes(c.k, c.lj, c.Nmax);
        }
        int st = shape_class(b, c);
        if (st != ROSEN_OK) return st;
        st = upload_items(c, make_items(b, c, 1.0));
        if (st != ROSEN_OK) return st;
    }
    return ROSEN_OK;
}

}  // namespace

extern "C" int rosen_batch_create(const rosen_ensemble *ens, int32_t n, rosen_batch **out)
{
    if (!ens || !out || n < 1) return set_error(ROSEN_EINVAL, "rosen_batch_create: bad arguments");
    for (int e = 0; e < n; ++e) {
        const int st = validate_ensemble(ens[e], e);
        if (st != ROSEN_OK) return st;
    }
    rosen_batch *b = new rosen_batch();
    const int st = create(b, ens, n);
    if (st != ROSEN_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return ROSEN_OK;
}

extern "C" int rosen_batch_tune(rosen_batch *b, void *stream)
{
    (void)stream;
    if (!b) return set_error(ROSEN_EINVAL, "rosen_batch_tune: NULL batch");
    for (ClassPlan &c : b->classes) {
        if (c.longc) continue;       // nothing to choose: fixed kernels
        const int st = tune_class(b, c);
        if (st != ROSEN_OK) return st;
    }
    b->tuned = true;
    return capture(b);
}

extern "C" int rosen_batch_run(rosen_batch *b, void *stream)
{
    if (!b) return set_error(ROSEN_EINVAL, "rosen_batch_run: NULL batch");
    if (!b->exec) {
        const int st = b->tuned ? capture(b) : rosen_batch_tune(b, stream);
        if (st != ROSEN_OK) return st;
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail("cudaGraphLaunch", e);
    return ROSEN_OK;
}

extern "C" int rosen_batch_stats(rosen_batch *b, rosen_stats **stats)
{
    if (!b || !stats) return set_error(ROSEN_EINVAL, "rosen_batch_stats: NULL argument");
    *stats = b->d_stats;
    return ROSEN_OK;
}

extern "C" int rosen_batch_lattice_outputs(rosen_batch *b, int32_t e, rosen_lattice_out *out)
{
    if (!b || !out || e < 0 || e >= (int)b->ens.size() || b->ens[e].model != ROSEN_MODEL_LATTICE)
        return set_error(ROSEN_EINVAL, "rosen_batch_lattice_outputs: bad ensemble %d", e);
    *out = b->lat_out[e];
    return ROSEN_OK;
}

extern "C" int rosen_batch_offlattice_outputs(rosen_batch *b, int32_t e, rosen_offlattice_out *out)
{
    if (!b || !out || e < 0 || e >= (int)b->ens.size() ||
        b->ens[e].model != ROSEN_MODEL_OFFLATTICE)
        return set_error(ROSEN_EINVAL, "rosen_batch_offlattice_outputs: bad ensemble %d", e);
    *out = b->off_out[e];
    return ROSEN_OK;
}

extern "C" int rosen_batch_describe(rosen_batch *b, char *buf, size_t len)
{
    if (!b || !buf || len == 0) return set_error(ROSEN_EINVAL, "rosen_batch_describe: bad arguments");
    std::string s = "[";
    for (size_t q = 0; q < b->classes.size(); ++q) {
        const ClassPlan &c = b->classes[q];
        char line[448];
        snprintf(line, sizeof line,
                 "%s{\"model\":\"%s\",\"k\":%d,\"Nmax\":%d,\"ensembles\":%zu,\"items\":%d,"
                 "\"threads\":%d,\"lanes_per_chain\":%d,\"chains_per_block\":%d,\"grid\":%d,"
                 "\"smem\":%zu,\"long\":%s,\"workspace\":%zu,\"tuned\":%s,\"members\":[",
                 q ? "," : "", c.lattice ? "lattice" : (c.lj ? "lj" : "hard_sphere"), c.k, c.Nmax,
                 c.members.size(), c.n_items, c.lattice ? c.B : c.cpb * c.G, c.lattice ? 1 : c.G,
                 c.cpb, c.grid, c.smem, c.longc ? "true" : "false", c.ws_bytes,
                 b->tuned ? "true" : "false");
        s += line;
        for (size_t m = 0; m < c.members.size(); ++m)
            s += (m ? "," : "") + std::to_string(c.members[m]);
        // Lanes per chain each member is grown with: the class's, or (own
        // launch) the single-ensemble default.
        s += "],\"own_launch\":[";
        for (size_t m = 0; m < c.members.size(); ++m)
            s += std::string(m ? "," : "") + ((!c.own.empty() && c.own[m]) ? "1" : "0");
        s += "],\"member_lanes\":[";
        for (size_t m = 0; m < c.members.size(); ++m) {
            const rosen_ensemble &x = b->ens[c.members[m]];
            int lanes = c.lattice ? 1 : c.G;
            if (!c.lattice && !c.own.empty() && c.own[m])
                lanes = offlattice_default_lanes(x.k, x.potential == ROSEN_LJ, x.N);
            if (c.longc) lanes = 0;      // the long-chain kernel's own default
            s += (m ? "," : "") + std::to_string(lanes);
        }
        s += "]}";
    }
    s += "]";
    snprintf(buf, len, "%s", s.c_str());
    return ROSEN_OK;
}

extern "C" int rosen_batch_destroy(rosen_batch *b)
{
    if (!b) return ROSEN_OK;
    free_batch(b);
    return ROSEN_OK;
}

extern "C" int rosen_batch_copy_stats(rosen_batch *b, rosen_stats *dst, void *stream)
{
    if (!b || !dst) return set_error(ROSEN_EINVAL, "rosen_batch_copy_stats: NULL argument");
    const cudaError_t e = cudaMemcpyAsync(dst, b->d_stats, sizeof(rosen_stats) * b->ens.size(),
                                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? ROSEN_OK : cuda_fail("rosen_batch_copy_stats", e);
}

extern "C" int rosen_batch_copy_lattice(rosen_batch *b, int32_t e, const rosen_lattice_out *dst,
                                        void *stream)
{
    rosen_lattice_out src;
    int st = rosen_batch_lattice_outputs(b, e, &src);
    if (st != ROSEN_OK) return st;
    if (!dst) return set_error(ROSEN_EINVAL, "rosen_batch_copy_lattice: NULL destination");
    const size_t C = (size_t)b->ens[e].C;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t r = cudaSuccess;
    if (dst->counts && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->counts, src.counts, 16 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->logw && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->logw, src.logw, 4 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->r2 && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->r2, src.r2, 4 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->n2rg2 && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->n2rg2, src.n2rg2, 8 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->attempts && src.attempts && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->attempts, src.attempts, 2 * C, cudaMemcpyDeviceToDevice, s);
    return r == cudaSuccess ? ROSEN_OK : cuda_fail("rosen_batch_copy_lattice", r);
}

extern "C" int rosen_batch_copy_offlattice(rosen_batch *b, int32_t e, const rosen_offlattice_out *dst,
                                           void *stream)
{
    rosen_offlattice_out src;
    int st = rosen_batch_offlattice_outputs(b, e, &src);
    if (st != ROSEN_OK) return st;
    if (!dst) return set_error(ROSEN_EINVAL, "rosen_batch_copy_offlattice: NULL destination");
    const size_t C = (size_t)b->ens[e].C;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t r = cudaSuccess;
    if (dst->logw && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->logw, src.logw, 4 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->r2 && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->r2, src.r2, 4 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->rg2 && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->rg2, src.rg2, 4 * C, cudaMemcpyDeviceToDevice, s);
    if (dst->alive && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->alive, src.alive, C, cudaMemcpyDeviceToDevice, s);
    if (dst->attempts && src.attempts && r == cudaSuccess)
        r = cudaMemcpyAsync(dst->attempts, src.attempts, 2 * C, cudaMemcpyDeviceToDevice, s);
    return r == cudaSuccess ? ROSEN_OK : cuda_fail("rosen_batch_copy_offlattice", r);
}

extern "C" int rosen_batch_counters(rosen_batch *b, uint64_t *dst, void *stream)
{
    if (!b || !dst) return set_error(ROSEN_EINVAL, "rosen_batch_counters: NULL argument");
    const cudaError_t e = cudaMemcpyAsync(dst, b->d_counters, 3 * sizeof(unsigned long long),
                                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? ROSEN_OK : cuda_fail("rosen_batch_counters", e);
}
