// reduce.cu -- FP64 ensemble reduction of Rosenbluth-weighted observables
// (Guo & Baulin, Eq. 2 with W as the importance weight; Eq. 9 for Z_N).
//
// Rosenbluth weights span hundreds of orders of magnitude, so the sums are
// formed in FP64 relative to a running maximum (log-sum-exp).  The chains
// are cut into fixed tiles of kTile chains; one block reduces one tile to a
// partial (its max M_t and the sums scaled by exp(-M_t)), and a single block
// merges the partials.  Tiles, the in-tile order and the merge tree depend
// only on C, so the result is bit-for-bit deterministic.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace rosen {
namespace {

constexpr int kTile = 2048;
constexpr int kThreads = 256;
constexpr int kPerThread = kTile / kThreads;
constexpr int kFinalThreads = 256;

struct Partial {
    double M;          // max log W in the tile (-inf: no live chain)
    double s[8];       // S0 S1 S2 Q0 Q1a Q2a Q1b Q2b, scaled by exp(-M) / exp(-2M)
    double alive;
    double n;          // growths in the tile: chains, or their attempts (restart mode)
    double pad;
};

struct ReduceArgs {
    int32_t kind, N, k, use_counts;
    int64_t C;
    const float *logw;
    const uint4 *counts;
    const int32_t *r2_i;
    const int64_t *n2rg2;
    const float *r2_f;
    const float *rg2_f;
    const uint16_t *attempts;   // optional: growths per chain (restart mode)
    double logm[8];     // log(m) in FP64, m = 0..6
    double inv_n2;      // 1 / N^2
};

__device__ __forceinline__ void load_chain(const ReduceArgs &a, int64_t c, double &lw,
                                           double &A1, double &A2)
{
    if (a.kind == ROSEN_REDUCE_LATTICE) {
        if (a.use_counts) {
            const uint4 v = a.counts[c];
            if (v.x & 0xFFFFu) {
                lw = -INFINITY;
            } else {
                // log W = sum_m counts[m] log m, exact up to FP64 rounding.
                const uint32_t cm[7] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16,
                                        v.z & 0xFFFFu, v.z >> 16, v.w & 0xFFFFu};
                double s = 0.0;
#pragma unroll
                for (int q = 2; q <= 6; ++q) s = fma((double)cm[q], a.logm[q], s);
                lw = s;
            }
        } else {
            lw = (double)a.logw[c];
        }
        A1 = (double)a.r2_i[c];
        A2 = (double)a.n2rg2[c] * a.inv_n2;
    } else {
        lw = (double)a.logw[c];
        A1 = (double)a.r2_f[c];
        A2 = (double)a.rg2_f[c];
    }
}

// Merge partial b into a (same max-shift convention).  Host and device: the
// multi-GPU merge (rosen_stats_merge) uses the same arithmetic.
__host__ __device__ __forceinline__ void merge(double &Ma, double *sa, double &na, double Mb,
                                               const double *sb, double nb)
{
    const double M = fmax(Ma, Mb);
    if (M == -INFINITY) {
        na += nb;
        return;
    }
    const double fa = (Ma == -INFINITY) ? 0.0 : exp(Ma - M);
    const double fb = (Mb == -INFINITY) ? 0.0 : exp(Mb - M);
#pragma unroll
    for (int q = 0; q < 3; ++q) sa[q] = sa[q] * fa + sb[q] * fb;
#pragma unroll
    for (int q = 3; q < 8; ++q) sa[q] = sa[q] * (fa * fa) + sb[q] * (fb * fb);
    Ma = M;
    na += nb;
}

// The statistics of an ensemble from its merged sums: Eq. 9's log Z (mean
// weight over the n growths), Eq. 2's W-weighted means of R_ee^2 and R_g^2,
// their ratio standard errors sqrt(sum w^2 (A - mean)^2) / sum w, and the
// effective sample size (sum w)^2 / sum w^2.
__host__ __device__ __forceinline__ rosen_stats finish(double M, const double *S, double alive,
                                                       double n, int N, int k)
{
    rosen_stats r;
    r.n = n;
    r.n_alive = alive;
    r.log_max = M;
    r.S0 = S[0];
    r.S1 = S[1];
    r.S2 = S[2];
    r.Q0 = S[3];
    r.Q1_r2 = S[4];
    r.Q2_r2 = S[5];
    r.Q1_rg2 = S[6];
    r.Q2_rg2 = S[7];
    if (alive == 0.0) {
        r.logZ = -INFINITY;
        r.logZ_norm = -INFINITY;
        r.mean_r2 = r.se_r2 = r.mean_rg2 = r.se_rg2 = NAN;
        r.ess = 0.0;
    } else {
        r.logZ = r.log_max + log(r.S0 / r.n);
        r.logZ_norm = k > 0 ? r.logZ - (double)(N - 1) * log((double)k) : r.logZ;
        const double m1 = r.S1 / r.S0, m2 = r.S2 / r.S0;
        const double v1 = r.Q2_r2 - 2.0 * m1 * r.Q1_r2 + m1 * m1 * r.Q0;
        const double v2 = r.Q2_rg2 - 2.0 * m2 * r.Q1_rg2 + m2 * m2 * r.Q0;
        r.mean_r2 = m1;
        r.se_r2 = sqrt(v1 > 0.0 ? v1 : 0.0) / r.S0;
        r.mean_rg2 = m2;
        r.se_rg2 = sqrt(v2 > 0.0 ? v2 : 0.0) / r.S0;
        r.ess = r.S0 * r.S0 / r.Q0;
    }
    return r;
}

// Reduce tile `tile` of the ensemble a into *out (one block of kThreads).
__device__ __forceinline__ void reduce_tile(const ReduceArgs &a, int64_t tile, Partial *out)
{
    __shared__ double red[kThreads / 32][10];   // 9 sums + the growth count
    __shared__ double tileM;
    const int64_t c0 = tile * kTile;
    double lw[kPerThread], A1[kPerThread], A2[kPerThread];
    double m = -INFINITY;
    double growths = 0.0;   // Eq. 9's sample size: chains, or attempts in restart mode
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
        const int64_t c = c0 + threadIdx.x + (int64_t)q * kThreads;
        if (c < a.C) {
            load_chain(a, c, lw[q], A1[q], A2[q]);
            growths += a.attempts ? (double)a.attempts[c] : 1.0;
        } else {
            lw[q] = -INFINITY;
            A1[q] = A2[q] = 0.0;
        }
        m = fmax(m, lw[q]);
    }
    // Block maximum.
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp][0] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = -INFINITY;
        for (int w = 0; w < kThreads / 32; ++w) mm = fmax(mm, red[w][0]);
        tileM = mm;
    }
    __syncthreads();
    const double M = tileM;
    double s[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) s[q] = 0.0;
    if (M > -INFINITY) {
#pragma unroll
        for (int q = 0; q < kPerThread; ++q) {
            if (lw[q] == -INFINITY) continue;
            const double w = exp(lw[q] - M), w2 = w * w;
            s[0] += w;
            s[1] += w * A1[q];
            s[2] += w * A2[q];
            s[3] += w2;
            s[4] += w2 * A1[q];
            s[5] += w2 * A1[q] * A1[q];
            s[6] += w2 * A2[q];
            s[7] += w2 * A2[q] * A2[q];
            s[8] += 1.0;
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) growths += __shfl_xor_sync(0xffffffffu, growths, off);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) red[warp][q] = s[q];
        red[warp][9] = growths;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial P;
        P.M = M;
        for (int q = 0; q < 8; ++q) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w][q];
            P.s[q] = t;
        }
        double al = 0.0, ng = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            al += red[w][8];
            ng += red[w][9];
        }
        P.alive = al;
        P.n = ng;
        P.pad = 0.0;
        *out = P;
    }
}

__global__ void __launch_bounds__(kThreads) reduce_tiles_kernel(const ReduceArgs a, Partial *part)
{
    reduce_tile(a, blockIdx.x, &part[blockIdx.x]);
}

// Merge the ntiles partials of one ensemble in a fixed tree (one block).
__device__ __forceinline__ void reduce_final(const Partial *part, int64_t ntiles,
                                             const ReduceArgs &a, rosen_stats *out)
{
    __shared__ double sM[kFinalThreads], sS[kFinalThreads][8], sN[kFinalThreads];
    __shared__ double sG[kFinalThreads];
    double M = -INFINITY, S[8] = {0, 0, 0, 0, 0, 0, 0, 0}, na = 0.0, ng = 0.0;
    for (int64_t t = threadIdx.x; t < ntiles; t += kFinalThreads) {
        merge(M, S, na, part[t].M, part[t].s, part[t].alive);
        ng += part[t].n;
    }
    sM[threadIdx.x] = M;
    for (int q = 0; q < 8; ++q) sS[threadIdx.x][q] = S[q];
    sN[threadIdx.x] = na;
    sG[threadIdx.x] = ng;
    __syncthreads();
    for (int half = kFinalThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half) {
            double Mb = sM[threadIdx.x + half], Sb[8];
            for (int q = 0; q < 8; ++q) Sb[q] = sS[threadIdx.x + half][q];
            double Ma = sM[threadIdx.x], Sa[8], nA = sN[threadIdx.x];
            for (int q = 0; q < 8; ++q) Sa[q] = sS[threadIdx.x][q];
            merge(Ma, Sa, nA, Mb, Sb, sN[threadIdx.x + half]);
            sM[threadIdx.x] = Ma;
            for (int q = 0; q < 8; ++q) sS[threadIdx.x][q] = Sa[q];
            sN[threadIdx.x] = nA;
            sG[threadIdx.x] += sG[threadIdx.x + half];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    // The growth count is a sum of integer-valued partials: exact in FP64.
    *out = finish(sM[0], sS[0], sN[0], sG[0], a.N, a.k);
}

__global__ void __launch_bounds__(kFinalThreads) reduce_final_kernel(const Partial *part,
                                                                     int64_t ntiles,
                                                                     const ReduceArgs a,
                                                                     rosen_stats *out)
{
    reduce_final(part, ntiles, a, out);
}

// Batched: block b reduces global tile b; tile_off[e] .. tile_off[e+1]-1 are
// the tiles of ensemble e.
__global__ void __launch_bounds__(kThreads) reduce_tiles_batch_kernel(const ReduceArgs *args,
                                                                      const int64_t *tile_off,
                                                                      int n_ens, Partial *part)
{
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n_ens;            // largest e with tile_off[e] <= b
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (tile_off[mid] <= b) lo = mid;
        else hi = mid;
    }
    reduce_tile(args[lo], b - tile_off[lo], &part[b]);
}

__global__ void __launch_bounds__(kFinalThreads) reduce_final_batch_kernel(const Partial *part,
                                                                           const int64_t *tile_off,
                                                                           const ReduceArgs *args,
                                                                           rosen_stats *out)
{
    const int e = blockIdx.x;
    reduce_final(part + tile_off[e], tile_off[e + 1] - tile_off[e], args[e], out + e);
}

}  // namespace

// Shared with the other translation units that reduce on the device.
int64_t reduce_tiles(int64_t C) { return (C + kTile - 1) / kTile; }

size_t reduce_args_size() { return sizeof(ReduceArgs); }
size_t reduce_partial_bytes() { return sizeof(Partial); }

void reduce_make_args(const rosen_reduce_in *in, void *out)
{
    ReduceArgs a;
    memset(&a, 0, sizeof a);
    a.kind = in->kind;
    a.N = in->N;
    a.k = in->k;
    a.use_counts = in->use_counts;
    a.C = in->C;
    a.logw = in->logw;
    a.counts = reinterpret_cast<const uint4 *>(in->counts);
    a.r2_i = in->r2_i;
    a.n2rg2 = in->n2rg2;
    a.r2_f = in->r2_f;
    a.rg2_f = in->rg2_f;
    a.attempts = in->attempts;
    for (int q = 0; q < 8; ++q) a.logm[q] = q >= 1 ? log((double)q) : 0.0;
    a.inv_n2 = 1.0 / ((double)in->N * (double)in->N);
    memcpy(out, &a, sizeof a);
}

void reduce_batch_launch(const void *dev_args, const int64_t *dev_tile_off, int n_ens,
                         int64_t total_tiles, void *part, rosen_stats *out, cudaStream_t s)
{
    const ReduceArgs *args = reinterpret_cast<const ReduceArgs *>(dev_args);
    Partial *p = reinterpret_cast<Partial *>(part);
    reduce_tiles_batch_kernel<<<(unsigned)total_tiles, kThreads, 0, s>>>(args, dev_tile_off, n_ens, p);
    reduce_final_batch_kernel<<<n_ens, kFinalThreads, 0, s>>>(p, dev_tile_off, args, out);
}

int reduce_launch(const rosen_reduce_in *in, rosen_stats *out, void *part_ws, cudaStream_t s)
{
    ReduceArgs a;
    memset(&a, 0, sizeof a);
    a.kind = in->kind;
    a.N = in->N;
    a.k = in->k;
    a.use_counts = in->use_counts;
    a.C = in->C;
    a.logw = in->logw;
    a.counts = reinterpret_cast<const uint4 *>(in->counts);
    a.r2_i = in->r2_i;
    a.n2rg2 = in->n2rg2;
    a.r2_f = in->r2_f;
    a.rg2_f = in->rg2_f;
    a.attempts = in->attempts;
    for (int q = 0; q < 8; ++q) a.logm[q] = q >= 1 ? log((double)q) : 0.0;
    a.inv_n2 = 1.0 / ((double)in->N * (double)in->N);
    const int64_t tiles = reduce_tiles(in->C);
    Partial *part = reinterpret_cast<Partial *>(part_ws);
    reduce_tiles_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(a, part);
    reduce_final_kernel<<<1, kFinalThreads, 0, s>>>(part, tiles, a, out);
    return check_launch("rosen_reduce");
}

int reduce_validate(const rosen_reduce_in *in, const rosen_stats *out)
{
    if (!in || !out) return set_error(ROSEN_EINVAL, "rosen_reduce: NULL input or output");
    if (in->C < 1) return set_error(ROSEN_EINVAL, "rosen_reduce: C must be >= 1");
    if (in->N < 1) return set_error(ROSEN_EINVAL, "rosen_reduce: N must be >= 1");
    if (in->k < 0) return set_error(ROSEN_EINVAL, "rosen_reduce: k must be >= 0");
    if (in->kind == ROSEN_REDUCE_LATTICE) {
        if (in->use_counts ? !in->counts : !in->logw)
            return set_error(ROSEN_EINVAL, "rosen_reduce: missing counts/logw");
        if (in->use_counts && (reinterpret_cast<uintptr_t>(in->counts) & 15u))
            return set_error(ROSEN_EINVAL, "rosen_reduce: counts must be 16-byte aligned");
        if (!in->r2_i || !in->n2rg2)
            return set_error(ROSEN_EINVAL, "rosen_reduce: lattice needs r2_i and n2rg2");
    } else if (in->kind == ROSEN_REDUCE_OFFLATTICE) {
        if (!in->logw || !in->r2_f || !in->rg2_f)
            return set_error(ROSEN_EINVAL, "rosen_reduce: real space needs logw, r2_f, rg2_f");
    } else {
        return set_error(ROSEN_EINVAL, "rosen_reduce: unknown kind %d", in->kind);
    }
    return ROSEN_OK;
}

size_t reduce_workspace_bytes(int64_t C)
{
    return (size_t)reduce_tiles(C < 1 ? 1 : C) * sizeof(Partial);
}

}  // namespace rosen

// ---------------------------------------------------------------------------
// Allocation-free variant.  Its scratch (the per-tile partials) lives in a
// fixed array in this file; every GPU that loads the library holds it until
// the process exits.  In host code the array's name is only a stand-in, so
// the device address is looked up with cudaGetSymbolAddress, with the
// device current, on every call made outside stream capture.
// ---------------------------------------------------------------------------
namespace rosen {
namespace {

constexpr int64_t kNoallocTiles = ((int64_t)ROSEN_REDUCE_NOALLOC_MAX_CHAINS + kTile - 1) / kTile;
static __device__ __align__(256) Partial g_noalloc_partials[kNoallocTiles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// The device address of the scratch on the current device.  A call whose
// stream is not being captured looks it up again every time (cheap), so a
// module reloaded after cudaDeviceReset is followed; a call made while its
// stream is captured uses the address the last uncaptured call on this
// device found.
int noalloc_scratch(cudaStream_t s, void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_reduce_noalloc: cudaGetDevice: %s",
                         cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(ROSEN_EINVAL, "rosen_reduce_noalloc: device %d out of range", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_reduce_noalloc: cudaStreamIsCapturing: %s",
                         cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return set_error(ROSEN_ECUDA, "rosen_reduce_noalloc: cudaGetSymbolAddress: %s",
                             cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    } else if (!g_noalloc_addr[dev]) {
        return set_error(ROSEN_EINVAL, "rosen_reduce_noalloc: the first call on device %d must "
                                       "come before any stream capture", dev);
    }
    *out = g_noalloc_addr[dev];
    return ROSEN_OK;
}

}  // namespace
}  // namespace rosen

extern "C" int rosen_reduce_noalloc(const rosen_reduce_in *in, rosen_stats *out, void *stream)
{
    int st = rosen::reduce_validate(in, out);
    if (st != ROSEN_OK) return st;
    if (in->C > (int64_t)ROSEN_REDUCE_NOALLOC_MAX_CHAINS)
        return rosen::set_error(ROSEN_ENOMEM,
                                "rosen_reduce_noalloc: C = %lld exceeds the built-in scratch "
                                "limit of %d chains; use rosen_reduce with a workspace",
                                (long long)in->C, (int)ROSEN_REDUCE_NOALLOC_MAX_CHAINS);
    void *ws = nullptr;
    st = rosen::noalloc_scratch((cudaStream_t)stream, &ws);
    if (st != ROSEN_OK) return st;
    // Every partial the final merge reads is rewritten by this call's tile
    // kernel, so nothing in the shared scratch has to be cleared first.
    return rosen::reduce_launch(in, out, ws, (cudaStream_t)stream);
}

using namespace rosen;

extern "C" size_t rosen_reduce_workspace_size(int64_t C) { return reduce_workspace_bytes(C); }

extern "C" int rosen_reduce(const rosen_reduce_in *in, rosen_stats *out, void *workspace,
                            size_t workspace_bytes, void *stream)
{
    int st = reduce_validate(in, out);
    if (st != ROSEN_OK) return st;
    if (!workspace || workspace_bytes < reduce_workspace_bytes(in->C))
        return set_error(ROSEN_ENOMEM, "rosen_reduce: workspace of %zu bytes < %zu needed",
                         workspace_bytes, reduce_workspace_bytes(in->C));
    if (reinterpret_cast<uintptr_t>(workspace) & 15u)
        return set_error(ROSEN_EINVAL, "rosen_reduce: workspace must be 16-byte aligned");
    return reduce_launch(in, out, workspace, (cudaStream_t)stream);
}

extern "C" int rosen_stats_merge(const rosen_stats *parts, int32_t n, int32_t N, int32_t k,
                                 rosen_stats *out)
{
    if (!parts || !out || n < 1)
        return set_error(ROSEN_EINVAL, "rosen_stats_merge: NULL argument or n < 1");
    if (N < 1 || k < 0) return set_error(ROSEN_EINVAL, "rosen_stats_merge: N >= 1, k >= 0");
    double M = -INFINITY, S[8] = {0, 0, 0, 0, 0, 0, 0, 0}, alive = 0.0, growths = 0.0;
    for (int32_t p = 0; p < n; ++p) {
        const rosen_stats &b = parts[p];
        const double Sb[8] = {b.S0, b.S1, b.S2, b.Q0, b.Q1_r2, b.Q2_r2, b.Q1_rg2, b.Q2_rg2};
        merge(M, S, alive, b.n_alive > 0.0 ? b.log_max : -INFINITY, Sb, b.n_alive);
        growths += b.n;
    }
    *out = finish(M, S, alive, growths, N, k);
    return ROSEN_OK;
}
