// offlattice.cu -- Rosenbluth growth in real space (Guo & Baulin, Section
// 3.3.3, Algorithm 2): k trial positions on the unit sphere around the chain
// end, scored against every earlier non-bonded bead by hard-sphere overlap or
// a truncated Lennard-Jones energy; W is multiplied by the sum of the trial
// weights and one trial is drawn in proportion to its weight.
//
// GB300 mapping: a group of G lanes (G = 8, 16 or 32) grows one chain, so a
// warp holds 32/G chains; each lane owns T = ceil(k/G) trials.  Each step:
//  1. the group scans the earlier beads G at a time and keeps, in ballot
//     order (ascending bead index), those within 1 + R of the end (R = sigma
//     or the cutoff); only those can reach a trial.  The kept displacement
//     g = end - r_j and c = 1 + |g|^2 go to a shared list;
//  2. every lane draws its trial directions u (Philox, 24-bit uniforms; one
//     call gives two trials) and evaluates d^2 = |g + u|^2 = c + 2 g.u against
//     the list (three FMAs per pair, entries broadcast from shared memory);
//  3. free flags / weights are combined with group ballots and scans, and the
//     selection draw picks the trial.
// Positions are float-float (hi + lo) sums of the FP32 directions, so they
// carry only the directions' own rounding.  Every FP32 decision comes with a
// bound on its distance from the FP64 result (d^2 within G_i of sigma^2 or of
// the cutoff, or the selection draw within E of a prefix-sum boundary); when
// the bound is not met the group replays the chain's positions in FP64 from
// its chosen trials, stores them back (so later steps start from exact
// positions), and re-decides the step with the sequential FP64 arithmetic of
// the definition.  The grown path is the one an FP64 implementation takes.
//
// Scheduling: the grid is what the GPU holds at once, and every group takes
// its next chain from a counter (chains differ in cost by their re-decisions
// and dead ends).  Short hard-sphere chains grow in two passes, the second
// regrowing, with the FP64 path, the few chains the first could not decide.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "internal.cuh"
#include "offlattice_chain.cuh"

namespace rosen {
namespace {


template <int G, int T, bool LJ>
__global__ void __launch_bounds__(256, 4) offlattice_group_kernel(const OffArgs a, int chains_per_block)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *logm = reinterpret_cast<float *>(smem_raw);
    fill_log_table(logm);
    __syncthreads();

    const Group<G> g;
    const int cib = threadIdx.x / G;
    const int64_t c = (int64_t)blockIdx.x * chains_per_block + cib;
    if (c >= a.C) return;     // whole groups leave together
    const ChainSmem w = carve(smem_raw + kTable * sizeof(float) +
                                  (size_t)cib * chain_smem_bytes(a.N, LJ), a.N, LJ);
    off_chain<G, T, LJ>(a, c, w, g, logm);
}

// The same growth with chains handed out one at a time: every group takes
// its next chain from a counter as soon as it is done with the last, so a
// block holds no lanes idle while its slowest chain finishes (chains differ
// in their number of FP64 re-decisions and dead ends).  The grid is what the
// GPU holds at once.
template <int G, int T, bool LJ, bool kDefer = false>
__global__ void __launch_bounds__(256, 4) offlattice_queue_kernel(const OffArgs a,
                                                                  int chains_per_block,
                                                                  unsigned long long *next,
                                                                  int64_t c_lo, int64_t c_hi)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *logm = reinterpret_cast<float *>(smem_raw);
    fill_log_table(logm);
    __syncthreads();

    const Group<G> g;
    const int cib = threadIdx.x / G;
    const ChainSmem w = carve(smem_raw + kTable * sizeof(float) +
                                  (size_t)cib * chain_smem_bytes(a.N, LJ), a.N, LJ);
    for (;;) {
        unsigned long long c = 0;
        if (g.gl == 0) c = (unsigned long long)c_lo + atomicAdd(next, 1ull);
        c = g.bcast(c, 0);
        if (c >= (unsigned long long)c_hi) break;
        off_chain<G, T, LJ, ChainSmem, kDefer>(a, (int64_t)c, w, g, logm);
    }
}

// Second pass of two-pass growth: the chains of [c_lo, c_hi) whose bits the
// first pass set, grown again from the start with the FP64 re-decision
// compiled in.  Warps take 32-chain words of the bit mask from a counter, so
// the few deferred chains spread evenly; the groups of a warp take a word's
// set bits together, one each per round, so they step in lock-step as in
// the first pass instead of diverging.
template <int G, int T, bool LJ>
__global__ void __launch_bounds__(256, 4) offlattice_deferred_kernel(const OffArgs a,
                                                                     int chains_per_block,
                                                                     unsigned int *next,
                                                                     int64_t c_lo, int64_t c_hi)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *logm = reinterpret_cast<float *>(smem_raw);
    fill_log_table(logm);
    __syncthreads();

    const Group<G> g;
    const int cib = threadIdx.x / G;
    const ChainSmem w = carve(smem_raw + kTable * sizeof(float) +
                                  (size_t)cib * chain_smem_bytes(a.N, LJ), a.N, LJ);
    const int64_t w_lo = c_lo / 32, w_hi = (c_hi + 31) / 32;
    const int gw = (threadIdx.x & 31) / G;     // this group's place in its warp
    for (;;) {
        int64_t q = 0;
        if ((threadIdx.x & 31) == 0) q = w_lo + (int64_t)atomicAdd(next, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= w_hi) break;
        // Only the chains of this range (the words at its ends may hold
        // chains of neighbouring ranges).
        const int64_t b0 = q * 32;
        uint32_t m = a.deferred[q];
        if (b0 < c_lo) m &= ~0u << (uint32_t)(c_lo - b0);
        if (b0 + 32 > c_hi) m &= (c_hi - b0 >= 32) ? ~0u : ((1u << (uint32_t)(c_hi - b0)) - 1u);
        while (m) {
            uint32_t mine = m;                   // the gw-th set bit of m, if any
            for (int t = 0; t < gw && mine; ++t) mine &= mine - 1u;
            if (mine) off_chain<G, T, LJ>(a, b0 + __ffs(mine) - 1, w, g, logm);
            for (int t = 0; t < 32 / G && m; ++t) m &= m - 1u;
            __syncwarp();
        }
    }
}

// Persistent batch kernel for one (G, T, potential) class.  The queue holds
// (ensemble, chain range) items of up to chains_per_block chains, sorted by
// decreasing cost; ticket t of a counter is chain t % chains_per_block of
// item t / chains_per_block.  Every group takes its own tickets, keeps the
// arguments of its current ensemble in shared memory, and grows each chain
// with the same off_chain code as the single-ensemble kernels -- no group
// waits for the others of its block.
template <int G, int T, bool LJ>
__global__ void __launch_bounds__(256, 4) offlattice_batch_kernel(const OffArgs *__restrict__ ens,
                                                                  const BatchItem *__restrict__ items,
                                                                  int n_items, int *head,
                                                                  int chains_per_block, int Nmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ OffArgs sa[256 / G];
    float *logm = reinterpret_cast<float *>(smem_raw);
    fill_log_table(logm);
    __syncthreads();
    const Group<G> g;
    const int cib = threadIdx.x / G;
    const ChainSmem w = carve(smem_raw + kTable * sizeof(float) +
                                  (size_t)cib * chain_smem_bytes(Nmax, LJ), Nmax, LJ);
    OffArgs &my = sa[cib];
    const unsigned int tickets = (unsigned int)n_items * (unsigned int)chains_per_block;
    unsigned int *next = reinterpret_cast<unsigned int *>(head);
    int cur = -1;     // the ensemble whose arguments are in my
    for (;;) {
        unsigned int t = 0;
        if (g.gl == 0) t = atomicAdd(next, 1u);
        t = g.bcast(t, 0);
        if (t >= tickets) break;
        const BatchItem bi = items[t / (unsigned int)chains_per_block];
        const unsigned int off = t % (unsigned int)chains_per_block;
        if (off >= bi.n) continue;
        if ((int)bi.ens != cur) {
            constexpr int kWords = (int)(sizeof(OffArgs) / 4);
            for (int q = g.gl; q < kWords; q += G)
                reinterpret_cast<uint32_t *>(&my)[q] =
                    reinterpret_cast<const uint32_t *>(&ens[bi.ens])[q];
            __syncwarp(g.mask);
            cur = (int)bi.ens;
        }
        off_chain<G, T, LJ, ChainSmem, false, true>(my, bi.c0 + off, w, g, logm);
    }
}

// Directions exactly as the growth kernels compute them (for verification).
__global__ void sphere_points_kernel(const uint2 *words, int64_t n, float *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint2 v = words[q];
    const float3 u = dir32(v.x, v.y);
    out[3 * q + 0] = u.x;
    out[3 * q + 1] = u.y;
    out[3 * q + 2] = u.z;
}

// Float-float directions as the Lennard-Jones kernels commit them.
__global__ void sphere_points_ff_kernel(const uint2 *words, int64_t n, float *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint2 v = words[q];
    float xh, xl, yh, yl, z;
    dir_ff(v.x, v.y, xh, xl, yh, yl, z);
    out[5 * q + 0] = xh;
    out[5 * q + 1] = xl;
    out[5 * q + 2] = yh;
    out[5 * q + 3] = yl;
    out[5 * q + 4] = z;
}

// Chains per block: 256 threads, fewer if the chains' shared memory would
// exceed 96 KB (at least one warp).
int chains_per_block_for(int G, int N, bool lj)
{
    const size_t per_chain = chain_smem_bytes(N, lj);
    int chains = 256 / G;
    while (chains > 32 / G && (size_t)chains * per_chain > 96 * 1024) chains -= 32 / G;
    return chains;
}

// Scratch of a range launch: 16 bytes of counters (the chain counter, 8
// bytes, and the second pass's word counter, 4 bytes), zeroed by every
// launch, and the deferral mask, one bit per chain of the ensemble, which
// must be zero before the first launch over an ensemble's chains.  Launches
// that may run at the same time need counters of their own; they can share
// the mask (their chain ranges are disjoint).
constexpr size_t kScratchHeader = 16;

size_t mask_bytes(int64_t C) { return (size_t)((C + 31) / 32) * sizeof(uint32_t); }

// Growth of local chains [c_lo, c_hi).  Groups take chains from a counter
// (offlattice_queue_kernel); the grid is what the GPU holds at once.  Short
// hard-sphere chains (N <= 128) grow in two passes: their FP32 decisions are
// almost never ambiguous (about 2% of N = 64, k = 32 chains meet one such
// step), but the FP64 re-decision path, compiled into the growth kernel,
// costs every chain registers and time (the kernel without it runs 11%
// faster).  So the first pass has no FP64 path and defers the chains that
// need it; the second regrows only those, with it.  Longer chains meet
// ambiguous steps more often (a third of N = 512 chains), and regrowing them
// costs more than the first pass saves, so they grow in one pass.  Every
// chain's outputs are those of the one-pass kernel, bit for bit.
template <int G, int T, bool LJ>
int launch_range(const OffArgs &a, int N, int64_t c_lo, int64_t c_hi, void *counters,
                 uint32_t *mask, cudaStream_t s)
{
    const int chains = chains_per_block_for(G, N, LJ);
    const size_t smem = kTable * sizeof(float) + (size_t)chains * chain_smem_bytes(N, LJ);
    const int threads = chains * G;
    const int64_t n = c_hi - c_lo;
    const int64_t blocks = (n + chains - 1) / chains;
    const bool two_pass = !LJ && N <= 128;
    unsigned char *sc = static_cast<unsigned char *>(counters);
    unsigned long long *next = reinterpret_cast<unsigned long long *>(sc);
    unsigned int *wnext = reinterpret_cast<unsigned int *>(sc + 8);
    OffArgs d = a;
    if (two_pass) d.deferred = mask;
    cudaError_t e = cudaMemsetAsync(sc, 0, kScratchHeader, s);
    int dev = 0, sms = 0, bps = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // The first pass without the FP64 path, or the one pass with it.
    auto first = two_pass ? offlattice_queue_kernel<G, T, LJ, !LJ>
                          : offlattice_queue_kernel<G, T, LJ, false>;
    if (e == cudaSuccess) e = allow_max_smem(first);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, first, threads, smem);
    if (e == cudaSuccess) {
        int64_t grid = (int64_t)(bps > 0 ? bps : 1) * sms;
        if (grid > blocks) grid = blocks;
        first<<<(unsigned)grid, threads, smem, s>>>(d, chains, next, c_lo, c_hi);
        if constexpr (!LJ) {
            if (two_pass) {
                int bps2 = 0;
                e = allow_max_smem(offlattice_deferred_kernel<G, T, LJ>);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &bps2, offlattice_deferred_kernel<G, T, LJ>, threads, smem);
                const int64_t words = (c_hi + 31) / 32 - c_lo / 32;
                int64_t grid2 = (int64_t)(bps2 > 0 ? bps2 : 1) * sms;
                if (grid2 > (words + chains - 1) / chains) grid2 = (words + chains - 1) / chains;
                if (e == cudaSuccess)
                    offlattice_deferred_kernel<G, T, LJ>
                        <<<(unsigned)grid2, threads, smem, s>>>(d, chains, wnext, c_lo, c_hi);
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_offlattice_grow: %s", cudaGetErrorString(e));
    return ROSEN_OK;
}

// A whole ensemble: the scratch comes from the stream-ordered allocator; if
// that fails, the one-pass kernel runs with one block per chains_per_block
// chains (same outputs).
template <int G, int T, bool LJ>
int launch_one(const OffArgs &a, int N, cudaStream_t s)
{
    const bool two_pass = !LJ && N <= 128;
    const size_t bytes = kScratchHeader + (two_pass ? mask_bytes(a.C) : 0);
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, s) == cudaSuccess) {
        cudaError_t e = two_pass ? cudaMemsetAsync(static_cast<unsigned char *>(buf) +
                                                       kScratchHeader, 0, bytes - kScratchHeader, s)
                                 : cudaSuccess;
        uint32_t *mask = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(buf) +
                                                      kScratchHeader);
        int st = e == cudaSuccess ? launch_range<G, T, LJ>(a, N, 0, a.C, buf, mask, s)
                                  : set_error(ROSEN_ECUDA, "rosen_offlattice_grow: %s",
                                              cudaGetErrorString(e));
        const cudaError_t f = cudaFreeAsync(buf, s);
        if (st != ROSEN_OK) return st;
        if (f != cudaSuccess)
            return set_error(ROSEN_ECUDA, "rosen_offlattice_grow: freeing the work counter: %s",
                             cudaGetErrorString(f));
        return ROSEN_OK;
    }
    cudaGetLastError();   // clear the failed allocation; grow in one pass
    const int chains = chains_per_block_for(G, N, LJ);
    const size_t smem = kTable * sizeof(float) + (size_t)chains * chain_smem_bytes(N, LJ);
    const int64_t blocks = (a.C + chains - 1) / chains;
    allow_max_smem(offlattice_group_kernel<G, T, LJ>);
    offlattice_group_kernel<G, T, LJ><<<(unsigned)blocks, chains * G, smem, s>>>(a, chains);
    return check_launch("rosen_offlattice_grow");
}

// Chains the GPU grows at once with the first-pass (or only) kernel.
template <int G, int T, bool LJ>
int64_t resident(int N)
{
    const int chains = chains_per_block_for(G, N, LJ);
    const size_t smem = kTable * sizeof(float) + (size_t)chains * chain_smem_bytes(N, LJ);
    auto first = (!LJ && N <= 128) ? offlattice_queue_kernel<G, T, LJ, !LJ>
                                   : offlattice_queue_kernel<G, T, LJ, false>;
    int dev = 0, sms = 0, bps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        allow_max_smem(first) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, first, chains * G, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int64_t)bps * sms * chains;
}

// launch_one (counters == nullptr: a whole ensemble, scratch allocated
// here), launch_range, or the resident chain count (resident_out != nullptr).
template <int G, bool LJ>
int launch_g(const OffArgs &a, int N, int k, int64_t c_lo, int64_t c_hi, void *counters,
             uint32_t *mask, cudaStream_t s, int64_t *resident_out = nullptr)
{
    const int T = (k + G - 1) / G;
    if (resident_out) {
        *resident_out = T <= 1 ? resident<G, 1, LJ>(N) : T <= 2 ? resident<G, 2, LJ>(N)
                                                                  : resident<G, 4, LJ>(N);
        return ROSEN_OK;
    }
    if (!counters) {
        if (T <= 1) return launch_one<G, 1, LJ>(a, N, s);
        if (T <= 2) return launch_one<G, 2, LJ>(a, N, s);
        return launch_one<G, 4, LJ>(a, N, s);
    }
    if (T <= 1) return launch_range<G, 1, LJ>(a, N, c_lo, c_hi, counters, mask, s);
    if (T <= 2) return launch_range<G, 2, LJ>(a, N, c_lo, c_hi, counters, mask, s);
    return launch_range<G, 4, LJ>(a, N, c_lo, c_hi, counters, mask, s);
}

template <bool LJ>
int launch_lj(const OffArgs &a, int G, int N, int k, int64_t c_lo, int64_t c_hi, void *counters,
              uint32_t *mask, cudaStream_t s, int64_t *resident_out = nullptr)
{
    if (G == 8) return launch_g<8, LJ>(a, N, k, c_lo, c_hi, counters, mask, s, resident_out);
    if (G == 16) return launch_g<16, LJ>(a, N, k, c_lo, c_hi, counters, mask, s, resident_out);
    return launch_g<32, LJ>(a, N, k, c_lo, c_hi, counters, mask, s, resident_out);
}

// The batch kernel of class (G, T, LJ) through one function pointer type.
using BatchFn = void (*)(const OffArgs *, const BatchItem *, int, int *, int, int);

template <int G, int T, bool LJ>
BatchFn batch_fn()
{
    return offlattice_batch_kernel<G, T, LJ>;
}

BatchFn pick_batch(int G, int T, bool lj)
{
#define ROSEN_PICK(GG, TT)                                                              \
    if (G == GG && T == TT) return lj ? batch_fn<GG, TT, true>() : batch_fn<GG, TT, false>();
    ROSEN_PICK(8, 1) ROSEN_PICK(8, 2) ROSEN_PICK(8, 4)
    ROSEN_PICK(16, 1) ROSEN_PICK(16, 2) ROSEN_PICK(16, 4)
    ROSEN_PICK(32, 1) ROSEN_PICK(32, 2) ROSEN_PICK(32, 4)
#undef ROSEN_PICK
    return nullptr;
}

}  // namespace

int offlattice_validate(const rosen_offlattice_params *p, const rosen_offlattice_out *o, int nmax,
                        const char *fn)
{
    if (!p || !o) return set_error(ROSEN_EINVAL, "%s: NULL params or outputs", fn);
    if (p->N < 2 || p->N > nmax)
        return set_error(ROSEN_EINVAL, "%s: N = %d outside [2, %d]", fn, p->N,
                         nmax);
    if (p->k < 1 || p->k > ROSEN_KMAX)
        return set_error(ROSEN_EINVAL, "%s: k = %d outside [1, %d]", fn, p->k,
                         ROSEN_KMAX);
    if (p->C < 0 || p->chain0 < 0 || p->chain0 + p->C > (int64_t(1) << 32))
        return set_error(ROSEN_EINVAL,
                         "%s: chains [%lld, %lld) outside [0, 2^32)", fn,
                         (long long)p->chain0, (long long)(p->chain0 + p->C));
    if (p->potential != ROSEN_HARD_SPHERE && p->potential != ROSEN_LJ)
        return set_error(ROSEN_EINVAL, "%s: unknown potential %d", fn, p->potential);
    if (!(p->sigma >= 0.0) || !isfinite(p->sigma) || p->sigma > 4.0)
        return set_error(ROSEN_EINVAL, "%s: sigma must lie in [0, 4]", fn);
    if (p->potential == ROSEN_LJ &&
        (!(p->cutoff > 0.0) || !isfinite(p->cutoff) || p->cutoff > 8.0 || p->sigma <= 0.0))
        return set_error(ROSEN_EINVAL,
                         "%s: LJ needs sigma > 0 and 0 < cutoff <= 8", fn);
    if (!(p->beta_eps >= 0.0) || !isfinite(p->beta_eps))
        return set_error(ROSEN_EINVAL, "%s: beta_eps must be finite and >= 0", fn);
    if (p->flags & ~(ROSEN_STORE_TRACE | ROSEN_STORE_COORDS))
        return set_error(ROSEN_EINVAL, "%s: unknown flags 0x%x", fn, p->flags);
    if ((p->flags & ROSEN_STORE_TRACE) && !o->trace)
        return set_error(ROSEN_EINVAL, "%s: ROSEN_STORE_TRACE without trace", fn);
    if ((p->flags & ROSEN_STORE_COORDS) && !o->coords)
        return set_error(ROSEN_EINVAL, "%s: ROSEN_STORE_COORDS without coords", fn);
    const int G = p->lanes_per_chain;
    if (G != 0 && G != 8 && G != 16 && G != 32)
        return set_error(ROSEN_EINVAL,
                         "%s: lanes_per_chain must be 0, 8, 16 or 32", fn);
    if (G != 0 && (p->k + G - 1) / G > 4)
        return set_error(ROSEN_EINVAL,
                         "%s: k = %d needs more than 4 trials per lane", fn, p->k);
    if (p->max_attempts < 0 || p->max_attempts > ROSEN_MAX_ATTEMPTS)
        return set_error(ROSEN_EINVAL, "%s: max_attempts = %d outside [0, %d]", fn,
                         p->max_attempts, ROSEN_MAX_ATTEMPTS);
    return ROSEN_OK;
}

// Default lanes per chain for the shared-memory kernels (measured on GB300):
// at N = 64 hard spheres run best with two chains per warp (16 lanes) and
// Lennard-Jones -- whose pair work is several times heavier -- with a whole
// warp per chain once k > 16.  Longer chains spend more of each step in the
// scan of earlier beads, which a whole warp does twice as fast: from N = 100
// every k takes 32 lanes (N = 128 / 256, hard spheres k = 32: 11.4 / 17.2 ms
// with 32 lanes against 13.7 / 38.0 ms with 16; LJ k = 16: 25.9 / 46.0
// against 29.3 / 71.8 ms).  N = 0: the chain length is not known (the
// long-chain kernel, whose near lists come from cells).
int offlattice_default_lanes(int k, bool lj, int N)
{
    if (N >= 100) return 32;
    if (lj) return k <= 16 ? 16 : 32;
    if (k <= 64) return 16;
    return 32;
}

size_t offlattice_args_size() { return sizeof(OffArgs); }

void offlattice_make_args(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                          unsigned long long *counters, void *out)
{
    OffArgs a;
    memset(&a, 0, sizeof a);
    a.key = philox_keys(p->seed);
    a.ens = p->ensemble;
    a.chain0 = (uint32_t)p->chain0;
    a.N = p->N;
    a.k = p->k;
    a.C = p->C;
    const bool lj = p->potential == ROSEN_LJ;
    const double sig = p->sigma;
    const double R = lj ? p->cutoff : sig;
    a.sig2 = (float)(sig * sig);
    a.rc2 = lj ? (float)(p->cutoff * p->cutoff) : 0.f;
    a.rf2 = (float)((1.0 + R) * (1.0 + R) * 1.001 + 1e-3);
    a.rf = (float)sqrt((double)a.rf2 * 1.0001);
    a.beta4 = lj ? (float)(4.0 * p->beta_eps) : 0.f;
    a.dband = (float)(lj ? p->cutoff : sig * 1.001);
    if (lj) {
        const double sc = (sig * sig) / (p->cutoff * p->cutoff), s3 = sc * sc * sc;
        a.ucut2 = (float)(2.0 * fabs(s3 * (s3 - 1.0)));
    }
    a.sig2d = sig * sig;
    a.rc2d = lj ? p->cutoff * p->cutoff : 0.0;
    a.beta_eps = p->beta_eps;
    a.logw = o->logw;
    a.r2 = o->r2;
    a.rg2 = o->rg2;
    a.alive = o->alive;
    a.trace = (p->flags & ROSEN_STORE_TRACE) ? o->trace : nullptr;
    a.coords = (p->flags & ROSEN_STORE_COORDS) ? o->coords : nullptr;
    // Position drift from exact per step for chains that commit float-float
    // directions (1.5e-12 per component) with float-float adds whose rounding
    // grows with |r| <= N (7e-15 N), both with margin; kernels that commit
    // FP32 directions use 4e-7 instead.
    a.drift = (float)(4e-12 + 1e-14 * p->N);
    a.counters = counters;
    a.attempts = o->attempts;
    a.max_att = p->max_attempts > 1 ? (uint32_t)p->max_attempts : 1u;
    memcpy(out, &a, sizeof a);
}

int offlattice_launch(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                      unsigned long long *counters, cudaStream_t s)
{
    OffArgs a;
    offlattice_make_args(p, o, counters, &a);
    const bool lj = p->potential == ROSEN_LJ;
    const int G =
        p->lanes_per_chain ? p->lanes_per_chain : offlattice_default_lanes(p->k, lj, p->N);
    return lj ? launch_lj<true>(a, G, p->N, p->k, 0, p->C, nullptr, nullptr, s)
              : launch_lj<false>(a, G, p->N, p->k, 0, p->C, nullptr, nullptr, s);
}

size_t offlattice_range_counter_bytes() { return kScratchHeader; }
size_t offlattice_range_mask_bytes(int64_t C) { return mask_bytes(C); }

int offlattice_grow_range(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                          int64_t c_lo, int64_t c_hi, void *counters, uint32_t *mask,
                          cudaStream_t s)
{
    if (c_hi <= c_lo) return ROSEN_OK;
    OffArgs a;
    offlattice_make_args(p, o, reinterpret_cast<unsigned long long *>(o->counters), &a);
    const bool lj = p->potential == ROSEN_LJ;
    const int G =
        p->lanes_per_chain ? p->lanes_per_chain : offlattice_default_lanes(p->k, lj, p->N);
    return lj ? launch_lj<true>(a, G, p->N, p->k, c_lo, c_hi, counters, mask, s)
              : launch_lj<false>(a, G, p->N, p->k, c_lo, c_hi, counters, mask, s);
}

int64_t offlattice_resident_chains(const rosen_offlattice_params *p)
{
    OffArgs a;
    memset(&a, 0, sizeof a);
    const bool lj = p->potential == ROSEN_LJ;
    const int G =
        p->lanes_per_chain ? p->lanes_per_chain : offlattice_default_lanes(p->k, lj, p->N);
    int64_t r = 0;
    if (lj) launch_lj<true>(a, G, p->N, p->k, 0, 0, nullptr, nullptr, nullptr, &r);
    else launch_lj<false>(a, G, p->N, p->k, 0, 0, nullptr, nullptr, nullptr, &r);
    return r;
}

int offlattice_batch_prepare(int G, int T, bool lj, int Nmax, int *chains_per_block, size_t *smem,
                             int *blocks_per_sm)
{
    const BatchFn fn = pick_batch(G, T, lj);
    if (!fn) return set_error(ROSEN_EINVAL, "no real-space batch kernel for G=%d T=%d", G, T);
    *chains_per_block = chains_per_block_for(G, Nmax, lj);
    *smem = kTable * sizeof(float) + (size_t)(*chains_per_block) * chain_smem_bytes(Nmax, lj);
    cudaError_t e = allow_max_smem(fn);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn,
                                                          (*chains_per_block) * G, *smem);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "real-space batch set-up: %s", cudaGetErrorString(e));
    return ROSEN_OK;
}

void offlattice_batch_launch(int G, int T, bool lj, const void *dev_args, const BatchItem *items,
                             int n_items, int *head, int chains_per_block, int Nmax, size_t smem,
                             int grid, cudaStream_t s)
{
    const BatchFn fn = pick_batch(G, T, lj);
    fn<<<grid, chains_per_block * G, smem, s>>>(reinterpret_cast<const OffArgs *>(dev_args), items,
                                               n_items, head, chains_per_block, Nmax);
}

}  // namespace rosen

using namespace rosen;

extern "C" int rosen_offlattice_grow(const rosen_offlattice_params *p,
                                     const rosen_offlattice_out *o, void *stream)
{
    const int st = offlattice_validate(p, o);
    if (st != ROSEN_OK) return st;
    if (p->C == 0) return ROSEN_OK;
    return offlattice_launch(p, o, reinterpret_cast<unsigned long long *>(o->counters),
                             (cudaStream_t)stream);
}

extern "C" int rosen_sphere_points(const uint32_t *words, int64_t n, float *out, void *stream)
{
    if (n < 0) return set_error(ROSEN_EINVAL, "rosen_sphere_points: n < 0");
    if (n > 0 && (!words || !out)) return set_error(ROSEN_EINVAL, "rosen_sphere_points: NULL");
    if (reinterpret_cast<uintptr_t>(words) & 7u)
        return set_error(ROSEN_EINVAL, "rosen_sphere_points: words must be 8-byte aligned");
    if (n == 0) return ROSEN_OK;
    const int threads = 256;
    sphere_points_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0,
                           (cudaStream_t)stream>>>(reinterpret_cast<const uint2 *>(words), n, out);
    return check_launch("rosen_sphere_points");
}

extern "C" int rosen_sphere_points_ff(const uint32_t *words, int64_t n, float *out, void *stream)
{
    if (n < 0) return set_error(ROSEN_EINVAL, "rosen_sphere_points_ff: n < 0");
    if (n > 0 && (!words || !out)) return set_error(ROSEN_EINVAL, "rosen_sphere_points_ff: NULL");
    if (reinterpret_cast<uintptr_t>(words) & 7u)
        return set_error(ROSEN_EINVAL, "rosen_sphere_points_ff: words must be 8-byte aligned");
    if (n == 0) return ROSEN_OK;
    const int threads = 256;
    sphere_points_ff_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0,
                              (cudaStream_t)stream>>>(reinterpret_cast<const uint2 *>(words), n,
                                                      out);
    return check_launch("rosen_sphere_points_ff");
}
