// perm.cu -- PERM, the pruned-enriched Rosenbluth method (Grassberger, Phys.
// Rev. E 56, 3682 (1997)), on the simple cubic lattice, breadth first: a
// population of chains grows one step at a time (the Rosenbluth step of
// Algorithm 1 with the weight of Eq. 3), and after step i a chain whose
// weight W exceeds c_hi mu^i is enriched (two copies sharing W), one whose
// weight is below c_lo mu^i is pruned (removed with probability 1/2, its
// weight doubled if it survives).  Both keep the expected total weight of
// every length, so (1/M0) sum W over the chains grown at step i is an
// unbiased estimate of Z_i (Eq. 9) and the W-weighted means are those of
// Eq. 2.  The paper's conclusion names a GPU PERM whose text is not
// available; the readings taken here are stated at rosen_perm_run.
//
// GB300 mapping.  A chain's packed monomer keys stay in one storage slot of
// device memory for as long as the chain lives: a slot holds the keys of
// even monomers, then those of odd monomers, 4 to a 16-byte word, so a lane
// reads the keys its step scans with 16-byte loads of its own slot.  The
// population is an array of slot numbers in population order (two buffers:
// this step's and the next), beside each chain's end key and its weight as
// an FP64 mantissa in [1, 2) and an int32 exponent, so every update is one
// correctly rounded product and every threshold comparison is exact.  (The
// end key sits beside the population, not only in the slot: a step then
// reads one half of the slot, of the parity it scans.)  A chain that leaves
// returns its slot to a stack of free slots, and an enrichment copy takes a
// slot from it and copies the keys there: only copies move keys, not the
// chains that stay.  A step is three launches, with no host synchronisation
// (the population size stays on the device):
//  1. perm_grow_kernel: one lane per chain (whole blocks step through the
//     population in chunks of 256 chains) scans the chain's earlier keys
//     with the displacement table of the lattice kernels, takes the step
//     (same draw, selection and weight as rosen_lattice_grow), appends the
//     new key to its slot and decides its fate; the slots of chains that
//     leave go to the free stack; per chunk the chains kept and the
//     enrichment requests; per-block partial sums of W and W R^2 for
//     Eq. 9 / Eq. 2;
//  2. perm_top_kernel (one block): the exclusive scan of the chunk counts,
//     the population cap (the first max_pop - kept enrichment requests in
//     population order are granted), the next population size, the free
//     slots the copies take, and the step's estimates from the partial sums;
//  3. perm_scatter_kernel: per chunk, a block scan of the fates places
//     every kept chain's slot, end key and weight (and its copy's) in the
//     next population, in order; a copy's keys go to a free slot.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"
#include "lattice_step.cuh"

namespace rosen {
namespace {

constexpr int kPermThreads = 256;        // also the chains of a scan chunk
constexpr int kPermWarps = kPermThreads / 32;
constexpr int kTopThreads = 1024;
constexpr int kMaxParts = 8192;          // grow-kernel blocks (partial sums)

struct PermArgs {
    PhiloxKeys key;
    uint32_t ens;
    int32_t N;
    int64_t max_pop;
    float wt32[8];     // exp(beta_eps c), c = 0..5 (FP32 selection)
    double wt64[8];    // the same in FP64 (weights, exact selection)
    int32_t isaw;
};

// Threshold of one step as m 2^e with m in [1, 2); mode 0: compare,
// 1: never exceeded / never undercut, 2: always exceeded.
struct Threshold {
    double m;
    int32_t e;
    int32_t mode;
};

struct PermPartial {
    double s, sr;      // sum of W 2^-e and W R^2 2^-e over the block's grown chains
    int32_t e;         // the block's largest weight exponent (INT_MIN: none grown)
    int32_t pad;
    double grown;
};

struct PermWs {
    uint32_t *keys;             // [max_pop slots][2][H]: key q of a slot at [q & 1][q >> 1]
    int32_t *ord[2];            // population position -> slot (this step's, the next)
    uint32_t *endk[2];          // the end key of the chain at each position
    double *wm[2];
    int32_t *we[2];
    int32_t *free_slots;        // stack of the slots no chain holds
    int8_t *fate;               // 0 gone, 1 kept, 2 enrichment request, -1 pruning survivor
    unsigned long long *chunks; // per chunk: kept | requests << 32, then the exclusive offset
    PermPartial *parts;
    long long *ctl;             // [0], [1]: population of the two buffers; [2]: grants;
                                // [3]: free slots; [4]: free slots after the step's returns
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Words per half slot: the keys of one parity, rounded up to 16-byte words.
__host__ __device__ inline int perm_half_words(int N) { return (((N + 1) / 2) + 3) & ~3; }
// Words per slot: the two halves.
__host__ __device__ inline int64_t perm_slot_words(int H) { return 2 * (int64_t)H; }

// Carve the workspace (or, with base == nullptr, measure it).
size_t perm_carve(void *base, int N, int64_t max_pop, PermWs *w)
{
    unsigned char *p = static_cast<unsigned char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *r = p ? p + off : nullptr;
        off += a256(bytes);
        return r;
    };
    const size_t P = (size_t)max_pop;
    const size_t chunks = (P + kPermThreads - 1) / kPermThreads;
    PermWs t;
    t.keys = static_cast<uint32_t *>(take(4 * (size_t)perm_slot_words(perm_half_words(N)) * P));
    for (int b = 0; b < 2; ++b) t.ord[b] = static_cast<int32_t *>(take(4 * P));
    for (int b = 0; b < 2; ++b) t.endk[b] = static_cast<uint32_t *>(take(4 * P));
    for (int b = 0; b < 2; ++b) t.wm[b] = static_cast<double *>(take(8 * P));
    for (int b = 0; b < 2; ++b) t.we[b] = static_cast<int32_t *>(take(4 * P));
    t.free_slots = static_cast<int32_t *>(take(4 * P));
    t.fate = static_cast<int8_t *>(take(P));
    t.chunks = static_cast<unsigned long long *>(take(8 * chunks));
    t.parts = static_cast<PermPartial *>(take(sizeof(PermPartial) * kMaxParts));
    t.ctl = static_cast<long long *>(take(8 * 8));
    if (w) *w = t;
    return off;
}

// x = m 2^e with m in [1, 2), for a positive normal double (bit fields).
__device__ __forceinline__ void norm_weight(double x, double &m, int32_t &e)
{
    const long long b = __double_as_longlong(x);
    e = (int32_t)((b >> 52) & 0x7FF) - 1023;
    m = __longlong_as_double((b & 0x800FFFFFFFFFFFFFll) | (1023ll << 52));
}

// Weight against threshold.  Mantissas in [1, 2) are positive normal
// doubles, which order like their bit patterns: the comparisons stay off the
// FP64 pipe (a small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ bool above(double wm, int32_t we, const Threshold &t)
{
    if (t.mode == 1) return false;
    if (t.mode == 2) return true;
    return we > t.e || (we == t.e && __double_as_longlong(wm) > __double_as_longlong(t.m));
}

__device__ __forceinline__ bool below(double wm, int32_t we, const Threshold &t)
{
    if (t.mode != 0) return false;
    return we < t.e || (we == t.e && __double_as_longlong(wm) < __double_as_longlong(t.m));
}

// wm m for wm in [1, 2) and a small integer m (1..6: an athermal step),
// rounded to the nearest double (ties to even) exactly as one FP64 multiply
// rounds it, and renormalised to (mantissa in [1, 2), exponent): in integer
// arithmetic, off the FP64 pipe.  The 53-bit significand times m is exact in
// 64 bits (< 2^56); its top 53 bits are kept, rounded on the k bits below.
__device__ __forceinline__ void mul_small(double wm, uint32_t m, double &m_out, int32_t &e_out)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(wm);
    const unsigned long long X = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) * (unsigned long long)m;
    int k = 11 - __clzll((long long)X);           // X in [2^(52+k), 2^(53+k))
    unsigned long long q = X >> k;
    if (k > 0) {
        const unsigned long long r = X & ((1ull << k) - 1ull), half = 1ull << (k - 1);
        if (r > half || (r == half && (q & 1ull))) ++q;
        if (q >> 53) {                            // rounded up to 2^53
            q >>= 1;
            ++k;
        }
    }
    m_out = __longlong_as_double((long long)((q & 0xFFFFFFFFFFFFFull) | (1023ull << 52)));
    e_out = k;
}

// m 2^d for m in [1, 2) and d <= 0 by its exponent field; 0 below the
// normal range (a relative weight under 2^-1022, far below the estimates'
// rounding).
__device__ __forceinline__ double scale_down(double m, int d)
{
    if (d < -1022) return 0.0;
    return __longlong_as_double(__double_as_longlong(m) + ((long long)d << 52));
}

// Chain j of the first population in slot j, at the origin; the other
// slots on the free stack.
__global__ void perm_init_kernel(int64_t M0, int64_t max_pop, int H, uint32_t *keys,
                                 int32_t *ord, uint32_t *endk, double *wm, int32_t *we,
                                 int32_t *free_slots, long long *ctl, long long *population,
                                 double *logz, double *mean_r2)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < max_pop; j += stride) {
        if (j < M0) {
            ord[j] = (int32_t)j;
            endk[j] = kOriginKey;
            keys[j * perm_slot_words(H)] = kOriginKey;
            wm[j] = 1.0;
            we[j] = 0;
        } else {
            free_slots[j - M0] = (int32_t)j;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl[0] = M0;
        ctl[1] = 0;
        ctl[2] = 0;
        ctl[3] = max_pop - M0;
        ctl[4] = 0;
        population[0] = M0;
        logz[0] = 0.0;
        if (mean_r2) mean_r2[0] = 0.0;
    }
}

// Sum of the table entries of the first n keys at ks (16-byte aligned) for
// the end whose bias is kb; the entries' fields never carry into one
// another, so the order of the sum does not matter.
__device__ __forceinline__ uint32_t scan_keys(const uint32_t *lut, const uint32_t *ks, int n,
                                              uint32_t kb)
{
    const uint4 *g = reinterpret_cast<const uint4 *>(ks);
    uint32_t acc = 0u;
    const int full = n >> 2;
#pragma unroll 4
    for (int t = 0; t < full; ++t) {
        const uint4 v = g[t];
        acc += lut_at(lut, lut_off(v.x + kb)) + lut_at(lut, lut_off(v.y + kb)) +
               lut_at(lut, lut_off(v.z + kb)) + lut_at(lut, lut_off(v.w + kb));
    }
    const int r = n & 3;
    if (r) {
        const uint4 v = g[full];
        acc += lut_at(lut, lut_off(v.x + kb));
        if (r > 1) acc += lut_at(lut, lut_off(v.y + kb));
        if (r > 2) acc += lut_at(lut, lut_off(v.z + kb));
    }
    return acc;
}

// Step i of every chain of the population (ord / endk / wm / we of this
// step's buffer, population *pcount): growth, weight, fate, chunk counts,
// partial sums; the slots of chains that leave go to the free stack (*nfree
// entries).
template <bool kIsaw>
__global__ void __launch_bounds__(kPermThreads) perm_grow_kernel(
    const PermArgs a, int i, Threshold hi, Threshold lo, uint32_t *keys, int H,
    const int32_t *ord, uint32_t *endk, double *wm, int32_t *we, int8_t *fate,
    unsigned long long *chunks, const long long *pcount, PermPartial *parts,
    int32_t *free_slots, long long *nfree)
{
    __shared__ uint32_t lut[kLutWords];
    __shared__ uint8_t seltab[kSelBytes];
    __shared__ float wt32[8];
    __shared__ double wt64[8];
    __shared__ double red_s[kPermThreads / 32], red_r[kPermThreads / 32], red_g[kPermThreads / 32];
    __shared__ int32_t red_e[kPermThreads / 32];
    __shared__ unsigned wk[kPermWarps], wr[kPermWarps];
    fill_tables(lut, seltab);
    if (threadIdx.x < 8) {
        wt32[threadIdx.x] = a.wt32[threadIdx.x];
        wt64[threadIdx.x] = a.wt64[threadIdx.x];
    }
    __syncthreads();
    const int64_t P = *pcount;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t emax = INT_MIN;     // running largest exponent of this lane's grown chains
    double s = 0.0, sr = 0.0;
    int grown_n = 0;
    // Whole blocks step through the population together, one chunk of
    // kPermThreads chains at a time; the next chunk's slot numbers are loaded
    // a chunk ahead, and the half slots its scans read are prefetched to L2
    // while this chunk grows.
    const int64_t j_first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t slot_next = j_first < P ? ord[j_first] : 0;
    const int half = i & 1;     // the half slot an athermal step scans
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < P; j0 += stride) {
        const int64_t j = j0 + threadIdx.x;
        const bool valid = j < P;
        int8_t f = 0;
        int32_t slot = slot_next;
        if (j + stride < P) slot_next = ord[j + stride];
        if (valid) {
            uint32_t *ks = keys + slot * perm_slot_words(H);
            const uint32_t key = endk[j];
            const uint32_t kb = kNearBias - key;
            // Monomers 0 .. i-2 (ISAW), or those of the parity of i, the only
            // ones that can be neighbours of the new site (athermal).
            uint32_t acc;
            if (kIsaw) {
                acc = scan_keys(lut, ks, i / 2, kb) + scan_keys(lut, ks + H, (i - 1) / 2, kb);
            } else {
                const int p = i & 1;
                acc = scan_keys(lut, ks + p * H, (i - p) / 2, kb);
            }
            const uint32_t freem = ~acc & 63u;
            const int m = __popc(freem);
            if (m > 0) {
                const uint32_t x =
                    philox(make_uint4((uint32_t)j, a.ens, (uint32_t)i, 0u), a.key).x;
                LogW lw_unused;
                const int sel = choose<kIsaw>(freem, m, acc, x, seltab, wt32, wt64, lw_unused);
                // The step's weight factor: m (athermal: the product in
                // integer arithmetic, mul_small), or the FP64 sum of the free
                // neighbours' Boltzmann factors in slot order.
                double S = 0.0;
                if (kIsaw) {
#pragma unroll
                    for (int d = 0; d < 6; ++d) {
                        const uint32_t cd = (acc >> (8 + 3 * d)) & 7u;
                        S = __dadd_rn(S, ((freem >> d) & 1u) ? wt64[cd] : 0.0);
                    }
                }
                const uint32_t axis_step = 1u << (10 * (sel >> 1));
                const uint32_t nk = (sel & 1) ? key - axis_step : key + axis_step;
                ks[(i & 1) * H + (i >> 1)] = nk;
                endk[j] = nk;
                double m_;
                int32_t e_;
                if (kIsaw)
                    norm_weight(__dmul_rn(wm[j], S), m_, e_);
                else
                    mul_small(wm[j], (uint32_t)m, m_, e_);
                const int32_t e_new = we[j] + e_;
                wm[j] = m_;
                we[j] = e_new;
                if (above(m_, e_new, hi)) {
                    f = 2;
                } else if (below(m_, e_new, lo)) {
                    const uint32_t y =
                        philox(make_uint4((uint32_t)j, a.ens, (uint32_t)i, 1u), a.key).x;
                    f = (y >> 31) ? -1 : 0;
                } else {
                    f = 1;
                }
                // Partial sums of W and W R^2, relative to 2^emax.
                const int ex = (int)(nk & 1023u) - 512, ey = (int)((nk >> 10) & 1023u) - 512,
                          ez = (int)(nk >> 20) - 512;
                const double R2 = (double)(ex * ex + ey * ey + ez * ez);
                if (e_new > emax) {
                    const double sc = emax == INT_MIN ? 0.0 : scale_down(1.0, emax - e_new);
                    s *= sc;
                    sr *= sc;
                    emax = e_new;
                }
                const double w = scale_down(m_, e_new - emax);
                s += w;
                sr = fma(w, R2, sr);
                ++grown_n;
            }
            fate[j] = f;
        }
        if (j + stride < P) {
            const uint32_t *nx = keys + slot_next * perm_slot_words(H);
            if (kIsaw) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nx));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + H));
            } else {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + half * H));
            }
        }
        // The slots of the chains that leave, back to the free stack (one
        // atomic per warp; the stack's order does not matter).
        const bool leaves = valid && f == 0;
        const unsigned gone = __ballot_sync(0xffffffffu, leaves);
        if (gone) {
            unsigned long long at = 0;
            if (lane == 0)
                at = atomicAdd(reinterpret_cast<unsigned long long *>(nfree),
                               (unsigned long long)__popc(gone));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (leaves) free_slots[at + __popc(gone & ((1u << lane) - 1u))] = slot;
        }
        // The chunk's counts: chains kept, enrichment requests.
        const unsigned kept_m = __ballot_sync(0xffffffffu, valid && f != 0);
        const unsigned req_m = __ballot_sync(0xffffffffu, valid && f == 2);
        if (lane == 0) {
            wk[warp] = __popc(kept_m);
            wr[warp] = __popc(req_m);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long kept = 0, req = 0;
            for (int q = 0; q < kPermWarps; ++q) {
                kept += wk[q];
                req += wr[q];
            }
            chunks[j0 / kPermThreads] = kept | (req << 32);
        }
        __syncthreads();
    }
    // Block partial: the largest exponent, then the sums rescaled to it.
    int32_t bm = emax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bm = max(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    if (lane == 0) red_e[warp] = bm;
    __syncthreads();
    int32_t E = INT_MIN;
    for (int q = 0; q < kPermThreads / 32; ++q) E = max(E, red_e[q]);
    const double sc = (emax == INT_MIN) ? 0.0 : ldexp(1.0, emax - E);
    s *= sc;
    sr *= sc;
    double grown = (double)grown_n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        grown += __shfl_xor_sync(0xffffffffu, grown, o);
    }
    if (lane == 0) {
        red_s[warp] = s;
        red_r[warp] = sr;
        red_g[warp] = grown;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        PermPartial pp;
        pp.s = pp.sr = pp.grown = 0.0;
        for (int q = 0; q < kPermThreads / 32; ++q) {
            pp.s += red_s[q];
            pp.sr += red_r[q];
            pp.grown += red_g[q];
        }
        pp.e = E;
        pp.pad = 0;
        parts[blockIdx.x] = pp;
    }
}

// One block: the chunks' offsets, the cap, the next population size, the
// free slots the copies take, and the estimates of length i from the grow
// kernel's partials.
__global__ void __launch_bounds__(kTopThreads) perm_top_kernel(
    int i, int64_t max_pop, double log_m0, unsigned long long *chunks, const long long *pcount,
    long long *pnext, long long *grants, long long *nfree, long long *pop_top,
    const PermPartial *parts, int nparts, long long *population, double *logz,
    double *mean_r2)
{
    __shared__ unsigned long long wsum[kTopThreads / 32 + 1];
    __shared__ double rs[kTopThreads / 32], rr[kTopThreads / 32], rg[kTopThreads / 32];
    __shared__ int32_t re[kTopThreads / 32];
    const int64_t P = *pcount;
    const int64_t nchunks = (P + kPermThreads - 1) / kPermThreads;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Exclusive scan in rounds of kTopThreads x 4 chunks, four consecutive
    // chunks per thread (two 16-byte loads; the next round's are issued
    // before this round is scanned).
    constexpr int kPer = 4;
    constexpr int64_t kRound = (int64_t)kTopThreads * kPer;
    unsigned long long total = 0;
    unsigned long long v4[kPer], n4[kPer];
    auto load4 = [&](int64_t r0, unsigned long long (&d)[kPer]) {
        const int64_t t = r0 + (int64_t)threadIdx.x * kPer;
        if (t + kPer <= nchunks) {
            const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(chunks + t);
            const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(chunks + t + 2);
            d[0] = a.x;
            d[1] = a.y;
            d[2] = b.x;
            d[3] = b.y;
        } else {
#pragma unroll
            for (int c = 0; c < kPer; ++c) d[c] = t + c < nchunks ? chunks[t + c] : 0ull;
        }
    };
    load4(0, v4);
    for (int64_t r0 = 0; r0 < nchunks; r0 += kRound) {
        const int64_t t = r0 + (int64_t)threadIdx.x * kPer;
        if (r0 + kRound < nchunks) load4(r0 + kRound, n4);
        const unsigned long long v = v4[0] + v4[1] + v4[2] + v4[3];
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long ws = wsum[lane];
            unsigned long long wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            wsum[lane] = wi - ws;            // exclusive offset of warp `lane`
            if (lane == 31) wsum[32] = wi;   // the round's total
        }
        __syncthreads();
        unsigned long long off = total + wsum[warp] + incl - v;
#pragma unroll
        for (int c = 0; c < kPer; ++c) {
            if (t + c < nchunks) chunks[t + c] = off;
            off += v4[c];
        }
        total += wsum[32];
        __syncthreads();                     // wsum is rewritten by the next round
#pragma unroll
        for (int c = 0; c < kPer; ++c) v4[c] = n4[c];
    }
    // Estimates: the largest exponent over the partials, then the sums.
    int32_t E = INT_MIN;
    for (int q = threadIdx.x; q < nparts; q += kTopThreads)
        if (parts[q].grown > 0.0) E = max(E, parts[q].e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) re[warp] = E;
    __syncthreads();
    E = INT_MIN;
    for (int q = 0; q < kTopThreads / 32; ++q) E = max(E, re[q]);
    double s = 0.0, sr = 0.0, g = 0.0;
    for (int q = threadIdx.x; q < nparts; q += kTopThreads) {
        const PermPartial pp = parts[q];
        if (pp.grown > 0.0) {
            const double sc = ldexp(1.0, pp.e - E);
            s += pp.s * sc;
            sr += pp.sr * sc;
            g += pp.grown;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
    }
    if (lane == 0) {
        rs[warp] = s;
        rr[warp] = sr;
        rg[warp] = g;
    }
    __syncthreads();
    if (warp == 0) {
        s = rs[lane];
        sr = rr[lane];
        g = rg[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
        }
    }
    if (threadIdx.x == 0) {
        const long long base = (long long)(total & 0xFFFFFFFFull);
        const long long extra = (long long)(total >> 32);
        const long long G = max_pop - base > 0 ? max_pop - base : 0;
        const long long Pn = base + (extra < G ? extra : G);
        *pnext = Pn;
        *grants = G;
        // The granted copies take the top Pn - base slots of the free stack.
        const long long top = *nfree;
        *pop_top = top;
        *nfree = top - (Pn - base);
        population[i] = Pn;
        if (g > 0.0) {
            logz[i] = log(s) + (double)E * 0.69314718055994530942 - log_m0;
            if (mean_r2) mean_r2[i] = sr / s;
        } else {
            logz[i] = -INFINITY;
            if (mean_r2) mean_r2[i] = NAN;
        }
    }
}

// Kept chains, in population order, to their places in the next buffer
// (per chunk: the chunk's offset from the top kernel plus a block scan of
// its fates); the copy granted to the enrichment request of rank r takes
// free slot free_slots[top - 1 - r] and the keys 0..i of its original.
__global__ void __launch_bounds__(kPermThreads) perm_scatter_kernel(
    int i, int H, uint32_t *keys, const int32_t *ord, int32_t *ord_n, const uint32_t *endk,
    uint32_t *endk_n, const double *wm, const int32_t *we, double *wm_n, int32_t *we_n,
    const int8_t *fate, const unsigned long long *chunks, const long long *pcount,
    const long long *grants, const int32_t *free_slots, const long long *pop_top)
{
    __shared__ unsigned wk[kPermWarps], wr[kPermWarps];
    const int64_t P = *pcount;
    const long long G = *grants;
    const long long top = *pop_top;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below_me = (1u << lane) - 1u;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < P; j0 += stride) {
        const int64_t j = j0 + threadIdx.x;
        const int f = j < P ? fate[j] : 0;
        const unsigned kept_m = __ballot_sync(0xffffffffu, f != 0);
        const unsigned req_m = __ballot_sync(0xffffffffu, f == 2);
        if (lane == 0) {
            wk[warp] = __popc(kept_m);
            wr[warp] = __popc(req_m);
        }
        __syncthreads();
        unsigned kb = 0, rb = 0;
        for (int q = 0; q < warp; ++q) {
            kb += wk[q];
            rb += wr[q];
        }
        __syncthreads();
        int32_t slot = 0, s2 = -1;
        if (f != 0) {
            const unsigned long long c = chunks[j0 / kPermThreads];
            const long long kept_before =
                (long long)(c & 0xFFFFFFFFull) + kb + __popc(kept_m & below_me);
            const long long rank = (long long)(c >> 32) + rb + __popc(req_m & below_me);
            const long long dst = kept_before + (rank < G ? rank : G);
            const int copies = (f == 2 && rank < G) ? 2 : 1;
            const int32_t w_e = we[j] + (copies == 2 ? -1 : (f == -1 ? 1 : 0));
            slot = ord[j];
            const uint32_t ek = endk[j];
            const double w_m = wm[j];
            ord_n[dst] = slot;
            endk_n[dst] = ek;
            wm_n[dst] = w_m;
            we_n[dst] = w_e;
            if (copies == 2) {
                s2 = free_slots[top - 1 - rank];
                ord_n[dst + 1] = s2;
                endk_n[dst + 1] = ek;
                wm_n[dst + 1] = w_m;
                we_n[dst + 1] = w_e;
            }
        }
        // The copies' keys 0..i (i/2 + 1 even and (i + 1)/2 odd monomers, in
        // whole 16-byte words; the words past them are never read unmasked):
        // the warp copies one copy at a time, a word per lane.
        unsigned cm = __ballot_sync(0xffffffffu, s2 >= 0);
        const int g0 = (i / 2 + 4) >> 2, g1 = ((i + 1) / 2 + 3) >> 2, h4 = H >> 2;
        while (cm) {
            const int from = __ffs(cm) - 1;
            cm &= cm - 1u;
            const int64_t a = __shfl_sync(0xffffffffu, slot, from);
            const int64_t b = __shfl_sync(0xffffffffu, s2, from);
            const uint4 *src = reinterpret_cast<const uint4 *>(keys + a * perm_slot_words(H));
            uint4 *dstk = reinterpret_cast<uint4 *>(keys + b * perm_slot_words(H));
            for (int t = lane; t < g0 + g1; t += 32) {
                const int q = t < g0 ? t : h4 + (t - g0);
                dstk[q] = src[q];
            }
        }
    }
}

// The final population to the caller's arrays.
__global__ void perm_final_kernel(int N, int64_t max_pop, int H, const uint32_t *keys,
                                  const int32_t *ord, const double *wm, const int32_t *we,
                                  const long long *pcount, long long *final_n, double *w_m,
                                  int32_t *w_e, int32_t *coords)
{
    const int64_t P = *pcount;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *final_n = P;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P; c += stride) {
        if (w_m) w_m[c] = wm[c];
        if (w_e) w_e[c] = we[c];
        if (coords) {
            const uint32_t *ks = keys + ord[c] * perm_slot_words(H);
            for (int q = 0; q < N; ++q) {
                const uint32_t k = ks[(q & 1) * H + (q >> 1)];
                coords[((int64_t)q * 3 + 0) * max_pop + c] = (int32_t)(k & 1023u) - 512;
                coords[((int64_t)q * 3 + 1) * max_pop + c] = (int32_t)((k >> 10) & 1023u) - 512;
                coords[((int64_t)q * 3 + 2) * max_pop + c] = (int32_t)(k >> 20) - 512;
            }
        }
    }
}

// c tm 2^te as a threshold (host: the same exact operations as the device
// comparisons need).
Threshold make_threshold(double c, double tm, int32_t te, bool upper)
{
    Threshold t;
    t.m = 1.0;
    t.e = 0;
    t.mode = 0;
    const double x = c * tm;
    if (isinf(c) || isinf(x)) {
        t.mode = 1;                      // never exceeded (never undercut: c_lo < c_hi)
    } else if (x == 0.0) {
        t.mode = upper ? 2 : 1;          // every weight exceeds it / none is below it
    } else {
        const int k = ilogb(x);
        t.m = ldexp(x, -k);
        t.e = te + k;
    }
    return t;
}

int perm_validate(const rosen_perm_params *p, const rosen_perm_out *o)
{
    if (!p || !o) return set_error(ROSEN_EINVAL, "rosen_perm_run: NULL params or outputs");
    if (p->N < 2 || p->N > ROSEN_LATTICE_NMAX)
        return set_error(ROSEN_EINVAL, "rosen_perm_run: N = %d outside [2, %d]", p->N,
                         ROSEN_LATTICE_NMAX);
    if (p->M0 < 1 || p->max_population < p->M0 || p->max_population > ROSEN_PERM_MAX_POP)
        return set_error(ROSEN_EINVAL, "rosen_perm_run: need 1 <= M0 <= max_population <= %d",
                         (int)ROSEN_PERM_MAX_POP);
    if (!(p->beta_eps >= 0.0) || !(p->beta_eps <= 16.0))
        return set_error(ROSEN_EINVAL, "rosen_perm_run: beta_eps must lie in [0, 16]");
    if (!(p->mu > 0.0) || !isfinite(p->mu))
        return set_error(ROSEN_EINVAL, "rosen_perm_run: mu must be finite and > 0");
    if (!(p->c_lo >= 0.0) || !(p->c_hi > p->c_lo) || isinf(p->c_lo))
        return set_error(ROSEN_EINVAL, "rosen_perm_run: need 0 <= c_lo < c_hi");
    if (p->flags & ~ROSEN_STORE_COORDS)
        return set_error(ROSEN_EINVAL, "rosen_perm_run: unknown flags 0x%x", p->flags);
    if ((p->flags & ROSEN_STORE_COORDS) && !o->coords)
        return set_error(ROSEN_EINVAL, "rosen_perm_run: ROSEN_STORE_COORDS without coords");
    if (!o->population || !o->logz || !o->final_n)
        return set_error(ROSEN_EINVAL, "rosen_perm_run: population, logz and final_n are required");
    return ROSEN_OK;
}

}  // namespace
}  // namespace rosen

using namespace rosen;

extern "C" size_t rosen_perm_workspace_size(int32_t N, int64_t max_population)
{
    if (N < 2 || N > ROSEN_LATTICE_NMAX || max_population < 1 ||
        max_population > ROSEN_PERM_MAX_POP)
        return 0;
    return perm_carve(nullptr, N, max_population, nullptr);
}

extern "C" int rosen_perm_run(const rosen_perm_params *p, const rosen_perm_out *o,
                              void *workspace, size_t workspace_bytes, void *stream)
{
    int st = perm_validate(p, o);
    if (st != ROSEN_OK) return st;
    const size_t need = perm_carve(nullptr, p->N, p->max_population, nullptr);
    if (!workspace || workspace_bytes < need)
        return set_error(ROSEN_ENOMEM, "rosen_perm_run: workspace of %zu bytes < %zu needed",
                         workspace_bytes, need);
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return set_error(ROSEN_EINVAL, "rosen_perm_run: workspace must be 256-byte aligned");
    PermWs w;
    perm_carve(workspace, p->N, p->max_population, &w);
    cudaStream_t s = (cudaStream_t)stream;
    PermArgs a;
    memset(&a, 0, sizeof a);
    a.key = philox_keys(p->seed);
    a.ens = p->ensemble;
    a.N = p->N;
    a.max_pop = p->max_population;
    a.isaw = p->beta_eps != 0.0;
    for (int q = 0; q < 8; ++q) {
        a.wt64[q] = exp(p->beta_eps * (double)q);
        a.wt32[q] = (float)a.wt64[q];
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_perm_run: %s", cudaGetErrorString(e));
    const int64_t MP = p->max_population;
    const int H = perm_half_words(p->N);
    // Grid-stride kernels: the blocks the GPU holds at once.
    int resident = 0;
    e = a.isaw ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, perm_grow_kernel<true>,
                                                               kPermThreads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, perm_grow_kernel<false>,
                                                               kPermThreads, 0);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_perm_run: %s", cudaGetErrorString(e));
    const int grid = (int)std::min<int64_t>(
        std::min<int64_t>((int64_t)sms * std::max(resident, 1), kMaxParts),
        (MP + kPermThreads - 1) / kPermThreads);
    long long *population = reinterpret_cast<long long *>(o->population);
    perm_init_kernel<<<grid, kPermThreads, 0, s>>>(p->M0, MP, H, w.keys, w.ord[0], w.endk[0],
                                                   w.wm[0], w.we[0], w.free_slots, w.ctl,
                                                   population, o->logz, o->mean_r2);
    const double log_m0 = log((double)p->M0);
    double tm = 1.0;   // mu^i = tm 2^te
    int32_t te = 0;
    for (int i = 1; i < p->N; ++i) {
        {
            const double x = tm * p->mu;
            const int k = ilogb(x);
            tm = ldexp(x, -k);
            te += k;
        }
        const Threshold hi = make_threshold(p->c_hi, tm, te, true);
        const Threshold lo = make_threshold(p->c_lo, tm, te, false);
        const int b = (i - 1) & 1;      // this step's buffer; the next one is b ^ 1
        if (a.isaw)
            perm_grow_kernel<true><<<grid, kPermThreads, 0, s>>>(
                a, i, hi, lo, w.keys, H, w.ord[b], w.endk[b], w.wm[b], w.we[b], w.fate, w.chunks,
                w.ctl + b, w.parts, w.free_slots, w.ctl + 3);
        else
            perm_grow_kernel<false><<<grid, kPermThreads, 0, s>>>(
                a, i, hi, lo, w.keys, H, w.ord[b], w.endk[b], w.wm[b], w.we[b], w.fate, w.chunks,
                w.ctl + b, w.parts, w.free_slots, w.ctl + 3);
        perm_top_kernel<<<1, kTopThreads, 0, s>>>(i, MP, log_m0, w.chunks, w.ctl + b,
                                                  w.ctl + (b ^ 1), w.ctl + 2, w.ctl + 3,
                                                  w.ctl + 4, w.parts, grid, population, o->logz,
                                                  o->mean_r2);
        perm_scatter_kernel<<<grid, kPermThreads, 0, s>>>(
            i, H, w.keys, w.ord[b], w.ord[b ^ 1], w.endk[b], w.endk[b ^ 1], w.wm[b], w.we[b],
            w.wm[b ^ 1], w.we[b ^ 1], w.fate, w.chunks, w.ctl + b, w.ctl + 2, w.free_slots,
            w.ctl + 4);
    }
    const int fb = (p->N - 1) & 1;      // the buffer the last step wrote
    perm_final_kernel<<<grid, kPermThreads, 0, s>>>(
        p->N, MP, H, w.keys, w.ord[fb], w.wm[fb], w.we[fb], w.ctl + fb,
        reinterpret_cast<long long *>(o->final_n), o->w_m, o->w_e,
        (p->flags & ROSEN_STORE_COORDS) ? o->coords : nullptr);
    return check_launch("rosen_perm_run");
}
