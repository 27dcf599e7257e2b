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
// GB300 mapping.  The population lives in device memory as packed monomer
// keys [monomer][chain] (two buffers: the population of this step and the
// next), with each chain's weight as an FP64 mantissa in [1, 2) and an int32
// exponent, so every update is one correctly rounded product and every
// threshold comparison is exact.  A step is four launches, with no host
// synchronisation (the population size stays on the device):
//  1. perm_grow_kernel: one lane per chain (grid-stride over the
//     population) scans the chain's earlier keys with the displacement
//     table of the lattice kernels, takes the step (same draw, selection
//     and weight as rosen_lattice_grow), and decides its fate; per-block
//     partial sums of W and W R^2 for Eq. 9 / Eq. 2;
//  2. perm_tiles_kernel: an exclusive scan, per tile of 1024 chains, of the
//     packed counts (chains kept, enrichment requests);
//  3. perm_top_kernel (one block): the scan of the tile totals, the
//     population cap (the first max_pop - kept enrichment requests in
//     population order are granted), the next population size, and the
//     step's estimates from the partial sums;
//  4. perm_scatter_kernel: every kept chain (and its copy) is written to its
//     place in the next population, in order.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"
#include "lattice_step.cuh"

namespace rosen {
namespace {

constexpr int kPermThreads = 256;
constexpr int kScanTile = 1024;          // chains per scan tile (4 per thread)
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
    uint32_t *keys[2];          // [N][max_pop]
    double *wm[2];
    int32_t *we[2];
    int8_t *fate;               // 0 gone, 1 kept, 2 enrichment request, -1 pruning survivor
    unsigned long long *packed; // kept | enrichment request << 32
    unsigned long long *excl;   // in-tile exclusive prefix of packed
    unsigned long long *tiles;  // per tile: total, then exclusive offset
    PermPartial *parts;
    long long *ctl;             // [0], [1]: population of the two buffers; [2]: grants
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

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
    const size_t tiles = (P + kScanTile - 1) / kScanTile;
    PermWs t;
    for (int b = 0; b < 2; ++b) t.keys[b] = static_cast<uint32_t *>(take(4 * (size_t)N * P));
    for (int b = 0; b < 2; ++b) t.wm[b] = static_cast<double *>(take(8 * P));
    for (int b = 0; b < 2; ++b) t.we[b] = static_cast<int32_t *>(take(4 * P));
    t.fate = static_cast<int8_t *>(take(P));
    t.packed = static_cast<unsigned long long *>(take(8 * P));
    t.excl = static_cast<unsigned long long *>(take(8 * P));
    t.tiles = static_cast<unsigned long long *>(take(8 * tiles));
    t.parts = static_cast<PermPartial *>(take(sizeof(PermPartial) * kMaxParts));
    t.ctl = static_cast<long long *>(take(8 * 4));
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

__device__ __forceinline__ bool above(double wm, int32_t we, const Threshold &t)
{
    if (t.mode == 1) return false;
    if (t.mode == 2) return true;
    return we > t.e || (we == t.e && wm > t.m);
}

__device__ __forceinline__ bool below(double wm, int32_t we, const Threshold &t)
{
    if (t.mode != 0) return false;
    return we < t.e || (we == t.e && wm < t.m);
}

__global__ void perm_init_kernel(int64_t M0, int64_t max_pop, uint32_t *keys, double *wm,
                                 int32_t *we, long long *ctl, long long *population,
                                 double *logz, double *mean_r2)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M0; j += stride) {
        keys[j] = kOriginKey;
        wm[j] = 1.0;
        we[j] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl[0] = M0;
        ctl[1] = 0;
        ctl[2] = 0;
        population[0] = M0;
        logz[0] = 0.0;
        if (mean_r2) mean_r2[0] = 0.0;
    }
    (void)max_pop;
}

// Step i of every chain of the population (keys / wm / we of this step's
// buffer, population *pcount): growth, weight, fate, partial sums.
template <bool kIsaw>
__global__ void __launch_bounds__(kPermThreads) perm_grow_kernel(
    const PermArgs a, int i, Threshold hi, Threshold lo, uint32_t *keys, double *wm, int32_t *we,
    int8_t *fate, unsigned long long *packed, const long long *pcount, PermPartial *parts)
{
    __shared__ uint32_t lut[kLutWords];
    __shared__ uint8_t seltab[kSelBytes];
    __shared__ float wt32[8];
    __shared__ double wt64[8];
    __shared__ double red_s[kPermThreads / 32], red_r[kPermThreads / 32], red_g[kPermThreads / 32];
    __shared__ int32_t red_e[kPermThreads / 32];
    fill_tables(lut, seltab);
    if (threadIdx.x < 8) {
        wt32[threadIdx.x] = a.wt32[threadIdx.x];
        wt64[threadIdx.x] = a.wt64[threadIdx.x];
    }
    __syncthreads();
    const int64_t P = *pcount;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t MP = a.max_pop;
    int32_t emax = INT_MIN;     // running largest exponent of this lane's grown chains
    double s = 0.0, sr = 0.0, grown = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += stride) {
        uint32_t *col = keys + j;
        const uint32_t key = col[(int64_t)(i - 1) * MP];
        const uint32_t kb = kNearBias - key;
        uint32_t acc = 0u;
        if (kIsaw) {
            for (int q = 0; q <= i - 2; ++q) acc += lut_at(lut, lut_off(col[(int64_t)q * MP] + kb));
        } else {
            for (int q = i & 1; q <= i - 2; q += 2) acc += lut_at(lut, lut_off(col[(int64_t)q * MP] + kb));
        }
        const uint32_t freem = ~acc & 63u;
        const int m = __popc(freem);
        int8_t f = 0;
        if (m > 0) {
            const uint32_t x =
                philox(make_uint4((uint32_t)j, a.ens, (uint32_t)i, 0u), a.key).x;
            LogW lw_unused;
            const int sel = choose<kIsaw>(freem, m, acc, x, seltab, wt32, wt64, lw_unused);
            // The step's weight factor in FP64: m, or the sum of the free
            // neighbours' Boltzmann factors in slot order.
            double S;
            if (kIsaw) {
                S = 0.0;
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    const uint32_t cd = (acc >> (8 + 3 * d)) & 7u;
                    S = __dadd_rn(S, ((freem >> d) & 1u) ? wt64[cd] : 0.0);
                }
            } else {
                S = (double)m;
            }
            const uint32_t axis_step = 1u << (10 * (sel >> 1));
            const uint32_t nk = (sel & 1) ? key - axis_step : key + axis_step;
            col[(int64_t)i * MP] = nk;
            double m_;
            int32_t e_;
            norm_weight(__dmul_rn(wm[j], S), m_, e_);
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
                const double sc = emax == INT_MIN ? 0.0 : ldexp(1.0, emax - e_new);
                s *= sc;
                sr *= sc;
                emax = e_new;
            }
            const double w = ldexp(m_, e_new - emax);
            s += w;
            sr += w * R2;
            grown += 1.0;
        }
        fate[j] = f;
        packed[j] = (unsigned long long)(f != 0) | ((unsigned long long)(f == 2) << 32);
    }
    // Block partial: the largest exponent, then the sums rescaled to it.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

// Exclusive scan of the packed counts inside tile blockIdx.x (1024 chains,
// 4 per thread); the tile's total goes to tiles[tile].
__global__ void __launch_bounds__(kPermThreads) perm_tiles_kernel(
    const unsigned long long *packed, const long long *pcount, unsigned long long *excl,
    unsigned long long *tiles)
{
    __shared__ unsigned long long wsum[kPermThreads / 32];
    const int64_t P = *pcount;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= P) return;
    const int64_t j0 = base + 4 * (int64_t)threadIdx.x;
    unsigned long long v[4], run = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[r] = (j0 + r < P) ? packed[j0 + r] : 0ull;
        const unsigned long long t = v[r];
        v[r] = run;               // exclusive within the thread
        run += t;
    }
    // Exclusive scan of the threads' totals.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned long long woff = 0, total = 0;
    for (int q = 0; q < kPermThreads / 32; ++q) {
        if (q < warp) woff += wsum[q];
        total += wsum[q];
    }
    const unsigned long long off = woff + incl - run;
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (j0 + r < P) excl[j0 + r] = off + v[r];
    if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

// One block: the tiles' offsets, the cap, the next population size, and the
// estimates of length i from the grow kernel's partials.
__global__ void __launch_bounds__(kTopThreads) perm_top_kernel(
    int i, int64_t max_pop, double log_m0, unsigned long long *tiles, const long long *pcount,
    long long *pnext, long long *grants, const PermPartial *parts, int nparts,
    long long *population, double *logz, double *mean_r2)
{
    __shared__ unsigned long long wsum[kTopThreads / 32];
    __shared__ double rs[kTopThreads / 32], rr[kTopThreads / 32], rg[kTopThreads / 32];
    __shared__ int32_t re[kTopThreads / 32];
    const int64_t P = *pcount;
    const int64_t ntiles = (P + kScanTile - 1) / kScanTile;
    const int64_t per = (ntiles + kTopThreads - 1) / kTopThreads;
    const int64_t t0 = (int64_t)threadIdx.x * per;
    unsigned long long run = 0;
    for (int64_t t = t0; t < t0 + per && t < ntiles; ++t) run += tiles[t];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned long long woff = 0, total = 0;
    for (int q = 0; q < kTopThreads / 32; ++q) {
        if (q < warp) woff += wsum[q];
        total += wsum[q];
    }
    unsigned long long off = woff + incl - run;
    for (int64_t t = t0; t < t0 + per && t < ntiles; ++t) {
        const unsigned long long v = tiles[t];
        tiles[t] = off;
        off += v;
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
    if (threadIdx.x == 0) {
        s = sr = g = 0.0;
        for (int q = 0; q < kTopThreads / 32; ++q) {
            s += rs[q];
            sr += rr[q];
            g += rg[q];
        }
        const long long base = (long long)(total & 0xFFFFFFFFull);
        const long long extra = (long long)(total >> 32);
        const long long G = max_pop - base > 0 ? max_pop - base : 0;
        const long long Pn = base + (extra < G ? extra : G);
        *pnext = Pn;
        *grants = G;
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

// Kept chains, in population order, to their places in the next buffer.
__global__ void __launch_bounds__(kPermThreads) perm_scatter_kernel(
    int i, int64_t max_pop, const uint32_t *keys, uint32_t *keys_n, const double *wm,
    const int32_t *we, double *wm_n, int32_t *we_n, const int8_t *fate,
    const unsigned long long *excl, const unsigned long long *tiles, const long long *pcount,
    const long long *grants)
{
    const int64_t P = *pcount;
    const long long G = *grants;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += stride) {
        const int f = fate[j];
        if (f == 0) continue;
        const unsigned long long e = excl[j] + tiles[j / kScanTile];
        const long long kept_before = (long long)(e & 0xFFFFFFFFull);
        const long long rank = (long long)(e >> 32);
        const long long dst = kept_before + (rank < G ? rank : G);
        const int copies = (f == 2 && rank < G) ? 2 : 1;
        const int32_t w_e = we[j] + (copies == 2 ? -1 : (f == -1 ? 1 : 0));
        for (int c = 0; c < copies; ++c) {
            wm_n[dst + c] = wm[j];
            we_n[dst + c] = w_e;
        }
        for (int q = 0; q <= i; ++q) {
            const uint32_t k = keys[(int64_t)q * max_pop + j];
            for (int c = 0; c < copies; ++c) keys_n[(int64_t)q * max_pop + dst + c] = k;
        }
    }
}

// The final population to the caller's arrays.
__global__ void perm_final_kernel(int N, int64_t max_pop, const uint32_t *keys, const double *wm,
                                  const int32_t *we, const long long *pcount, long long *final_n,
                                  double *w_m, int32_t *w_e, int32_t *coords)
{
    const int64_t P = *pcount;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *final_n = P;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P; c += stride) {
        if (w_m) w_m[c] = wm[c];
        if (w_e) w_e[c] = we[c];
        if (coords)
            for (int q = 0; q < N; ++q) {
                const uint32_t k = keys[(int64_t)q * max_pop + c];
                coords[((int64_t)q * 3 + 0) * max_pop + c] = (int32_t)(k & 1023u) - 512;
                coords[((int64_t)q * 3 + 1) * max_pop + c] = (int32_t)((k >> 10) & 1023u) - 512;
                coords[((int64_t)q * 3 + 2) * max_pop + c] = (int32_t)(k >> 20) - 512;
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
    const int grid = (int)std::min<int64_t>(std::min<int64_t>((int64_t)sms * 8, kMaxParts),
                                            (MP + kPermThreads - 1) / kPermThreads);
    const unsigned tiles = (unsigned)((MP + kScanTile - 1) / kScanTile);
    long long *population = reinterpret_cast<long long *>(o->population);
    perm_init_kernel<<<grid, kPermThreads, 0, s>>>(p->M0, MP, w.keys[0], w.wm[0], w.we[0], w.ctl,
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
                a, i, hi, lo, w.keys[b], w.wm[b], w.we[b], w.fate, w.packed, w.ctl + b, w.parts);
        else
            perm_grow_kernel<false><<<grid, kPermThreads, 0, s>>>(
                a, i, hi, lo, w.keys[b], w.wm[b], w.we[b], w.fate, w.packed, w.ctl + b, w.parts);
        perm_tiles_kernel<<<tiles, kPermThreads, 0, s>>>(w.packed, w.ctl + b, w.excl, w.tiles);
        perm_top_kernel<<<1, kTopThreads, 0, s>>>(i, MP, log_m0, w.tiles, w.ctl + b,
                                                  w.ctl + (b ^ 1), w.ctl + 2, w.parts, grid,
                                                  population, o->logz, o->mean_r2);
        perm_scatter_kernel<<<grid, kPermThreads, 0, s>>>(
            i, MP, w.keys[b], w.keys[b ^ 1], w.wm[b], w.we[b], w.wm[b ^ 1], w.we[b ^ 1], w.fate,
            w.excl, w.tiles, w.ctl + b, w.ctl + 2);
    }
    const int fb = (p->N - 1) & 1;      // the buffer the last step wrote
    perm_final_kernel<<<grid, kPermThreads, 0, s>>>(
        p->N, MP, w.keys[fb], w.wm[fb], w.we[fb], w.ctl + fb,
        reinterpret_cast<long long *>(o->final_n), o->w_m, o->w_e,
        (p->flags & ROSEN_STORE_COORDS) ? o->coords : nullptr);
    return check_launch("rosen_perm_run");
}
