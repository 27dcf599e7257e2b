// lattice.cu -- Rosenbluth growth on the simple cubic lattice
// (Guo & Baulin, Section 3.3.2, Algorithm 1; weight of Eq. 3).
//
// GB300 mapping: one chain per lane.  A warp grows 32 chains in lock-step
// (every chain is at the same step i), so the overlap scan over the earlier
// monomers has a warp-uniform trip count and no divergence.  The chain lives
// in shared memory as one packed 32-bit key per monomer,
//     key = (x + 512) | (y + 512) << 10 | (z + 512) << 20,
// stored [monomer][lane] so that a warp's 32 loads of monomer j hit 32
// different banks.  For every earlier monomer j the kernel forms
//     t = key_j - key_end + (2, 2, 2)
// with one integer add: t is the packed displacement (dx+2, dy+2, dz+2) and
// it fits three 3-bit fields exactly when the monomer lies in the 5x5x5 box
// around the end (|d| <= 511 on every axis keeps the fields from borrowing
// into each other).  One multiply gathers the three fields into the byte
// offset of an entry of a 512-entry table (lattice_step.cuh) that turns the
// displacement into "occupies neighbour d" bits and "touches neighbour d"
// contact increments.  Monomers outside the box read the all-zero entry
// 511, so the scan has no branch; the entries are simply added (a site holds
// one monomer, so the occupancy bits never carry).  Parity halves the
// athermal scan: only monomers j with j = i (mod 2) can sit on a neighbour
// of the end.
//
// Selection: athermal steps take the idx-th free neighbour with
// idx = floor(x * m / 2^32).  Interacting steps draw r = u24(x) * S in FP32
// and take the smallest slot whose prefix sum exceeds r; when r lies within
// 2^-18 S of one of the chosen slot's bounds the choice is recomputed in FP64
// with exactly the sequential FP64 arithmetic, so the path never depends on
// FP32 rounding.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"
#include "lattice_step.cuh"

namespace rosen {
namespace {

// 16-byte key groups per parity and lane: ceil(ceil(N / 2) / 4).
__host__ __device__ __forceinline__ int key_groups(int N) { return ((N + 1) / 2 + 3) / 4; }


// Growth number att of chain c (local index) of the ensemble described by a,
// in this lane.  The keys sit in 16-byte groups of four monomers, the lane's
// groups B apart, so one 128-bit load brings four keys and the 32 lanes of a
// warp read 512 contiguous bytes (no bank conflict).  The interacting scan
// reads every monomer: key j is word j % 4 of group j / 4 ([j / 4][lane]
// [j % 4]).  The athermal scan reads one parity: key j (p = j % 2, h = j / 2)
// is word h % 4 of group h / 4 of parity p, the parities key_groups(N)
// groups apart ([p][h / 4][lane][h % 4]).  my points at the lane's first
// group.  Returns true when the growth was trapped and another
// attempt is allowed (restart mode): the caller grows the chain again with
// att + 1 (the outputs then hold nothing final for it).  Otherwise the
// chain's outputs are written and false is returned.
// kB > 0 fixes the stride at compile time (immediate load offsets).
template <bool kIsaw, int kB = 0>
__device__ __forceinline__ bool lattice_attempt(const LatticeArgs &a, int64_t c, uint32_t att,
                                                uint32_t *my, int B_, const uint32_t *lut,
                                                const uint8_t *seltab, const float *wt32,
                                                const double *wt64)
{
    const int B = kB > 0 ? kB : B_;
    const uint32_t chain = a.chain0 + (uint32_t)c;
    const int N = a.N;
    const int64_t C = a.C;

    uint32_t key;
    int sx, sy, sz, sq;
    int ex, ey, ez;
    uint64_t cnt;      // 9-bit field m holds the number of steps with m free sites
    LogW lw;      // interacting: product of the step factors
    int dead_at;
    if (a.coords && att == 0) {
        a.coords[(0 * 3 + 0) * C + c] = 0;
        a.coords[(0 * 3 + 1) * C + c] = 0;
        a.coords[(0 * 3 + 2) * C + c] = 0;
    }
    {
        key = kOriginKey;
        my[0] = key;
        const uint4 *m4 = reinterpret_cast<const uint4 *>(my);
        const int pstride = key_groups(N) * B;   // groups between the parities
        sx = sy = sz = sq = 0;
        ex = ey = ez = 0;
        cnt = 0;
        lw = LogW();
        dead_at = 0;

        for (int i = 1; i < N; ++i) {
            uint32_t acc = 0u;
            const uint32_t kb = kNearBias - key;
            // Interacting: monomers 0 .. i-2.  Athermal: only monomers
            // j = i (mod 2) can sit on a neighbour of the end; of that parity
            // q, monomers 0 .. i-2 hold (i - q) / 2 keys.
            const int q = i & 1;
            const int n = kIsaw ? i - 1 : (i - q) >> 1;
            const uint4 *src = kIsaw ? m4 : m4 + q * pstride;
            const int full = n >> 2, rem = n & 3;
#pragma unroll 2
            for (int g = 0; g < full; ++g) {
                const uint4 v = src[g * B];
                acc += lut_at(lut, lut_off(v.x + kb)) + lut_at(lut, lut_off(v.y + kb)) +
                       lut_at(lut, lut_off(v.z + kb)) + lut_at(lut, lut_off(v.w + kb));
            }
            if (rem) {
                const uint4 v = src[full * B];
                acc += lut_at(lut, lut_off(v.x + kb));
                if (rem > 1) acc += lut_at(lut, lut_off(v.y + kb));
                if (rem > 2) acc += lut_at(lut, lut_off(v.z + kb));
            }
            const uint32_t freem = ~acc & 63u;
            const int m = __popc(freem);
            if (m == 0) {
                dead_at = i;
                break;
            }
            const uint32_t x = philox(make_uint4(chain, a.ens, (uint32_t)i | (att << 16), 0u), a.key).x;
            const int sel = choose<kIsaw>(freem, m, acc, x, seltab, wt32, wt64, lw);
            cnt += 1ull << (9 * m);
            const uint32_t axis_step = 1u << (10 * (sel >> 1));
            key = (sel & 1) ? key - axis_step : key + axis_step;
            if (kIsaw) my[(i >> 2) * 4 * B + (i & 3)] = key;
            else my[((i & 1) * pstride + (i >> 3) * B) * 4 + ((i >> 1) & 3)] = key;
            ex = (int)(key & 1023u) - 512;
            ey = (int)((key >> 10) & 1023u) - 512;
            ez = (int)(key >> 20) - 512;
            sx += ex;
            sy += ey;
            sz += ez;
            sq += ex * ex + ey * ey + ez * ez;
            if (a.trace) a.trace[(int64_t)(i - 1) * C + c] = (uint8_t)((m << 3) | sel);
            if (a.coords) {
                a.coords[((int64_t)i * 3 + 0) * C + c] = ex;
                a.coords[((int64_t)i * 3 + 1) * C + c] = ey;
                a.coords[((int64_t)i * 3 + 2) * C + c] = ez;
            }
        }
    }
    if (dead_at && att + 1 < a.max_att) return true;
    if (a.attempts) a.attempts[c] = (uint16_t)(att + 1);
    if (dead_at) cnt += 1ull;   // counts[0] = 1 marks the dead end
    uint32_t cm[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) cm[q] = (uint32_t)(cnt >> (9 * q)) & 511u;
    if (a.counts)
        a.counts[c] = make_uint4(cm[0] | (cm[1] << 16), cm[2] | (cm[3] << 16),
                                 cm[4] | (cm[5] << 16), cm[6]);
    if (dead_at) {
        // Trapped (in every attempt made): W = 0 is kept and the counts of
        // the steps before the dead end stay recorded.
        if (a.logw) a.logw[c] = -INFINITY;
        if (a.r2) a.r2[c] = 0;
        if (a.n2rg2) a.n2rg2[c] = 0;
        if (a.trace) {
            a.trace[(int64_t)(dead_at - 1) * C + c] = 7u;
            for (int i = dead_at + 1; i < N; ++i) a.trace[(int64_t)(i - 1) * C + c] = 0xFFu;
        }
        if (a.coords)
            for (int i = dead_at; i < N; ++i)
                for (int q = 0; q < 3; ++q) a.coords[((int64_t)i * 3 + q) * C + c] = 0;
        return false;
    }
    float logw;
    if (!kIsaw) {
        logw = 0.f;
#pragma unroll
        for (int q = 2; q <= 6; ++q) logw += (float)cm[q] * a.logm[q];
    } else {
        logw = lw.value();
    }
    if (a.logw) a.logw[c] = logw;
    if (a.r2) a.r2[c] = ex * ex + ey * ey + ez * ez;
    if (a.n2rg2)
        a.n2rg2[c] = (int64_t)N * sq -
                     ((int64_t)sx * sx + (int64_t)sy * sy + (int64_t)sz * sz);
    return false;
}

// Every growth of chain c in this lane (restart mode regrows in place).
template <bool kIsaw, int kB = 0>
__device__ __forceinline__ void lattice_chain(const LatticeArgs &a, int64_t c, uint32_t *my, int B,
                                              const uint32_t *lut, const uint8_t *seltab,
                                              const float *wt32, const double *wt64)
{
    uint32_t att = 0;
    while (lattice_attempt<kIsaw, kB>(a, c, att, my, B, lut, seltab, wt32, wt64)) ++att;
}


// Local chains [c_lo, c_hi) of the ensemble, one per lane (a call grows
// [0, C); the server grows a request in slices of chain ranges).  kB > 0:
// blocks of exactly kB threads (the key stride known at compile time).
template <bool kIsaw, int kB = 0>
__global__ void __launch_bounds__(256) lattice_lane_kernel(const LatticeArgs a, int64_t c_lo,
                                                           int64_t c_hi)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *lut = smem;
    uint8_t *seltab = reinterpret_cast<uint8_t *>(smem + kLutWords);
    float *wt32 = reinterpret_cast<float *>(smem + kLutWords + kSelBytes / 4);
    double *wt64 = reinterpret_cast<double *>(smem + kLutWords + kSelBytes / 4 + 8);
    uint32_t *keys = smem + kLutWords + kSelBytes / 4 + 8 + 16;

    fill_tables(lut, seltab);
    if (threadIdx.x < 8) {
        wt32[threadIdx.x] = a.wt32[threadIdx.x];
        wt64[threadIdx.x] = a.wt64[threadIdx.x];
    }
    __syncthreads();

    const int B = kB > 0 ? kB : (int)blockDim.x;
    const int64_t c = c_lo + (int64_t)blockIdx.x * B + threadIdx.x;
    if (c >= c_hi) return;
    lattice_chain<kIsaw, kB>(a, c, keys + 4 * threadIdx.x, B, lut, seltab, wt32, wt64);
}

// Restart mode, single ensemble: a persistent kernel in which every warp owns
// a contiguous range of chains and grows 32 of them per pass in lock-step.
// A chain whose growth is trapped goes into the warp's retry queue (at most
// 32 entries, in shared memory) and is grown again, with the next attempt
// index, in the warp's next pass next to fresh chains.  No lane waits for a
// regrowth while the others idle, and no block waits for one warp.
template <bool kIsaw>
__global__ void __launch_bounds__(256) lattice_retry_kernel(const LatticeArgs a, int64_t per_warp,
                                                            int64_t c_lo, int64_t c_hi)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *lut = smem;
    uint8_t *seltab = reinterpret_cast<uint8_t *>(smem + kLutWords);
    float *wt32 = reinterpret_cast<float *>(smem + kLutWords + kSelBytes / 4);
    double *wt64 = reinterpret_cast<double *>(smem + kLutWords + kSelBytes / 4 + 8);
    const int wpb = blockDim.x / 32, wib = threadIdx.x / 32, lane = threadIdx.x & 31;
    uint32_t *rq = smem + kLutWords + kSelBytes / 4 + 8 + 16 + (size_t)wib * 64;   // [2][32]
    uint32_t *keys = smem + kLutWords + kSelBytes / 4 + 8 + 16 + (size_t)wpb * 64 +
                     (size_t)wib * key_groups(a.N) * 2 * 4 * 32;

    fill_tables(lut, seltab);
    if (threadIdx.x < 8) {
        wt32[threadIdx.x] = a.wt32[threadIdx.x];
        wt64[threadIdx.x] = a.wt64[threadIdx.x];
    }
    __syncthreads();

    const int64_t w = (int64_t)blockIdx.x * wpb + wib;
    const int64_t hi = c_lo + (w + 1) * per_warp < c_hi ? c_lo + (w + 1) * per_warp : c_hi;
    int64_t next = c_lo + w * per_warp;
    int queued = 0;          // warp-uniform
    for (;;) {
        const int take = queued;
        const int64_t left = hi > next ? hi - next : 0;
        const int fresh = left < 32 - take ? (int)left : 32 - take;
        if (take + fresh == 0) break;
        int64_t c = -1;
        uint32_t att = 0;
        if (lane < take) {
            c = (int64_t)rq[lane];
            att = rq[32 + lane];
        } else if (lane < take + fresh) {
            c = next + (lane - take);
        }
        next += fresh;
        __syncwarp();
        const bool retry =
            c >= 0 && lattice_attempt<kIsaw, 32>(a, c, att, keys + 4 * lane, 32, lut, seltab,
                                                 wt32, wt64);
        const unsigned m = __ballot_sync(0xffffffffu, retry);
        if (retry) {
            const int pos = __popc(m & ((1u << lane) - 1u));
            rq[pos] = (uint32_t)c;
            rq[32 + pos] = att + 1;
        }
        queued = __popc(m);
        __syncwarp();
    }
}

// Persistent batch kernel: blocks take (ensemble, chain range) items from a
// queue (items sorted by decreasing cost) until it is empty; every chain is
// grown by the same lattice_chain code as in the single-ensemble kernel, so
// its results do not depend on the batch it is grown in.
__global__ void __launch_bounds__(256) lattice_batch_kernel(const LatticeArgs *__restrict__ ens,
                                                            const BatchItem *__restrict__ items,
                                                            int n_items, int *head)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ LatticeArgs sa;
    __shared__ int s_item;
    uint32_t *lut = smem;
    uint8_t *seltab = reinterpret_cast<uint8_t *>(smem + kLutWords);
    float *wt32 = reinterpret_cast<float *>(smem + kLutWords + kSelBytes / 4);
    double *wt64 = reinterpret_cast<double *>(smem + kLutWords + kSelBytes / 4 + 8);
    uint32_t *keys = smem + kLutWords + kSelBytes / 4 + 8 + 16;
    fill_tables(lut, seltab);
    const int B = blockDim.x;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const BatchItem bi = items[it];
        constexpr int kWords = (int)(sizeof(LatticeArgs) / 4);
        for (int q = threadIdx.x; q < kWords; q += B)
            reinterpret_cast<uint32_t *>(&sa)[q] = reinterpret_cast<const uint32_t *>(&ens[bi.ens])[q];
        __syncthreads();
        if (threadIdx.x < 8) {
            wt32[threadIdx.x] = sa.wt32[threadIdx.x];
            wt64[threadIdx.x] = sa.wt64[threadIdx.x];
        }
        __syncthreads();
        if (threadIdx.x < (int)bi.n) {
            if (sa.isaw)
                lattice_chain<true>(sa, bi.c0 + threadIdx.x, keys + 4 * threadIdx.x, B, lut, seltab,
                                    wt32, wt64);
            else
                lattice_chain<false>(sa, bi.c0 + threadIdx.x, keys + 4 * threadIdx.x, B, lut, seltab,
                                     wt32, wt64);
        }
        __syncthreads();
    }
}

// ---- long chains: occupancy bitmaps in a per-chain hash table in HBM -------
//
// Beyond a few hundred monomers the O(i) scan of the shared-memory kernel
// dominates and the packed 10-bit keys run out.  Here every lane keeps its
// chain's occupied sites in an open-addressing hash table (linear probing)
// in device memory, one 16-byte entry per 4x4x4 block of sites: the block's
// key and a 64-bit occupancy bitmap (bit (x & 3) | (y & 3) << 2 | (z & 3) << 4).
// A step reads only the blocks its neighbourhood touches: the end's block
// and, per axis, the neighbouring block the neighbours (athermal, about 2.5
// blocks per step on average) or the sites at lattice distance <= 2
// (interacting, about 4.75) cross into -- one 16-byte load each.  Block keys
// pack 16 bits per axis; bits 48..63 of the key word hold the generation of
// the growth that wrote it, so a lane reuses its table for the next chain
// without clearing it (older generations read as empty).  A chain occupies at
// most N blocks and a table holds more than N entries, so every probe
// sequence ends at an empty slot.
constexpr int kGenShift = 48;
constexpr uint64_t kBlockMask = (1ull << kGenShift) - 1ull;
constexpr uint32_t kGenMax = 65535;

__device__ __forceinline__ uint64_t block_key(int bx, int by, int bz)
{
    return (uint64_t)(uint32_t)(bx + 32768) | ((uint64_t)(uint32_t)(by + 32768) << 16) |
           ((uint64_t)(uint32_t)(bz + 32768) << 32);
}

__device__ __forceinline__ uint32_t block_slot(uint64_t key, int logH)
{
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - logH));
}

// A block found (or not) in the table: its bitmap, the slot holding it (or
// the empty slot where it would go) and whether it exists.
struct BlockRef {
    uint64_t bits;
    uint32_t h;
    bool found;
};

// Continue the probe for tagged key `want` that read entry e at slot h.
__device__ __forceinline__ BlockRef block_rest(const ulonglong2 *tab, uint32_t hmask, uint64_t want,
                                               uint64_t tag, uint32_t h, ulonglong2 e)
{
    while ((e.x & ~kBlockMask) == tag) {
        if (e.x == want) return BlockRef{e.y, h, true};
        h = (h + 1u) & hmask;
        e = tab[h];
    }
    return BlockRef{0ull, h, false};
}

// Bit of the site at offset (dx, dy, dz) from the end, whose position in its
// block is (qx, qy, qz); the block offset along an axis is 0 or the axis's
// side s (the neighbouring block the neighbourhood reaches on that axis).
__device__ __forceinline__ uint32_t site_bit(int qx, int qy, int qz, int dx, int dy, int dz,
                                             uint64_t b0, uint64_t bx, uint64_t by, uint64_t bz,
                                             uint64_t bxy, uint64_t bxz, uint64_t byz)
{
    const int px = qx + dx, py = qy + dy, pz = qz + dz;
    const bool ox = (unsigned)px > 3u, oy = (unsigned)py > 3u, oz = (unsigned)pz > 3u;
    const uint64_t m = ox ? (oy ? bxy : (oz ? bxz : bx)) : (oy ? (oz ? byz : by) : (oz ? bz : b0));
    return (uint32_t)(m >> ((px & 3) | ((py & 3) << 2) | ((pz & 3) << 4))) & 1u;
}

// Growth number att of chain c with the sites in the lane's table tab
// (2^logH entries).  Same rule, draws and outputs as lattice_attempt.
template <bool kIsaw>
__device__ __forceinline__ bool long_attempt(const LatticeArgs &a, int64_t c, uint32_t att,
                                             ulonglong2 *tab, int logH, uint32_t &gen,
                                             const uint8_t *seltab, const float *wt32,
                                             const double *wt64)
{
    const uint32_t chain = a.chain0 + (uint32_t)c;
    const int N = a.N;
    const int64_t C = a.C;
    const uint32_t hmask = (1u << logH) - 1u;

    if (++gen > kGenMax) {          // generation tags exhausted: clear the table
        for (uint32_t h = 0; h <= hmask; ++h) tab[h] = make_ulonglong2(0ull, 0ull);
        gen = 1;
    }
    const uint64_t tag = (uint64_t)gen << kGenShift;
    {
        const uint64_t want = block_key(0, 0, 0) | tag;
        uint32_t h = block_slot(want & kBlockMask, logH);
        while ((tab[h].x & ~kBlockMask) == tag) h = (h + 1u) & hmask;
        tab[h] = make_ulonglong2(want, 1ull);     // site (0,0,0): bit 0
    }
    if (a.coords && att == 0) {
        a.coords[(0 * 3 + 0) * C + c] = 0;
        a.coords[(0 * 3 + 1) * C + c] = 0;
        a.coords[(0 * 3 + 2) * C + c] = 0;
    }
    int ex = 0, ey = 0, ez = 0;
    int64_t sx = 0, sy = 0, sz = 0, sq = 0;
    uint64_t cnt_lo = 0ull, cnt_hi = 0ull;   // 16-bit fields: m = 0..3 | 4..7
    LogW lw;      // interacting: product of the step factors
    int dead_at = 0;

    for (int i = 1; i < N; ++i) {
        const int bx0 = ex >> 2, by0 = ey >> 2, bz0 = ez >> 2;
        const int qx = ex & 3, qy = ey & 3, qz = ez & 3;
        // The neighbouring block per axis: athermal steps need it only when
        // the end sits on a face of its block, interacting steps always.
        const int sx_ = qx <= 1 ? -1 : 1, sy_ = qy <= 1 ? -1 : 1, sz_ = qz <= 1 ? -1 : 1;
        const bool need_x = kIsaw || qx == 0 || qx == 3;
        const bool need_y = kIsaw || qy == 0 || qy == 3;
        const bool need_z = kIsaw || qz == 0 || qz == 3;
        const bool fx = qx == 0 || qx == 3, fy = qy == 0 || qy == 3, fz = qz == 0 || qz == 3;
        const bool need_xy = kIsaw && fx && fy, need_xz = kIsaw && fx && fz,
                   need_yz = kIsaw && fy && fz;
        uint64_t want[7];
        bool need[7];
        want[0] = block_key(bx0, by0, bz0) | tag;
        want[1] = block_key(bx0 + sx_, by0, bz0) | tag;
        want[2] = block_key(bx0, by0 + sy_, bz0) | tag;
        want[3] = block_key(bx0, by0, bz0 + sz_) | tag;
        want[4] = block_key(bx0 + sx_, by0 + sy_, bz0) | tag;
        want[5] = block_key(bx0 + sx_, by0, bz0 + sz_) | tag;
        want[6] = block_key(bx0, by0 + sy_, bz0 + sz_) | tag;
        need[0] = true;
        need[1] = need_x;
        need[2] = need_y;
        need[3] = need_z;
        need[4] = need_xy;
        need[5] = need_xz;
        need[6] = need_yz;
        uint32_t h[7];
        ulonglong2 e[7];
        constexpr int kB = kIsaw ? 7 : 4;
#pragma unroll
        for (int q = 0; q < kB; ++q) {
            h[q] = block_slot(want[q] & kBlockMask, logH);
            e[q] = need[q] ? tab[h[q]] : make_ulonglong2(0ull, 0ull);
        }
        BlockRef ref[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q)
            ref[q] = need[q] ? block_rest(tab, hmask, want[q], tag, h[q], e[q])
                             : BlockRef{0ull, 0u, false};
        const uint64_t b0 = ref[0].bits, bxm = ref[1].bits, bym = ref[2].bits, bzm = ref[3].bits;
        const uint64_t bxy = kIsaw ? ref[4 < kB ? 4 : 0].bits : 0ull;
        const uint64_t bxz = kIsaw ? ref[5 < kB ? 5 : 0].bits : 0ull;
        const uint64_t byz = kIsaw ? ref[6 < kB ? 6 : 0].bits : 0ull;

        uint32_t occ = 0u, acc;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const int ux = d == 0 ? 1 : (d == 1 ? -1 : 0);
            const int uy = d == 2 ? 1 : (d == 3 ? -1 : 0);
            const int uz = d == 4 ? 1 : (d == 5 ? -1 : 0);
            occ |= site_bit(qx, qy, qz, ux, uy, uz, b0, bxm, bym, bzm, bxy, bxz, byz) << d;
        }
        acc = occ;
        if (kIsaw) {
            // Contacts of neighbour d: occupied sites next to it other than
            // the end (its far site and the four beside it).
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const int ux = d == 0 ? 1 : (d == 1 ? -1 : 0);
                const int uy = d == 2 ? 1 : (d == 3 ? -1 : 0);
                const int uz = d == 4 ? 1 : (d == 5 ? -1 : 0);
                uint32_t cd = 0u;
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    if (f == (d ^ 1)) continue;    // back to the end
                    const int vx = f == 0 ? 1 : (f == 1 ? -1 : 0);
                    const int vy = f == 2 ? 1 : (f == 3 ? -1 : 0);
                    const int vz = f == 4 ? 1 : (f == 5 ? -1 : 0);
                    cd += site_bit(qx, qy, qz, ux + vx, uy + vy, uz + vz, b0, bxm, bym, bzm, bxy,
                                   bxz, byz);
                }
                acc |= cd << (8 + 3 * d);
            }
        }
        const uint32_t freem = ~occ & 63u;
        const int m = __popc(freem);
        if (m == 0) {
            dead_at = i;
            break;
        }
        const uint32_t x = philox(make_uint4(chain, a.ens, (uint32_t)i | (att << 16), 0u), a.key).x;
        const int sel = choose<kIsaw>(freem, m, acc, x, seltab, wt32, wt64, lw);
        if (m < 4) cnt_lo += 1ull << (16 * m);
        else cnt_hi += 1ull << (16 * (m - 4));
        const int step = (sel & 1) ? -1 : 1;
        if ((sel >> 1) == 0) ex += step;
        else if ((sel >> 1) == 1) ey += step;
        else ez += step;
        // Set the new site's bit in its block (the end's block or the
        // neighbouring block of the axis moved along).
        const int ax = sel >> 1;
        const bool out = ax == 0 ? (unsigned)(qx + step) > 3u
                                 : (ax == 1 ? (unsigned)(qy + step) > 3u : (unsigned)(qz + step) > 3u);
        BlockRef r = ref[0];
        uint64_t key = want[0];
        if (out) {
            r = ax == 0 ? ref[1] : (ax == 1 ? ref[2] : ref[3]);
            key = ax == 0 ? want[1] : (ax == 1 ? want[2] : want[3]);
        }
        const uint64_t bit = 1ull << ((ex & 3) | ((ey & 3) << 2) | ((ez & 3) << 4));
        if (r.found) tab[r.h].y = r.bits | bit;
        else tab[r.h] = make_ulonglong2(key, bit);
        sx += ex;
        sy += ey;
        sz += ez;
        sq += (int64_t)ex * ex + (int64_t)ey * ey + (int64_t)ez * ez;
        if (a.trace) a.trace[(int64_t)(i - 1) * C + c] = (uint8_t)((m << 3) | sel);
        if (a.coords) {
            a.coords[((int64_t)i * 3 + 0) * C + c] = ex;
            a.coords[((int64_t)i * 3 + 1) * C + c] = ey;
            a.coords[((int64_t)i * 3 + 2) * C + c] = ez;
        }
    }
    if (dead_at && att + 1 < a.max_att) return true;
    if (a.attempts) a.attempts[c] = (uint16_t)(att + 1);
    if (dead_at) cnt_lo += 1ull;   // counts[0] = 1 marks the dead end
    if (a.counts)
        a.counts[c] = make_uint4((uint32_t)cnt_lo, (uint32_t)(cnt_lo >> 32), (uint32_t)cnt_hi,
                                 (uint32_t)(cnt_hi >> 32));
    if (dead_at) {
        if (a.logw) a.logw[c] = -INFINITY;
        if (a.r2) a.r2[c] = 0;
        if (a.n2rg2) a.n2rg2[c] = 0;
        if (a.trace) {
            a.trace[(int64_t)(dead_at - 1) * C + c] = 7u;
            for (int i = dead_at + 1; i < N; ++i) a.trace[(int64_t)(i - 1) * C + c] = 0xFFu;
        }
        if (a.coords)
            for (int i = dead_at; i < N; ++i)
                for (int q = 0; q < 3; ++q) a.coords[((int64_t)i * 3 + q) * C + c] = 0;
        return false;
    }
    float logw;
    if (!kIsaw) {
        logw = 0.f;
#pragma unroll
        for (int q = 2; q <= 6; ++q) {
            const uint32_t cm = (uint32_t)(((q < 4 ? cnt_lo : cnt_hi) >> (16 * (q & 3))) & 0xFFFFu);
            logw += (float)cm * a.logm[q];
        }
    } else {
        logw = lw.value();
    }
    if (a.logw) a.logw[c] = logw;
    if (a.r2) a.r2[c] = ex * ex + ey * ey + ez * ez;
    if (a.n2rg2) a.n2rg2[c] = (int64_t)N * sq - (sx * sx + sy * sy + sz * sz);
    return false;
}

// One lane per chain at a time, in its own table (2^logH entries at
// ws + l 2^logH for lane l); each lane takes its next chain from the counter
// *next as soon as it is done, so lanes whose chains die early take more.
template <bool kIsaw>
__global__ void __launch_bounds__(256) lattice_long_kernel(const LatticeArgs a, ulonglong2 *ws,
                                                           int64_t lanes, int logH,
                                                           unsigned long long *next)
{
    __shared__ uint8_t seltab[kSelBytes];
    __shared__ float wt32[8];
    __shared__ double wt64[8];
    for (int q = threadIdx.x; q < kSelBytes; q += blockDim.x)
        seltab[q] = nth_set_bit((uint32_t)q >> 3, (uint32_t)q & 7u);
    if (threadIdx.x < 8) {
        wt32[threadIdx.x] = a.wt32[threadIdx.x];
        wt64[threadIdx.x] = a.wt64[threadIdx.x];
    }
    __syncthreads();
    const int64_t lane = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (lane >= lanes) return;
    ulonglong2 *tab = ws + (lane << logH);
    uint32_t gen = 0;
    for (;;) {
        const unsigned long long c = atomicAdd(next, 1ull);
        if (c >= (unsigned long long)a.C) break;
        uint32_t att = 0;
        while (long_attempt<kIsaw>(a, (int64_t)c, att, tab, logH, gen, seltab, wt32, wt64)) ++att;
    }
}

}  // namespace

size_t lattice_smem_bytes(int N, int B)
{
    // Tables, then the keys: two parities of key_groups(N) 16-byte groups per lane.
    return (size_t)(kLutWords + kSelBytes / 4 + 8 + 16) * 4 + (size_t)key_groups(N) * 2 * 16 * B;
}

// Block size: the largest multiple of 32 (at most 256) whose coordinate
// tile fits in about half of an SM's shared memory, so that at least two
// blocks are resident per SM.
int lattice_block(int N)
{
    const size_t budget = 110 * 1024;
    int B = 256;
    while (B > 32 && lattice_smem_bytes(N, B) > budget) B -= 32;
    return B;
}

int lattice_validate(const rosen_lattice_params *p, const rosen_lattice_out *o, int nmax,
                     const char *fn)
{
    if (!p || !o) return set_error(ROSEN_EINVAL, "%s: NULL params or outputs", fn);
    if (p->N < 2 || p->N > nmax)
        return set_error(ROSEN_EINVAL, "%s: N = %d outside [2, %d]", fn, p->N,
                         nmax);
    if (p->C < 0 || p->chain0 < 0 || p->chain0 + p->C > (int64_t(1) << 32))
        return set_error(ROSEN_EINVAL, "%s: chains [%lld, %lld) outside [0, 2^32)", fn,
                         (long long)p->chain0, (long long)(p->chain0 + p->C));
    if (!(p->beta_eps >= 0.0) || !(p->beta_eps <= 16.0))
        return set_error(ROSEN_EINVAL, "%s: beta_eps must lie in [0, 16] (the FP32 Boltzmann "
                                       "factor of five contacts must be finite)", fn);
    if (p->flags & ~(ROSEN_STORE_TRACE | ROSEN_STORE_COORDS))
        return set_error(ROSEN_EINVAL, "%s: unknown flags 0x%x", fn, p->flags);
    if (p->lanes_per_chain != 0 && p->lanes_per_chain != 1)
        return set_error(ROSEN_EINVAL, "%s: lanes_per_chain must be 0 or 1", fn);
    if (p->max_attempts < 0 || p->max_attempts > ROSEN_MAX_ATTEMPTS)
        return set_error(ROSEN_EINVAL, "%s: max_attempts = %d outside [0, %d]", fn,
                         p->max_attempts, ROSEN_MAX_ATTEMPTS);
    if ((p->flags & ROSEN_STORE_TRACE) && !o->trace)
        return set_error(ROSEN_EINVAL, "%s: ROSEN_STORE_TRACE without trace", fn);
    if ((p->flags & ROSEN_STORE_COORDS) && !o->coords)
        return set_error(ROSEN_EINVAL, "%s: ROSEN_STORE_COORDS without coords", fn);
    if (o->counts && (reinterpret_cast<uintptr_t>(o->counts) & 15u))
        return set_error(ROSEN_EINVAL, "%s: counts must be 16-byte aligned", fn);
    return ROSEN_OK;
}

size_t lattice_args_size() { return sizeof(LatticeArgs); }

// Kernel arguments of one ensemble (params already validated).
void lattice_make_args(const rosen_lattice_params *p, const rosen_lattice_out *o, void *out)
{
    LatticeArgs a;
    memset(&a, 0, sizeof a);
    a.key = philox_keys(p->seed);
    a.ens = p->ensemble;
    a.chain0 = (uint32_t)p->chain0;
    a.N = p->N;
    a.isaw = p->beta_eps != 0.0;
    a.C = p->C;
    for (int q = 0; q < 8; ++q) {
        a.wt64[q] = exp(p->beta_eps * (double)q);
        a.wt32[q] = (float)a.wt64[q];
        a.logm[q] = q >= 1 ? (float)log((double)q) : 0.f;
    }
    a.counts = reinterpret_cast<uint4 *>(o->counts);
    a.logw = o->logw;
    a.r2 = o->r2;
    a.n2rg2 = o->n2rg2;
    a.trace = (p->flags & ROSEN_STORE_TRACE) ? o->trace : nullptr;
    a.coords = (p->flags & ROSEN_STORE_COORDS) ? o->coords : nullptr;
    a.attempts = o->attempts;
    a.max_att = p->max_attempts > 1 ? (uint32_t)p->max_attempts : 1u;
    memcpy(out, &a, sizeof a);
}

int lattice_batch_prepare(int B, int Nmax, size_t *smem, int *blocks_per_sm)
{
    *smem = lattice_smem_bytes(Nmax, B);
    cudaError_t e = allow_max_smem(lattice_batch_kernel);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, lattice_batch_kernel, B,
                                                          *smem);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "lattice batch set-up: %s", cudaGetErrorString(e));
    return ROSEN_OK;
}

void lattice_batch_launch(const void *dev_args, const BatchItem *items, int n_items, int *head,
                          int B, size_t smem, int grid, cudaStream_t s)
{
    lattice_batch_kernel<<<grid, B, smem, s>>>(reinterpret_cast<const LatticeArgs *>(dev_args),
                                               items, n_items, head);
}

// Restart mode: as many warps as fit on the GPU at once (at most one per 32
// chains), each with a contiguous range of the chains [c_lo, c_hi).
int lattice_retry_launch(const LatticeArgs &a, int N, int B, int64_t c_lo, int64_t c_hi,
                         cudaStream_t s)
{
    const int wpb = B / 32;
    const size_t smem = (size_t)(kLutWords + kSelBytes / 4 + 8 + 16) * 4 +
                        (size_t)wpb * (64 * 4 + (size_t)key_groups(N) * 2 * 16 * 32);
    auto kern = a.isaw ? lattice_retry_kernel<true> : lattice_retry_kernel<false>;
    cudaError_t e = allow_max_smem(kern);
    int bps = 0, dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, B, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_lattice_grow: %s", cudaGetErrorString(e));
    if (bps < 1) return set_error(ROSEN_ECUDA, "rosen_lattice_grow: kernel does not fit an SM");
    const int64_t n = c_hi - c_lo;
    const int64_t warps = std::min<int64_t>((int64_t)bps * sms * wpb, (n + 31) / 32);
    const int64_t per_warp = (n + warps - 1) / warps;
    const int64_t grid = ((n + per_warp - 1) / per_warp + wpb - 1) / wpb;
    kern<<<(unsigned)grid, B, smem, s>>>(a, per_warp, c_lo, c_hi);
    return check_launch("rosen_lattice_grow");
}

// Grow local chains [c_lo, c_hi) of a validated ensemble (shared-memory
// kernels, N <= 512).  Every chain's outputs are those of a call over all C
// chains, bit for bit: a chain is grown by one lane whatever its block.
int lattice_grow_range(const rosen_lattice_params *p, const rosen_lattice_out *o, int64_t c_lo,
                       int64_t c_hi, cudaStream_t s)
{
    if (c_hi <= c_lo) return ROSEN_OK;
    LatticeArgs a;
    lattice_make_args(p, o, &a);
    const int B = lattice_block(p->N);
    if (a.max_att > 1) return lattice_retry_launch(a, p->N, B, c_lo, c_hi, s);
    const size_t smem = lattice_smem_bytes(p->N, B);
    const int64_t blocks = (c_hi - c_lo + B - 1) / B;
    // Blocks of 256 (N up to about 100) with the stride fixed at compile time.
    auto kern = p->beta_eps == 0.0
                    ? (B == 256 ? lattice_lane_kernel<false, 256> : lattice_lane_kernel<false, 0>)
                    : (B == 256 ? lattice_lane_kernel<true, 256> : lattice_lane_kernel<true, 0>);
    allow_max_smem(kern);
    kern<<<(unsigned)blocks, B, smem, s>>>(a, c_lo, c_hi);
    return check_launch("rosen_lattice_grow");
}

int64_t lattice_resident_chains(const rosen_lattice_params *p)
{
    const int B = lattice_block(p->N);
    const size_t smem = lattice_smem_bytes(p->N, B);
    auto kern = p->beta_eps != 0.0
                    ? (B == 256 ? lattice_lane_kernel<true, 256> : lattice_lane_kernel<true, 0>)
                    : (B == 256 ? lattice_lane_kernel<false, 256> : lattice_lane_kernel<false, 0>);
    int dev = 0, sms = 0, bps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        allow_max_smem(kern) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, B, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int64_t)bps * sms * B;
}

}  // namespace rosen

using namespace rosen;

extern "C" int rosen_lattice_grow(const rosen_lattice_params *p, const rosen_lattice_out *o,
                                  void *stream)
{
    const int st = lattice_validate(p, o);
    if (st != ROSEN_OK) return st;
    if (p->C == 0) return ROSEN_OK;
    return lattice_grow_range(p, o, 0, p->C, (cudaStream_t)stream);
}

// ---- long chains -------------------------------------------------------------
namespace {

constexpr int64_t kLongLanes = 1 << 17;   // tables the default workspace holds
constexpr size_t kLongHeader = 256;       // the chain counter, at the head of the workspace

// log2 of the table entries per lane: more than N (a chain fills at most N
// blocks) and at least 64.
int long_log_entries(int N)
{
    int lg = 6;
    while ((int64_t(1) << lg) < (int64_t)N + 1) ++lg;
    return lg;
}

}  // namespace

extern "C" size_t rosen_lattice_long_workspace_size(int32_t N, int64_t C)
{
    if (N < 2 || N > ROSEN_LATTICE_LONG_NMAX || C < 1) return 0;
    const int64_t lanes = C < kLongLanes ? C : kLongLanes;
    return kLongHeader + (size_t)lanes * (sizeof(ulonglong2) << long_log_entries(N));
}

extern "C" int rosen_lattice_grow_long(const rosen_lattice_params *p, const rosen_lattice_out *o,
                                       void *workspace, size_t workspace_bytes, void *stream)
{
    const int st = lattice_validate(p, o, ROSEN_LATTICE_LONG_NMAX, "rosen_lattice_grow_long");
    if (st != ROSEN_OK) return st;
    if (p->C == 0) return ROSEN_OK;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 15u))
        return set_error(ROSEN_EINVAL, "rosen_lattice_grow_long: workspace must be a non-NULL, "
                                       "16-byte aligned device pointer");
    const int logH = long_log_entries(p->N);
    const size_t table = sizeof(ulonglong2) << logH;
    int64_t lanes = workspace_bytes > kLongHeader
                        ? (int64_t)((workspace_bytes - kLongHeader) / table) : 0;
    if (lanes > p->C) lanes = p->C;
    if (lanes < 1)
        return set_error(ROSEN_ENOMEM,
                         "rosen_lattice_grow_long: workspace of %zu bytes holds no table of %zu "
                         "bytes after its %zu-byte header (N = %d)", workspace_bytes, table,
                         kLongHeader, p->N);
    LatticeArgs a;
    lattice_make_args(p, o, &a);
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = cudaMemsetAsync(workspace, 0, kLongHeader + (size_t)lanes * table, s);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_lattice_grow_long: clearing %lld tables of %zu bytes: %s",
                         (long long)lanes, table, cudaGetErrorString(e));
    const unsigned grid = (unsigned)((lanes + 255) / 256);
    unsigned long long *next = static_cast<unsigned long long *>(workspace);
    ulonglong2 *ws = reinterpret_cast<ulonglong2 *>(static_cast<unsigned char *>(workspace) +
                                                    kLongHeader);
    if (a.isaw) lattice_long_kernel<true><<<grid, 256, 0, s>>>(a, ws, lanes, logH, next);
    else lattice_long_kernel<false><<<grid, 256, 0, s>>>(a, ws, lanes, logH, next);
    return check_launch("rosen_lattice_grow_long (kernel launch)");
}

