// offlattice_chain.cuh -- the device code that grows one real-space chain
// (Guo & Baulin, Section 3.3.3, Algorithm 2), shared by the shared-memory
// kernels (offlattice.cu) and the long-chain kernel (offlattice_long.cu):
// the kernel arguments, the per-chain storage, trial directions, the group
// primitives, the FP64 replay and re-decision, and off_chain itself.
#pragma once

#include <limits.h>
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "turn_table.cuh"

namespace rosen {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct OffArgs {
    PhiloxKeys key;
    uint32_t ens, chain0;
    int32_t N, k;
    int64_t C;
    float sig2, rc2, rf2, rf;  // sigma^2, cutoff^2, list radius^2 (with margin), list radius
    float beta4;               // 4 beta eps (LJ)
    float dband;               // HS: sigma (the distance at which decisions flip); LJ: cutoff
    float ucut2;               // 2 |s^6 (s^6 - 1)| at the cutoff: energy jump (doubled)
    double sig2d, rc2d, beta_eps;
    float *logw, *r2, *rg2;
    uint8_t *alive, *trace;
    float *coords;
    float drift;                    // bound on a position's drift from exact, per step
    unsigned long long *counters;   // optional [3]: steps re-decided, chains, listed beads
    uint16_t *attempts;             // optional [C]
    uint32_t max_att;               // growths per chain (1: no restart)
    uint32_t *deferred;             // two-pass hard-sphere growth: bit c = chain c deferred
};

// Per-chain shared memory: float-float positions, the near list, the trace.
// Rounded up to 16 bytes so that every chain's float4 arrays stay aligned.
// (The per-bead band array exists only for Lennard-Jones chains.)
__host__ __device__ inline size_t chain_smem_bytes(int N, bool lj)
{
    const size_t n = (size_t)N;
    const size_t b = 3 * n * sizeof(float4) + n * sizeof(int) + (lj ? n * sizeof(float) : 0) + n;
    return (b + 15) & ~size_t(15);
}

struct ChainSmem {
    float4 *hi, *lo;   // positions (x, y, z, -)
    float4 *nl;        // near list: g.x, g.y, g.z, 1 + |g|^2
    int *nj;           // near list: bead index
    float *nb;         // near list: bound on |d^2 (FP32) - d^2 (FP64)| for this bead
    uint8_t *tr;       // chosen trial of each step
};

// A long chain's storage (all in device memory): the arrays above, the near
// list as gathered (before it is put in bead order), and the cell grid -- a
// hash table of the cells that hold beads, each heading a list of its beads.
// The list link of bead j is kept in hi[j].w (its bits), so one 16-byte load
// gives a bead's position and the next bead of its cell.
struct ChainLong : ChainSmem {
    float4 *nls;
    int *njs;
    float *nbs;
    uint4 *cells;      // {key with generation (2 words), head bead, -}
    int logH;          // log2 of the cell-table entries
    float inv_cell;    // 1 / cell side
    float pre2;        // coarse test: beads with hi-only |g|^2 >= pre2 are not near
};

__device__ inline ChainSmem carve(unsigned char *base, int N, bool lj)
{
    ChainSmem w;
    w.hi = reinterpret_cast<float4 *>(base);
    w.lo = w.hi + N;
    w.nl = w.lo + N;
    w.nj = reinterpret_cast<int *>(w.nl + N);
    w.nb = reinterpret_cast<float *>(w.nj + N);
    w.tr = reinterpret_cast<uint8_t *>(lj ? w.nb + N : w.nb);
    return w;
}

// ---- the cell grid of long chains --------------------------------------------
// A bead belongs to the cell floor(hi / side) on each axis, with the side a
// little above the list radius (plus twice the largest position drift), so
// every bead that can be listed at a step lies in the 27 cells around the
// end's cell.  Cell keys pack 16 bits per axis; bits 48..63 of an entry hold
// the generation of the growth that wrote it (older generations read as
// empty, so a chain slot is reused without clearing its table).
constexpr int kCellGenShift = 48;
constexpr uint64_t kCellKeyMask = (1ull << kCellGenShift) - 1ull;
constexpr uint32_t kCellGenMax = 65535;

__device__ __forceinline__ uint64_t cell_key(int cx, int cy, int cz)
{
    return (uint64_t)(uint32_t)(cx + 32768) | ((uint64_t)(uint32_t)(cy + 32768) << 16) |
           ((uint64_t)(uint32_t)(cz + 32768) << 32);
}

__device__ __forceinline__ int cell_coord(float x, float inv) { return (int)floorf(x * inv); }

// First probe of a cell: the low bits of its three coordinates side by side
// (x fastest), so the 27 cells around the end sit in 9 runs of 3 adjacent
// entries and a moving end reuses the entries it read at the last steps.
// Distant cells whose low bits agree share a probe sequence; the table holds
// at most half as many cells as entries, so every sequence ends at an empty
// entry.
__device__ __forceinline__ uint32_t cell_slot(uint64_t key, int logH)
{
    const int bx = (logH + 2) / 3, by = (logH + 1) / 3, bz = logH - bx - by;
    const uint32_t x = (uint32_t)key & ((1u << bx) - 1u);
    const uint32_t y = (uint32_t)(key >> 16) & ((1u << by) - 1u);
    const uint32_t z = (uint32_t)(key >> 32) & ((1u << bz) - 1u);
    return x | (y << bx) | (z << (bx + by));
}

// First bead of the cell whose tagged key is `want` (-1: no bead there),
// going on from entry h, already loaded as e.
__device__ __forceinline__ int cell_find(const uint4 *cells, int logH, uint64_t want,
                                         uint64_t tag, uint32_t h, uint4 e)
{
    const uint32_t hmask = (1u << logH) - 1u;
    for (;;) {
        const uint64_t k = (uint64_t)e.x | ((uint64_t)e.y << 32);
        if ((k & ~kCellKeyMask) != tag) return -1;
        if (k == want) return (int)e.z;
        h = (h + 1u) & hmask;
        e = cells[h];
    }
}

// First beads of two cells (the second only if `two`), their first probes
// loaded together.
__device__ __forceinline__ void cell_heads2(const uint4 *cells, int logH, uint64_t want0,
                                            uint64_t want1, bool two, uint64_t tag, int &b0,
                                            int &b1)
{
    const uint32_t h0 = cell_slot(want0 & kCellKeyMask, logH);
    const uint32_t h1 = cell_slot(want1 & kCellKeyMask, logH);
    const uint4 e0 = cells[h0];
    const uint4 e1 = two ? cells[h1] : make_uint4(0u, 0u, 0u, 0u);
    b0 = cell_find(cells, logH, want0, tag, h0, e0);
    b1 = two ? cell_find(cells, logH, want1, tag, h1, e1) : -1;
}

// Put bead j at the head of the list of its cell (key `want`); returns the
// bead it now links to (-1: the cell was empty).
__device__ __forceinline__ int cell_push(uint4 *cells, int logH, uint64_t want, uint64_t tag,
                                         int j)
{
    const uint32_t hmask = (1u << logH) - 1u;
    uint32_t h = cell_slot(want & kCellKeyMask, logH);
    for (;;) {
        const uint4 e = cells[h];
        const uint64_t k = (uint64_t)e.x | ((uint64_t)e.y << 32);
        if ((k & ~kCellKeyMask) != tag) {
            cells[h] = make_uint4((uint32_t)want, (uint32_t)(want >> 32), (uint32_t)j, 0u);
            return -1;
        }
        if (k == want) {
            reinterpret_cast<int *>(&cells[h])[2] = j;
            return (int)e.z;
        }
        h = (h + 1u) & hmask;
    }
}

// Bound on |d^2 (FP32) - d^2 (FP64)| for a trial against a listed bead with
// displacement g (|g| = gn, 1 + |g|^2 = c) whose position drifted for D steps
// since it was last exact.  d^2 = c + 2 u.g differs from the exact value by
// 2 (g + u).dg + 2 g.du + rounding, with |du| <= 4e-7 per direction (the
// exhaustively measured component error is 2.7e-7; z is exact), |dg| <=
// D drift + 2.1e-7 |g| (drift plus the rounding of g), |g + u| <= dmax (sigma
// at the hard-sphere decision, min(1 + |g|, cutoff) for LJ), and three FMA
// roundings of values up to 2c.  Doubled for safety.  The drift per step is
// 4e-7 when positions sum the FP32 directions and about 1e-12 when they sum
// float-float directions (dir_ff; Lennard-Jones with k > 32).
__device__ __forceinline__ float pair_band(float gn, float c, int D, float dmax, float drift)
{
    // Explicit FMAs: the same rounding in every kernel that inlines this.
    const float dg = fmaf((float)D, drift, 2.1e-7f * gn);
    return 2.f * fmaf(2.f * dmax, dg, fmaf(8e-7f, gn, 3.6e-7f * c));
}

// sin and cos of 2 pi V / 2^24 for a 24-bit integer V.  The quarter-turn
// reduction is exact integer arithmetic: V = q 2^22 + r with r in
// [-2^21, 2^21), so the angle is q (pi/2) + pi y with y = r / 2^23 exact in
// FP32 and |y| <= 1/4.  sin(pi y) and cos(pi y) are their Taylor series
// truncated after y^9 and y^10 (remainders below 2e-9), evaluated by Horner's
// rule in FP32; the quadrant q only swaps and negates.
__device__ __forceinline__ void sincos_turn24(uint32_t V, float &sn, float &cs)
{
    constexpr float S1 = (float)kPi;
    constexpr float S3 = (float)(-kPi * kPi * kPi / 6.0);
    constexpr float S5 = (float)(kPi * kPi * kPi * kPi * kPi / 120.0);
    constexpr float S7 = (float)(-kPi * kPi * kPi * kPi * kPi * kPi * kPi / 5040.0);
    constexpr float S9 = (float)(kPi * kPi * kPi * kPi * kPi * kPi * kPi * kPi * kPi / 362880.0);
    constexpr float C2 = (float)(-kPi * kPi / 2.0);
    constexpr float C4 = (float)(kPi * kPi * kPi * kPi / 24.0);
    constexpr float C6 = (float)(-kPi * kPi * kPi * kPi * kPi * kPi / 720.0);
    constexpr float C8 = (float)(kPi * kPi * kPi * kPi * kPi * kPi * kPi * kPi / 40320.0);
    constexpr float C10 =
        (float)(-kPi * kPi * kPi * kPi * kPi * kPi * kPi * kPi * kPi * kPi / 3628800.0);
    const uint32_t qn = (V + (1u << 21)) >> 22;
    const int32_t r = (int32_t)V - (int32_t)(qn << 22);
    const float y = (float)r * 0x1p-23f;
    const float y2 = y * y;
    const float ps = fmaf(fmaf(fmaf(fmaf(S9, y2, S7), y2, S5), y2, S3), y2, S1) * y;
    const float pc = fmaf(fmaf(fmaf(fmaf(fmaf(C10, y2, C8), y2, C6), y2, C4), y2, C2), y2, 1.f);
    const uint32_t q = qn & 3u;
    const float a = (q & 1u) ? pc : ps;
    const float b = (q & 1u) ? ps : pc;
    sn = (q & 2u) ? -a : a;
    cs = ((q + 1u) & 2u) ? -b : b;
}

// Trial direction from two words (the reading of "rngonsphere"):
// z = 1 - 2 u24(a), phi = 2 pi u24(b), s = sqrt((1-z)(1+z)).  (1-z), (1+z) are
// exact in FP32; sqrtf is correctly rounded.  dir32x2 returns twice the
// direction, as the pair test uses it, with the factor folded in:
// 2z = 2 - 4 u24(a), 2s = sqrt((2 - 2z)(2 + 2z)).  Every factor of 2 (and 4
// under the root) is exact and commutes with the rounding of a product or
// a correctly rounded root, so dir32x2 is 2 dir32, bit for bit.  In FP32:
// 2z = 2 - (a >> 8) 2^-22 is one fused multiply-add of exact terms, and
// since 2 - 2z and 2 + 2z are exact, their product is the single rounding
// of 4 - (2z)^2, which is what fmaf(-2z, 2z, 4) rounds too.
__device__ __forceinline__ float3 dir32x2(uint32_t a, uint32_t b)
{
    const float z2 = fmaf(-0x1p-22f, (float)(a >> 8), 2.f);
    const float s2 = sqrtf(fmaf(-z2, z2, 4.f));
    float sn, cs;
    sincos_turn24(b >> 8, sn, cs);
    return make_float3(s2 * cs, s2 * sn, z2);
}

__device__ __forceinline__ float3 dir32(uint32_t a, uint32_t b)
{
    const float3 u = dir32x2(a, b);
    return make_float3(0.5f * u.x, 0.5f * u.y, 0.5f * u.z);
}

__device__ __forceinline__ void dir64(uint32_t a, uint32_t b, double &x, double &y, double &z)
{
    z = 1.0 - 2.0 * u24d(a);
    const double s = sqrt((1.0 - z) * (1.0 + z));
    double sn, cs;
    sincospi(2.0 * u24d(b), &sn, &cs);
    x = s * cs;
    y = s * sn;
}

// Words of trial t inside its draw: slot 1 + t/2, pair (0,1) or (2,3).
__device__ __forceinline__ void trial_words(const uint4 &x, int t, uint32_t &a, uint32_t &b)
{
    a = (t & 1) ? x.z : x.x;
    b = (t & 1) ? x.w : x.y;
}

// Error-free sum of a float into a float-float value (Knuth's TwoSum).
__device__ __forceinline__ void ff_add(float &hi, float &lo, float v)
{
    const float s = hi + v;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (v - bp);
    const float t = lo + e;
    hi = s + t;
    lo = t - (hi - s);
}

// ff_add of v = w / 2: the halving is exact, so each sum with v is one
// fused multiply-add with 0.5 and rounds exactly as the sum does.
__device__ __forceinline__ void ff_add_half(float &hi, float &lo, float w)
{
    const float s = fmaf(0.5f, w, hi);
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + fmaf(0.5f, w, -bp);
    const float t = lo + e;
    hi = s + t;
    lo = t - (hi - s);
}

// ---- float-float arithmetic (Knuth's TwoSum, Dekker's product with FMA) ----
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Renormalise s + e with |e| small against s.
__device__ __forceinline__ void quick_sum(float &s, float &e)
{
    const float t = s + e;
    e = e - (t - s);
    s = t;
}

__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    ph = ah * bh;
    pl = fmaf(ah, bh, -ph);            // exact error of the leading product
    pl = fmaf(ah, bl, fmaf(al, bh, pl));
    quick_sum(ph, pl);
}

__device__ __forceinline__ void ff_sum(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    two_sum(ah, bh, sh, sl);
    sl += al + bl;
    quick_sum(sh, sl);
}

// The unit vector of words (a, b) as float-float components (z is exact).
// With the turn fraction V = b >> 8 = 2^16 m + v, the angle 2 pi V / 2^24 is
// 2 pi m / 256 (cos and sin from the float-float table kTurn) plus
// t = 2 pi v / 2^24 < 0.0246, whose sin and cos come from their Taylor series:
// sin t = t + d with d = -t^3/6 (1 - t^2/20 (1 - t^2/42)) in FP32 (|d| <
// 2.5e-6, so its FP32 rounding is below 1e-12), cos t = 1 + e with
// e = -q/2 + q^2/24 (1 - q/30), q = t^2 float-float.  The rotation and the
// scaling by s = sqrt((1 - z)(1 + z)) are float-float products.  Each
// component is within 1.5e-12 of the exact value (the FP32 part of d
// dominates; the table and the truncations are below 3e-15).
__device__ __forceinline__ void dir_ff(uint32_t a, uint32_t b, float &xh, float &xl, float &yh,
                                       float &yl, float &z)
{
    z = 1.f - 2.f * u24f(a);
    const float om = 1.f - z, op = 1.f + z;           // exact
    const float ph = om * op, pl = fmaf(om, op, -ph);  // (1 - z)(1 + z), exactly
    const float sh0 = sqrtf(ph);
    float sh = sh0, sl = 0.f;
    if (sh0 > 0.f) {
        sl = __fdividef(fmaf(-sh0, sh0, ph) + pl, 2.f * sh0);
        quick_sum(sh, sl);
    }
    const uint32_t V = b >> 8;
    const float4 tb = kTurn[V >> 16];
    const float v = (float)(V & 0xFFFFu);              // exact
    float th = v * kTurnUnitHi;
    float tl = fmaf(v, kTurnUnitHi, -th);
    tl = fmaf(v, kTurnUnitLo, tl);
    quick_sum(th, tl);
    float qh = th * th;
    float ql = fmaf(th, th, -qh);
    ql = fmaf(2.f * th, tl, ql);
    quick_sum(qh, ql);
    const float d = -(th * qh) * (1.f / 6.f) *
                    fmaf(-qh * (1.f / 20.f), fmaf(-qh, 1.f / 42.f, 1.f), 1.f);
    float s2h, s2l;
    two_sum(th, d, s2h, s2l);
    s2l += tl;
    quick_sum(s2h, s2l);
    const float r = qh * qh * (1.f / 24.f) * fmaf(-qh, 1.f / 30.f, 1.f);
    float c2h, c2l;
    two_sum(1.f, -0.5f * qh, c2h, c2l);
    c2l += fmaf(-0.5f, ql, r);
    quick_sum(c2h, c2l);
    float ah, al, bh, bl, ch, cl, nh, nl;
    ff_mul(tb.x, tb.z, c2h, c2l, ah, al);              // cos(2 pi m/256) cos t
    ff_mul(tb.y, tb.w, s2h, s2l, bh, bl);              // sin(2 pi m/256) sin t
    ff_sum(ah, al, -bh, -bl, ch, cl);
    ff_mul(tb.y, tb.w, c2h, c2l, ah, al);
    ff_mul(tb.x, tb.z, s2h, s2l, bh, bl);
    ff_sum(ah, al, bh, bl, nh, nl);
    ff_mul(sh, sl, ch, cl, xh, xl);
    ff_mul(sh, sl, nh, nl, yh, yl);
}

template <int G>
struct Group {
    unsigned mask;   // the group's lanes in the warp
    unsigned below;  // the group's lanes below this one (warp lane bits)
    int gl;          // lane within the group
    int base;        // first lane of the group in the warp

    __device__ Group()
    {
        const int lane = threadIdx.x & 31;
        gl = lane & (G - 1);
        base = lane - gl;
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
        below = ((1u << lane) - 1u) & mask;
    }
    __device__ unsigned ballot(bool p) const
    {
        const unsigned b = __ballot_sync(mask, p);
        return (G == 32) ? b : (b >> base) & ((1u << G) - 1u);
    }
    // The group's votes at their warp lane positions (for counts and ranks
    // with `below`, without shifting them down).
    __device__ unsigned vote(bool p) const { return __ballot_sync(mask, p) & mask; }
    template <class V>
    __device__ V bcast(V v, int src) const
    {
        return __shfl_sync(mask, v, src, G);
    }
    __device__ float min(float v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(mask, v, o, G));
        return v;
    }
    __device__ double min(double v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(mask, v, o, G));
        return v;
    }
    __device__ float max(float v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, G));
        return v;
    }
    __device__ float sum(float v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
        return v;
    }
    template <class V>
    __device__ V scan(V v) const   // inclusive prefix sum over the group
    {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const V u = __shfl_up_sync(mask, v, o, G);
            if (gl >= o) v += u;
        }
        return v;
    }
};

// Philox draw of counter c under the ensemble's key.  kFly computes the round
// keys on the fly from the first (two adds per round) instead of reading the
// precomputed schedule: kernels whose OffArgs live in shared memory (the
// batch kernels) would otherwise hold 20 key words in registers.
template <bool kFly>
__device__ __forceinline__ uint4 draw(const OffArgs &a, uint4 c)
{
    if constexpr (kFly)
        return philox(c, a.key.k0[0], a.key.k1[0]);
    else
        return philox(c, a.key);
}

// FP64 replay of r_{b+1} .. r_{i-1} from the chosen trials, starting at bead
// b, the last bead replayed before (its float-float position is its FP64 one
// to 2^-48 relative); the positions are stored back into the float-float
// arrays and the end returned.  Only the steps since the last replay are
// summed, so the cost does not grow with i.  The G lanes add their
// directions with a group prefix scan: the sums differ from the sequential
// order of the definition by a few FP64 roundings, far below the 2^-48 of
// the float-float storage.
template <int G, bool kFly = false>
__device__ __noinline__ void replay_positions(const OffArgs &a, const ChainSmem &w,
                                              const Group<G> &g, uint32_t chain, uint32_t aw,
                                              int b, int i, double &ex, double &ey, double &ez)
{
    const float4 bh = w.hi[b], bl = w.lo[b];
    double cx = (double)bh.x + (double)bl.x, cy = (double)bh.y + (double)bl.y,
           cz = (double)bh.z + (double)bl.z;
    for (int b0 = b + 1; b0 <= i - 1; b0 += G) {
        const int s = b0 + g.gl;
        double x = 0.0, y = 0.0, z = 0.0;
        if (s <= i - 1) {
            const int t = w.tr[s];
            const uint4 q =
                draw<kFly>(a, make_uint4(chain, a.ens, (uint32_t)s | aw, 1u + (uint32_t)(t >> 1)));
            uint32_t wa, wb;
            trial_words(q, t, wa, wb);
            dir64(wa, wb, x, y, z);
        }
        x = g.scan(x) + cx;
        y = g.scan(y) + cy;
        z = g.scan(z) + cz;
        if (s <= i - 1) {
            const float hx = (float)x, hy = (float)y, hz = (float)z;
            w.hi[s] = make_float4(hx, hy, hz, w.hi[s].w);   // .w: a long chain's cell link
            w.lo[s] = make_float4((float)(x - hx), (float)(y - hy), (float)(z - hz), 0.f);
        }
        cx = g.bcast(x, G - 1);
        cy = g.bcast(y, G - 1);
        cz = g.bcast(z, G - 1);
    }
    __syncwarp(g.mask);
    ex = cx;
    ey = cy;
    ez = cz;
}

// FP64 re-decision of step i: replay the exact positions, recompute every
// trial's free flag or energy in FP64 from the listed beads, and select with
// the sequential FP64 arithmetic of the definition.
template <int G, int T, bool LJ, bool kFly = false>
__device__ __forceinline__ void redecide(const OffArgs &a, const ChainSmem &w, const Group<G> &g,
                                      uint32_t chain, uint32_t aw, int b, int i, int nn,
                                      uint32_t selw,
                                      const float *logm, float &ehx, float &ehy, float &ehz,
                                      float &elx, float &ely, float &elz, int &sel, float &logS,
                                      int &dead_at)
{
    const int k = a.k;
    double ex, ey, ez;
    replay_positions<G, kFly>(a, w, g, chain, aw, b, i, ex, ey, ez);
    // The exact end, back into the float-float registers.
    ehx = (float)ex;
    elx = (float)(ex - ehx);
    ehy = (float)ey;
    ely = (float)(ey - ehy);
    ehz = (float)ez;
    elz = (float)(ez - ehz);
    double val[T];
#pragma unroll
    for (int s = 0; s < T; ++s) {
        const int t = T * g.gl + s;
        const uint4 xx =
            draw<kFly>(a, make_uint4(chain, a.ens, (uint32_t)i | aw, 1u + (uint32_t)(t >> 1)));
        uint32_t wa, wb;
        trial_words(xx, t, wa, wb);
        double dx, dy, dz;
        dir64(wa, wb, dx, dy, dz);
        // The definition's arithmetic in its order, each operation rounded
        // once (no contraction into FMAs, a true division): the trial
        // position end + u, the displacement to bead j, d^2 = (dx^2 + dy^2)
        // + dz^2, and 4 s3 (s3 - 1) with s3 = (sigma^2 / d^2)^3 summed over
        // the beads within the cutoff.
        const double tx = __dadd_rn(ex, dx), ty = __dadd_rn(ey, dy), tz = __dadd_rn(ez, dz);
        double acc = 0.0;
        bool fr = true;
        for (int q = 0; q < nn; ++q) {
            const int j = w.nj[q];
            const float4 h = w.hi[j], l = w.lo[j];
            // (hi + lo of a float-float position is exact in FP64.)
            const double rx = __dsub_rn(tx, (double)h.x + (double)l.x);
            const double ry = __dsub_rn(ty, (double)h.y + (double)l.y);
            const double rz = __dsub_rn(tz, (double)h.z + (double)l.z);
            const double d2 =
                __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
            if (!LJ) {
                if (d2 < a.sig2d) fr = false;
            } else if (d2 < a.rc2d) {
                const double sr = __ddiv_rn(a.sig2d, d2);
                const double s3 = __dmul_rn(__dmul_rn(sr, sr), sr);
                acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(4.0, s3), __dsub_rn(s3, 1.0)));
            }
        }
        const bool valid = t < k;
        if (!valid) val[s] = LJ ? INFINITY : 0.0;
        else if (!LJ) val[s] = fr ? 1.0 : 0.0;
        else val[s] = (a.beta_eps == 0.0) ? 0.0 : __dmul_rn(a.beta_eps, acc);
    }
    if (!LJ) {
        int cnt = 0;
#pragma unroll
        for (int s = 0; s < T; ++s) cnt += val[s] > 0.0;
        const int incl = g.scan(cnt);
        const int m = g.bcast(incl, G - 1);
        if (m == 0) {
            dead_at = i;
        } else {
            const int idx = (int)__umulhi(selw, (uint32_t)m);
            int mine = -1, seen = incl - cnt;
#pragma unroll
            for (int s = 0; s < T; ++s)
                if (val[s] > 0.0) {
                    if (seen == idx) mine = T * g.gl + s;
                    ++seen;
                }
            const unsigned who = g.ballot(mine >= 0);
            sel = g.bcast(mine, __ffs(who) - 1);
            logS = logm[m];
        }
    } else {
        double bmin = INFINITY;
#pragma unroll
        for (int s = 0; s < T; ++s) bmin = fmin(bmin, val[s]);
        bmin = g.min(bmin);
        if (bmin == INFINITY) {
            dead_at = i;
        } else {
            double wv[T];
#pragma unroll
            for (int s = 0; s < T; ++s) wv[s] = exp(-(val[s] - bmin));
            // Sequential FP64 sum and prefix in trial order, as the
            // definition states them; every lane walks the trials.
            double S = 0.0, r = 0.0, P = 0.0;
            int pick = -1, lastpos = -1;
            for (int pass = 0; pass < 2; ++pass) {
                for (int t = 0; t < k; ++t) {
                    double v = 0.0;
#pragma unroll
                    for (int s = 0; s < T; ++s)
                        if (s == t % T) v = wv[s];
                    v = g.bcast(v, t / T);
                    if (pass == 0) {
                        S += v;
                        if (v > 0.0) lastpos = t;
                    } else if (pick < 0) {
                        P += v;
                        if (P > r) pick = t;
                    }
                }
                if (pass == 0) r = __dmul_rn(u24d(selw), S);
            }
            sel = pick >= 0 ? pick : lastpos;
            logS = (float)(log(S) - bmin);
        }
    }
}

// Near list of step i for a long chain: the beads 0..i-2 that lie within the
// list radius of the end, in ascending bead order -- the order in which the
// full scan lists them, so the step's arithmetic is the same as in the
// shared-memory kernels.
// A bead is filed in the cell grid only once it is G steps old: the G most
// recent non-bonded beads (i-1-G .. i-2), which are the ones most often near
// the end and would make the end's own cell list long, are tested directly
// (one per lane, independent loads); the lists of the 27 cells around the
// end's cell then hold only beads 0..i-2-G, few of them near, and are walked
// cell by cell (lanes on different cells).
// The heads of the 27 cells are kept between steps (cell[], heads[2] per
// lane: cells gl and gl + G): while the end stays in one cell the only change
// to those lists is the bead filed at this step, which heads its cell's list.
// When the end changes cell, a lane's two cells are probed together.
template <int G, bool LJ>
__device__ __forceinline__ int long_near_list(const OffArgs &a, const ChainLong &w,
                                              const Group<G> &g, int i, uint64_t tag, float ehx,
                                              float ehy, float ehz, float elx, float ely, float elz,
                                              int exact_upto, float drift, int (&cell)[3],
                                              int (&heads)[2])
{
    // File bead i-2-G in the cell of its current position.
    const int fb = i - 2 - G;
    if (fb >= 0) {
        const float4 hb = w.hi[fb];
        const int bx = cell_coord(hb.x, w.inv_cell), by = cell_coord(hb.y, w.inv_cell),
                  bz = cell_coord(hb.z, w.inv_cell);
        if (g.gl == 0) {
            const int link = cell_push(w.cells, w.logH, cell_key(bx, by, bz) | tag, tag, fb);
            reinterpret_cast<float *>(w.hi + fb)[3] = __int_as_float(link);
        }
        const int dx = bx - cell[0], dy = by - cell[1], dz = bz - cell[2];
        if (cell[0] != INT_MIN && dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 &&
            dz <= 1) {
            const int qb = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (g.gl + r * G == qb) heads[r] = fb;
        }
        __syncwarp(g.mask);
    }
    const int cx = cell_coord(ehx, w.inv_cell), cy = cell_coord(ehy, w.inv_cell),
              cz = cell_coord(ehz, w.inv_cell);
    if (cx != cell[0] || cy != cell[1] || cz != cell[2]) {
        const int q0 = g.gl, q1 = g.gl + G;
        cell_heads2(w.cells, w.logH,
                    cell_key(cx + q0 % 3 - 1, cy + (q0 / 3) % 3 - 1, cz + q0 / 9 - 1) | tag,
                    cell_key(cx + q1 % 3 - 1, cy + (q1 / 3) % 3 - 1, cz + q1 / 9 - 1) | tag,
                    q1 < 27, tag, heads[0], heads[1]);
        cell[0] = cx;
        cell[1] = cy;
        cell[2] = cz;
    }
    int q = g.gl;
    int j = heads[0];
    int nn = 0;
    for (;;) {
        if (j < 0 && q == g.gl) {
            q += G;
            j = q < 27 ? heads[1] : -1;
        }
        const bool has = j >= 0;
        if (!g.vote(has)) break;
        float4 L = make_float4(0.f, 0.f, 0.f, 0.f);
        bool near = false;
        float4 h = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        if (has) h = w.hi[j];
        if (has && j <= i - 2) {
            // Coarse test on hi alone (the lo words are below 6e-8 |x|; pre2
            // covers them), then the exact test of the full scan.
            const float px = (ehx - h.x) + elx, py = (ehy - h.y) + ely, pz = (ehz - h.z) + elz;
            if (fmaf(px, px, fmaf(py, py, pz * pz)) < w.pre2) {
                const float4 l = w.lo[j];
                const float gx = (ehx - h.x) + (elx - l.x);
                const float gy = (ehy - h.y) + (ely - l.y);
                const float gz = (ehz - h.z) + (elz - l.z);
                const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
                L = make_float4(gx, gy, gz, 1.f + g2);
                near = g2 < a.rf2;
            }
        }
        const unsigned m = g.vote(near);
        if (near) {
            const int slot = nn + __popc(m & g.below);
            w.nls[slot] = L;
            w.njs[slot] = j;
            if (LJ) {
                const float gn = fmaf(sqrtf(L.w - 1.f), 1.001f, 1e-6f);
                w.nbs[slot] = pair_band(gn, L.w, i - 1 - max(j, exact_upto),
                                        fminf(1.f + gn, a.dband), drift);
            }
        }
        nn += __popc(m);
        if (has) j = __float_as_int(h.w);
    }
    {
        // The G most recent non-bonded beads, one per lane.
        const int j = i - 1 - G + g.gl;
        float4 L = make_float4(0.f, 0.f, 0.f, 0.f);
        bool near = false;
        if (j >= 0) {
            const float4 h = w.hi[j], l = w.lo[j];
            const float gx = (ehx - h.x) + (elx - l.x);
            const float gy = (ehy - h.y) + (ely - l.y);
            const float gz = (ehz - h.z) + (elz - l.z);
            const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            L = make_float4(gx, gy, gz, 1.f + g2);
            near = g2 < a.rf2;
        }
        const unsigned m = g.vote(near);
        if (near) {
            const int slot = nn + __popc(m & g.below);
            w.nls[slot] = L;
            w.njs[slot] = j;
            if (LJ) {
                const float gn = fmaf(sqrtf(L.w - 1.f), 1.001f, 1e-6f);
                w.nbs[slot] = pair_band(gn, L.w, i - 1 - max(j, exact_upto),
                                        fminf(1.f + gn, a.dband), drift);
            }
        }
        nn += __popc(m);
    }
    __syncwarp(g.mask);
    for (int p = g.gl; p < nn; p += G) {
        const int jp = w.njs[p];
        int r = 0;
        for (int t = 0; t < nn; ++t) r += w.njs[t] < jp;
        w.nl[r] = w.nls[p];
        w.nj[r] = jp;
        if (LJ) w.nb[r] = w.nbs[p];
    }
    return nn;
}

// Grow chain c (local index) of the ensemble a with the G lanes of group g,
// in the per-chain storage w (shared memory; for kLong, device memory with a
// cell grid, generation counter *genp).  With kDefer the FP64 re-decision is
// not compiled in: a chain that meets a step its FP32 arithmetic cannot
// decide sets its bit in a.deferred and stops without writing anything; a
// second pass grows it again, from the start, with the FP64 path.  In restart mode a growth that
// reaches a dead end is thrown away and the chain grown again from bead 0,
// with the attempt index in the high half of the step word.
template <int G, int T, bool LJ, class W = ChainSmem, bool kDefer = false, bool kFly = false>
__device__ __forceinline__ void off_chain(const OffArgs &a, int64_t c, const W &w,
                                          const Group<G> &g, const float *logm,
                                          uint32_t *genp = nullptr)
{
    constexpr bool kLong = !std::is_same<W, ChainSmem>::value;
    // Lennard-Jones groups whose lanes hold several trials (k > 32) commit
    // float-float directions: their many trials make FP64 re-decisions the
    // larger cost, and the positions then drift by ~1e-12 per step instead
    // of 4e-7, so the error bands shrink.  (At k <= 32 the extra commit work
    // costs about what the saved re-decisions gain.)  The drift of the band
    // follows the commit mode of this instantiation.
    constexpr bool kFF = LJ && G * T > 32;
    const float drift = kFF ? a.drift : 4e-7f;
    const int N = a.N, k = a.k;
    const uint32_t chain = a.chain0 + (uint32_t)c;

    if (g.gl == 0) {
        w.hi[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        w.lo[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float ehx, ehy, ehz, elx, ely, elz;
    float lw;
    int dead_at;
    int exact_upto;   // beads 0..exact_upto are exact (r_0; after a replay at step i: all < i)
    unsigned rechecks = 0;
    unsigned long long listed = 0;
    uint32_t att = 0;
    for (;;) {
        const uint32_t aw = att << 16;
        ehx = ehy = ehz = elx = ely = elz = 0.f;
        lw = 0.f;
        dead_at = 0;
        exact_upto = 0;
        uint64_t tag = 0;
        int cell[3] = {INT_MIN, 0, 0}, heads[2] = {-1, -1};   // long chains: cached cell heads
        if constexpr (kLong) {
            // A fresh generation of the cell grid for this growth (beads are
            // filed G steps after they are placed).
            if (++*genp > kCellGenMax) {
                for (int h = g.gl; h < (1 << w.logH); h += G) w.cells[h] = make_uint4(0u, 0u, 0u, 0u);
                *genp = 1;
                __syncwarp(g.mask);
            }
            tag = (uint64_t)*genp << kCellGenShift;
        }

        for (int i = 1; i < N; ++i) {
            // ---- 1. near list (ascending bead index) --------------------------
            int nn = 0;
            float band = 0.f;    // largest bead band of the step (hard spheres)
            if constexpr (kLong)
                nn = long_near_list<G, LJ>(a, w, g, i, tag, ehx, ehy, ehz, elx, ely, elz,
                                           exact_upto, drift, cell, heads);
            for (int b0 = 0; !kLong && b0 <= i - 2; b0 += G) {
                const int j = b0 + g.gl;
                float4 L = make_float4(0.f, 0.f, 0.f, 0.f);
                bool near = false;
                if (j <= i - 2) {
                    const float4 h = w.hi[j], l = w.lo[j];
                    const float gx = (ehx - h.x) + (elx - l.x);
                    const float gy = (ehy - h.y) + (ely - l.y);
                    const float gz = (ehz - h.z) + (elz - l.z);
                    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
                    L = make_float4(gx, gy, gz, 1.f + g2);
                    near = g2 < a.rf2;
                }
                const unsigned m = g.vote(near);
                if (near) {
                    const int slot = nn + __popc(m & g.below);
                    w.nl[slot] = L;
                    w.nj[slot] = j;
                    if (LJ) {
                        const float gn = fmaf(sqrtf(L.w - 1.f), 1.001f, 1e-6f);
                        w.nb[slot] =
                            pair_band(gn, L.w, i - 1 - max(j, exact_upto),
                                      fminf(1.f + gn, a.dband), drift);
                    }
                }
                nn += __popc(m);
            }
            listed += (unsigned)nn;
            __syncwarp(g.mask);
            if (!LJ && nn > 0) {
                // One band for the step: the oldest listed bead drifted longest, and
                // |g| <= sqrt(rf2), c <= 1 + rf2 for every listed bead.
                const int D = i - 1 - max(w.nj[0], exact_upto);
                band = pair_band(a.rf, 1.f + a.rf2, D, a.dband, drift);
            }

            // ---- 2. trials ----------------------------------------------------
            float ux[T], uy[T], uz[T];
            uint32_t twa[T], twb[T];   // the trials' words (for float-float commits)
            bool valid[T];
            uint32_t selw = 0;
            uint4 x = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int s = 0; s < T; ++s) {
                const int t = T * g.gl + s;
                valid[s] = t < k;
                if (T == 1 || (s & 1) == 0)
                    x = draw<kFly>(
                        a, make_uint4(chain, a.ens, (uint32_t)i | aw, 1u + (uint32_t)(t >> 1)));
                if (s == 0)
                    // The low bytes of the four words, x.x's lowest:
                    // (x.x & 0xFF) | (x.y & 0xFF) << 8 | (x.z & 0xFF) << 16 | ...
                    selw = __byte_perm(__byte_perm(x.x, x.y, 0x0040u),
                                       __byte_perm(x.z, x.w, 0x0040u), 0x5410u);
                uint32_t wa, wb;
                trial_words(x, t, wa, wb);
                twa[s] = wa;
                twb[s] = wb;
                const float3 u = dir32x2(wa, wb);   // 2u: d^2 = c + (2u).g
                ux[s] = u.x;
                uy[s] = u.y;
                uz[s] = u.z;
            }
            selw = g.bcast(selw, 0);

            // ---- 3. pair loop -----------------------------------------------
            float mind[T], U[T], Ub[T], Ua[T];
            int ncut[T];
#pragma unroll
            for (int s = 0; s < T; ++s) {
                mind[s] = INFINITY;
                U[s] = 0.f;
                Ub[s] = 0.f;
                Ua[s] = 0.f;
                ncut[s] = 0;
            }
#pragma unroll 2
            for (int q = 0; q < nn; ++q) {
                const float4 L = w.nl[q];
                const float bq = LJ ? w.nb[q] : 0.f;
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    const float d2 = fmaf(ux[s], L.x, fmaf(uy[s], L.y, fmaf(uz[s], L.z, L.w)));
                    if (!LJ) {
                        mind[s] = fminf(mind[s], d2);
                    } else {
                        if (d2 < a.rc2) {
                            const float sr = __fdividef(a.sig2, d2);
                            const float s3 = sr * sr * sr;
                            const float e = s3 * (s3 - 1.f);
                            U[s] += e;
                            Ua[s] += fabsf(e);
                            Ub[s] = fmaf(sr * s3, fabsf(2.f * s3 - 1.f) * bq, Ub[s]);
                        }
                        ncut[s] += fabsf(d2 - a.rc2) < bq;
                    }
                }
            }

            // ---- 4. weights, selection, error bounds ---------------------------
            int sel = -1;
            float logS = 0.f;
            bool ok = true;
            if (!LJ) {
                bool fr[T], flag = false;
                int cnt = 0;
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    fr[s] = valid[s] && mind[s] >= a.sig2;
                    flag |= valid[s] && fabsf(mind[s] - a.sig2) < band;
                    cnt += fr[s];
                }
                if (g.vote(flag)) {
                    ok = false;
                } else {
                    const int incl = g.scan(cnt);
                    const int m = g.bcast(incl, G - 1);
                    if (m == 0) {
                        dead_at = i;
                    } else {
                        const int idx = (int)__umulhi(selw, (uint32_t)m);
                        int mine = -1, seen = incl - cnt;
#pragma unroll
                        for (int s = 0; s < T; ++s)
                            if (fr[s]) {
                                if (seen == idx) mine = T * g.gl + s;
                                ++seen;
                            }
                        const unsigned who = g.ballot(mine >= 0);
                        sel = g.bcast(mine, __ffs(who) - 1);
                        logS = logm[m];
                    }
                }
            } else {
                float bu[T], bmin = INFINITY;
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    bu[s] = valid[s] ? (a.beta4 == 0.f ? 0.f : a.beta4 * U[s]) : INFINITY;
                    bmin = fminf(bmin, bu[s]);
                }
                bmin = g.min(bmin);
                if (bmin == INFINITY) {
                    dead_at = i;
                } else {
                    float wt[T], own = 0.f, err = 0.f;
#pragma unroll
                    for (int s = 0; s < T; ++s) {
                        wt[s] = exp2f(-(bu[s] - bmin) * 1.4426950408889634f);
                        own += wt[s];
                        // |d(bu)/d(d^2)| = 4 beta eps (3 / sigma^2) s^4 |2 s^6 - 1| per
                        // pair, the FP32 rounding of the pair terms, and the jump of
                        // pairs within the band of the cutoff; doubled.
                        // (Ub already carries each bead's own band.)  Trials of
                        // zero weight contribute no error (and would give 0 * inf).
                        const float dbu =
                            a.beta4 * fmaf(6.f / a.sig2, Ub[s],
                                           fmaf(1e-6f, Ua[s], a.ucut2 * (float)ncut[s]));
                        if (wt[s] > 0.f)
                            err = fmaf(wt[s], dbu + fmaf(1.2e-7f, bu[s] - bmin, 3e-7f), err);
                    }
                    const float incl = g.scan(own);
                    const float S = g.bcast(incl, G - 1);
                    const float E = fmaf(S * 6e-8f, (float)(k + 2), g.sum(err));
                    const float r = u24f(selw) * S;
                    float P = incl - own;
                    int mine = -1;
                    float lo = 0.f, hi = 0.f;
#pragma unroll
                    for (int s = 0; s < T; ++s) {
                        const float Pn = P + wt[s];
                        if (mine < 0 && Pn > r && wt[s] > 0.f) {
                            mine = T * g.gl + s;
                            lo = P;
                            hi = Pn;
                        }
                        P = Pn;
                    }
                    const unsigned who = g.ballot(mine >= 0);
                    if (who == 0u) {
                        ok = false;
                    } else {
                        const int src = __ffs(who) - 1;
                        sel = g.bcast(mine, src);
                        lo = g.bcast(lo, src);
                        hi = g.bcast(hi, src);
                        if (!(r - lo > E) || !(hi - r > E)) ok = false;
                        logS = __logf(S) - bmin;
                    }
                }
            }

            // ---- 5. FP64 re-decision of an ambiguous step -------------------
            if (!ok) {
                if constexpr (kDefer) {
                    if (g.gl == 0) atomicOr(&a.deferred[c >> 5], 1u << (c & 31));
                    return;
                } else {
                    ++rechecks;
                    redecide<G, T, LJ, kFly>(a, w, g, chain, aw, exact_upto, i, nn, selw, logm, ehx,
                                       ehy, ehz, elx, ely, elz, sel, logS, dead_at);
                    exact_upto = i - 1;
                }
            }
            if (dead_at) break;

            // ---- 6. commit ----------------------------------------------------
            {
                const int ss = sel % T;
                const int src = sel / T;
                if constexpr (kFF) {
                    // The chosen trial's direction in float-float, so that
                    // positions drift by ~1e-12 per step instead of 4e-7.
                    uint32_t wa = 0u, wb = 0u;
#pragma unroll
                    for (int s = 0; s < T; ++s)
                        if (s == ss) {
                            wa = twa[s];
                            wb = twb[s];
                        }
                    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, zz = 0.f;
                    if (g.gl == src) dir_ff(wa, wb, xh, xl, yh, yl, zz);
                    xh = g.bcast(xh, src);
                    xl = g.bcast(xl, src);
                    yh = g.bcast(yh, src);
                    yl = g.bcast(yl, src);
                    zz = g.bcast(zz, src);
                    ff_sum(ehx, elx, xh, xl, ehx, elx);
                    ff_sum(ehy, ely, yh, yl, ehy, ely);
                    ff_add(ehz, elz, zz);
                } else {
                    float vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
                    for (int s = 0; s < T; ++s)
                        if (s == ss) {
                            vx = ux[s];
                            vy = uy[s];
                            vz = uz[s];
                        }
                    // (ux holds 2u: the commit adds half of it.)
                    ff_add_half(ehx, elx, g.bcast(vx, src));
                    ff_add_half(ehy, ely, g.bcast(vy, src));
                    ff_add_half(ehz, elz, g.bcast(vz, src));
                }
                if (g.gl == 0) {
                    // (.w: a long chain's cell link, set when the bead is filed)
                    w.hi[i] = make_float4(ehx, ehy, ehz, 0.f);
                    w.lo[i] = make_float4(elx, ely, elz, 0.f);
                    w.tr[i] = (uint8_t)sel;
                }
                lw += logS;
            }
            __syncwarp(g.mask);
        }
        if (!dead_at || att + 1 >= a.max_att) break;
        ++att;
        __syncwarp(g.mask);
    }

    if (a.attempts && g.gl == 0) a.attempts[c] = (uint16_t)(att + 1);
    if (a.counters && g.gl == 0) {
        if (rechecks) atomicAdd(&a.counters[0], (unsigned long long)rechecks);
        atomicAdd(&a.counters[1], 1ull);
        atomicAdd(&a.counters[2], listed);
    }
    const int64_t C = a.C;
    if (dead_at) {
        if (g.gl == 0) {
            if (a.logw) a.logw[c] = -INFINITY;
            if (a.r2) a.r2[c] = 0.f;
            if (a.rg2) a.rg2[c] = 0.f;
            if (a.alive) a.alive[c] = 0;
        }
        if (a.trace)
            for (int s = 1 + g.gl; s < N; s += G)
                a.trace[(int64_t)(s - 1) * C + c] =
                    s < dead_at ? w.tr[s] : (s == dead_at ? 0xFEu : 0xFFu);
        if (a.coords)
            for (int s = g.gl; s < N; s += G) {
                const bool keep = s < dead_at;
                const float4 h = w.hi[s], l = w.lo[s];
                a.coords[((int64_t)s * 3 + 0) * C + c] = keep ? h.x + l.x : 0.f;
                a.coords[((int64_t)s * 3 + 1) * C + c] = keep ? h.y + l.y : 0.f;
                a.coords[((int64_t)s * 3 + 2) * C + c] = keep ? h.z + l.z : 0.f;
            }
        return;
    }
    // Observables: R_ee^2 and R_g^2 about the centre of mass.
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int s = g.gl; s < N; s += G) {
        const float4 h = w.hi[s], l = w.lo[s];
        sx += h.x + l.x;
        sy += h.y + l.y;
        sz += h.z + l.z;
    }
    const float inv = 1.f / (float)N;
    const float mx = g.sum(sx) * inv, my = g.sum(sy) * inv, mz = g.sum(sz) * inv;
    float gg = 0.f;
    for (int s = g.gl; s < N; s += G) {
        const float4 h = w.hi[s], l = w.lo[s];
        const float dx = (h.x - mx) + l.x, dy = (h.y - my) + l.y, dz = (h.z - mz) + l.z;
        gg += fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    }
    gg = g.sum(gg) * inv;
    if (g.gl == 0) {
        const float xe = ehx + elx, ye = ehy + ely, ze = ehz + elz;
        if (a.logw) a.logw[c] = lw;
        if (a.r2) a.r2[c] = fmaf(xe, xe, fmaf(ye, ye, ze * ze));
        if (a.rg2) a.rg2[c] = gg;
        if (a.alive) a.alive[c] = 1;
    }
    if (a.trace)
        for (int s = 1 + g.gl; s < N; s += G) a.trace[(int64_t)(s - 1) * C + c] = w.tr[s];
    if (a.coords)
        for (int s = g.gl; s < N; s += G) {
            const float4 h = w.hi[s], l = w.lo[s];
            a.coords[((int64_t)s * 3 + 0) * C + c] = h.x + l.x;
            a.coords[((int64_t)s * 3 + 1) * C + c] = h.y + l.y;
            a.coords[((int64_t)s * 3 + 2) * C + c] = h.z + l.z;
        }
}


constexpr int kTable = 132;   // log m, m = 0..131: 528 bytes keep per-chain areas aligned

__device__ __forceinline__ void fill_log_table(float *logm)
{
    for (int q = threadIdx.x; q < kTable; q += blockDim.x) logm[q] = q ? logf((float)q) : 0.f;
}

}  // namespace
}  // namespace rosen
