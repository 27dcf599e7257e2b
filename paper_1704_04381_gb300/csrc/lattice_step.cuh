// lattice_step.cuh -- the device code of one cubic-lattice growth step
// (Guo & Baulin, Section 3.3.2, Algorithm 1; weight of Eq. 3), shared by the
// lattice kernels (lattice.cu) and the PERM kernels (perm.cu): the packed
// monomer keys, the displacement table that turns a packed displacement into
// occupancy and contact increments, the kernel arguments of an ensemble, and
// the neighbour selection (FP32 with an exact FP64 fallback).
#pragma once

#include <math.h>

#include "common.cuh"

namespace rosen {
namespace {

constexpr uint32_t kFieldMask = 0x00701C07u;                  // 3-bit fields at 0, 10, 20
constexpr uint32_t kNearBias = 2u | (2u << 10) | (2u << 20);  // +2 on every axis
constexpr uint32_t kOriginKey = 512u | (512u << 10) | (512u << 20);
constexpr int kLutWords = 512;
constexpr int kSelBytes = 512;

// One multiply gathers the three 3-bit fields of an in-box displacement into
// bits 23..31 of the product -- y at 23..25, z at 26..28, x at 29..31 -- and
// a shift by 21 leaves them at bits 2..10: the byte offset of table entry
// y + 8 z + 64 x.  The other partial products (x 2^13, x 2^6, y 2^6; the
// rest overflow past bit 31) sum to less than 2^19, so nothing carries into
// bits 19 and up.
constexpr uint32_t kGather = (1u << 29) | (1u << 13) | (1u << 6);
constexpr uint32_t kZeroOff = 511u * 4u;   // fields (7,7,7): outside the box, entry 0

// Byte offset of displacement t's table entry if the monomer lies in the
// 5x5x5 box around the end, else of the zero entry.
__device__ __forceinline__ uint32_t lut_off(uint32_t t)
{
    const uint32_t off = (t * kGather) >> 21;
    return ((t & ~kFieldMask) == 0u) ? off : kZeroOff;
}

__device__ __forceinline__ uint32_t lut_at(const uint32_t *lut, uint32_t off)
{
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const unsigned char *>(lut) + off);
}

// Table entry for an earlier monomer at displacement d from the chain end.
// Bits 0..5: d is neighbour n of the end (neighbour n is occupied).
// Bits 8+3n..10+3n: the monomer is at lattice distance 1 from neighbour n
// (one non-bonded contact for a monomer placed there).
__device__ uint32_t lut_entry(int idx)
{
    const int dy = (idx & 7) - 2, dz = ((idx >> 3) & 7) - 2, dx = ((idx >> 6) & 7) - 2;
    if (dx > 2 || dy > 2 || dz > 2) return 0u;
    if (dx == 0 && dy == 0 && dz == 0) return 0u;
    uint32_t e = 0u;
    for (int n = 0; n < 6; ++n) {
        const int ex = (n == 0) - (n == 1), ey = (n == 2) - (n == 3), ez = (n == 4) - (n == 5);
        const int l1 = abs(dx - ex) + abs(dy - ey) + abs(dz - ez);
        if (l1 == 0) e |= 1u << n;
        else if (l1 == 1) e += 1u << (8 + 3 * n);
    }
    return e;
}

// Position of the (idx+1)-th set bit of a 6-bit mask (selection table).
__device__ uint8_t nth_set_bit(uint32_t mask, uint32_t idx)
{
    uint32_t seen = 0;
    for (int n = 0; n < 6; ++n)
        if ((mask >> n) & 1u) {
            if (seen == idx) return (uint8_t)n;
            ++seen;
        }
    return 0xFFu;
}

__device__ __forceinline__ void fill_tables(uint32_t *lut, uint8_t *seltab)
{
    for (int q = threadIdx.x; q < kLutWords; q += blockDim.x) {
        lut[q] = lut_entry(q);
        seltab[q] = nth_set_bit((uint32_t)q >> 3, (uint32_t)q & 7u);
    }
}

struct LatticeArgs {
    PhiloxKeys key;
    uint32_t ens, chain0;
    int32_t N, isaw;
    int64_t C;
    float wt32[8];    // exp(beta_eps * c), c = 0..5, rounded to FP32
    double wt64[8];   // the same in FP64
    float logm[8];    // log(m), m = 0..6 (athermal log W from counts)
    uint4 *counts;    // [C] packed 8 x u16
    float *logw;
    int32_t *r2;
    int64_t *n2rg2;
    uint8_t *trace;   // [N-1][C]
    int32_t *coords;  // [N][3][C]
    uint16_t *attempts;   // [C]
    uint32_t max_att;     // growths per chain (1: no restart)
};

// The FP64 selection, in exactly the order of the sequential definition:
// S = sum of the weights in slot order, r = u24(x) * S, first slot whose
// running prefix exceeds r, else the last slot with a positive weight.
__device__ __noinline__ int select_fp64(uint32_t freem, uint32_t acc, uint32_t x,
                                        const double *wt64)
{
    double w[6], S = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const uint32_t cd = (acc >> (8 + 3 * d)) & 7u;
        w[d] = ((freem >> d) & 1u) ? wt64[cd] : 0.0;
        S = __dadd_rn(S, w[d]);
    }
    const double r = __dmul_rn(u24d(x), S);
    double P = 0.0;
    int sel = -1;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        P = __dadd_rn(P, w[d]);
        if (sel < 0 && P > r) sel = d;
    }
    if (sel < 0)
#pragma unroll
        for (int d = 0; d < 6; ++d)
            if (w[d] > 0.0) sel = d;
    return sel;
}

// log W of an interacting chain: the running product of its step factors S
// (each >= 1, finite: beta_eps <= 16) as an FP32 mantissa in [1, 2) and an
// integer exponent, so that a step costs a multiply and an exact rescale
// instead of a logarithm; log W = log(mantissa) + exponent ln 2 once, at the
// end.  Each product rounds by at most 2^-24, so log W is within
// (N - 1) 6e-8 of the exact sum of the logarithms, plus the final rounding.
struct LogW {
    float m = 1.f;
    int e = 0;
    __device__ __forceinline__ void mul(float S)
    {
        const int b = __float_as_int(m * S);
        const int k = ((b >> 23) & 0xFF) - 127;
        m = __int_as_float(b - (k << 23));
        e += k;
    }
    __device__ __forceinline__ float value() const
    {
        constexpr float kLn2Hi = 0.693145751953125f;        // ln 2 to 16 bits
        constexpr float kLn2Lo = 1.428606820309417e-6f;     // ln 2 - kLn2Hi
        const float E = (float)e;
        return fmaf(E, kLn2Hi, fmaf(E, kLn2Lo, logf(m)));
    }
};

// The neighbour taken at one step, in slot order, from the free mask, the
// contact fields of acc (bits 8+3d..10+3d: contacts of neighbour d) and the
// step's draw x.  Athermal: the idx-th free neighbour, idx = floor(x m / 2^32).
// Interacting: the smallest slot whose FP32 prefix sum of exp(beta_eps c_d)
// exceeds r = u24(x) S, re-taken in FP64 when r lies within 2^-18 S of the
// slot's bounds; S goes into the chain's weight product lw.
template <bool kIsaw>
__device__ __forceinline__ int choose(uint32_t freem, int m, uint32_t acc, uint32_t x,
                                      const uint8_t *seltab, const float *wt32,
                                      const double *wt64, LogW &lw)
{
    if (!kIsaw) return seltab[(freem << 3) | __umulhi(x, (uint32_t)m)];
    float w[6], S = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const uint32_t cd = (acc >> (8 + 3 * d)) & 7u;
        w[d] = ((freem >> d) & 1u) ? wt32[cd] : 0.f;
        S += w[d];
    }
    const float r = u24f(x) * S;
    float P = 0.f, lo = 0.f, hi = 0.f;
    int sel = -1;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const float Pn = P + w[d];
        if (sel < 0 && Pn > r) {
            sel = d;
            lo = P;
            hi = Pn;
        }
        P = Pn;
    }
    const float tol = S * 0x1p-18f;
    if (sel < 0 || !(r - lo > tol) || !(hi - r > tol)) sel = select_fp64(freem, acc, x, wt64);
    lw.mul(S);
    return sel;
}

}  // namespace
}  // namespace rosen
