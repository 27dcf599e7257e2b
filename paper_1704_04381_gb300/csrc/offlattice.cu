// offlattice.cu -- Rosenbluth growth in real space (Guo & Baulin, Section
// 3.3.3, Algorithm 2): k trial positions on the unit sphere around the chain
// end, scored against every earlier non-bonded bead by hard-sphere overlap or
// a truncated Lennard-Jones energy; W is multiplied by the sum of the trial
// weights and one trial is drawn in proportion to its weight.
//
// GB300 mapping: one warp per chain, lanes = trials (T = k/32 trials per
// lane beyond 32).  Each step:
//  1. lanes scan the earlier beads 32 at a time and keep, in ballot order
//     (ascending bead index), those within 1 + R of the end (R = sigma or
//     the cutoff); only those can reach a trial.  The kept displacement
//     g = end - r_j and c = 1 + |g|^2 go to a shared list;
//  2. every lane draws its trial direction u (Philox, 24-bit uniforms) and
//     evaluates d^2 = |g + u|^2 = c + 2 g.u against the list (three FMAs per
//     pair, list entries broadcast from shared memory);
//  3. free flags / weights are combined with ballots and a warp scan, and the
//     selection draw picks the trial.
// Positions are float-float (hi + lo) sums of the FP32 directions, so they
// carry only the directions' own rounding.  Every FP32 decision comes with a
// bound on its distance from the FP64 result (d^2 within G_i of sigma^2 or
// of the cutoff, or the selection draw within E of a prefix-sum boundary);
// when the bound is not met the warp replays the chain's exact positions in
// FP64 and re-decides the step with the sequential FP64 arithmetic, so the
// grown path is the one an FP64 implementation of the same rule takes.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace rosen {
namespace {

constexpr int kWarp = 32;

struct OffArgs {
    PhiloxKeys key;
    uint32_t ens, chain0;
    int32_t N, k, lj;
    int64_t C;
    float sig2, rc2, rf2;      // sigma^2, cutoff^2, list radius^2 (with margin)
    float beta4;               // 4 beta eps (LJ)
    float band0, band1;        // decision band G_i = band0 + band1 * i on d^2
    float ucut2;               // 2 |s^6 (s^6 - 1)| at the cutoff: energy jump (doubled)
    double sig2d, rc2d, beta_eps;
    float *logw, *r2, *rg2;
    uint8_t *alive, *trace;
    float *coords;
    unsigned long long *counters;   // optional [3]: steps re-decided, chains, list entries
};

// Per-warp shared memory layout (N = chain length).
struct WarpSmem {
    float *hx, *hy, *hz, *lx, *ly, *lz;   // float-float positions [N]
    float4 *nl;                           // near list: g.x, g.y, g.z, 1 + |g|^2
    int *nj;                              // near list: bead index
    uint8_t *tr;                          // chosen trial per step
    double *R;                            // FP64 replay scratch [N][3]
};

__host__ __device__ inline size_t warp_smem_bytes(int N)
{
    const size_t n = (size_t)N;
    size_t b = 0;
    b += 6 * n * sizeof(float);
    b = (b + 15) & ~size_t(15);
    b += n * sizeof(float4) + n * sizeof(int);
    b += (n + 15) & ~size_t(15);
    b = (b + 15) & ~size_t(15);
    b += 3 * n * sizeof(double);
    return (b + 15) & ~size_t(15);
}

__device__ inline WarpSmem carve(unsigned char *base, int N)
{
    WarpSmem w;
    float *f = reinterpret_cast<float *>(base);
    w.hx = f;
    w.hy = f + N;
    w.hz = f + 2 * N;
    w.lx = f + 3 * N;
    w.ly = f + 4 * N;
    w.lz = f + 5 * N;
    size_t off = (6 * (size_t)N * sizeof(float) + 15) & ~size_t(15);
    w.nl = reinterpret_cast<float4 *>(base + off);
    off += (size_t)N * sizeof(float4);
    w.nj = reinterpret_cast<int *>(base + off);
    off += (size_t)N * sizeof(int);
    w.tr = base + off;
    off += ((size_t)N + 15) & ~size_t(15);
    off = (off + 15) & ~size_t(15);
    w.R = reinterpret_cast<double *>(base + off);
    return w;
}

// Trial direction from two words (the reading of "rngonsphere"):
// z = 1 - 2 u24(a) and phi = 2 pi u24(b); (1-z), (1+z) and 2 u24(b) are exact
// in FP32, sincospif is within 1 ulp and sqrtf is correctly rounded, so each
// component is within 2.7e-7 of the exact direction.
__device__ __forceinline__ float3 dir32(uint32_t a, uint32_t b)
{
    const float z = 1.f - 2.f * u24f(a);
    const float s = sqrtf((1.f - z) * (1.f + z));
    float sn, cs;
    sincospif(2.f * u24f(b), &sn, &cs);
    return make_float3(s * cs, s * sn, z);
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

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_min_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// FP64 replay of the chain's positions r_0 .. r_{i-1} from the chosen trials:
// every lane recomputes the FP64 directions of its steps, then a warp scan
// accumulates them.  Writes R[3*j + axis].
__device__ __noinline__ void replay_positions(const OffArgs &a, const WarpSmem &w,
                                              uint32_t chain, int i, int lane)
{
    if (lane == 0) {
        w.R[0] = 0.0;
        w.R[1] = 0.0;
        w.R[2] = 0.0;
    }
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int base = 1; base <= i - 1; base += kWarp) {
        const int s = base + lane;
        double x = 0.0, y = 0.0, z = 0.0;
        if (s <= i - 1) {
            const int t = w.tr[s];
            const uint4 q = philox(make_uint4(chain, a.ens, (uint32_t)s, 1u + (uint32_t)(t >> 1)), a.key);
            uint32_t wa, wb;
            trial_words(q, t, wa, wb);
            dir64(wa, wb, x, y, z);
        }
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const double px = __shfl_up_sync(0xffffffffu, x, o);
            const double py = __shfl_up_sync(0xffffffffu, y, o);
            const double pz = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) {
                x += px;
                y += py;
                z += pz;
            }
        }
        x += cx;
        y += cy;
        z += cz;
        if (s <= i - 1) {
            w.R[3 * s + 0] = x;
            w.R[3 * s + 1] = y;
            w.R[3 * s + 2] = z;
        }
        cx = __shfl_sync(0xffffffffu, x, kWarp - 1);
        cy = __shfl_sync(0xffffffffu, y, kWarp - 1);
        cz = __shfl_sync(0xffffffffu, z, kWarp - 1);
    }
    __syncwarp();
}

template <int T>
__global__ void __launch_bounds__(256) offlattice_warp_kernel(const OffArgs a, int warps)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * warps + wib;
    if (c >= a.C) return;     // whole warps leave together
    const int N = a.N, k = a.k;
    const WarpSmem w = carve(smem_raw + (size_t)wib * warp_smem_bytes(N), N);
    const uint32_t chain = a.chain0 + (uint32_t)c;

    if (lane == 0) {
        w.hx[0] = w.hy[0] = w.hz[0] = 0.f;
        w.lx[0] = w.ly[0] = w.lz[0] = 0.f;
    }
    float ehx = 0.f, ehy = 0.f, ehz = 0.f, elx = 0.f, ely = 0.f, elz = 0.f;
    float lw = 0.f;
    int dead_at = 0;
    unsigned rechecks = 0;
    unsigned long long listed = 0;

    for (int i = 1; i < N; ++i) {
        // ---- 1. near list (ascending bead index) --------------------------
        int nn = 0;
        for (int base = 0; base <= i - 2; base += kWarp) {
            const int j = base + lane;
            float gx = 0.f, gy = 0.f, gz = 0.f, g2 = 0.f;
            bool near = false;
            if (j <= i - 2) {
                gx = (ehx - w.hx[j]) + (elx - w.lx[j]);
                gy = (ehy - w.hy[j]) + (ely - w.ly[j]);
                gz = (ehz - w.hz[j]) + (elz - w.lz[j]);
                g2 = gx * gx + gy * gy + gz * gz;
                near = g2 < a.rf2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, near);
            if (near) {
                const int slot = nn + __popc(m & ((1u << lane) - 1u));
                w.nl[slot] = make_float4(gx, gy, gz, 1.f + g2);
                w.nj[slot] = j;
            }
            nn += __popc(m);
        }
        listed += (unsigned)nn;
        __syncwarp();

        // ---- 2. trials ----------------------------------------------------
        float ux[T], uy[T], uz[T];
        bool valid[T];
        uint32_t selw;
        {
            uint4 x;
            int last_call = -1;
#pragma unroll
            for (int s = 0; s < T; ++s) {
                const int t = (T == 1) ? lane : T * lane + s;
                valid[s] = t < k;
                const int call = t >> 1;
                if (call != last_call) {
                    x = philox(make_uint4(chain, a.ens, (uint32_t)i, 1u + (uint32_t)call), a.key);
                    last_call = call;
                }
                if (s == 0 && lane == 0)
                    selw = (x.x & 0xFFu) | ((x.y & 0xFFu) << 8) | ((x.z & 0xFFu) << 16) |
                           ((x.w & 0xFFu) << 24);
                uint32_t wa, wb;
                trial_words(x, t, wa, wb);
                const float3 u = dir32(wa, wb);
                ux[s] = 2.f * u.x;   // 2u: d^2 = c + (2u).g
                uy[s] = 2.f * u.y;
                uz[s] = 2.f * u.z;
            }
            selw = __shfl_sync(0xffffffffu, selw, 0);
        }

        // ---- 3. pair loop -----------------------------------------------
        const float G = a.band0 + a.band1 * (float)i;
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
        if (!a.lj) {
            for (int q = 0; q < nn; ++q) {
                const float4 L = w.nl[q];
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    const float d2 = fmaf(ux[s], L.x, fmaf(uy[s], L.y, fmaf(uz[s], L.z, L.w)));
                    mind[s] = fminf(mind[s], d2);
                }
            }
        } else {
            for (int q = 0; q < nn; ++q) {
                const float4 L = w.nl[q];
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    const float d2 = fmaf(ux[s], L.x, fmaf(uy[s], L.y, fmaf(uz[s], L.z, L.w)));
                    if (d2 < a.rc2) {
                        const float sr = a.sig2 / d2;
                        const float s3 = sr * sr * sr;
                        const float e = s3 * (s3 - 1.f);
                        U[s] += e;
                        Ua[s] += fabsf(e);
                        Ub[s] += sr * s3 * fabsf(2.f * s3 - 1.f);
                    }
                    ncut[s] += fabsf(d2 - a.rc2) < G;
                }
            }
        }

        // ---- 4. weights, selection, error bounds ---------------------------
        int sel = -1;
        float logS = 0.f;
        bool ok = true;
        if (!a.lj) {
            bool fr[T], flag = false;
            int cnt = 0;
#pragma unroll
            for (int s = 0; s < T; ++s) {
                fr[s] = valid[s] && mind[s] >= a.sig2;
                flag |= valid[s] && fabsf(mind[s] - a.sig2) < G;
                cnt += fr[s];
            }
            if (__any_sync(0xffffffffu, flag)) {
                ok = false;
            } else {
                // Free trials in trial order: lane-major with T per lane.
                int pre = cnt;
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += v;
                }
                const int m = __shfl_sync(0xffffffffu, pre, kWarp - 1);
                pre -= cnt;
                if (m == 0) {
                    dead_at = i;
                } else {
                    const int idx = (int)__umulhi(selw, (uint32_t)m);
                    int mine = -1, seen = pre;
#pragma unroll
                    for (int s = 0; s < T; ++s)
                        if (fr[s]) {
                            if (seen == idx) mine = (T == 1) ? lane : T * lane + s;
                            ++seen;
                        }
                    const unsigned who = __ballot_sync(0xffffffffu, mine >= 0);
                    sel = __shfl_sync(0xffffffffu, mine, __ffs(who) - 1);
                    logS = logf((float)m);
                }
            }
        } else {
            float bu[T], bmin = INFINITY;
#pragma unroll
            for (int s = 0; s < T; ++s) {
                bu[s] = valid[s] ? a.beta4 * U[s] : INFINITY;
                if (a.beta4 == 0.f && valid[s]) bu[s] = 0.f;
                bmin = fminf(bmin, bu[s]);
            }
            bmin = warp_min(bmin);
            if (bmin == INFINITY) {
                dead_at = i;
            } else {
                float wt[T], own = 0.f, err = 0.f;
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    wt[s] = exp2f(-(bu[s] - bmin) * 1.4426950408889634f);
                    own += wt[s];
                    // |d(bu)/d(d^2)| = 4 beta eps (3 / sigma^2) s^4 |2 s^6 - 1| per pair,
                    // plus FP32 rounding of the pair terms and the jump of
                    // pairs that sit within the band of the cutoff; doubled.
                    const float dbu = a.beta4 * (6.f / a.sig2 * G * Ub[s] + 1e-6f * Ua[s] +
                                                 a.ucut2 * (float)ncut[s]);
                    err += wt[s] * (dbu + 1.2e-7f * (bu[s] - bmin) + 3e-7f);
                }
                float pre = own;
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const float v = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += v;
                }
                const float S = __shfl_sync(0xffffffffu, pre, kWarp - 1);
                const float E = warp_sum(err) + S * 6e-8f * (float)(k + 2);
                const float r = u24f(selw) * S;
                // Inclusive prefix of each of this lane's trials.
                float P = pre - own;
                int mine = -1;
                float lo = 0.f, hi = 0.f;
#pragma unroll
                for (int s = 0; s < T; ++s) {
                    const float Pn = P + wt[s];
                    if (mine < 0 && Pn > r && wt[s] > 0.f) {
                        mine = (T == 1) ? lane : T * lane + s;
                        lo = P;
                        hi = Pn;
                    }
                    P = Pn;
                }
                const unsigned who = __ballot_sync(0xffffffffu, mine >= 0);
                if (who == 0u) {
                    ok = false;
                } else {
                    const int src = __ffs(who) - 1;
                    sel = __shfl_sync(0xffffffffu, mine, src);
                    lo = __shfl_sync(0xffffffffu, lo, src);
                    hi = __shfl_sync(0xffffffffu, hi, src);
                    if (!(r - lo > E) || !(hi - r > E)) ok = false;
                    logS = logf(S) - bmin;
                }
            }
        }

        // ---- 5. FP64 re-decision of an ambiguous step -------------------
        if (!ok) {
            ++rechecks;
            replay_positions(a, w, chain, i, lane);
            const double ex = w.R[3 * (i - 1)], ey = w.R[3 * (i - 1) + 1], ez = w.R[3 * (i - 1) + 2];
            double val[T];
            uint4 x;
            int last_call = -1;
#pragma unroll
            for (int s = 0; s < T; ++s) {
                const int t = (T == 1) ? lane : T * lane + s;
                const int call = t >> 1;
                if (call != last_call) {
                    x = philox(make_uint4(chain, a.ens, (uint32_t)i, 1u + (uint32_t)call), a.key);
                    last_call = call;
                }
                uint32_t wa, wb;
                trial_words(x, t, wa, wb);
                double dx, dy, dz;
                dir64(wa, wb, dx, dy, dz);
                const double tx = ex + dx, ty = ey + dy, tz = ez + dz;
                double acc = 0.0;
                bool fr = true;
                for (int q = 0; q < nn; ++q) {
                    const int j = w.nj[q];
                    const double rx = tx - w.R[3 * j], ry = ty - w.R[3 * j + 1],
                                 rz = tz - w.R[3 * j + 2];
                    const double d2 = rx * rx + ry * ry + rz * rz;
                    if (!a.lj) {
                        if (d2 < a.sig2d) fr = false;
                    } else if (d2 < a.rc2d) {
                        const double sr = a.sig2d / d2;
                        const double s3 = sr * sr * sr;
                        acc += 4.0 * s3 * (s3 - 1.0);
                    }
                }
                if (!valid[s]) val[s] = a.lj ? INFINITY : 0.0;
                else if (!a.lj) val[s] = fr ? 1.0 : 0.0;
                else val[s] = (a.beta_eps == 0.0) ? 0.0 : a.beta_eps * acc;
            }
            if (!a.lj) {
                int cnt = 0;
#pragma unroll
                for (int s = 0; s < T; ++s) cnt += val[s] > 0.0;
                int pre = cnt;
#pragma unroll
                for (int o = 1; o < kWarp; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += v;
                }
                const int m = __shfl_sync(0xffffffffu, pre, kWarp - 1);
                pre -= cnt;
                if (m == 0) {
                    dead_at = i;
                } else {
                    const int idx = (int)__umulhi(selw, (uint32_t)m);
                    int mine = -1, seen = pre;
#pragma unroll
                    for (int s = 0; s < T; ++s)
                        if (val[s] > 0.0) {
                            if (seen == idx) mine = (T == 1) ? lane : T * lane + s;
                            ++seen;
                        }
                    const unsigned who = __ballot_sync(0xffffffffu, mine >= 0);
                    sel = __shfl_sync(0xffffffffu, mine, __ffs(who) - 1);
                    logS = logf((float)m);
                }
            } else {
                double bmin = INFINITY;
#pragma unroll
                for (int s = 0; s < T; ++s) bmin = fmin(bmin, val[s]);
                bmin = warp_min_d(bmin);
                if (bmin == INFINITY) {
                    dead_at = i;
                } else {
                    double wv64[T];
#pragma unroll
                    for (int s = 0; s < T; ++s) wv64[s] = exp(-(val[s] - bmin));
                    // Sequential FP64 sum and prefix in trial order, as the
                    // definition states them; every lane walks the trials.
                    double S = 0.0, r = 0.0, P = 0.0;
                    int pick = -1, lastpos = -1;
                    for (int pass = 0; pass < 2; ++pass) {
                        for (int t = 0; t < k; ++t) {
                            const int src = (T == 1) ? t : t / T;
                            const int ss = (T == 1) ? 0 : t % T;
                            double v = 0.0;
#pragma unroll
                            for (int s = 0; s < T; ++s)
                                if (s == ss) v = wv64[s];
                            const double wv = __shfl_sync(0xffffffffu, v, src);
                            if (pass == 0) {
                                S += wv;
                                if (wv > 0.0) lastpos = t;
                            } else if (pick < 0) {
                                P += wv;
                                if (P > r) pick = t;
                            }
                        }
                        if (pass == 0) r = u24d(selw) * S;
                    }
                    sel = pick >= 0 ? pick : lastpos;
                    logS = (float)(log(S) - bmin);
                }
            }
        }
        if (dead_at) break;

        // ---- 6. commit ----------------------------------------------------
        {
            const int src = (T == 1) ? sel : sel / T;
            const int ss = (T == 1) ? 0 : sel % T;
            float vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
            for (int s = 0; s < T; ++s)
                if (s == ss) {
                    vx = ux[s];
                    vy = uy[s];
                    vz = uz[s];
                }
            vx = 0.5f * __shfl_sync(0xffffffffu, vx, src);
            vy = 0.5f * __shfl_sync(0xffffffffu, vy, src);
            vz = 0.5f * __shfl_sync(0xffffffffu, vz, src);
            ff_add(ehx, elx, vx);
            ff_add(ehy, ely, vy);
            ff_add(ehz, elz, vz);
            if (lane == 0) {
                w.hx[i] = ehx;
                w.hy[i] = ehy;
                w.hz[i] = ehz;
                w.lx[i] = elx;
                w.ly[i] = ely;
                w.lz[i] = elz;
                w.tr[i] = (uint8_t)sel;
            }
            lw += logS;
        }
        __syncwarp();
    }

    if (a.counters && lane == 0) {
        if (rechecks) atomicAdd(&a.counters[0], (unsigned long long)rechecks);
        atomicAdd(&a.counters[1], 1ull);
        atomicAdd(&a.counters[2], listed);
    }
    const int64_t C = a.C;
    if (dead_at) {
        if (lane == 0) {
            if (a.logw) a.logw[c] = -INFINITY;
            if (a.r2) a.r2[c] = 0.f;
            if (a.rg2) a.rg2[c] = 0.f;
            if (a.alive) a.alive[c] = 0;
        }
        if (a.trace)
            for (int s = 1 + lane; s < N; s += kWarp)
                a.trace[(int64_t)(s - 1) * C + c] =
                    s < dead_at ? w.tr[s] : (s == dead_at ? 0xFEu : 0xFFu);
        if (a.coords)
            for (int s = lane; s < N; s += kWarp) {
                const bool keep = s < dead_at;
                a.coords[((int64_t)s * 3 + 0) * C + c] = keep ? w.hx[s] + w.lx[s] : 0.f;
                a.coords[((int64_t)s * 3 + 1) * C + c] = keep ? w.hy[s] + w.ly[s] : 0.f;
                a.coords[((int64_t)s * 3 + 2) * C + c] = keep ? w.hz[s] + w.lz[s] : 0.f;
            }
        return;
    }
    // Observables: R_ee^2 and R_g^2 about the centre of mass.
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int s = lane; s < N; s += kWarp) {
        sx += w.hx[s] + w.lx[s];
        sy += w.hy[s] + w.ly[s];
        sz += w.hz[s] + w.lz[s];
    }
    const float inv = 1.f / (float)N;
    const float mx = warp_sum(sx) * inv, my = warp_sum(sy) * inv, mz = warp_sum(sz) * inv;
    float g = 0.f;
    for (int s = lane; s < N; s += kWarp) {
        const float dx = (w.hx[s] - mx) + w.lx[s];
        const float dy = (w.hy[s] - my) + w.ly[s];
        const float dz = (w.hz[s] - mz) + w.lz[s];
        g += dx * dx + dy * dy + dz * dz;
    }
    g = warp_sum(g) * inv;
    if (lane == 0) {
        const float x = ehx + elx, y = ehy + ely, z = ehz + elz;
        if (a.logw) a.logw[c] = lw;
        if (a.r2) a.r2[c] = x * x + y * y + z * z;
        if (a.rg2) a.rg2[c] = g;
        if (a.alive) a.alive[c] = 1;
    }
    if (a.trace)
        for (int s = 1 + lane; s < N; s += kWarp) a.trace[(int64_t)(s - 1) * C + c] = w.tr[s];
    if (a.coords)
        for (int s = lane; s < N; s += kWarp) {
            a.coords[((int64_t)s * 3 + 0) * C + c] = w.hx[s] + w.lx[s];
            a.coords[((int64_t)s * 3 + 1) * C + c] = w.hy[s] + w.ly[s];
            a.coords[((int64_t)s * 3 + 2) * C + c] = w.hz[s] + w.lz[s];
        }
}

}  // namespace

int offlattice_validate(const rosen_offlattice_params *p, const rosen_offlattice_out *o)
{
    if (!p || !o) return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: NULL params or outputs");
    if (p->N < 2 || p->N > ROSEN_OFFLATTICE_NMAX)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: N = %d outside [2, %d]", p->N,
                         ROSEN_OFFLATTICE_NMAX);
    if (p->k < 1 || p->k > ROSEN_KMAX)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: k = %d outside [1, %d]", p->k,
                         ROSEN_KMAX);
    if (p->C < 0 || p->chain0 < 0 || p->chain0 + p->C > (int64_t(1) << 32))
        return set_error(ROSEN_EINVAL,
                         "rosen_offlattice_grow: chains [%lld, %lld) outside [0, 2^32)",
                         (long long)p->chain0, (long long)(p->chain0 + p->C));
    if (p->potential != ROSEN_HARD_SPHERE && p->potential != ROSEN_LJ)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: unknown potential %d", p->potential);
    if (!(p->sigma >= 0.0) || !isfinite(p->sigma) || p->sigma > 4.0)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: sigma must lie in [0, 4]");
    if (p->potential == ROSEN_LJ &&
        (!(p->cutoff > 0.0) || !isfinite(p->cutoff) || p->cutoff > 8.0 || p->sigma <= 0.0))
        return set_error(ROSEN_EINVAL,
                         "rosen_offlattice_grow: LJ needs sigma > 0 and 0 < cutoff <= 8");
    if (!(p->beta_eps >= 0.0) || !isfinite(p->beta_eps))
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: beta_eps must be finite and >= 0");
    if (p->flags & ~(ROSEN_STORE_TRACE | ROSEN_STORE_COORDS))
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: unknown flags 0x%x", p->flags);
    if ((p->flags & ROSEN_STORE_TRACE) && !o->trace)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: ROSEN_STORE_TRACE without trace");
    if ((p->flags & ROSEN_STORE_COORDS) && !o->coords)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: ROSEN_STORE_COORDS without coords");
    if (p->lanes_per_chain != 0 && p->lanes_per_chain != 32)
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow: lanes_per_chain must be 0 or 32");
    return ROSEN_OK;
}

static int warps_per_block(int N)
{
    const size_t budget = 100 * 1024;
    int W = 8;
    while (W > 1 && (size_t)W * warp_smem_bytes(N) > budget) --W;
    return W;
}

int offlattice_launch(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                      unsigned long long *counters, cudaStream_t s)
{
    OffArgs a;
    memset(&a, 0, sizeof a);
    a.key = philox_keys(p->seed);
    a.ens = p->ensemble;
    a.chain0 = (uint32_t)p->chain0;
    a.N = p->N;
    a.k = p->k;
    a.lj = p->potential == ROSEN_LJ;
    a.C = p->C;
    const double sig = p->sigma;
    const double R = a.lj ? p->cutoff : sig;
    a.sig2 = (float)(sig * sig);
    a.rc2 = a.lj ? (float)(p->cutoff * p->cutoff) : 0.f;
    a.rf2 = (float)((1.0 + R) * (1.0 + R) * 1.001 + 1e-3);
    a.beta4 = a.lj ? (float)(4.0 * p->beta_eps) : 0.f;
    // Decision band: |d^2 (FP32) - d^2 (FP64)| <= 2 (1+R) (i e_u + e_g) + e_eval
    // with e_u = 4e-7 (per-step direction error), e_g = 4.1e-7 (rounding of g)
    // and e_eval the three FMA roundings of values up to (1+R)^2; doubled.
    const double f = 2.0 * (1.0 + R);
    const double ev = 3.0 * 0.5 * 1.19209290e-7 * (1.0 + R) * (1.0 + R) * 2.0;
    a.band1 = (float)(2.0 * f * 4e-7);
    a.band0 = (float)(2.0 * (f * (4e-7 + 4.1e-7) + ev));
    if (a.lj) {
        const double sc = (sig * sig) / (p->cutoff * p->cutoff), s3 = sc * sc * sc;
        a.ucut2 = (float)(2.0 * fabs(s3 * (s3 - 1.0)));
    }
    a.sig2d = sig * sig;
    a.rc2d = a.lj ? p->cutoff * p->cutoff : 0.0;
    a.beta_eps = p->beta_eps;
    a.logw = o->logw;
    a.r2 = o->r2;
    a.rg2 = o->rg2;
    a.alive = o->alive;
    a.trace = (p->flags & ROSEN_STORE_TRACE) ? o->trace : nullptr;
    a.coords = (p->flags & ROSEN_STORE_COORDS) ? o->coords : nullptr;
    a.counters = counters;

    const int W = warps_per_block(p->N);
    const size_t smem = (size_t)W * warp_smem_bytes(p->N);
    const int64_t blocks = (p->C + W - 1) / W;
    if (p->k <= 32) {
        cudaFuncSetAttribute(offlattice_warp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        offlattice_warp_kernel<1><<<(unsigned)blocks, 32 * W, smem, s>>>(a, W);
    } else if (p->k <= 64) {
        cudaFuncSetAttribute(offlattice_warp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        offlattice_warp_kernel<2><<<(unsigned)blocks, 32 * W, smem, s>>>(a, W);
    } else {
        cudaFuncSetAttribute(offlattice_warp_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        offlattice_warp_kernel<4><<<(unsigned)blocks, 32 * W, smem, s>>>(a, W);
    }
    return check_launch("rosen_offlattice_grow");
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
