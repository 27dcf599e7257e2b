/*
 * rosen_oracle.c -- plain, slow CPU oracle for Rosenbluth chain growth.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (the CUDA library and its Python binding) never calls it.
 *
 * Everything here is FP64 and follows the method step by step, in the
 * order Guo & Baulin describe it (arxiv 1704.04381):
 *   - Eq. 3: the Rosenbluth weight W_n is the product over growth steps of
 *     the number of ways the chain can continue (Section 2).
 *   - Algorithm 1 (Section 3.3.2): cubic-lattice growth; we score all six
 *     neighbours of the chain end instead of blind trials (reading G4).
 *   - Algorithm 2 (Section 3.3.3): real-space growth with k trial positions
 *     on the unit sphere around the end; W is multiplied by the sum of the
 *     trial weights (reading G5).
 *   - Eq. 1-2 (Section 2): the W-weighted estimator of an ensemble mean.
 *   - Eq. 9 (Section 4.2): Z_N estimated by the mean Rosenbluth weight.
 * The readings where the paper is silent or garbled (energies, selection
 * rule, RNG stream layout, dead ends) are stated in the comments below where
 * they are used.
 *
 * Random numbers: Philox4x32-10 from Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11), keyed by the
 * 64-bit seed and indexed by (chain, ensemble, step, slot).  Written here
 * from that published definition; it shares no code with the GPU library.
 *
 * Parity status of each function (what pins it to something other than
 * itself; the pins are the -m "not gpu" tests):
 *   orc_philox4x32_10      pinned on the GPU against cuRAND's
 *                          Philox4_32_10 generator (a library routine)
 *   orc_lattice_chain      pinned by exact enumeration (c_n, <R^2>, Z_n)
 *   orc_offlattice_chain   pinned by closed forms (trimer), the ideal limit,
 *                          direction moments and simple sampling
 *   *_chain_restart        pinned by the trimer in restart mode (closed-form
 *                          attempt law, E[W] and <R^2>) and the exact c_n
 *   orc_reduce             pinned against exact rational sums
 *   orc_enumerate          pinned against brute force over all 6^n walks
 *   orc_perm_run           pinned by exact reduction to orc_lattice_run
 *                          without thresholds, and by the exact c_n (n <= 12)
 *                          and Z_n(beta eps) (n <= 10) that its mean estimate
 *                          must equal with pruning and enrichment active
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Section 3.2).                                  */
/* ------------------------------------------------------------------ */
ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                  uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key bumps    */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One draw of the stream: counter = (chain, ensemble, step, slot). */
static void draw(uint64_t seed, uint32_t ens, uint32_t chain, uint32_t step,
                 uint32_t slot, uint32_t out[4])
{
    uint32_t ctr[4] = {chain, ens, step, slot};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* A uniform in [0,1) from the top 24 bits of a word; exact in FP32 and FP64. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------ */
/* Cubic lattice (Algorithm 1, Eq. 3).                                  */
/* ------------------------------------------------------------------ */
/* Neighbour order (the slot order used by the selection rule). */
static const int DIRS[6][3] = {
    {+1, 0, 0}, {-1, 0, 0}, {0, +1, 0}, {0, -1, 0}, {0, 0, +1}, {0, 0, -1}};

static int l1(const int32_t *a, const int32_t *b)
{
    return abs(a[0] - b[0]) + abs(a[1] - b[1]) + abs(a[2] - b[2]);
}

/*
 * Grow one cubic-lattice chain of N monomers.
 *
 * Monomer 0 sits at the origin (Section 3.3.2 allows any start).  Step i
 * (1 <= i <= N-1) places monomer i on one of the six neighbours t_d of the
 * end r_{i-1}.  Trial d is free when no earlier non-bonded monomer
 * r_0..r_{i-2} sits on t_d (Algorithm 1's overlap test).  Its contact count
 * c_d is the number of those monomers at lattice distance 1 from t_d.
 *
 * beta_eps == 0 (athermal SAW, Eq. 3): m = number of free neighbours,
 *   W *= m, and the idx-th free neighbour is taken with
 *   idx = floor(x * m / 2^32), x the step's 32-bit draw.
 * beta_eps > 0 (interacting SAW, U = -eps per non-bonded contact, so the
 *   Boltzmann factor of Eq. 1 is exp(+beta_eps * c_d)): w_d = free_d *
 *   exp(beta_eps * c_d), S = sum_d w_d, W *= S, and the chosen d is the
 *   smallest slot whose inclusive prefix sum exceeds r = u24(x) * S (the
 *   last slot with w_d > 0 if rounding leaves none).
 * m = 0 (or S = 0) is a dead end: the chain keeps W = 0 (reading G10).
 *
 * Outputs: counts[m] = number of steps with m free neighbours (counts[0]=1
 * marks a dead chain), *logw = log W (-inf when dead), *r2 = R_ee^2,
 * *n2rg2 = N^2 R_g^2 = N sum|r_i|^2 - |sum r_i|^2 (exact integers), trace
 * byte per step = (m << 3) | d (7 at the dead step, 0xFF after it), and the
 * positions in pos[N][3].  Returns 1 if the chain is alive, else 0.
 *
 * attempt numbers the growths of one chain in restart mode (below); its draws
 * use the step word i + 2^16 * attempt, so attempt 0 is the plain stream.
 */
static int lattice_attempt(uint64_t seed, uint32_t ens, uint32_t chain, uint32_t attempt,
                           int N, double beta_eps, int32_t *pos, uint8_t *trace,
                           uint16_t counts[8], double *logw, int64_t *r2, int64_t *n2rg2)
{
    memset(counts, 0, sizeof(uint16_t) * 8);
    memset(pos, 0, sizeof(int32_t) * 3 * (size_t)N);
    if (trace) memset(trace, 0xFF, (size_t)(N - 1));
    double lw = 0.0;
    int alive = 1;
    for (int i = 1; i < N && alive; ++i) {
        const int32_t *end = &pos[3 * (i - 1)];
        int free_[6], contact[6], m = 0;
        for (int d = 0; d < 6; ++d) {
            int32_t t[3] = {end[0] + DIRS[d][0], end[1] + DIRS[d][1],
                            end[2] + DIRS[d][2]};
            free_[d] = 1;
            contact[d] = 0;
            for (int j = 0; j <= i - 2; ++j) {       /* non-bonded monomers */
                int dist = l1(&pos[3 * j], t);
                if (dist == 0) free_[d] = 0;
                else if (dist == 1) contact[d]++;
            }
            m += free_[d];
        }
        uint32_t x[4];
        draw(seed, ens, chain, (uint32_t)i | (attempt << 16), 0u, x);
        int sel = -1;
        if (m == 0) {
            alive = 0;
        } else if (beta_eps == 0.0) {
            lw += log((double)m);
            uint32_t idx = (uint32_t)(((uint64_t)x[0] * (uint64_t)m) >> 32);
            uint32_t seen = 0;
            for (int d = 0; d < 6; ++d) {
                if (!free_[d]) continue;
                if (seen == idx) { sel = d; break; }
                seen++;
            }
        } else {
            double w[6], S = 0.0;
            for (int d = 0; d < 6; ++d) {
                w[d] = free_[d] ? exp(beta_eps * (double)contact[d]) : 0.0;
                S += w[d];
            }
            lw += log(S);
            double r = u24(x[0]) * S, P = 0.0;
            for (int d = 0; d < 6; ++d) {
                P += w[d];
                if (P > r) { sel = d; break; }
            }
            if (sel < 0)
                for (int d = 0; d < 6; ++d)
                    if (w[d] > 0.0) sel = d;
        }
        if (!alive) {
            counts[0] = 1;
            if (trace) trace[i - 1] = 7;
            break;
        }
        counts[m]++;
        int32_t *nxt = &pos[3 * i];
        nxt[0] = end[0] + DIRS[sel][0];
        nxt[1] = end[1] + DIRS[sel][1];
        nxt[2] = end[2] + DIRS[sel][2];
        if (trace) trace[i - 1] = (uint8_t)((m << 3) | sel);
    }
    if (!alive) {
        *logw = -INFINITY;
        *r2 = 0;
        *n2rg2 = 0;
        return 0;
    }
    *logw = lw;
    const int32_t *last = &pos[3 * (N - 1)];
    *r2 = (int64_t)last[0] * last[0] + (int64_t)last[1] * last[1] +
          (int64_t)last[2] * last[2];
    int64_t sx = 0, sy = 0, sz = 0, sq = 0;
    for (int i = 0; i < N; ++i) {
        const int32_t *p = &pos[3 * i];
        sx += p[0]; sy += p[1]; sz += p[2];
        sq += (int64_t)p[0] * p[0] + (int64_t)p[1] * p[1] + (int64_t)p[2] * p[2];
    }
    *n2rg2 = (int64_t)N * sq - (sx * sx + sy * sy + sz * sz);
    return 1;
}

/* One growth from the plain stream (attempt 0): a dead end keeps W = 0. */
ORC_EXPORT int orc_lattice_chain(uint64_t seed, uint32_t ens, uint32_t chain,
                                 int N, double beta_eps, int32_t *pos,
                                 uint8_t *trace, uint16_t counts[8],
                                 double *logw, int64_t *r2, int64_t *n2rg2)
{
    return lattice_attempt(seed, ens, chain, 0u, N, beta_eps, pos, trace, counts, logw, r2,
                           n2rg2);
}

/*
 * Restart mode (Section 3.3.2: a chain that runs into a dead end is thrown
 * away and grown again from the first monomer).  Attempts a = 0, 1, ... are
 * made until one survives or max_attempts have been made; the outputs are
 * those of the last attempt (a dead chain after max_attempts failures) and
 * *attempts = the number of attempts made.  Every attempt is an independent
 * growth, so the mean weight over all attempts, dead ones counted as 0, is
 * the unbiased estimate of Z (Eq. 9 with the number of growths started).
 */
ORC_EXPORT int orc_lattice_chain_restart(uint64_t seed, uint32_t ens, uint32_t chain,
                                         int N, double beta_eps, int max_attempts,
                                         int32_t *pos, uint8_t *trace, uint16_t counts[8],
                                         double *logw, int64_t *r2, int64_t *n2rg2,
                                         uint32_t *attempts)
{
    int alive = 0;
    uint32_t a = 0;
    while (!alive && a < (uint32_t)max_attempts) {
        alive = lattice_attempt(seed, ens, chain, a, N, beta_eps, pos, trace, counts, logw, r2,
                                n2rg2);
        a++;
    }
    *attempts = a;
    return alive;
}

/* ------------------------------------------------------------------ */
/* Real space (Algorithm 2).                                            */
/* ------------------------------------------------------------------ */
enum { ORC_HARD_SPHERE = 0, ORC_LJ = 1 };

/*
 * Trial direction t of step i (reading of "rngonsphere", Algorithm 2):
 * draw slot 1 + t/2; trial t uses words (0,1) if t is even, (2,3) if odd.
 * z = 1 - 2 u24(a), phi = 2 pi u24(b), s = sqrt((1-z)(1+z)),
 * u = (s cos phi, s sin phi, z): uniform on the unit sphere
 * (Archimedes' hat-box theorem).
 */
static void trial_direction(const uint32_t x[4], int t, double u[3])
{
    uint32_t a = x[2 * (t & 1)], b = x[2 * (t & 1) + 1];
    double z = 1.0 - 2.0 * u24(a);
    double phi = 2.0 * ORC_PI * u24(b);
    double s = sqrt((1.0 - z) * (1.0 + z));
    u[0] = s * cos(phi);
    u[1] = s * sin(phi);
    u[2] = z;
}

/* The step's selection word: the low bytes of the four words of slot 1. */
static uint32_t selection_word(const uint32_t x[4])
{
    return (x[0] & 0xFFu) | ((x[1] & 0xFFu) << 8) | ((x[2] & 0xFFu) << 16) |
           ((x[3] & 0xFFu) << 24);
}

/*
 * Grow one real-space chain of N beads with bond length 1 and k trials per
 * step.  Non-bonded beads are j = 0..i-2 (Algorithm 2 would also test the
 * bonded bead r_{i-1}, which always sits at distance 1; reading G6).
 *
 * HARD_SPHERE: trial t is free when every non-bonded bead lies at squared
 *   distance >= sigma^2 (strict d^2 < sigma^2 is an overlap).  m = number of
 *   free trials, W *= m, and the idx-th free trial is taken with
 *   idx = floor(x * m / 2^32).
 * LJ: U_t = sum over non-bonded beads with d^2 < cutoff^2 of
 *   4 [(sigma/d)^12 - (sigma/d)^6] in units of eps (truncated, not
 *   shifted).  With bu_t = beta_eps * U_t and bmin = min_t bu_t, the trial
 *   weights are w_t = exp(-(bu_t - bmin)), S = sum_t w_t,
 *   log W += log S - bmin, and the trial is the smallest t whose inclusive
 *   prefix sum exceeds r = u24(x) * S (last t with w_t > 0 if none).
 *   beta_eps == 0 gives w_t = 1 for every trial (ideal chain).
 * No trial available (m = 0, or every bu_t infinite) is a dead end: W = 0.
 *
 * Outputs: *logw = log W (-inf when dead), *r2 = R_ee^2,
 * *rg2 = (1/N) sum_i |r_i - r_cm|^2, trace byte per step = chosen trial
 * (0xFE at the dead step, 0xFF after it), positions in pos[N][3].  The
 * normalised weight W / k^(N-1) estimates the fraction of ideal chains that
 * are self-avoiding (hard spheres) or their mean Boltzmann factor (LJ).
 *
 * attempt numbers the growths of one chain in restart mode; its draws use the
 * step word i + 2^16 * attempt (attempt 0 is the plain stream).
 */
static int offlattice_attempt(uint64_t seed, uint32_t ens, uint32_t chain, uint32_t attempt,
                              int N, int k, int potential, double sigma, double cutoff,
                              double beta_eps, double *pos, double *trial, double *wbuf,
                              uint8_t *trace, double *logw, double *r2, double *rg2)
{
    memset(pos, 0, sizeof(double) * 3 * (size_t)N);
    if (trace) memset(trace, 0xFF, (size_t)(N - 1));
    const double sig2 = sigma * sigma, rc2 = cutoff * cutoff;
    double lw = 0.0;
    int alive = 1;
    for (int i = 1; i < N && alive; ++i) {
        const double *end = &pos[3 * (i - 1)];
        uint32_t sel_word = 0;
        for (int t = 0; t < k; ++t) {
            uint32_t x[4];
            draw(seed, ens, chain, (uint32_t)i | (attempt << 16), 1u + (uint32_t)(t / 2), x);
            if (t == 0) sel_word = selection_word(x);
            double u[3];
            trial_direction(x, t, u);
            double *tt = &trial[3 * t];
            tt[0] = end[0] + u[0];
            tt[1] = end[1] + u[1];
            tt[2] = end[2] + u[2];
            if (potential == ORC_HARD_SPHERE) {
                int free_ = 1;
                for (int j = 0; j <= i - 2; ++j) {
                    const double *rj = &pos[3 * j];
                    double dx = tt[0] - rj[0], dy = tt[1] - rj[1],
                           dz = tt[2] - rj[2];
                    if (dx * dx + dy * dy + dz * dz < sig2) free_ = 0;
                }
                wbuf[t] = free_ ? 1.0 : 0.0;
            } else {
                double U = 0.0;
                for (int j = 0; j <= i - 2; ++j) {
                    const double *rj = &pos[3 * j];
                    double dx = tt[0] - rj[0], dy = tt[1] - rj[1],
                           dz = tt[2] - rj[2];
                    double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 < rc2) {
                        double s = sig2 / d2;          /* (sigma/d)^2     */
                        double s3 = s * s * s;         /* (sigma/d)^6     */
                        U += 4.0 * s3 * (s3 - 1.0);    /* 4(s^12 - s^6)   */
                    }
                }
                wbuf[t] = U;   /* energy for now, turned into a weight below */
            }
        }
        int sel = -1;
        if (potential == ORC_HARD_SPHERE) {
            int m = 0;
            for (int t = 0; t < k; ++t) m += (wbuf[t] > 0.0);
            if (m == 0) {
                alive = 0;
            } else {
                lw += log((double)m);
                uint32_t idx = (uint32_t)(((uint64_t)sel_word * (uint64_t)m) >> 32);
                uint32_t seen = 0;
                for (int t = 0; t < k; ++t) {
                    if (wbuf[t] == 0.0) continue;
                    if (seen == idx) { sel = t; break; }
                    seen++;
                }
            }
        } else {
            double bmin = INFINITY;
            if (beta_eps == 0.0) {
                for (int t = 0; t < k; ++t) wbuf[t] = 0.0;  /* bu_t = 0 */
                bmin = 0.0;
            } else {
                for (int t = 0; t < k; ++t) {
                    wbuf[t] = beta_eps * wbuf[t];
                    if (wbuf[t] < bmin) bmin = wbuf[t];
                }
            }
            if (bmin == INFINITY) {
                alive = 0;
            } else {
                double S = 0.0;
                for (int t = 0; t < k; ++t) {
                    wbuf[t] = exp(-(wbuf[t] - bmin));   /* exp(-inf) = 0 */
                    S += wbuf[t];
                }
                lw += log(S) - bmin;
                double r = u24(sel_word) * S, P = 0.0;
                for (int t = 0; t < k; ++t) {
                    P += wbuf[t];
                    if (P > r) { sel = t; break; }
                }
                if (sel < 0)
                    for (int t = 0; t < k; ++t)
                        if (wbuf[t] > 0.0) sel = t;
            }
        }
        if (!alive) {
            if (trace) trace[i - 1] = 0xFE;
            break;
        }
        double *nxt = &pos[3 * i];
        nxt[0] = trial[3 * sel + 0];
        nxt[1] = trial[3 * sel + 1];
        nxt[2] = trial[3 * sel + 2];
        if (trace) trace[i - 1] = (uint8_t)sel;
    }
    if (!alive) {
        *logw = -INFINITY;
        *r2 = 0.0;
        *rg2 = 0.0;
        return 0;
    }
    *logw = lw;
    const double *last = &pos[3 * (N - 1)];
    *r2 = last[0] * last[0] + last[1] * last[1] + last[2] * last[2];
    double cx = 0, cy = 0, cz = 0;
    for (int i = 0; i < N; ++i) {
        cx += pos[3 * i]; cy += pos[3 * i + 1]; cz += pos[3 * i + 2];
    }
    cx /= N; cy /= N; cz /= N;
    double g = 0.0;
    for (int i = 0; i < N; ++i) {
        double dx = pos[3 * i] - cx, dy = pos[3 * i + 1] - cy,
               dz = pos[3 * i + 2] - cz;
        g += dx * dx + dy * dy + dz * dz;
    }
    *rg2 = g / N;
    return 1;
}

/* One growth from the plain stream (attempt 0): a dead end keeps W = 0. */
ORC_EXPORT int orc_offlattice_chain(uint64_t seed, uint32_t ens, uint32_t chain,
                                    int N, int k, int potential, double sigma,
                                    double cutoff, double beta_eps, double *pos,
                                    double *trial /* [k][3] scratch */,
                                    double *wbuf /* [k] scratch */,
                                    uint8_t *trace, double *logw, double *r2,
                                    double *rg2)
{
    return offlattice_attempt(seed, ens, chain, 0u, N, k, potential, sigma, cutoff, beta_eps,
                              pos, trial, wbuf, trace, logw, r2, rg2);
}

/*
 * Restart mode (Section 3.3.3: when no trial position is free the growth
 * starts again from the first bead): attempts a = 0, 1, ... until one
 * survives or max_attempts have been made; outputs of the last attempt and
 * *attempts = the number made (see orc_lattice_chain_restart).
 */
ORC_EXPORT int orc_offlattice_chain_restart(uint64_t seed, uint32_t ens, uint32_t chain,
                                            int N, int k, int potential, double sigma,
                                            double cutoff, double beta_eps, int max_attempts,
                                            double *pos, double *trial, double *wbuf,
                                            uint8_t *trace, double *logw, double *r2,
                                            double *rg2, uint32_t *attempts)
{
    int alive = 0;
    uint32_t a = 0;
    while (!alive && a < (uint32_t)max_attempts) {
        alive = offlattice_attempt(seed, ens, chain, a, N, k, potential, sigma, cutoff,
                                   beta_eps, pos, trial, wbuf, trace, logw, r2, rg2);
        a++;
    }
    *attempts = a;
    return alive;
}

/* ------------------------------------------------------------------ */
/* Whole ensembles: chains chain0 .. chain0+C-1, split over threads.    */
/* Every chain is independent (Section 3.3.1: one chain per thread), so  */
/* splitting the index range changes nothing in the results.            */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind;                 /* 0 lattice, 1 real space */
    uint64_t seed;
    uint32_t ens;
    int64_t chain0, lo, hi;
    int N, k, potential;
    double sigma, cutoff, beta_eps;
    /* outputs, indexed by local chain c (0 .. C-1) */
    uint16_t *counts;         /* [C][8]        lattice   */
    double *logw;             /* [C]                      */
    int64_t *r2_i;            /* [C]           lattice   */
    int64_t *n2rg2;           /* [C]           lattice   */
    double *r2_d;             /* [C]           real space */
    double *rg2_d;            /* [C]           real space */
    uint8_t *alive;           /* [C]                      */
    uint8_t *trace;           /* [C][N-1] or NULL         */
    double *coords;           /* [C][N][3] or NULL        */
    int max_attempts;         /* 1 = no restart           */
    uint32_t *attempts;       /* [C] or NULL              */
} run_job;

static void *run_range(void *arg)
{
    run_job *J = (run_job *)arg;
    const int N = J->N;
    if (J->kind == 0) {
        int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)N);
        for (int64_t c = J->lo; c < J->hi; ++c) {
            uint16_t cnt[8];
            double lw;
            int64_t r2, g2;
            uint32_t att;
            int ok = orc_lattice_chain_restart(
                J->seed, J->ens, (uint32_t)(J->chain0 + c), N, J->beta_eps, J->max_attempts,
                pos, J->trace ? J->trace + (size_t)c * (N - 1) : NULL, cnt, &lw, &r2, &g2,
                &att);
            if (J->attempts) J->attempts[c] = att;
            if (J->counts) memcpy(J->counts + 8 * (size_t)c, cnt, sizeof cnt);
            if (J->logw) J->logw[c] = lw;
            if (J->r2_i) J->r2_i[c] = r2;
            if (J->n2rg2) J->n2rg2[c] = g2;
            if (J->alive) J->alive[c] = (uint8_t)ok;
            if (J->coords)
                for (int q = 0; q < 3 * N; ++q)
                    J->coords[(size_t)c * 3 * N + q] = (double)pos[q];
        }
        free(pos);
    } else {
        double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)N);
        double *trial = (double *)malloc(sizeof(double) * 3 * (size_t)J->k);
        double *wbuf = (double *)malloc(sizeof(double) * (size_t)J->k);
        for (int64_t c = J->lo; c < J->hi; ++c) {
            double lw, r2, g2;
            uint32_t att;
            int ok = orc_offlattice_chain_restart(
                J->seed, J->ens, (uint32_t)(J->chain0 + c), N, J->k, J->potential,
                J->sigma, J->cutoff, J->beta_eps, J->max_attempts, pos, trial, wbuf,
                J->trace ? J->trace + (size_t)c * (N - 1) : NULL, &lw, &r2, &g2, &att);
            if (J->attempts) J->attempts[c] = att;
            if (J->logw) J->logw[c] = lw;
            if (J->r2_d) J->r2_d[c] = r2;
            if (J->rg2_d) J->rg2_d[c] = g2;
            if (J->alive) J->alive[c] = (uint8_t)ok;
            if (J->coords)
                memcpy(J->coords + (size_t)c * 3 * N, pos, sizeof(double) * 3 * N);
        }
        free(pos);
        free(trial);
        free(wbuf);
    }
    return NULL;
}

static void run_threads(run_job *base, int64_t C, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > C) nthreads = (int)(C > 0 ? C : 1);
    pthread_t th[256];
    run_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *base;
        jobs[t].lo = C * t / nthreads;
        jobs[t].hi = C * (t + 1) / nthreads;
    }
    if (nthreads == 1) {
        run_range(&jobs[0]);
        return;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, run_range, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* max_attempts: 1 = a dead end keeps W = 0; > 1 = restart mode.  attempts
 * (may be NULL) receives the number of growths made per chain. */
ORC_EXPORT void orc_lattice_run_restart(uint64_t seed, uint32_t ens, int64_t chain0,
                                        int64_t C, int N, double beta_eps, int max_attempts,
                                        int nthreads, uint16_t *counts, double *logw,
                                        int64_t *r2, int64_t *n2rg2, uint8_t *alive,
                                        uint8_t *trace, double *coords, uint32_t *attempts)
{
    run_job J;
    memset(&J, 0, sizeof J);
    J.kind = 0; J.seed = seed; J.ens = ens; J.chain0 = chain0; J.N = N;
    J.beta_eps = beta_eps; J.counts = counts; J.logw = logw; J.r2_i = r2;
    J.n2rg2 = n2rg2; J.alive = alive; J.trace = trace; J.coords = coords;
    J.max_attempts = max_attempts < 1 ? 1 : max_attempts;
    J.attempts = attempts;
    run_threads(&J, C, nthreads);
}

ORC_EXPORT void orc_lattice_run(uint64_t seed, uint32_t ens, int64_t chain0,
                                int64_t C, int N, double beta_eps, int nthreads,
                                uint16_t *counts, double *logw, int64_t *r2,
                                int64_t *n2rg2, uint8_t *alive, uint8_t *trace,
                                double *coords)
{
    orc_lattice_run_restart(seed, ens, chain0, C, N, beta_eps, 1, nthreads, counts, logw, r2,
                            n2rg2, alive, trace, coords, NULL);
}

ORC_EXPORT void orc_offlattice_run_restart(uint64_t seed, uint32_t ens, int64_t chain0,
                                           int64_t C, int N, int k, int potential,
                                           double sigma, double cutoff, double beta_eps,
                                           int max_attempts, int nthreads, double *logw,
                                           double *r2, double *rg2, uint8_t *alive,
                                           uint8_t *trace, double *coords, uint32_t *attempts)
{
    run_job J;
    memset(&J, 0, sizeof J);
    J.kind = 1; J.seed = seed; J.ens = ens; J.chain0 = chain0; J.N = N; J.k = k;
    J.potential = potential; J.sigma = sigma; J.cutoff = cutoff;
    J.beta_eps = beta_eps; J.logw = logw; J.r2_d = r2; J.rg2_d = rg2;
    J.alive = alive; J.trace = trace; J.coords = coords;
    J.max_attempts = max_attempts < 1 ? 1 : max_attempts;
    J.attempts = attempts;
    run_threads(&J, C, nthreads);
}

ORC_EXPORT void orc_offlattice_run(uint64_t seed, uint32_t ens, int64_t chain0,
                                   int64_t C, int N, int k, int potential,
                                   double sigma, double cutoff, double beta_eps,
                                   int nthreads, double *logw, double *r2,
                                   double *rg2, uint8_t *alive, uint8_t *trace,
                                   double *coords)
{
    orc_offlattice_run_restart(seed, ens, chain0, C, N, k, potential, sigma, cutoff, beta_eps,
                               1, nthreads, logw, r2, rg2, alive, trace, coords, NULL);
}

/* ------------------------------------------------------------------ */
/* Ensemble statistics (Eq. 2 with W as importance weight, Eq. 9).      */
/* ------------------------------------------------------------------ */
/*
 * out[] (18 doubles):
 *  0 n            number of growths (Eq. 9's sample size: the chains, dead
 *                 ones included, or in restart mode every attempt made)
 *  1 n_alive
 *  2 log_max      M = max log W over live chains
 *  3 S0 = sum w,  w = exp(log W - M)
 *  4 S1 = sum w A1          (A1 = R_ee^2)
 *  5 S2 = sum w A2          (A2 = R_g^2)
 *  6 Q0 = sum w^2
 *  7 Q1_r2  = sum w^2 A1    8 Q2_r2  = sum w^2 A1^2
 *  9 Q1_rg2 = sum w^2 A2   10 Q2_rg2 = sum w^2 A2^2
 * 11 logZ      = M + log(S0 / n)          (log of Eq. 9's mean weight)
 * 12 logZ_norm = logZ - (N-1) log k       (k = trials per step; 0 skips)
 * 13 mean_r2   = S1 / S0                  (Eq. 2)
 * 14 se_r2     = sqrt(sum w^2 (A1 - mean)^2) / S0
 * 15 mean_rg2  = S2 / S0
 * 16 se_rg2
 * 17 ess      = S0^2 / Q0   (Kish effective sample size)
 * Written plainly: one pass for the maximum, one pass for the sums.
 */
ORC_EXPORT void orc_reduce_n(int64_t C, const double *logw, const double *A1,
                             const double *A2, int N, int k, double n, double *out)
{
    double M = -INFINITY;
    int64_t alive = 0;
    for (int64_t c = 0; c < C; ++c)
        if (logw[c] > -INFINITY) {
            alive++;
            if (logw[c] > M) M = logw[c];
        }
    double S0 = 0, S1 = 0, S2 = 0, Q0 = 0, Q1a = 0, Q2a = 0, Q1b = 0, Q2b = 0;
    if (alive > 0)
        for (int64_t c = 0; c < C; ++c) {
            if (!(logw[c] > -INFINITY)) continue;
            double w = exp(logw[c] - M);
            double a = A1[c], b = A2[c];
            S0 += w; S1 += w * a; S2 += w * b;
            Q0 += w * w; Q1a += w * w * a; Q2a += w * w * a * a;
            Q1b += w * w * b; Q2b += w * w * b * b;
        }
    out[0] = n;
    out[1] = (double)alive;
    out[2] = M;
    out[3] = S0; out[4] = S1; out[5] = S2; out[6] = Q0;
    out[7] = Q1a; out[8] = Q2a; out[9] = Q1b; out[10] = Q2b;
    if (alive == 0) {
        out[11] = -INFINITY;
        out[12] = -INFINITY;
        out[13] = out[14] = out[15] = out[16] = NAN;
        out[17] = 0.0;
        return;
    }
    out[11] = M + log(S0 / n);
    out[12] = k > 0 ? out[11] - (double)(N - 1) * log((double)k) : out[11];
    double m1 = S1 / S0, m2 = S2 / S0;
    double v1 = Q2a - 2.0 * m1 * Q1a + m1 * m1 * Q0;
    double v2 = Q2b - 2.0 * m2 * Q1b + m2 * m2 * Q0;
    out[13] = m1;
    out[14] = sqrt(v1 > 0 ? v1 : 0) / S0;
    out[15] = m2;
    out[16] = sqrt(v2 > 0 ? v2 : 0) / S0;
    out[17] = S0 * S0 / Q0;
}

/* The statistics with n = C (one growth per chain). */
ORC_EXPORT void orc_reduce(int64_t C, const double *logw, const double *A1,
                           const double *A2, int N, int k, double *out)
{
    orc_reduce_n(C, logw, A1, A2, N, k, (double)C, out);
}

/* ------------------------------------------------------------------ */
/* Exact enumeration of cubic-lattice SAWs (test fixture).              */
/* ------------------------------------------------------------------ */
/*
 * For every walk of n = 1..nmax steps from the origin that visits no site
 * twice, record by its number of non-bonded nearest-neighbour contacts c:
 *   cnt[n][c]    number of walks,
 *   sr2[n][c]    sum of R_ee^2,
 *   sg2[n][c]    sum of (n+1)^2 R_g^2 = (n+1) sum|r|^2 - |sum r|^2.
 * Arrays are (nmax+1) x (nmax+1), row n, column c.  The Rosenbluth weight
 * is an unbiased estimator of sum over walks of exp(beta_eps c) (Eq. 3 with
 * Eq. 1), so these give the exact Z_n(beta_eps), <R^2>_n and <R_g^2>_n.
 */
typedef struct {
    int nmax, L, off;
    uint8_t *occ;
    int32_t (*path)[3];
    int64_t *cnt, *sr2, *sg2;
} enum_state;

static int site(const enum_state *E, int x, int y, int z)
{
    return ((x + E->off) * E->L + (y + E->off)) * E->L + (z + E->off);
}

static void dfs(enum_state *E, int n, int contacts, int64_t sx, int64_t sy,
                int64_t sz, int64_t sq)
{
    if (n >= 1) {
        const int32_t *e = E->path[n];
        int64_t r2 = (int64_t)e[0] * e[0] + (int64_t)e[1] * e[1] + (int64_t)e[2] * e[2];
        int64_t g2 = (int64_t)(n + 1) * sq - (sx * sx + sy * sy + sz * sz);
        size_t idx = (size_t)n * (E->nmax + 1) + contacts;
        E->cnt[idx] += 1;
        E->sr2[idx] += r2;
        E->sg2[idx] += g2;
    }
    if (n == E->nmax) return;
    const int32_t *e = E->path[n];
    for (int d = 0; d < 6; ++d) {
        int x = e[0] + DIRS[d][0], y = e[1] + DIRS[d][1], z = e[2] + DIRS[d][2];
        int s = site(E, x, y, z);
        if (E->occ[s]) continue;
        int c = 0;
        for (int q = 0; q < 6; ++q) {
            int xx = x + DIRS[q][0], yy = y + DIRS[q][1], zz = z + DIRS[q][2];
            if (xx == e[0] && yy == e[1] && zz == e[2]) continue;   /* bonded */
            if (E->occ[site(E, xx, yy, zz)]) c++;
        }
        E->occ[s] = 1;
        E->path[n + 1][0] = x; E->path[n + 1][1] = y; E->path[n + 1][2] = z;
        dfs(E, n + 1, contacts + c, sx + x, sy + y, sz + z,
            sq + (int64_t)x * x + (int64_t)y * y + (int64_t)z * z);
        E->occ[s] = 0;
    }
}

ORC_EXPORT int orc_enumerate(int nmax, int64_t *cnt, int64_t *sr2, int64_t *sg2)
{
    if (nmax < 1 || nmax > 16) return -1;
    enum_state E;
    E.nmax = nmax;
    E.off = nmax + 2;
    E.L = 2 * E.off + 1;
    E.occ = (uint8_t *)calloc((size_t)E.L * E.L * E.L, 1);
    E.path = malloc(sizeof(int32_t[3]) * (size_t)(nmax + 1));
    size_t sz = (size_t)(nmax + 1) * (nmax + 1);
    memset(cnt, 0, sizeof(int64_t) * sz);
    memset(sr2, 0, sizeof(int64_t) * sz);
    memset(sg2, 0, sizeof(int64_t) * sz);
    E.cnt = cnt; E.sr2 = sr2; E.sg2 = sg2;
    E.path[0][0] = E.path[0][1] = E.path[0][2] = 0;
    E.occ[site(&E, 0, 0, 0)] = 1;
    dfs(&E, 0, 0, 0, 0, 0, 0);
    free(E.occ);
    free(E.path);
    return 0;
}

/* ------------------------------------------------------------------ */
/* PERM: pruned-enriched Rosenbluth growth, breadth first.              */
/* ------------------------------------------------------------------ */
/*
 * The paper's conclusion names a GPU PERM; its text is not available, so
 * this follows the published method (Grassberger, Phys. Rev. E 56, 3682
 * (1997)): Rosenbluth growth in which a chain whose weight has grown well
 * above the typical weight of its length is copied (enrichment, the copies
 * share its weight) and a chain whose weight has fallen well below it is
 * removed with probability 1/2, its weight doubled if it survives (pruning).
 * Both keep the expected total weight of every length unchanged, so the
 * mean weight over the tours started is still an unbiased estimate of Z_n
 * (Eq. 9) and W-weighted means are still those of Eq. 2.
 *
 * Readings (the listing is not available):
 *  - Breadth first: all chains grow step i together, as one population,
 *    instead of Grassberger's depth-first recursion.  The expectations are
 *    the same.
 *  - Thresholds per step: enrich when W > c_hi mu^i, prune when
 *    W < c_lo mu^i, with mu a caller-chosen growth constant (a chain's fate
 *    depends on its own weight only).  c_hi = +inf never enriches,
 *    c_lo = 0 never prunes; then the method is plain Rosenbluth growth.
 *  - Two copies per enrichment.  A population cap max_pop bounds memory:
 *    enrichments are granted in population order while the population stays
 *    <= max_pop; a chain denied its copy keeps its whole weight.
 *  - Dead ends (no free neighbour) leave the population.
 *  - The growth step is the Rosenbluth step of the lattice chains above
 *    (same free/contact rule, weight, selection and draw); the chain at
 *    position j of the population before step i draws from the counter
 *    (j, ens, i, 0), and its pruning coin is the top bit of word 0 of
 *    (j, ens, i, 1) (kept when set).  Without pruning, enrichment or dead
 *    ends the chain at position j is chain j of orc_lattice_run.
 *  - Weights are kept as W = wm 2^we with wm in [1, 2) (FP64 mantissa,
 *    integer exponent): every update is one correctly rounded product and
 *    an exact rescaling, and every comparison with a threshold is exact.
 *    The threshold mu^i is kept the same way, multiplied by mu each step.
 *
 * Outputs per length (i = 0 .. N-1, i steps):
 *   pop[i]   chains in the population after step i (pop[0] = M0);
 *   logz[i]  log of (1/M0) sum W over the chains grown at step i (Eq. 9);
 *   r2[i]    W-weighted mean R_ee^2 of those chains (Eq. 2);
 * and the final population: its size *final_n, weights (fw_m, fw_e) and
 * positions fpos[c][N][3] (optional).  Returns 0, or -1 on bad arguments.
 */
typedef struct perm_chain {
    double wm;
    int32_t we;
    int32_t *pos;      /* [N][3] */
} perm_chain;

/* x = m 2^e with m in [1, 2); x > 0 finite. */
static void perm_norm(double x, double *m, int32_t *e)
{
    int k = ilogb(x);
    *m = ldexp(x, -k);
    *e = k;
}

/* Is wm 2^we > c tm 2^te ?  (c >= 0; c = +inf is never exceeded.) */
static int perm_above(double wm, int32_t we, double c, double tm, int32_t te)
{
    if (isinf(c)) return 0;
    double x = c * tm;
    if (x == 0.0) return 1;
    double xm;
    int32_t xe;
    perm_norm(x, &xm, &xe);
    xe += te;
    return we > xe || (we == xe && wm > xm);
}

/* Is wm 2^we < c tm 2^te ? */
static int perm_below(double wm, int32_t we, double c, double tm, int32_t te)
{
    if (isinf(c)) return 1;
    double x = c * tm;
    if (x == 0.0) return 0;
    double xm;
    int32_t xe;
    perm_norm(x, &xm, &xe);
    xe += te;
    return we < xe || (we == xe && wm < xm);
}

ORC_EXPORT int orc_perm_run(uint64_t seed, uint32_t ens, int N, double beta_eps, int64_t M0,
                            int64_t max_pop, double mu, double c_hi, double c_lo,
                            int64_t *pop, double *logz, double *r2, int64_t *final_n,
                            double *fw_m, int32_t *fw_e, int32_t *fpos)
{
    if (N < 2 || M0 < 1 || max_pop < M0 || !(mu > 0.0) || !(c_lo >= 0.0) || !(c_hi > c_lo))
        return -1;
    perm_chain *cur = calloc((size_t)max_pop, sizeof(perm_chain));
    perm_chain *nxt = calloc((size_t)max_pop, sizeof(perm_chain));
    int *grew = calloc((size_t)max_pop, sizeof(int));    /* grown at this step         */
    int *fate = calloc((size_t)max_pop, sizeof(int));    /* 0 gone, 1 kept, 2 enriched,
                                                            -1 pruning survivor         */
    int32_t *posbuf = malloc(sizeof(int32_t) * 3 * (size_t)N * (size_t)max_pop * 2);
    for (int64_t c = 0; c < max_pop; ++c) {
        cur[c].pos = posbuf + (size_t)3 * N * (size_t)c;
        nxt[c].pos = posbuf + (size_t)3 * N * (size_t)(max_pop + c);
    }
    double wt[8];
    for (int c = 0; c < 8; ++c) wt[c] = exp(beta_eps * (double)c);
    int64_t P = M0;
    for (int64_t c = 0; c < P; ++c) {
        cur[c].wm = 1.0;
        cur[c].we = 0;
        memset(cur[c].pos, 0, sizeof(int32_t) * 3 * (size_t)N);
    }
    pop[0] = M0;
    logz[0] = 0.0;
    r2[0] = 0.0;
    double tm = 1.0;   /* mu^i = tm 2^te */
    int32_t te = 0;
    int i = 1;
    for (; i < N && P > 0; ++i) {
        double m_;
        int32_t e_;
        perm_norm(tm * mu, &m_, &e_);
        tm = m_;
        te += e_;

        /* 1. One Rosenbluth step of every chain, in population order. */
        for (int64_t j = 0; j < P; ++j) {
            perm_chain *ch = &cur[j];
            const int32_t *end = &ch->pos[3 * (i - 1)];
            int free_[6], contact[6], m = 0;
            for (int d = 0; d < 6; ++d) {
                int32_t t[3] = {end[0] + DIRS[d][0], end[1] + DIRS[d][1], end[2] + DIRS[d][2]};
                free_[d] = 1;
                contact[d] = 0;
                for (int q = 0; q <= i - 2; ++q) {
                    int dist = l1(&ch->pos[3 * q], t);
                    if (dist == 0) free_[d] = 0;
                    else if (dist == 1) contact[d]++;
                }
                m += free_[d];
            }
            grew[j] = m > 0;
            if (m == 0) continue;          /* dead end: leaves the population */
            uint32_t x[4];
            draw(seed, ens, (uint32_t)j, (uint32_t)i, 0u, x);
            int sel = -1;
            double S;
            if (beta_eps == 0.0) {
                S = (double)m;
                uint32_t idx = (uint32_t)(((uint64_t)x[0] * (uint64_t)m) >> 32);
                uint32_t seen = 0;
                for (int d = 0; d < 6; ++d) {
                    if (!free_[d]) continue;
                    if (seen == idx) { sel = d; break; }
                    seen++;
                }
            } else {
                double w[6];
                S = 0.0;
                for (int d = 0; d < 6; ++d) {
                    w[d] = free_[d] ? wt[contact[d]] : 0.0;
                    S += w[d];
                }
                double r = u24(x[0]) * S, Pf = 0.0;
                for (int d = 0; d < 6; ++d) {
                    Pf += w[d];
                    if (Pf > r) { sel = d; break; }
                }
                if (sel < 0)
                    for (int d = 0; d < 6; ++d)
                        if (w[d] > 0.0) sel = d;
            }
            int32_t *p = &ch->pos[3 * i];
            p[0] = end[0] + DIRS[sel][0];
            p[1] = end[1] + DIRS[sel][1];
            p[2] = end[2] + DIRS[sel][2];
            perm_norm(ch->wm * S, &m_, &e_);
            ch->wm = m_;
            ch->we += e_;
        }

        /* 2. Estimates of length i over the grown chains (Eq. 9, Eq. 2). */
        int32_t emax = INT32_MIN;
        for (int64_t j = 0; j < P; ++j)
            if (grew[j] && cur[j].we > emax) emax = cur[j].we;
        if (emax == INT32_MIN) {
            logz[i] = -INFINITY;
            r2[i] = NAN;
        } else {
            double sw = 0.0, swr = 0.0;
            for (int64_t j = 0; j < P; ++j) {
                if (!grew[j]) continue;
                const int32_t *e = &cur[j].pos[3 * i];
                const double R2 = (double)((int64_t)e[0] * e[0] + (int64_t)e[1] * e[1] +
                                           (int64_t)e[2] * e[2]);
                const double w = ldexp(cur[j].wm, cur[j].we - emax);
                sw += w;
                swr += w * R2;
            }
            logz[i] = log(sw) + (double)emax * log(2.0) - log((double)M0);
            r2[i] = swr / sw;
        }

        /* 3. Fate of every grown chain against the thresholds of length i. */
        int64_t base = 0;
        for (int64_t j = 0; j < P; ++j) {
            if (!grew[j]) {
                fate[j] = 0;
            } else if (perm_above(cur[j].wm, cur[j].we, c_hi, tm, te)) {
                fate[j] = 2;
            } else if (perm_below(cur[j].wm, cur[j].we, c_lo, tm, te)) {
                uint32_t y[4];
                draw(seed, ens, (uint32_t)j, (uint32_t)i, 1u, y);
                fate[j] = (y[0] >> 31) ? -1 : 0;
            } else {
                fate[j] = 1;
            }
            base += fate[j] != 0;
        }

        /* 4. The next population, in order; the first max_pop - base
         *    enrichment requests are granted. */
        const int64_t G = max_pop - base;
        int64_t rank = 0, n = 0;
        for (int64_t j = 0; j < P; ++j) {
            if (fate[j] == 0) continue;
            int copies = 1;
            int32_t we = cur[j].we;
            if (fate[j] == 2) {
                if (rank < G) {
                    copies = 2;
                    we -= 1;         /* the copies share the weight */
                }
                ++rank;
            } else if (fate[j] == -1) {
                we += 1;             /* a pruning survivor carries twice the weight */
            }
            for (int c = 0; c < copies; ++c) {
                nxt[n].wm = cur[j].wm;
                nxt[n].we = we;
                memcpy(nxt[n].pos, cur[j].pos, sizeof(int32_t) * 3 * (size_t)(i + 1));
                ++n;
            }
        }
        perm_chain *t = cur;
        cur = nxt;
        nxt = t;
        P = n;
        pop[i] = P;
    }
    for (; i < N; ++i) {             /* the population died out */
        pop[i] = 0;
        logz[i] = -INFINITY;
        r2[i] = NAN;
    }
    *final_n = P;
    for (int64_t c = 0; c < P; ++c) {
        if (fw_m) fw_m[c] = cur[c].wm;
        if (fw_e) fw_e[c] = cur[c].we;
        if (fpos) memcpy(fpos + (size_t)3 * N * (size_t)c, cur[c].pos, sizeof(int32_t) * 3 * (size_t)N);
    }
    free(cur);
    free(nxt);
    free(grew);
    free(fate);
    free(posbuf);
    return 0;
}
