/*
 * rosen.h -- C ABI of the GB300 Rosenbluth chain-growth library (librosen.so).
 *
 * The library grows very many independent polymer chains with the
 * Rosenbluth method of Guo & Baulin, "GPU Implementation of the Rosenbluth
 * Generation Method for Static Monte Carlo Simulations" (arxiv 1704.04381),
 * on the simple cubic lattice (Section 3.3.2, Algorithm 1) and in real space
 * (Section 3.3.3, Algorithm 2), and reduces W-weighted ensemble averages
 * (Eq. 2, Eq. 9).  Every step runs in the library's own CUDA kernels for
 * sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point:
 *  - Return value: a ROSEN_* status.  ROSEN_OK on success.  On failure a
 *    description is available from rosen_last_error() (thread-local).
 *  - Array pointers are DEVICE pointers owned by the caller, unless a
 *    comment says otherwise.  The library never frees them and keeps no
 *    reference after the call returns (the serving API is the exception and
 *    says so).  Output pointers that may be NULL are marked "optional".
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream).  Parameters are checked on
 *    the host first: a bad parameter returns ROSEN_EINVAL and enqueues
 *    nothing.  ROSEN_ECUDA reports a CUDA launch error.
 *  - Per-chain arrays are indexed by the local chain index c in [0, C); the
 *    chain's random stream is keyed by its global index chain0 + c, so a
 *    range of chains can be grown in pieces (or on several GPUs) with
 *    identical results.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = the 64-bit
 *    seed (low word first), counter = (chain, ensemble, step, slot).
 */
#ifndef ROSEN_H
#define ROSEN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ROSEN_API __attribute__((visibility("default")))
#else
#define ROSEN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define ROSEN_OK 0
#define ROSEN_EINVAL 1    /* bad argument; nothing was enqueued            */
#define ROSEN_ENOMEM 2    /* workspace too small / budget exceeded         */
#define ROSEN_ECUDA 3     /* a CUDA call failed                            */
#define ROSEN_ETIMEOUT 4  /* a bounded wait ran out                        */
#define ROSEN_EBUSY 5     /* queue full, try again                         */
#define ROSEN_EAGAIN 6    /* result not ready yet                          */
#define ROSEN_ECLOSED 7   /* server shut down / request cancelled          */
#define ROSEN_ENOTFOUND 8 /* unknown ticket                                */

/* ---- limits and flags ------------------------------------------------ */
#define ROSEN_LATTICE_NMAX 512    /* packed 10-bit lattice coordinates      */
#define ROSEN_LATTICE_LONG_NMAX 32768 /* rosen_lattice_grow_long            */
#define ROSEN_OFFLATTICE_NMAX 1024
#define ROSEN_OFFLATTICE_LONG_NMAX 16384 /* rosen_offlattice_grow_long      */
#define ROSEN_KMAX 128            /* real-space trials per step             */

#define ROSEN_MAX_ATTEMPTS 65535  /* restart mode: growths per chain        */
#define ROSEN_STORE_TRACE 1u      /* write the per-step trace bytes         */
#define ROSEN_STORE_COORDS 2u     /* write the chain coordinates            */

#define ROSEN_HARD_SPHERE 0
#define ROSEN_LJ 1

/* Human-readable name of a status code (static string). */
ROSEN_API const char *rosen_status_string(int status);
/* Last error message of the calling thread ("" if none). */
ROSEN_API const char *rosen_last_error(void);
/* Library version string, e.g. "rosen 0.1 sm_103a". */
ROSEN_API const char *rosen_version(void);

/* ---- Philox stream (exposed for verification) ------------------------ */
/*
 * out[4*q + w] = word w of Philox4x32-10(counter = (chain0 + q, ensemble,
 * step, slot), key = seed), for q in [0, n).  out: device, 4*n uint32.
 * This is the generator every growth kernel draws from (it replaces the
 * paper's per-thread cuRAND state, Section 3.2).
 */
ROSEN_API int rosen_philox(uint64_t seed, uint32_t ensemble, uint32_t step, uint32_t slot,
                 int64_t chain0, int64_t n, uint32_t *out, void *stream);

/* ---- cubic lattice growth (Section 3.3.2, Algorithm 1, Eq. 3) --------- */
typedef struct rosen_lattice_params {
    uint64_t seed;
    uint32_t ensemble;        /* ensemble id, part of the Philox counter    */
    int32_t N;                /* monomers per chain, 2 <= N <= 512          */
    int64_t C;                /* chains, C >= 0                             */
    int64_t chain0;           /* global index of chain 0; chain0+C <= 2^32  */
    double beta_eps;          /* 0 <= beta_eps <= 16.  0: athermal SAW.  > 0:
                                 each non-bonded nearest-neighbour contact has
                                 energy -eps (interacting SAW); the bound
                                 keeps the FP32 factor exp(5 beta_eps) of a
                                 site with five contacts finite             */
    uint32_t flags;           /* ROSEN_STORE_TRACE | ROSEN_STORE_COORDS     */
    int32_t lanes_per_chain;  /* 0 = automatic; else 1 (one chain per lane) */
    int32_t max_attempts;     /* 0 or 1: a trapped chain keeps W = 0.  2 ..
                                 ROSEN_MAX_ATTEMPTS: restart mode (Section
                                 3.3.2): a trapped chain is grown again from
                                 monomer 0, at most max_attempts growths in
                                 all; growth a draws from the step word
                                 i + 2^16 a (a = 0 is the plain stream)    */
} rosen_lattice_params;

typedef struct rosen_lattice_out {
    uint16_t *counts; /* [C][8] optional: counts[c][m] = steps with m free
                         neighbours (m = 1..6); counts[c][0] = 1 marks a dead
                         chain (trapped: W = 0; the other entries keep the
                         steps before the dead end).  For beta_eps = 0 the exact
                         weight is W = prod_m m^counts[c][m].              */
    float *logw;      /* [C] optional: log W, -inf for a dead chain.  FP32
                         sum of FP32 logs (athermal: from the exact counts) */
    int32_t *r2;      /* [C] optional: R_ee^2 (exact)                       */
    int64_t *n2rg2;   /* [C] optional: N^2 R_g^2 = N sum|r_i|^2 - |sum r_i|^2
                         (exact)                                            */
    uint8_t *trace;   /* [N-1][C] optional (needs ROSEN_STORE_TRACE):
                         byte (m << 3) | d for step i at [i-1][c], d the
                         chosen neighbour in the order +x,-x,+y,-y,+z,-z;
                         7 at the step that dead-ends, 0xFF after it        */
    int32_t *coords;  /* [N][3][C] optional (needs ROSEN_STORE_COORDS):
                         monomer i, axis a of chain c at [i][a][c]; zero
                         after a dead end                                   */
    uint16_t *attempts; /* [C] optional: growths made (1 unless restart
                         mode); every other output is the last growth's.
                         Eq. 9's sample size is the sum (rosen_reduce_in) */
} rosen_lattice_out;

/*
 * Grow chains chain0 .. chain0+C-1 on the simple cubic lattice.  Monomer 0
 * is at the origin; step i scores the six neighbours of monomer i-1 against
 * monomers 0..i-2 (free / number of contacts), multiplies W by the number of
 * free neighbours (athermal) or by the sum of their Boltzmann factors
 * exp(beta_eps * contacts) (interacting), and picks one neighbour in
 * proportion to its weight.  Results are identical, bit for bit, to a
 * sequential implementation of the same rule in FP64 (the FP32 selection
 * falls back to FP64 whenever rounding could change the choice).
 * Errors: EINVAL for N outside [2, 512], C < 0, chain0 + C > 2^32,
 * beta_eps outside [0, 16], unknown flags or lanes_per_chain,
 * max_attempts outside [0, ROSEN_MAX_ATTEMPTS].
 */
ROSEN_API int rosen_lattice_grow(const rosen_lattice_params *p, const rosen_lattice_out *o,
                       void *stream);

/*
 * Long chains (Section 4: chains that do not fit in shared memory keep
 * their coordinates in global memory).  Same rule, draws, parameters and
 * outputs as rosen_lattice_grow, bit for bit, for 2 <= N <= 32768.  Each
 * chain's occupied sites live in an open-addressing hash table in
 * `workspace`, one 16-byte entry (key and occupancy bitmap) per 4x4x4 block
 * of sites, so a step costs a few block lookups, not a scan of the chain.  A
 * lane owns one table of 16 * 2^ceil(log2(max(N + 1, 64))) bytes and grows
 * chains one after another, taking the next from a counter as soon as it is
 * done.  The call grows min(C, (workspace_bytes - 256) / table) chains at a
 * time, so a smaller workspace means fewer chains in flight and no other
 * change.
 * workspace: caller-owned device memory, 16-byte aligned: a 256-byte header
 * (the chain counter), then the tables; the call zeroes the part it uses on
 * the stream first, so its contents need not be kept between calls.
 * rosen_lattice_long_workspace_size gives the size for min(C, 131072)
 * tables in flight.
 * Errors: those of rosen_lattice_grow with N <= 32768; EINVAL for a NULL or
 * misaligned workspace; ENOMEM if the workspace holds no table after the
 * header.
 */
ROSEN_API size_t rosen_lattice_long_workspace_size(int32_t N, int64_t C);
ROSEN_API int rosen_lattice_grow_long(const rosen_lattice_params *p, const rosen_lattice_out *o,
                                      void *workspace, size_t workspace_bytes, void *stream);

/* ---- real-space growth (Section 3.3.3, Algorithm 2) ------------------- */
typedef struct rosen_offlattice_params {
    uint64_t seed;
    uint32_t ensemble;        /* ensemble id, part of the Philox counter    */
    int32_t N;                /* beads per chain, 2 <= N <= 1024            */
    int64_t C;                /* chains, C >= 0                             */
    int64_t chain0;           /* global index of chain 0; chain0+C <= 2^32  */
    int32_t k;                /* trial directions per step, 1 <= k <= 128   */
    int32_t potential;        /* ROSEN_HARD_SPHERE or ROSEN_LJ              */
    double sigma;             /* bead diameter (HS) / LJ sigma, bond = 1;
                                 0 <= sigma <= 4 (LJ: sigma > 0)            */
    double cutoff;            /* LJ truncation radius, 0 < cutoff <= 8      */
    double beta_eps;          /* LJ well depth over kT, >= 0, finite        */
    uint32_t flags;           /* ROSEN_STORE_TRACE | ROSEN_STORE_COORDS     */
    int32_t lanes_per_chain;  /* 0 = automatic; else 8, 16 or 32 lanes grow
                                 one chain (k <= 4 * lanes_per_chain)       */
    int32_t max_attempts;     /* 0 or 1: a dead end keeps W = 0.  2 ..
                                 ROSEN_MAX_ATTEMPTS: restart mode (Section
                                 3.3.3): the chain is grown again from bead
                                 0; growth a draws from the step word
                                 i + 2^16 a                                 */
} rosen_offlattice_params;

typedef struct rosen_offlattice_out {
    float *logw;       /* [C] optional: log W (sum of log S_i), -inf if dead;
                          log W - (N-1) log k estimates log of the mean
                          Boltzmann factor of an ideal chain               */
    float *r2;         /* [C] optional: R_ee^2                              */
    float *rg2;        /* [C] optional: R_g^2 about the centre of mass      */
    uint8_t *alive;    /* [C] optional: 1 = grown to N beads, 0 = dead end  */
    uint8_t *trace;    /* [N-1][C] optional (needs ROSEN_STORE_TRACE): the
                          chosen trial of step i at [i-1][c]; 0xFE at the
                          dead step, 0xFF after it                          */
    float *coords;     /* [N][3][C] optional (needs ROSEN_STORE_COORDS)     */
    uint64_t *counters;/* [3] optional, accumulated with atomics (the
                          caller zeroes them): steps re-decided in FP64,
                          chains grown, beads listed near the chain end
                          (each listed bead is tested against all k trials) */
    uint16_t *attempts;/* [C] optional: growths made (1 unless restart mode);
                          the other outputs are the last growth's           */
} rosen_offlattice_out;

/*
 * Grow chains chain0 .. chain0+C-1 in real space.  Bead 0 is at the origin;
 * step i draws k unit vectors u_t uniformly on the sphere and scores the
 * trial positions r_{i-1} + u_t against beads 0..i-2: hard spheres are free
 * when no bead lies closer than sigma (W *= number of free trials, one free
 * trial taken uniformly); Lennard-Jones trials get w_t = exp(-beta U_t) with
 * U_t the sum of 4 eps [(sigma/d)^12 - (sigma/d)^6] over beads with
 * d < cutoff (W *= sum_t w_t, trial t taken with probability w_t / sum).
 * Coordinates are FP32 (float-float sums); decisions that FP32 rounding
 * could flip are re-taken in FP64 with the definition's arithmetic in its
 * order (no contraction, a true division).  The FP64 positions they use
 * differ from those of a sequential FP64 implementation by the float-float
 * storage of earlier re-decisions (at most 2^-48 |r|), the FP64 sin/cos of
 * the directions (a few 1e-16 per step) and the order of the position sums,
 * together below 1e-14 i after i steps.  So the path equals that of an FP64
 * implementation of the same rule except at a step where a squared
 * distance lies within about 1e-13 N of sigma^2 or of cutoff^2, or the
 * selection draw within a relative 1e-13 N of a prefix-sum boundary (the
 * tests require >= 99.9% equal paths; all tested chains take them).
 * Scratch: the call takes 8 bytes (plus, for hard spheres with N <= 128, a
 * bit per chain) from the device's stream-ordered allocator on `stream` and
 * frees it there: a chain counter for the persistent grid and the mask of
 * chains deferred to the FP64 second pass.  If that allocation fails, the
 * chains grow in one pass with one block per few chains; the results are
 * the same bit for bit.
 * Errors: EINVAL for N outside [2, 1024], k outside [1, 128], bad chain
 * range, unknown potential, sigma/cutoff/beta_eps out of range, unknown
 * flags or lanes_per_chain, max_attempts outside [0, ROSEN_MAX_ATTEMPTS].
 */
ROSEN_API int rosen_offlattice_grow(const rosen_offlattice_params *p,
                                    const rosen_offlattice_out *o, void *stream);

/*
 * Long real-space chains (Section 4: chains that do not fit in shared memory
 * keep their coordinates in global memory).  Same rule, draws, parameters,
 * exactness and outputs as rosen_offlattice_grow, for 2 <= N <= 16384 and
 * lanes_per_chain 0, 16 or 32.  Each chain slot keeps its positions, trace
 * and near list in `workspace`, and files its beads in a hash table of
 * spatial cells (side just above the list radius).  A step visits the 27
 * cells around the end instead of every earlier bead.  The near list is put
 * in bead order, so a chain's arithmetic is that of rosen_offlattice_grow
 * with the same lanes per chain, and its outputs are identical.
 * As many chains are grown at once as the workspace holds slots
 * (rosen_offlattice_long_workspace_size(N, 1) - 256 bytes each) after its
 * 256-byte header, at most as many as are resident on the GPU; a slot takes
 * its next chain from a counter in the header as soon as it is done.
 * workspace: caller-owned device memory, 16-byte aligned; the call zeroes
 * the part it uses on the stream first.  rosen_offlattice_long_workspace_size
 * gives the size for min(C, 9728) slots.
 * Errors: those of rosen_offlattice_grow with N <= 16384; EINVAL for
 * lanes_per_chain 8 or a NULL or misaligned workspace; ENOMEM if the
 * workspace holds no slot.
 */
ROSEN_API size_t rosen_offlattice_long_workspace_size(int32_t N, int64_t C);
ROSEN_API int rosen_offlattice_grow_long(const rosen_offlattice_params *p,
                                         const rosen_offlattice_out *o, void *workspace,
                                         size_t workspace_bytes, void *stream);

/*
 * The FP32 unit vectors the real-space kernels use as trial directions
 * (Algorithm 2's "rngonsphere"): for each pair of words (a, b) = words[2q],
 * words[2q+1], z = 1 - 2 u24(a), phi = 2 pi u24(b), s = sqrt((1-z)(1+z)),
 * out[3q..3q+2] = (s cos phi, s sin phi, z).  words: device, 8-byte aligned,
 * 2n uint32; out: device, 3n floats.  Exposed so the direction error bound
 * the kernels rely on can be checked exhaustively.
 */
ROSEN_API int rosen_sphere_points(const uint32_t *words, int64_t n, float *out, void *stream);

/*
 * The same unit vectors as float-float components, as the Lennard-Jones
 * kernels add them to the chain's position (no paper counterpart: it keeps
 * positions within ~1e-12 per step of exact).  out: device, 5n floats per
 * pair: x hi, x lo, y hi, y lo, z.  Each component is within 1.5e-12 of the
 * exact value; exposed so that bound can be checked exhaustively.
 */
ROSEN_API int rosen_sphere_points_ff(const uint32_t *words, int64_t n, float *out, void *stream);

/* ---- ensemble reduction (Eq. 2 with W as weight, Eq. 9) --------------- */
#define ROSEN_REDUCE_LATTICE 0    /* inputs: counts or logw, r2 (int32), n2rg2 */
#define ROSEN_REDUCE_OFFLATTICE 1 /* inputs: logw, r2 (float), rg2 (float)     */

typedef struct rosen_reduce_in {
    int32_t kind;            /* ROSEN_REDUCE_LATTICE / ROSEN_REDUCE_OFFLATTICE */
    int32_t N;               /* monomers per chain                           */
    int32_t k;               /* trials per step for logZ_norm (0: none)      */
    int32_t use_counts;      /* lattice only: 1 = take log W from counts in
                                FP64 (exact athermal weights), 0 = from logw */
    int64_t C;               /* chains, >= 1                                 */
    const float *logw;       /* [C] log W, -inf = dead (ignored if use_counts) */
    const uint16_t *counts;  /* [C][8] (lattice, use_counts = 1)             */
    const int32_t *r2_i;     /* [C] lattice R_ee^2                           */
    const int64_t *n2rg2;    /* [C] lattice N^2 R_g^2                        */
    const float *r2_f;       /* [C] real-space R_ee^2                        */
    const float *rg2_f;      /* [C] real-space R_g^2                         */
    const uint16_t *attempts;/* [C] optional (restart mode): growths made per
                                chain; Eq. 9's n is then their sum (every
                                discarded growth counts with W = 0), else C */
} rosen_reduce_in;

/* Ensemble statistics, all FP64.  With w_c = exp(log W_c - log_max):     */
typedef struct rosen_stats {
    double n;          /* growths: chains, dead ones included (Eq. 9), or
                          the sum of attempts in restart mode              */
    double n_alive;
    double log_max;    /* max log W over live chains                       */
    double S0, S1, S2; /* sum w, sum w R_ee^2, sum w R_g^2                 */
    double Q0;         /* sum w^2                                          */
    double Q1_r2, Q2_r2;   /* sum w^2 R_ee^2, sum w^2 R_ee^4               */
    double Q1_rg2, Q2_rg2; /* sum w^2 R_g^2,  sum w^2 R_g^4                */
    double logZ;       /* log((1/n) sum W), Eq. 9                          */
    double logZ_norm;  /* logZ - (N-1) log k (k > 0), else logZ            */
    double mean_r2, se_r2;   /* S1/S0 (Eq. 2) and its ratio standard error */
    double mean_rg2, se_rg2;
    double ess;        /* S0^2 / Q0                                        */
} rosen_stats;

/* Bytes of device workspace rosen_reduce needs for C chains. */
ROSEN_API size_t rosen_reduce_workspace_size(int64_t C);

/*
 * Reduce per-chain outputs to ensemble statistics in FP64 with a max-shifted
 * (log-sum-exp) sum, in a fixed order that depends only on C: the result is
 * deterministic.  out: DEVICE pointer to one rosen_stats.  workspace: device,
 * at least rosen_reduce_workspace_size(C) bytes, contents need not be
 * initialised.  All chains dead gives logZ = -inf, means = NaN, ess = 0.
 * Errors: EINVAL (C < 1, missing input array, bad kind), ENOMEM (workspace
 * too small).
 */
ROSEN_API int rosen_reduce(const rosen_reduce_in *in, rosen_stats *out, void *workspace,
                 size_t workspace_bytes, void *stream);

/*
 * Merge the statistics of n disjoint chain sets of one ensemble -- e.g. the
 * chain ranges that several GPUs grew -- into the statistics of their union
 * (Eq. 2 with W as weight, Eq. 9), with the reduction's own tile merge:
 * the largest log_max M, every weighted sum rescaled by exp(M_p - M) and
 * every squared-weight sum by exp(2 (M_p - M)), growths and live chains
 * summed; the derived fields (logZ, logZ_norm, means, standard errors, ESS)
 * are then formed as rosen_reduce forms them.  parts and out are HOST
 * pointers; the parts are merged in the order given.  N and k are the
 * ensemble's monomers and trials per step (k = 0: logZ_norm = logZ).  Runs
 * on the host, with no CUDA call.  Errors: EINVAL (NULL pointer, n < 1,
 * N < 1 or k < 0).
 */
ROSEN_API int rosen_stats_merge(const rosen_stats *parts, int32_t n, int32_t N, int32_t k,
                                rosen_stats *out);

/* ---- PERM: pruned-enriched Rosenbluth growth (cubic lattice) ---------- */
/*
 * The paper's conclusion names a GPU implementation of PERM (Grassberger,
 * Phys. Rev. E 56, 3682 (1997)) whose text is not available; this is that
 * method, breadth first.  A population of M0 chains grows one step at a time
 * with the Rosenbluth step of rosen_lattice_grow (Section 3.3.2, Eq. 3).
 * After step i a chain with W > c_hi mu^i is enriched: it and a copy go on,
 * each with W/2.  A chain with W < c_lo mu^i is pruned: it is removed with
 * probability 1/2 and otherwise goes on with 2W.  Chains at a dead end leave.
 * Both operations keep the expected total weight, so logz[i] estimates
 * log Z_i (Eq. 9: the mean weight per chain started) and mean_r2[i] the
 * W-weighted <R_ee^2> (Eq. 2), for every length at once.
 * Readings: thresholds c mu^i with a caller-chosen growth constant mu
 * (c_hi = +inf: no enrichment, c_lo = 0: no pruning, which is plain
 * Rosenbluth growth); two copies per enrichment; at most max_population
 * chains -- enrichments are granted in population order while the cap
 * allows, and a chain denied its copy keeps its weight.  Random numbers: the
 * chain at position j of the population before step i draws its step from
 * the Philox counter (j, ensemble, i, 0), as chain j of rosen_lattice_grow
 * would, and its pruning coin from the top bit of word 0 of (j, ensemble,
 * i, 1) (kept when set).  Weights are FP64 mantissas in [1, 2) with int32
 * exponents, so every fate decision is exact and the run is deterministic.
 */
#define ROSEN_PERM_MAX_POP (1 << 24)

typedef struct rosen_perm_params {
    uint64_t seed;
    uint32_t ensemble;
    int32_t N;                /* monomers per chain, 2 <= N <= 512           */
    int64_t M0;               /* chains started, >= 1                        */
    int64_t max_population;   /* cap, M0 <= max_population <= 2^24            */
    double beta_eps;          /* contact attraction (0: athermal), [0, 16]    */
    double mu;                /* threshold growth per step, > 0               */
    double c_hi, c_lo;        /* enrichment / pruning factors, 0 <= c_lo < c_hi
                                 (c_hi may be +inf)                           */
    uint32_t flags;           /* ROSEN_STORE_COORDS: the final conformations  */
    int32_t reserved;         /* set to 0                                     */
} rosen_perm_params;

typedef struct rosen_perm_out {
    int64_t *population;      /* [N]: chains after step i (population[0] = M0) */
    double *logz;             /* [N]: log((1/M0) sum W) over the chains grown at
                                 step i, -inf if none (logz[0] = 0)            */
    double *mean_r2;          /* [N] optional: their W-weighted <R_ee^2>       */
    int64_t *final_n;         /* [1]: chains in the final population            */
    double *w_m;              /* [max_population] optional: final weights       */
    int32_t *w_e;             /*   W = w_m 2^w_e, w_m in [1, 2)                  */
    int32_t *coords;          /* [N][3][max_population] optional (needs
                                 ROSEN_STORE_COORDS): final chain c, monomer q,
                                 axis a at [q][a][c]                             */
} rosen_perm_out;

/* Bytes of workspace rosen_perm_run needs (a storage slot of packed keys per
 * chain of the cap, the population as slot numbers, weights, a stack of free
 * slots, scan counts): about 4 N + 45 bytes per chain of the cap; 0 for
 * arguments out of range. */
ROSEN_API size_t rosen_perm_workspace_size(int32_t N, int64_t max_population);
/*
 * Run PERM on the stream: all outputs are DEVICE pointers owned by the
 * caller; workspace: device, 256-byte aligned, at least
 * rosen_perm_workspace_size bytes, contents need not be initialised.  The
 * population size stays on the device (no host synchronisation); about
 * 3 N kernel launches.  Errors: EINVAL (N, M0, cap, beta_eps, mu, c_hi,
 * c_lo or flags out of range, a required output missing), ENOMEM (workspace
 * too small), ECUDA.
 */
ROSEN_API int rosen_perm_run(const rosen_perm_params *p, const rosen_perm_out *o,
                             void *workspace, size_t workspace_bytes, void *stream);

/* ---- batched growth: many ensembles, one graph launch ---------------- */
#define ROSEN_MODEL_LATTICE 0
#define ROSEN_MODEL_OFFLATTICE 1

typedef struct rosen_ensemble {
    int32_t model;       /* ROSEN_MODEL_LATTICE or ROSEN_MODEL_OFFLATTICE        */
    int32_t N;           /* monomers per chain: lattice <= 32768, real space
                            <= 16384; chains longer than 512 / 1024 are grown
                            by the long-chain kernels (their own classes)     */
    int64_t C;           /* chains, >= 1; chain indices 0 .. C-1                 */
    uint64_t seed;
    uint32_t ensemble;   /* ensemble id, part of the Philox counter              */
    int32_t k;           /* real space: trial directions per step                */
    int32_t potential;   /* real space: ROSEN_HARD_SPHERE or ROSEN_LJ            */
    int32_t max_attempts;/* 0 or 1: dead ends keep W = 0; else restart mode (see
                            the growth parameters); the batch then keeps the
                            attempts per chain and reduces over all growths   */
    double beta_eps;     /* lattice: contact attraction; LJ: well depth / kT     */
    double sigma;        /* real space: bead diameter / LJ sigma                 */
    double cutoff;       /* LJ truncation radius                                 */
} rosen_ensemble;

typedef struct rosen_batch rosen_batch;   /* opaque */

/*
 * Plan a batch: validate every ensemble (the rules of rosen_lattice_grow /
 * rosen_offlattice_grow), group them into classes that share a kernel shape,
 * and allocate (with cudaMalloc, on the current device) the per-chain outputs
 * of every ensemble, the work queues and the statistics.  The batch owns all
 * of it until rosen_batch_destroy.  Errors: EINVAL (names the ensemble),
 * ECUDA.
 */
ROSEN_API int rosen_batch_create(const rosen_ensemble *ens, int32_t n, rosen_batch **out);
/*
 * Pick each class's kernel shape by timing the candidates on a sample of its
 * chains (synchronous; writes sample outputs that the next run overwrites),
 * then capture the whole batch -- persistent growth kernels on forked
 * streams and the FP64 reduction of every ensemble -- into a CUDA graph.
 */
ROSEN_API int rosen_batch_tune(rosen_batch *b, void *stream);
/* Enqueue one pass over the batch (one graph launch) on stream; tunes and
 * captures first if that has not happened. */
ROSEN_API int rosen_batch_run(rosen_batch *b, void *stream);
/* Device pointer to the batch's statistics, one rosen_stats per ensemble,
 * valid after a run completes; identical to rosen_reduce of that ensemble
 * grown alone. */
ROSEN_API int rosen_batch_stats(rosen_batch *b, rosen_stats **stats);
/* Device views of ensemble e's per-chain outputs (owned by the batch). */
ROSEN_API int rosen_batch_lattice_outputs(rosen_batch *b, int32_t e, rosen_lattice_out *out);
ROSEN_API int rosen_batch_offlattice_outputs(rosen_batch *b, int32_t e, rosen_offlattice_out *out);
/* Enqueue copies of the statistics (dst: device, n rosen_stats) or of
 * ensemble e's per-chain outputs (the non-NULL fields of dst, device) on
 * stream.  attempts is copied only for an ensemble in restart mode (the
 * batch keeps no attempts otherwise; dst->attempts is then left as is). */
ROSEN_API int rosen_batch_copy_stats(rosen_batch *b, rosen_stats *dst, void *stream);
ROSEN_API int rosen_batch_copy_lattice(rosen_batch *b, int32_t e, const rosen_lattice_out *dst,
                                       void *stream);
ROSEN_API int rosen_batch_copy_offlattice(rosen_batch *b, int32_t e,
                                          const rosen_offlattice_out *dst, void *stream);
/* Enqueue a copy of the real-space counters (see rosen_offlattice_out),
 * accumulated over every run of the batch, into dst (device, 3 uint64). */
ROSEN_API int rosen_batch_counters(rosen_batch *b, uint64_t *dst, void *stream);
/* JSON description of the classes and their (tuned) shapes, into buf. */
ROSEN_API int rosen_batch_describe(rosen_batch *b, char *buf, size_t len);
ROSEN_API int rosen_batch_destroy(rosen_batch *b);

/* ---- serving: a request loop with continuous admission --------------- */
typedef struct rosen_serve_config {
    uint64_t mem_budget_bytes; /* device memory the requests may hold at once  */
    int32_t max_slots;         /* requests admitted (on the GPU) at once,
                                  1..1024                                      */
    int32_t max_queue;         /* waiting requests before submit says EBUSY     */
    int32_t device;            /* CUDA device                                   */
    int32_t shortest_first;    /* order in which admitted requests get GPU time
                                  slices: 0 = arrival order; 1 = least
                                  estimated remaining GPU time first, divided
                                  by 1 + the seconds the request has waited;
                                  a request admitted for longer than 1 s + 2x
                                  its own GPU time gets every other slice
                                  until done, every slice while requests wait
                                  for admission (so none starves)              */
    uint64_t pool_max_bytes;   /* cap of the server's device memory pool (0: no
                                  cap); a request whose memory the pool cannot
                                  supply fails with ROSEN_ENOMEM and gives its
                                  share of the budget back                     */
} rosen_serve_config;

typedef struct rosen_request {
    int32_t model;       /* ROSEN_MODEL_LATTICE or ROSEN_MODEL_OFFLATTICE        */
    int32_t N;           /* lattice <= 32768, real space <= 16384; longer than
                            512 / 1024: grown by the long-chain entry points,
                            with a workspace of at most 1 GiB from the budget */
    int64_t C;
    uint64_t seed;
    uint32_t ensemble;
    int32_t k;           /* real space: trial directions per step                */
    int32_t potential;   /* real space: ROSEN_HARD_SPHERE or ROSEN_LJ            */
    int32_t store_coords;/* 1: keep the conformations (FP32 / int32 [N][3][C])   */
    double beta_eps, sigma, cutoff;
    int32_t max_attempts;/* 0 or 1: dead ends keep W = 0; else restart mode      */
    int32_t reserved;    /* set to 0                                             */
} rosen_request;

typedef struct rosen_result {
    uint64_t ticket;
    int32_t status;      /* ROSEN_OK, ROSEN_ECLOSED (cancelled), or the failure  */
    int32_t reserved;
    rosen_stats stats;   /* the ensemble's statistics (rosen_reduce)             */
    int64_t t_submit_ns, t_admit_ns, t_done_ns;   /* steady-clock times          */
    void *coords;        /* device conformations if store_coords, owned by the
                            server until rosen_serve_release                     */
    char message[256];   /* failure detail                                       */
} rosen_result;

typedef struct rosen_serve_counters {
    uint64_t submitted, rejected, completed, failed;
    uint64_t queued, running, bytes_in_use;
} rosen_serve_counters;

typedef struct rosen_server rosen_server;   /* opaque */

/*
 * Start a server: a scheduler thread that
 *  - admits submitted requests in arrival order as soon as a slot and enough
 *    of the memory budget are free (a request that does not fit may be
 *    passed by later ones that do for at most one second; then nothing
 *    behind it is admitted until it fits);
 *  - grows every admitted request in slices of its chains (about 4 ms of GPU
 *    time each; long-chain requests in one piece) on a stream of its own,
 *    choosing the request of each next slice by the shortest_first policy,
 *    and keeps a few milliseconds of slices enqueued so the GPU does not
 *    idle; a request that arrives while others run starts within a slice or
 *    two and shares the GPU with them;
 *  - after a request's last slice, reduces it in FP64 (rosen_reduce).
 * Every chain is grown by the kernel and lanes per chain that
 * rosen_lattice_grow / rosen_offlattice_grow (or their long-chain forms)
 * use, so a request's statistics and conformations are those of the
 * single-ensemble entry points, bit for bit, alone or in any mix.  Device
 * memory (outputs, scratch, stored conformations) comes from the server's
 * own stream-ordered pool and is counted against the budget.
 * Errors: EINVAL, ECUDA.
 */
ROSEN_API int rosen_serve_create(const rosen_serve_config *cfg, rosen_server **out);
/* Submit from any thread.  EINVAL if the request is invalid or needs more
 * than the whole budget; EBUSY if max_queue requests are waiting; ECLOSED
 * after rosen_serve_destroy began. */
ROSEN_API int rosen_serve_submit(rosen_server *s, const rosen_request *r, uint64_t *ticket);
/* ROSEN_OK with the result once the request finished, ROSEN_EAGAIN while it
 * is queued or running, ROSEN_ENOTFOUND for an unknown ticket. */
ROSEN_API int rosen_serve_poll(rosen_server *s, uint64_t ticket, rosen_result *out);
/* Wait at most timeout_ns (host-side, bounded); ROSEN_ETIMEOUT if not done. */
ROSEN_API int rosen_serve_wait(rosen_server *s, uint64_t ticket, int64_t timeout_ns,
                               rosen_result *out);
/* Cancel a request that is still queued (ROSEN_EBUSY once admitted); its
 * result then has status ROSEN_ECLOSED. */
ROSEN_API int rosen_serve_cancel(rosen_server *s, uint64_t ticket);
/* Forget a finished ticket and free its stored conformations. */
ROSEN_API int rosen_serve_release(rosen_server *s, uint64_t ticket);
ROSEN_API int rosen_serve_info(rosen_server *s, rosen_serve_counters *out);
/* Stop accepting, cancel queued requests, let running ones finish, free. */
ROSEN_API int rosen_serve_destroy(rosen_server *s);

/* ---- reduction without device allocation ---------------------------- */
/*
 * No counterpart in the paper: this entry point exists for callers that
 * cannot allocate device memory themselves -- code running while a CUDA
 * stream is being captured into a graph (cudaMalloc is not allowed there),
 * real-time or serving threads that must not take the allocator's implicit
 * synchronisation, and hosts whose device memory is fully pre-reserved by
 * another owner.  It is rosen_reduce with its scratch (the per-tile partials)
 * taken from a fixed array inside librosen instead of a caller workspace:
 *  - limit: C <= ROSEN_REDUCE_NOALLOC_MAX_CHAINS (2^24 chains, 768 KiB of
 *    scratch, held by every GPU that loads the library until exit); larger C
 *    returns ROSEN_ENOMEM and enqueues nothing;
 *  - a call looks the scratch address up (cudaGetSymbolAddress) with the
 *    caller's device current, every time its stream is not being captured
 *    (so it follows a module reloaded after cudaDeviceReset); a call made
 *    while its stream is being captured reuses the address found by the last
 *    uncaptured call on that device, so make one call on each device before
 *    any stream capture (otherwise EINVAL);
 *  - every call shares the one array, which keeps the last call's contents;
 *    nothing in it needs clearing (each call rewrites what it reads), but
 *    calls whose kernels overlap on the GPU (e.g. on two streams) race;
 *  - it calls no cudaMalloc, cudaFree or allocating library routine.
 * Arguments, results and errors are otherwise those of rosen_reduce.
 */
#define ROSEN_REDUCE_NOALLOC_MAX_CHAINS (1 << 24)
ROSEN_API int rosen_reduce_noalloc(const rosen_reduce_in *in, rosen_stats *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ROSEN_H */
