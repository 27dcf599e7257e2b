// internal.cuh -- host-side entry points the translation units of librosen
// share with each other (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace rosen {

// ---- lattice.cu ------------------------------------------------------------
int lattice_validate(const rosen_lattice_params *p, const rosen_lattice_out *o,
                     int nmax = ROSEN_LATTICE_NMAX, const char *fn = "rosen_lattice_grow");
size_t lattice_args_size();
void lattice_make_args(const rosen_lattice_params *p, const rosen_lattice_out *o, void *out);
size_t lattice_smem_bytes(int N, int B);
// Local chains [c_lo, c_hi) of a validated ensemble (shared-memory kernels,
// N <= 512); outputs are those of rosen_lattice_grow, bit for bit.
int lattice_grow_range(const rosen_lattice_params *p, const rosen_lattice_out *o, int64_t c_lo,
                       int64_t c_hi, cudaStream_t s);
// Chains the GPU grows at the same time for this ensemble (0 on error).
int64_t lattice_resident_chains(const rosen_lattice_params *p);
int lattice_batch_prepare(int B, int Nmax, size_t *smem, int *blocks_per_sm);
void lattice_batch_launch(const void *dev_args, const BatchItem *items, int n_items, int *head,
                          int B, size_t smem, int grid, cudaStream_t s);

// ---- offlattice.cu ---------------------------------------------------------
int offlattice_validate(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                        int nmax = ROSEN_OFFLATTICE_NMAX,
                        const char *fn = "rosen_offlattice_grow");
size_t offlattice_args_size();
void offlattice_make_args(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                          unsigned long long *counters, void *out);
int offlattice_default_lanes(int k, bool lj, int N = 0);
// Local chains [c_lo, c_hi) of a validated ensemble (shared-memory kernels,
// N <= 1024), with caller-owned scratch: counters of
// offlattice_range_counter_bytes() (16-byte aligned, zeroed by the call; one
// set per range that may run concurrently with another) and the deferral
// mask of offlattice_range_mask_bytes(C) bytes (4-byte aligned, zero before
// the first range of the ensemble, shared by all its ranges).  For hard
// spheres, ranges that run at the same time must not share mask words: start
// them at multiples of 32 chains.  Outputs are those of
// rosen_offlattice_grow, bit for bit.
size_t offlattice_range_counter_bytes();
size_t offlattice_range_mask_bytes(int64_t C);
int offlattice_grow_range(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                          int64_t c_lo, int64_t c_hi, void *counters, uint32_t *mask,
                          cudaStream_t s);
// Chains the GPU grows at the same time for this ensemble (0 on error).
int64_t offlattice_resident_chains(const rosen_offlattice_params *p);
int offlattice_batch_prepare(int G, int T, bool lj, int Nmax, int *chains_per_block, size_t *smem,
                             int *blocks_per_sm);
void offlattice_batch_launch(int G, int T, bool lj, const void *dev_args, const BatchItem *items,
                             int n_items, int *head, int chains_per_block, int Nmax, size_t smem,
                             int grid, cudaStream_t s);

// ---- reduce.cu -------------------------------------------------------------
int reduce_validate(const rosen_reduce_in *in, const rosen_stats *out);
size_t reduce_args_size();
void reduce_make_args(const rosen_reduce_in *in, void *out);
int64_t reduce_tiles(int64_t C);
size_t reduce_partial_bytes();
// Every tile of every ensemble in one launch, then one block per ensemble
// merging its partials: the same tile and merge code as rosen_reduce, so the
// statistics of an ensemble do not depend on the batch it is reduced in.
void reduce_batch_launch(const void *dev_args, const int64_t *dev_tile_off, int n_ens,
                         int64_t total_tiles, void *part, rosen_stats *out, cudaStream_t s);

}  // namespace rosen
