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
// N <= 1024), with caller-owned scratch of offlattice_range_scratch_bytes(C)
// bytes (16-byte aligned) whose deferral mask (after a 16-byte header) is
// zero before the first range of the ensemble; ranges of one ensemble run
// in stream order and, for hard spheres, start at multiples of 32 chains
// (any others cost regrowths of shared mask words, same outputs).  Outputs
// are those of rosen_offlattice_grow, bit for bit.
size_t offlattice_range_scratch_bytes(int64_t C);
int offlattice_grow_range(const rosen_offlattice_params *p, const rosen_offlattice_out *o,
                          int64_t c_lo, int64_t c_hi, void *scratch, cudaStream_t s);
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
