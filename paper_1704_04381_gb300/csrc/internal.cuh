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
