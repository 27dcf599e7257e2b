"""rosen_reduce_noalloc: the ensemble reduction without device allocation.

Some callers cannot allocate device memory at the moment they reduce: code
that runs while a stream is captured into a CUDA graph (cudaMalloc is not
allowed there), serving threads that must not take the allocator's implicit
synchronisation, and hosts whose device memory is owned by someone else.
For them rosen_reduce_noalloc takes its scratch from a fixed array inside
the library (at most 2^24 chains).  These tests call it through the C ABI
and check it against rosen_reduce on two calls in a row, so a second call
cannot lean on what the first one left in the shared scratch.  Both entry
points run the same tile and merge kernels over the same tiles, so the
statistics must be identical bit for bit (NaNs in the same places); a
stale partial left in the scratch by an earlier, larger call would show as
a difference.  This file is collected last.
"""
import ctypes

import pytest
import torch

from paper_1704_04381_gb300 import build as pkg_build


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def assert_identical(got, ref):
    # Same kernels, same tiles, same merge tree: equal bit for bit, with NaN
    # (all chains dead) in the same fields.
    same_nan = torch.isnan(got) == torch.isnan(ref)
    assert bool(same_nan.all()), (got, ref)
    assert torch.equal(torch.nan_to_num(got, nan=0.0), torch.nan_to_num(ref, nan=0.0)), (got, ref)


def test_rejects_more_chains_than_the_scratch_holds(rosen):
    # Checked on the host before any CUDA call: runs without a GPU.
    inp = rosen.rosen_reduce_in(kind=rosen.ROSEN_REDUCE_OFFLATTICE, N=8, k=0, use_counts=0,
                                C=rosen.ROSEN_REDUCE_NOALLOC_MAX_CHAINS + 1,
                                logw=4096, r2_f=8192, rg2_f=16384)
    st = rosen.load().rosen_reduce_noalloc(ctypes.byref(inp), 1024, None)
    assert st == rosen.ROSEN_ENOMEM
    assert "limit" in rosen.last_error()


@pytest.mark.gpu
def test_matches_rosen_reduce_on_two_calls_in_a_row(rosen):
    cases = [
        # (kind, seed, N, C, beta_eps, use_counts): a large call, then a smaller
        # one over fewer tiles, then a real-space ensemble.
        ("lattice", 3, 64, 300_001, 0.2, 0),
        ("lattice", 4, 16, 40_000, 0.0, 1),
        ("offlattice", 5, 24, 20_000, 0.0, 0),
    ]
    for kind, seed, N, C, beps, use_counts in cases:
        if kind == "lattice":
            out = rosen.lattice_outputs(N, C)
            rosen.rosen_lattice_grow(rosen.lattice_params(seed, N, C, beta_eps=beps), out)
            inp = rosen.lattice_reduce_in(out, N, use_counts)
        else:
            out = rosen.offlattice_outputs(N, C)
            rosen.rosen_offlattice_grow(rosen.offlattice_params(seed, N, C, 32), out)
            inp = rosen.offlattice_reduce_in(out, N, 32)
        ref = rosen.stats_tensor()
        rosen.rosen_reduce(inp, ref, rosen.reduce_workspace(C))
        for _ in range(2):
            got = torch.full_like(ref, float("nan"))
            rosen.rosen_reduce_noalloc(inp, got)
            torch.cuda.synchronize()
            assert_identical(got, ref)
