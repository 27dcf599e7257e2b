"""rosen_reduce_noalloc: the ensemble reduction without device allocation.

Some callers cannot allocate device memory at the moment they reduce: code
that runs while a stream is captured into a CUDA graph (cudaMalloc is not
allowed there), serving threads that must not take the allocator's implicit
synchronisation, and hosts whose device memory is owned by someone else.
For them rosen_reduce_noalloc takes its scratch from a fixed array inside
the library (at most 2^24 chains).  These tests call it through the C ABI
and check it against rosen_reduce (the same tolerance as the reduction
parity tests) on two calls in a row, so a second call cannot lean on what
the first one left in the shared scratch.  This file is collected last.
"""
import ctypes
import math

import pytest
import torch

from paper_1704_04381_gb300 import build as pkg_build

EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def tolerance(ref, key):
    n = max(ref["n_alive"], 1.0)
    base = 4.0 * n * EPS + 1e-15
    if key in ("se_r2", "se_rg2"):
        q1, q2 = ("Q1_r2", "Q2_r2") if key == "se_r2" else ("Q1_rg2", "Q2_rg2")
        m = ref["mean_r2"] if key == "se_r2" else ref["mean_rg2"]
        var = (ref[key] * ref["S0"]) ** 2
        kappa = (ref[q2] + 2 * abs(m) * ref[q1] + m * m * ref["Q0"]) / var if var > 0 else 1.0
        return base * max(kappa, 1.0)
    return base


def assert_close(got, ref):
    for key in ref:
        g, r = got[key], ref[key]
        if math.isnan(r):
            assert math.isnan(g), key
        elif math.isinf(r) or key in ("n", "n_alive", "log_max"):
            assert g == r, key
        elif key in ("logZ", "logZ_norm"):
            assert abs(g - r) <= tolerance(ref, key), key
        else:
            assert abs(g - r) <= tolerance(ref, key) * abs(r), key


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
            assert_close(rosen.stats_dict(got), rosen.stats_dict(ref))
