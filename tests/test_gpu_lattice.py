"""GPU parity of rosen_lattice_grow with the FP64 oracle (Algorithm 1, Eq. 3).

Lattice chains must agree with the oracle bit for bit: the trace (every
step's free-site count and chosen neighbour), the factor counts, R_ee^2,
N^2 R_g^2 and the coordinates.  log W is FP32 on the GPU; it must lie
within the FP32 rounding bound (N-1) * (1e-6 + 6e-8 |log W|): each step adds
one logf rounding (<= 1 ulp of log S, and S itself carries <= 6 ulp from
its FP32 sum) and one rounding of the running sum (<= 2^-24 |log W|).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_04381_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def grow(rosen, seed, N, C, beta_eps=0.0, chain0=0, ensemble=0, trace=True, coords=False):
    flags = (rosen.ROSEN_STORE_TRACE if trace else 0) | (rosen.ROSEN_STORE_COORDS if coords else 0)
    out = rosen.lattice_outputs(N, C, trace=trace, coords=coords)
    rosen.rosen_lattice_grow(rosen.lattice_params(seed, N, C, beta_eps=beta_eps, chain0=chain0,
                                                  ensemble=ensemble, flags=flags), out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def logw_tol(N, lw):
    return (N - 1) * (1e-6 + 6e-8 * np.abs(np.where(np.isfinite(lw), lw, 0.0)))


def assert_same(g, o, N, coords=False):
    assert np.array_equal(g["counts"].astype(np.int64), o["counts"].astype(np.int64))
    assert np.array_equal(g["r2"].astype(np.int64), o["r2"])
    assert np.array_equal(g["n2rg2"], o["n2rg2"])
    if "trace" in g:
        assert np.array_equal(g["trace"].T, o["trace"])
    dead = o["alive"] == 0
    assert np.array_equal(np.isneginf(g["logw"]), dead)
    lw = o["logw"][~dead]
    err = np.abs(g["logw"][~dead].astype(np.float64) - lw)
    assert (err <= logw_tol(N, lw)).all(), err.max()
    if coords:
        assert np.array_equal(np.transpose(g["coords"], (2, 0, 1)).astype(np.float64), o["coords"])


@pytest.mark.parametrize("beta_eps", [0.0, 0.2, 0.4])
def test_small_ensembles_bit_exact(rosen, beta_eps):
    N, C = 32, 4099          # several blocks and a ragged tail
    g = grow(rosen, 3, N, C, beta_eps, coords=True)
    o = oracle.lattice_run(3, N, C, beta_eps=beta_eps, trace=True, coords=True)
    assert_same(g, o, N, coords=True)


def test_config_athermal_n16_1e5(rosen):
    # Lattice athermal SAW, N = 16, 100,000 chains, seed 1: every chain.
    N, C = 16, 100_000
    g = grow(rosen, 1, N, C)
    o = oracle.lattice_run(1, N, C, trace=True)
    assert_same(g, o, N)
    # And the exact-enumeration pin carries over: mean prefix weight ~ c_n.
    cnt, _, _ = oracle.enumerate_saw(10)
    m = (g["trace"].T.astype(np.int64) >> 3)
    W = np.cumprod(m[:, :10].astype(np.float64), axis=1)
    for n in range(1, 11):
        se = W[:, n - 1].std(ddof=1) / np.sqrt(C) if n > 3 else 0.0
        assert abs(W[:, n - 1].mean() - cnt[n].sum()) <= 4.5 * se + 1e-9


@pytest.mark.parametrize("N", [2, 3, 4, 5, 64, 130, 257])
def test_lengths_and_offsets(rosen, N):
    C = 333 if N < 200 else 65
    g = grow(rosen, 77, N, C, beta_eps=0.3, chain0=123_456, ensemble=5)
    o = oracle.lattice_run(77, N, C, beta_eps=0.3, chain0=123_456, ensemble=5, trace=True)
    assert_same(g, o, N)


def test_maximum_length(rosen):
    N, C = 512, 40
    for beps in (0.0, 0.25):
        g = grow(rosen, 5, N, C, beps, coords=True)
        o = oracle.lattice_run(5, N, C, beta_eps=beps, trace=True, coords=True)
        assert_same(g, o, N, coords=True)


def test_dead_chains_marked(rosen):
    # N = 64 attrition is about half a percent: a few thousand chains contain dead ones.
    N, C = 64, 6000
    g = grow(rosen, 9, N, C)
    o = oracle.lattice_run(9, N, C, trace=True)
    assert (o["alive"] == 0).sum() > 0
    assert_same(g, o, N)
    dead = np.where(o["alive"] == 0)[0]
    assert (g["counts"][dead, 0] == 1).all() and (g["r2"][dead] == 0).all()


def test_sharding_is_invisible(rosen):
    # Growing [0, C) in one call or in two pieces gives the same chains.
    N, C = 40, 5000
    whole = grow(rosen, 21, N, C, beta_eps=0.2)
    a = grow(rosen, 21, N, 1800, beta_eps=0.2)
    b = grow(rosen, 21, N, C - 1800, beta_eps=0.2, chain0=1800)
    for k in ("counts", "logw", "r2", "n2rg2"):
        assert np.array_equal(whole[k], np.concatenate([a[k], b[k]]))


@pytest.mark.parametrize("beta_eps,seed", [(0.0, 2), (0.2, 3), (0.4, 4)])
def test_full_size_sampled(rosen, beta_eps, seed):
    # Interacting SAW, N = 64, 10^7 chains, one launch as timed by the bench;
    # windows at the start, middle and ragged end are checked chain by chain.
    N, C = 64, 10_000_000
    out = rosen.lattice_outputs(N, C)
    rosen.rosen_lattice_grow(rosen.lattice_params(seed, N, C, beta_eps=beta_eps), out)
    torch.cuda.synchronize()
    for lo in (0, C // 2 + 17, C - 1500):
        hi = min(C, lo + 1500)
        o = oracle.lattice_run(seed, N, hi - lo, beta_eps=beta_eps, chain0=lo)
        g = {k: v[lo:hi].cpu().numpy() for k, v in out.items()}
        assert_same(g, o, N)
    # Properties that hold at any size: R^2 parity, counts sum to N-1 steps.
    r2 = out["r2"].cpu().numpy()
    cnt = out["counts"].cpu().numpy().astype(np.int64)
    alive = cnt[:, 0] == 0
    assert ((r2[alive] - (N - 1)) % 2 == 0).all()
    assert (cnt[alive, 1:7].sum(1) == N - 1).all()
    assert 0.98 < alive.mean() < 1.0
