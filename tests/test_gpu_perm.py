"""GPU parity of rosen_perm_run (breadth-first PERM, Grassberger 1997) with
the FP64 oracle.

Every fate decision is an exact comparison of an FP64 mantissa and an
integer exponent, the growth step is the lattice step (bit-exact on both
sides), and both sides draw from the same Philox counters, so the runs must
agree exactly: the population after every step, the final weights (mantissa
and exponent) and the final conformations.  The per-length estimates are
FP64 sums of up to max_population positive terms in different orders:
log Z_i within 4 n 2^-53 and <R^2>_i within 8 n 2^-53 relative.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1704_04381_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def run_gpu(rosen, seed, N, M0, max_pop, beta_eps, mu, c_hi, c_lo, coords=True):
    flags = rosen.ROSEN_STORE_COORDS if coords else 0
    p = rosen.perm_params(seed, N, M0, max_pop, beta_eps=beta_eps, mu=mu, c_hi=c_hi, c_lo=c_lo,
                          flags=flags)
    out = rosen.perm_outputs(N, max_pop, coords=coords)
    rosen.rosen_perm_run(p, out, rosen.perm_workspace(N, max_pop))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(g, o, N, max_pop):
    assert np.array_equal(g["population"], o["pop"])
    n = int(g["final_n"][0])
    assert n == o["n"]
    assert np.array_equal(g["w_m"][:n], o["w_m"])
    assert np.array_equal(g["w_e"][:n], o["w_e"])
    if "coords" in g:
        xyz = np.transpose(g["coords"][:, :, :n], (2, 0, 1))
        assert np.array_equal(xyz, o["pos"])
    tol = 4.0 * max_pop * EPS
    fin = np.isfinite(o["logz"])
    assert np.array_equal(np.isfinite(g["logz"]), fin)
    assert np.abs(g["logz"][fin] - o["logz"][fin]).max() <= tol * np.maximum(1.0, np.abs(o["logz"][fin])).max()
    rel = np.abs(g["mean_r2"][fin] - o["r2"][fin]) / np.maximum(o["r2"][fin], 1e-300)
    assert rel.max() <= 2 * tol


@pytest.mark.parametrize("seed,N,M0,max_pop,beta_eps,mu,c_hi,c_lo", [
    (1, 40, 3000, 12000, 0.0, 4.684, 1.3, 0.6),      # both operations, athermal
    (2, 32, 2000, 8000, 0.3, 5.2, 1.4, 0.5),         # interacting SAW
    (3, 24, 1500, 1500, 0.0, 4.684, 1.1, 0.6),       # the cap binds
    (4, 11, 800, 800, 0.2, 4.684, math.inf, 0.0),    # no thresholds: plain Rosenbluth
    (5, 200, 20000, 60000, 0.0, 4.684, 2.0, 0.5),    # long chains, many scan tiles
    (6, 2, 37, 100, 0.0, 4.684, 1.3, 0.6),           # a single step
    (8, 33, 2000, 6000, 0.35, 5.0, 1.3, 0.6),        # odd N: half slots of 20 words
    (9, 512, 300, 1200, 0.0, 4.684, 1.5, 0.5),       # the longest chains: 2 KiB slots
])
def test_matches_the_oracle(rosen, seed, N, M0, max_pop, beta_eps, mu, c_hi, c_lo):
    g = run_gpu(rosen, seed, N, M0, max_pop, beta_eps, mu, c_hi, c_lo)
    o = oracle.perm_run(seed, N, M0, max_pop, beta_eps=beta_eps, mu=mu, c_hi=c_hi, c_lo=c_lo,
                        positions=True)
    compare(g, o, N, max_pop)


def test_without_thresholds_equals_rosen_lattice_grow(rosen):
    # No pruning, enrichment or dead end (10 steps): chain j of the
    # population is chain j of rosen_lattice_grow.
    N, C = 11, 4096
    g = run_gpu(rosen, 7, N, C, C, 0.4, 4.684, math.inf, 0.0)
    out = rosen.lattice_outputs(N, C, coords=True)
    rosen.rosen_lattice_grow(rosen.lattice_params(7, N, C, beta_eps=0.4,
                                                  flags=rosen.ROSEN_STORE_COORDS), out)
    torch.cuda.synchronize()
    assert np.array_equal(g["coords"][:, :, :C], out["coords"].cpu().numpy())


def test_a_population_that_dies_out(rosen):
    # One chain, no enrichment: once it is trapped the population is empty.
    N = 300
    for seed in range(20):
        g = run_gpu(rosen, 100 + seed, N, 1, 1, 0.0, 4.684, math.inf, 0.0, coords=False)
        o = oracle.perm_run(100 + seed, N, 1, 1, c_hi=math.inf, c_lo=0.0)
        assert np.array_equal(g["population"], o["pop"])
        if o["n"] == 0:
            assert np.isneginf(g["logz"][-1])
            return
    pytest.fail("no trapped chain in 20 seeds")


def test_full_size_athermal_n64(rosen):
    # The bench's PERM configuration: N = 64, 10^6 chains started, cap 4x10^6.
    N, M0, cap = 64, 1_000_000, 4_000_000
    g = run_gpu(rosen, 9, N, M0, cap, 0.0, 4.684, 3.0, 1.0 / 3.0, coords=False)
    o = oracle.perm_run(9, N, M0, cap, mu=4.684, c_hi=3.0, c_lo=1.0 / 3.0)
    assert np.array_equal(g["population"], o["pop"])
    n = int(g["final_n"][0])
    assert n == o["n"]
    assert np.array_equal(g["w_m"][:n], o["w_m"]) and np.array_equal(g["w_e"][:n], o["w_e"])
    # The first three lengths are exact: every chain has W = 6, 30, 150.
    assert np.allclose(g["logz"][1:4], np.log([6.0, 30.0, 150.0]), rtol=0, atol=1e-12)
    assert np.abs(g["logz"] - o["logz"]).max() <= 4.0 * cap * EPS * abs(o["logz"]).max()
