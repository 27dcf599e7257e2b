"""GPU parity of rosen_offlattice_grow_long, the cell-grid kernel for long real-space chains.

It runs the same chain code as rosen_offlattice_grow; only the near list of a
step comes from the 27 cells around the end instead of a scan of every bead,
and it is put in the same bead order.  What is checked:
- With the same lanes per chain, every output is identical bit for bit:
  log W, R^2, R_g^2, alive, trace, coordinates, attempts, counters.
- Beyond N = 1024 the FP64 oracle decides: at least 99.9% of paths identical,
  within the FP32 bounds of the shorter-chain tests, up to N = 16384.
- Results do not depend on how many chain slots the workspace holds.
- A slot that outlives the 65535 generation tags clears its cell table and
  goes on unchanged.
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


def grow(rosen, seed, N, C, k, long=True, potential=0, beta_eps=0.0, sigma=1.0, lanes=16,
         max_attempts=0, chain0=0, ensemble=0, coords=True, ws_slots=None):
    flags = rosen.ROSEN_STORE_TRACE | (rosen.ROSEN_STORE_COORDS if coords else 0)
    out = rosen.offlattice_outputs(N, C, trace=True, coords=coords, counters=True, attempts=True)
    p = rosen.offlattice_params(seed, N, C, k, potential=potential, beta_eps=beta_eps,
                                sigma=sigma, chain0=chain0, ensemble=ensemble, flags=flags,
                                lanes_per_chain=lanes, max_attempts=max_attempts)
    if long:
        if ws_slots is None:
            ws = rosen.offlattice_long_workspace(N, C)
        else:
            per = rosen.rosen_offlattice_long_workspace_size(N, 1)
            ws = torch.empty(per * ws_slots // 8, dtype=torch.int64, device="cuda")
        rosen.rosen_offlattice_grow_long(p, out, ws)
    else:
        rosen.rosen_offlattice_grow(p, out)
    torch.cuda.synchronize()
    return {k_: v.cpu().numpy() for k_, v in out.items()}


def same(a, b):
    for key in ("logw", "r2", "rg2", "alive", "trace", "coords", "attempts", "counters"):
        assert (key in a) == (key in b), key
        if key in a:
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)


@pytest.mark.parametrize("N,k,pot,beta_eps,lanes", [
    (2, 32, 0, 0.0, 16), (3, 32, 0, 0.0, 16), (64, 32, 0, 0.0, 16), (300, 32, 0, 0.0, 16),
    (1024, 16, 0, 0.0, 32), (64, 32, 1, 1.0, 32), (500, 32, 1, 0.6, 32), (200, 16, 1, 0.8, 16),
    (300, 64, 1, 1.0, 32)])
def test_equals_shared_memory_kernel(rosen, N, k, pot, beta_eps, lanes):
    C = 600 if N >= 500 else 3001
    a = grow(rosen, 51, N, C, k, True, pot, beta_eps, lanes=lanes, chain0=77, ensemble=2)
    b = grow(rosen, 51, N, C, k, False, pot, beta_eps, lanes=lanes, chain0=77, ensemble=2)
    same(a, b)


def test_restart_mode_equals_shared_memory_kernel(rosen):
    a = grow(rosen, 52, 40, 3000, 8, True, sigma=1.5, max_attempts=4)
    b = grow(rosen, 52, 40, 3000, 8, False, sigma=1.5, max_attempts=4)
    assert (a["attempts"] > 1).any()
    same(a, b)


def compare_oracle(g, o, N, beta_eps=0.0):
    ok = (g["trace"].T == o["trace"]).all(1)
    assert ok.mean() >= 0.999, ok.mean()
    np.testing.assert_array_equal(g["alive"][ok], o["alive"][ok])
    al = ok & (o["alive"] == 1)
    lw = o["logw"][al]
    err = np.abs(g["logw"][al].astype(np.float64) - lw)
    assert (err <= (N - 1) * (2e-6 + 2e-7 * np.abs(lw) + 1e-5 * beta_eps)).all(), err.max()
    for key in ("r2", "rg2"):
        ref = o[key][al]
        err = np.abs(g[key][al].astype(np.float64) - ref)
        assert (err <= 2 * np.sqrt(ref) * (N - 1) * 4e-7 + 2e-6 * ref + 1e-7).all(), key


@pytest.mark.parametrize("N,C,k,pot,beta_eps", [(1500, 40, 16, 0, 0.0), (3000, 12, 32, 0, 0.0),
                                                (2000, 12, 16, 1, 0.7), (1200, 12, 64, 1, 1.0)])
def test_long_chains_follow_the_oracle(rosen, N, C, k, pot, beta_eps):
    g = grow(rosen, 53, N, C, k, True, pot, beta_eps, lanes=32 if pot else 16)
    o = oracle.offlattice_run(53, N, C, k, potential=pot, beta_eps=beta_eps, trace=True,
                              coords=True)
    compare_oracle(g, o, N, beta_eps)
    # Positions of identical paths: within the FP32 drift bound of the
    # oracle's, however many FP64 replays (each from the last replayed bead)
    # the chain went through.
    assert g["counters"][0] > 0
    same = (g["trace"].T == o["trace"]).all(1) & (o["alive"] == 1)
    xyz = np.transpose(g["coords"], (2, 0, 1))[same].astype(np.float64)
    assert np.abs(xyz - o["coords"][same]).max() <= (N - 1) * 4e-7 + 1e-6


def test_longest_chains(rosen):
    # k = 32: one of the four chains grows to step 16034 before a dead end.
    N, C, k = 16384, 4, 32
    g = grow(rosen, 54, N, C, k, True, coords=False)
    o = oracle.offlattice_run(54, N, C, k, trace=True)
    compare_oracle(g, o, N)


def test_results_do_not_depend_on_the_workspace(rosen):
    a = grow(rosen, 55, 1200, 40, 32, True)
    b = grow(rosen, 55, 1200, 40, 32, True, ws_slots=3)
    same(a, b)


def test_generation_wrap_clears_the_cell_table(rosen):
    # One slot grows all 66000 chains: growth 65536 clears the table.
    a = grow(rosen, 56, 4, 66_000, 8, True, ws_slots=1, coords=False)
    b = grow(rosen, 56, 4, 66_000, 8, False, coords=False)
    same(a, b)
