"""GPU parity of rosen_lattice_grow_long, the hash-table kernel for long lattice chains.

It follows the same rule and draws as rosen_lattice_grow (Algorithm 1, Eq. 3).
What is checked:
- Where both kernels apply (N <= 512), every output must be identical bit
  for bit: counts, log W, R^2, N^2 R_g^2, trace, coordinates, attempts.
- Beyond that the FP64 oracle decides, bit for bit, up to the maximum
  N = 32768.
- Results must not depend on how many tables the workspace holds.
- A lane that outlives the 65535 generation tags clears its table and goes
  on unchanged.
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


def grow(rosen, seed, N, C, beta_eps=0.0, long=True, chain0=0, ensemble=0, max_attempts=0,
         coords=True, ws_tables=None):
    flags = rosen.ROSEN_STORE_TRACE | (rosen.ROSEN_STORE_COORDS if coords else 0)
    out = rosen.lattice_outputs(N, C, trace=True, coords=coords, attempts=True)
    p = rosen.lattice_params(seed, N, C, beta_eps=beta_eps, chain0=chain0, ensemble=ensemble,
                             flags=flags, max_attempts=max_attempts)
    if long:
        if ws_tables is None:
            ws = rosen.lattice_long_workspace(N, C)
        else:
            per = rosen.rosen_lattice_long_workspace_size(N, 1)
            ws = torch.empty(per * ws_tables // 8, dtype=torch.int64, device="cuda")
        rosen.rosen_lattice_grow_long(p, out, ws)
    else:
        rosen.rosen_lattice_grow(p, out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def same(a, b, keys=("counts", "logw", "r2", "n2rg2", "trace", "coords", "attempts")):
    for k in keys:
        if k in a and k in b:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def vs_oracle(g, o, N):
    np.testing.assert_array_equal(g["counts"].astype(np.int64), o["counts"].astype(np.int64))
    np.testing.assert_array_equal(g["r2"].astype(np.int64), o["r2"])
    np.testing.assert_array_equal(g["n2rg2"], o["n2rg2"])
    np.testing.assert_array_equal(g["trace"].T, o["trace"])
    np.testing.assert_array_equal(g["attempts"].astype(np.uint16), o["attempts"])
    if "coords" in g and "coords" in o:
        np.testing.assert_array_equal(np.transpose(g["coords"], (2, 0, 1)).astype(np.float64),
                                      o["coords"])
    dead = o["alive"] == 0
    np.testing.assert_array_equal(np.isneginf(g["logw"]), dead)
    lw = o["logw"][~dead]
    err = np.abs(g["logw"][~dead].astype(np.float64) - lw)
    assert (err <= (N - 1) * (1e-6 + 6e-8 * np.abs(lw))).all(), err.max()


@pytest.mark.parametrize("N,beta_eps", [(2, 0.0), (3, 0.3), (64, 0.0), (64, 0.4), (257, 0.2),
                                        (512, 0.0), (512, 0.3)])
def test_equals_shared_memory_kernel(rosen, N, beta_eps):
    C = 5003
    a = grow(rosen, 41, N, C, beta_eps, long=True, chain0=999, ensemble=4)
    b = grow(rosen, 41, N, C, beta_eps, long=False, chain0=999, ensemble=4)
    same(a, b)


def test_restart_mode_equals_shared_memory_kernel(rosen):
    a = grow(rosen, 42, 300, 4000, 0.2, long=True, max_attempts=4)
    b = grow(rosen, 42, 300, 4000, 0.2, long=False, max_attempts=4)
    assert (a["attempts"] > 1).any()
    same(a, b)


@pytest.mark.parametrize("N,C,beta_eps,A", [(600, 300, 0.0, 0), (1500, 120, 0.3, 0),
                                            (1000, 200, 0.1, 3), (4096, 24, 0.0, 2),
                                            (4096, 24, 0.4, 0)])
def test_long_chains_bit_exact(rosen, N, C, beta_eps, A):
    g = grow(rosen, 43, N, C, beta_eps, max_attempts=A)
    o = oracle.lattice_run(43, N, C, beta_eps=beta_eps, trace=True, coords=True, max_attempts=A)
    vs_oracle(g, o, N)


def test_longest_chains(rosen):
    N, C = 32768, 3
    g = grow(rosen, 44, N, C, 0.0, coords=False)
    o = oracle.lattice_run(44, N, C, trace=True, max_attempts=1)
    vs_oracle(g, o, N)


def test_results_do_not_depend_on_the_workspace(rosen):
    N, C = 700, 600
    a = grow(rosen, 45, N, C, 0.2)
    b = grow(rosen, 45, N, C, 0.2, ws_tables=7)
    same(a, b)


def test_generation_wrap_clears_the_table(rosen):
    # One table grows all 66000 chains: growth 65536 clears the table and
    # restarts the generation tags.
    N, C = 8, 66_000
    a = grow(rosen, 46, N, C, 0.3, ws_tables=1)
    b = grow(rosen, 46, N, C, 0.3, long=False)
    same(a, b)
