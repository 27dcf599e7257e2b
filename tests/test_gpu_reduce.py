"""GPU parity of rosen_reduce with the oracle's FP64 reduction (Eq. 2, Eq. 9).

Both sides reduce the same per-chain inputs; they differ only in the order
of FP64 additions, so the statistics agree to 1e-12 relative.  The GPU
result is also deterministic: a second launch is bitwise identical.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1704_04381_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu
KEYS = ("n", "n_alive", "log_max", "logZ", "mean_r2", "se_r2", "mean_rg2", "se_rg2", "ess")


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def close(g, o, keys=KEYS, rel=1e-12):
    for k in keys:
        if isinstance(o[k], float) and math.isnan(o[k]):
            assert math.isnan(g[k]), k
        elif math.isinf(o[k]):
            assert g[k] == o[k], k
        else:
            assert g[k] == pytest.approx(o[k], rel=rel, abs=1e-300), (k, g[k], o[k])


def lattice_case(rosen, seed, N, C, beta_eps):
    out = rosen.lattice_outputs(N, C)
    rosen.rosen_lattice_grow(rosen.lattice_params(seed, N, C, beta_eps=beta_eps), out)
    return out


@pytest.mark.parametrize("N,C,beta_eps,use_counts", [
    (16, 100_000, 0.0, 1), (16, 100_000, 0.0, 0), (64, 20_001, 0.4, 0), (64, 1, 0.2, 0),
    (64, 2048, 0.0, 1), (64, 2049, 0.0, 1)])
def test_lattice_reduce_matches_oracle(rosen, N, C, beta_eps, use_counts):
    out = lattice_case(rosen, 4, N, C, beta_eps)
    st = rosen.stats_tensor()
    ws = rosen.reduce_workspace(C)
    rosen.rosen_reduce(rosen.lattice_reduce_in(out, N, use_counts), st, ws)
    g = rosen.stats_dict(st)
    if use_counts:
        lw = oracle.lattice_logw_from_counts(out["counts"].cpu().numpy().astype(np.int64))
    else:
        lw = out["logw"].cpu().double().numpy()
    o = oracle.reduce(lw, out["r2"].cpu().double().numpy(),
                      out["n2rg2"].cpu().double().numpy() / float(N * N), N)
    close(g, o)
    # Deterministic: the same launch again gives the same bits.
    st2 = rosen.stats_tensor()
    rosen.rosen_reduce(rosen.lattice_reduce_in(out, N, use_counts), st2, ws)
    assert torch.equal(st, st2)


def test_reduce_exact_weights_against_integers(rosen):
    # Athermal N = 16: W = prod m^counts is an exact integer; the FP64 device
    # reduction from counts must reproduce the exact rational mean.
    N, C = 16, 50_000
    out = lattice_case(rosen, 1, N, C, 0.0)
    st = rosen.stats_tensor()
    rosen.rosen_reduce(rosen.lattice_reduce_in(out, N, 1), st, rosen.reduce_workspace(C))
    g = rosen.stats_dict(st)
    cnt = out["counts"].cpu().numpy().astype(np.int64)
    r2 = out["r2"].cpu().numpy().astype(np.int64)
    W = [0 if c[0] else int(2 ** c[2] * 3 ** c[3] * 4 ** c[4] * 5 ** c[5] * 6 ** c[6]) for c in cnt]
    S0 = sum(W)
    S1 = sum(w * int(a) for w, a in zip(W, r2))
    assert g["mean_r2"] == pytest.approx(S1 / S0, rel=1e-13)
    assert g["logZ"] == pytest.approx(math.log(S0 / C), abs=1e-12)


def test_reduce_all_dead_and_mixed(rosen):
    C, N = 5000, 8
    logw = torch.full((C,), float("-inf"), dtype=torch.float32, device="cuda")
    r2 = torch.arange(C, dtype=torch.float32, device="cuda")
    rg2 = torch.ones(C, dtype=torch.float32, device="cuda")
    inp = rosen.rosen_reduce_in(kind=rosen.ROSEN_REDUCE_OFFLATTICE, N=N, k=16, use_counts=0, C=C,
                                logw=logw.data_ptr(), r2_f=r2.data_ptr(), rg2_f=rg2.data_ptr())
    st = rosen.stats_tensor()
    ws = rosen.reduce_workspace(C)
    rosen.rosen_reduce(inp, st, ws)
    g = rosen.stats_dict(st)
    assert g["n_alive"] == 0 and g["logZ"] == -math.inf and g["ess"] == 0
    assert math.isnan(g["mean_r2"])
    # Weights spanning hundreds of orders of magnitude, a dead chain per tile.
    gen = torch.Generator(device="cpu").manual_seed(5)
    lw = (torch.rand(C, generator=gen) * 600 - 300).to(torch.float32)
    lw[::2048] = float("-inf")
    logw.copy_(lw)
    rosen.rosen_reduce(inp, st, ws)
    g = rosen.stats_dict(st)
    o = oracle.reduce(lw.double().numpy(), r2.cpu().double().numpy(),
                      rg2.cpu().double().numpy(), N, k=16)
    close(g, o, KEYS + ("logZ_norm",))
