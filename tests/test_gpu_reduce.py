"""GPU parity of rosen_reduce with the oracle's FP64 reduction (Eq. 2, Eq. 9).

Both sides reduce the same per-chain inputs; they differ only in the order
of FP64 additions.  A sum of n non-negative terms carries a relative error of
at most (n-1) eps (eps = 2^-53) in any order, so sums, their ratios and logZ
agree within 4 n eps (relative; absolute for logZ).  The standard errors come
from sum w^2 (A - mean)^2 = Q2 - 2 mean Q1 + mean^2 Q0, whose cancellation
multiplies that bound by kappa = (Q2 + 2 |mean| Q1 + mean^2 Q0) / variance.
The GPU result is also deterministic: a second launch is bitwise identical.
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


EPS = 2.0 ** -53


def tolerance(o, key):
    """Relative (absolute for logZ) bound on the order-of-summation difference."""
    n = max(o["n_alive"], 1.0)
    base = 4.0 * n * EPS + 1e-15
    if key in ("se_r2", "se_rg2"):
        q1, q2 = ("Q1_r2", "Q2_r2") if key == "se_r2" else ("Q1_rg2", "Q2_rg2")
        m = o["mean_r2"] if key == "se_r2" else o["mean_rg2"]
        var = (o[key] * o["S0"]) ** 2
        kappa = (o[q2] + 2 * abs(m) * o[q1] + m * m * o["Q0"]) / var if var > 0 else 1.0
        return base * max(kappa, 1.0)
    return base


def close(g, o, keys=KEYS):
    for k in keys:
        if isinstance(o[k], float) and math.isnan(o[k]):
            assert math.isnan(g[k]), k
        elif math.isinf(o[k]) or k in ("n", "n_alive"):
            assert g[k] == o[k], k
        elif k == "log_max":
            # Equal inputs give the same maximum; log W recomputed from counts
            # may differ by a few ulp between the FMA chain and numpy's sum.
            assert abs(g[k] - o[k]) <= 8 * EPS * abs(o[k]), (k, g[k], o[k])
        elif k in ("logZ", "logZ_norm"):
            assert abs(g[k] - o[k]) <= tolerance(o, k), (k, g[k], o[k])
        else:
            assert abs(g[k] - o[k]) <= tolerance(o, k) * abs(o[k]), (k, g[k], o[k])


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
