"""GPU parity of restart mode (Sections 3.3.2 and 3.3.3) with the FP64 oracle.

In restart mode a chain that reaches a dead end is thrown away and grown
again from the first monomer, with the attempt index in the high half of the
Philox step word, for at most max_attempts growths.  The tests check:
- Lattice chains agree with the oracle bit for bit: the attempts, the trace of
  the last growth, the counts, R_ee^2, N^2 R_g^2 and the coordinates.
- Real-space chains take the oracle's path (trace and attempts equal) in at
  least 99.9% of chains, to the same bounds as without restarts.
- The reduction counts every growth: n = sum of attempts (Eq. 9).
- Batched and served ensembles in restart mode equal the single-ensemble
  path.
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


def grow_lattice(rosen, seed, N, C, beta_eps, max_attempts, coords=False):
    flags = rosen.ROSEN_STORE_TRACE | (rosen.ROSEN_STORE_COORDS if coords else 0)
    out = rosen.lattice_outputs(N, C, trace=True, coords=coords, attempts=True)
    rosen.rosen_lattice_grow(rosen.lattice_params(seed, N, C, beta_eps=beta_eps, flags=flags,
                                                  max_attempts=max_attempts), out)
    torch.cuda.synchronize()
    return out


def grow_off(rosen, seed, N, C, k, max_attempts, sigma=1.0, potential=0, beta_eps=0.0):
    out = rosen.offlattice_outputs(N, C, trace=True, attempts=True)
    rosen.rosen_offlattice_grow(
        rosen.offlattice_params(seed, N, C, k, potential=potential, beta_eps=beta_eps,
                                sigma=sigma, flags=rosen.ROSEN_STORE_TRACE,
                                max_attempts=max_attempts), out)
    torch.cuda.synchronize()
    return out


def host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def gpu_stats(rosen, inp, C):
    st = rosen.stats_tensor()
    rosen.rosen_reduce(inp, st, rosen.reduce_workspace(C))
    torch.cuda.synchronize()
    return rosen.stats_dict(st)


@pytest.mark.parametrize("N,C,beta_eps,A", [(64, 30_000, 0.0, 16), (64, 30_000, 0.4, 16),
                                            (200, 6000, 0.2, 2), (150, 5000, 0.0, 3)])
def test_lattice_restart_bit_exact(rosen, N, C, beta_eps, A):
    g = host(grow_lattice(rosen, 31, N, C, beta_eps, A, coords=True))
    o = oracle.lattice_run(31, N, C, beta_eps=beta_eps, trace=True, coords=True, max_attempts=A)
    assert (o["attempts"] > 1).any()
    np.testing.assert_array_equal(g["attempts"].astype(np.uint16), o["attempts"])
    np.testing.assert_array_equal(g["counts"].astype(np.int64), o["counts"].astype(np.int64))
    np.testing.assert_array_equal(g["r2"].astype(np.int64), o["r2"])
    np.testing.assert_array_equal(g["n2rg2"], o["n2rg2"])
    np.testing.assert_array_equal(g["trace"].T, o["trace"])
    np.testing.assert_array_equal(np.transpose(g["coords"], (2, 0, 1)).astype(np.float64),
                                  o["coords"])
    dead = o["alive"] == 0
    np.testing.assert_array_equal(np.isneginf(g["logw"]), dead)
    lw = o["logw"][~dead]
    err = np.abs(g["logw"][~dead].astype(np.float64) - lw)
    assert (err <= (N - 1) * (1e-6 + 6e-8 * np.abs(lw))).all()


@pytest.mark.parametrize("C", [1, 31, 33, 1000])
def test_lattice_restart_small_and_ragged(rosen, C):
    # The persistent restart kernel splits the chains into per-warp ranges;
    # tiny and ragged ensembles exercise its empty and partial ranges.  Wide
    # dead-end odds (N = 300) make every pass carry retries.
    N = 300
    g = host(grow_lattice(rosen, 37, N, C, 0.1, 5, coords=True))
    o = oracle.lattice_run(37, N, C, beta_eps=0.1, trace=True, coords=True, max_attempts=5)
    np.testing.assert_array_equal(g["attempts"].astype(np.uint16), o["attempts"])
    np.testing.assert_array_equal(g["counts"].astype(np.int64), o["counts"].astype(np.int64))
    np.testing.assert_array_equal(g["trace"].T, o["trace"])
    np.testing.assert_array_equal(g["n2rg2"], o["n2rg2"])


def test_single_attempt_equals_plain_growth(rosen):
    N, C = 64, 20_000
    a = host(grow_lattice(rosen, 32, N, C, 0.2, 1))
    b = host(grow_lattice(rosen, 32, N, C, 0.2, 0))
    for key in ("counts", "logw", "r2", "n2rg2", "trace"):
        np.testing.assert_array_equal(a[key], b[key])
    assert (a["attempts"] == 1).all()


def test_lattice_restart_reduction_counts_every_growth(rosen):
    N, C = 64, 50_000
    out = grow_lattice(rosen, 33, N, C, 0.0, 16)
    st = gpu_stats(rosen, rosen.lattice_reduce_in(out, N, use_counts=1), C)
    att = out["attempts"].cpu().numpy().astype(np.int64)
    assert st["n"] == att.sum() > C
    o = oracle.lattice_run(33, N, C, max_attempts=16)
    ref = oracle.reduce(o["logw"], o["r2"], o["n2rg2"] / N ** 2, N, n=o["attempts"].sum())
    for key in ("n", "n_alive", "logZ", "mean_r2", "mean_rg2", "se_r2", "ess"):
        assert abs(st[key] - ref[key]) <= 1e-9 * max(1.0, abs(ref[key])), (key, st, ref)


def test_trimer_restart_paths_and_closed_form(rosen):
    # Hard-sphere trimer with sigma = 1.8, k = 2: a growth dies with
    # probability q = (sigma^2/4)^k = 0.6561; E[W/k^2] = p = 1 - sigma^2/4.
    sigma, k, A, N, C = 1.8, 2, 6, 3, 200_000
    out = grow_off(rosen, 34, N, C, k, A, sigma=sigma)
    g = host(out)
    o = oracle.offlattice_run(34, N, C, k, sigma=sigma, trace=True, max_attempts=A)
    np.testing.assert_array_equal(g["attempts"].astype(np.uint16), o["attempts"])
    np.testing.assert_array_equal(g["trace"].T, o["trace"])
    np.testing.assert_array_equal(g["alive"], o["alive"])
    st = gpu_stats(rosen, rosen.offlattice_reduce_in(out, N, k), C)
    a = g["attempts"].astype(np.int64)
    assert st["n"] == a.sum()
    p = 1.0 - sigma ** 2 / 4.0
    wn = np.where(g["alive"] == 1, np.exp(g["logw"].astype(np.float64) - 2 * np.log(k)), 0.0)
    R = wn.sum() / a.sum()
    se = np.sqrt(((wn - R * a) ** 2).sum()) / a.sum()
    assert abs(np.exp(st["logZ_norm"]) - R) <= 1e-6 * R
    assert abs(R - p) < 4.5 * se, (R, p, se)
    assert abs(st["mean_r2"] - (2 + sigma ** 2 / 2)) < 4.5 * st["se_r2"]


@pytest.mark.parametrize("N,k,sigma,A", [(64, 32, 1.0, 8), (24, 8, 1.5, 4), (40, 16, 1.3, 3)])
def test_real_space_restart_paths(rosen, N, k, sigma, A):
    C = 3000
    g = host(grow_off(rosen, 35, N, C, k, A, sigma=sigma))
    o = oracle.offlattice_run(35, N, C, k, sigma=sigma, trace=True, max_attempts=A)
    assert (o["attempts"] > 1).any()
    same = (g["trace"].T == o["trace"]).all(1) & (g["attempts"] == o["attempts"])
    assert same.mean() >= 0.999, same.mean()
    np.testing.assert_array_equal(g["alive"][same], o["alive"][same])
    al = same & (o["alive"] == 1)
    lw = o["logw"][al]
    err = np.abs(g["logw"][al].astype(np.float64) - lw)
    assert (err <= (N - 1) * (2e-6 + 2e-7 * np.abs(lw))).all()
    ref = o["r2"][al]
    err = np.abs(g["r2"][al].astype(np.float64) - ref)
    assert (err <= 2 * np.sqrt(ref) * (N - 1) * 4e-7 + 2e-6 * ref + 1e-7).all()


def test_lennard_jones_restart_changes_nothing_without_dead_ends(rosen):
    # LJ trials never all have infinite energy at a finite distance, so no
    # growth is discarded: restart mode equals plain growth.
    N, C, k = 48, 4000, 16
    a = host(grow_off(rosen, 36, N, C, k, 8, potential=1, beta_eps=0.6))
    b = host(grow_off(rosen, 36, N, C, k, 0, potential=1, beta_eps=0.6))
    assert (a["attempts"] == 1).all()
    for key in ("logw", "r2", "rg2", "trace"):
        np.testing.assert_array_equal(a[key], b[key])


def test_batch_restart_equals_single(rosen):
    ens = [rosen.ensemble(rosen.ROSEN_MODEL_LATTICE, 150, 20_000, 40, 0, beta_eps=0.3,
                          max_attempts=4),
           rosen.ensemble(rosen.ROSEN_MODEL_OFFLATTICE, 30, 6000, 41, 1, k=8, sigma=1.5,
                          max_attempts=4),
           rosen.ensemble(rosen.ROSEN_MODEL_LATTICE, 64, 10_000, 42, 2)]
    b = rosen.RosenBatch(ens)
    b.tune()
    b.run()
    torch.cuda.synchronize()
    stats = b.stats().cpu().numpy()
    # Lattice ensemble 0: bitwise equal to growing and reducing it alone.
    out = grow_lattice(rosen, 40, 150, 20_000, 0.3, 4)
    lat = b.lattice_outputs(0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lat["attempts"].cpu().numpy(), out["attempts"].cpu().numpy())
    single = gpu_stats(rosen, rosen.lattice_reduce_in(out, 150, use_counts=0), 20_000)
    for q, key in enumerate(rosen.STAT_KEYS):
        assert stats[0, q] == single[key] or (np.isnan(stats[0, q]) and np.isnan(single[key])), key
    # Real-space ensemble 1: same attempts and paths as the oracle.
    off = b.offlattice_outputs(1)
    torch.cuda.synchronize()
    o = oracle.offlattice_run(41, 30, 6000, 8, sigma=1.5, ensemble=1, max_attempts=4)
    same = off["attempts"].cpu().numpy().astype(np.uint16) == o["attempts"]
    assert same.mean() >= 0.999
    assert stats[1, 0] == off["attempts"].cpu().numpy().astype(np.int64).sum()
    # Ensemble 2 is not in restart mode: n = C.
    assert stats[2, 0] == 10_000
    b.close()


def test_served_restart_request_equals_single(rosen):
    srv = rosen.RosenServer(mem_budget_bytes=2 << 30, max_slots=4, max_queue=16)
    try:
        t = srv.submit(rosen.request(rosen.ROSEN_MODEL_LATTICE, 150, 20_000, 40, 0,
                                     beta_eps=0.3, max_attempts=4))
        st, r = srv.wait(t, timeout_s=120)
        assert st == rosen.ROSEN_OK and r["status"] == rosen.ROSEN_OK
        out = grow_lattice(rosen, 40, 150, 20_000, 0.3, 4)
        single = gpu_stats(rosen, rosen.lattice_reduce_in(out, 150, use_counts=0), 20_000)
        for key in rosen.STAT_KEYS:
            a, b = r["stats"][key], single[key]
            assert a == b or (np.isnan(a) and np.isnan(b)), key
    finally:
        srv.close()
