"""The batched path (rosen_batch_*): many ensembles of uneven chain length and
model in one graph launch.

A chain is grown by the same device code whichever path runs it, and every
ensemble is reduced by the same tile and merge code as rosen_reduce.  So each
lattice ensemble's per-chain outputs and statistics are bitwise identical
alone and in the mix; a real-space ensemble is bitwise identical when grown
alone with the lanes per chain the batch chose, and otherwise takes the same
paths with per-chain values within the FP32 bounds of the single-ensemble
parity tests and statistics within 1e-5 relative.  The batch is also checked
against the oracle.
"""
import json

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


def mixed_ensembles(rosen):
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    return [
        rosen.ensemble(L, 64, 30_001, 2, 0, beta_eps=0.0),
        rosen.ensemble(L, 9, 5_000, 3, 1, beta_eps=0.3),
        rosen.ensemble(L, 150, 2_000, 4, 2, beta_eps=0.45),
        rosen.ensemble(L, 300, 700, 5, 3, beta_eps=0.1),
        rosen.ensemble(R, 64, 6_000, 6, 4, k=32, potential=rosen.ROSEN_HARD_SPHERE),
        rosen.ensemble(R, 40, 3_000, 7, 5, k=16, potential=rosen.ROSEN_LJ, beta_eps=0.8),
        rosen.ensemble(R, 130, 800, 8, 6, k=64, potential=rosen.ROSEN_LJ, beta_eps=0.4),
        rosen.ensemble(R, 20, 4_000, 9, 7, k=32, potential=rosen.ROSEN_LJ, beta_eps=0.0),
        rosen.ensemble(R, 12, 1_000, 10, 8, k=16, potential=rosen.ROSEN_HARD_SPHERE),
    ]


def single(rosen, e, lanes=0):
    """Grow and reduce ensemble e alone through the single-ensemble entry points."""
    st = rosen.stats_tensor()
    ws = rosen.reduce_workspace(e.C)
    if e.model == rosen.ROSEN_MODEL_LATTICE:
        out = rosen.lattice_outputs(e.N, e.C)
        rosen.rosen_lattice_grow(rosen.lattice_params(e.seed, e.N, e.C, beta_eps=e.beta_eps,
                                                      ensemble=e.ensemble), out)
        rosen.rosen_reduce(rosen.lattice_reduce_in(out, e.N, int(e.beta_eps == 0.0)), st, ws)
    else:
        out = rosen.offlattice_outputs(e.N, e.C)
        rosen.rosen_offlattice_grow(
            rosen.offlattice_params(e.seed, e.N, e.C, e.k, potential=e.potential,
                                    beta_eps=e.beta_eps, sigma=e.sigma, cutoff=e.cutoff,
                                    ensemble=e.ensemble, lanes_per_chain=lanes), out)
        rosen.rosen_reduce(rosen.offlattice_reduce_in(out, e.N, e.k), st, ws)
    return out, st


def test_alone_and_in_the_mix_are_identical(rosen):
    ens = mixed_ensembles(rosen)
    b = rosen.RosenBatch(ens)
    b.run()
    got = b.stats()
    torch.cuda.synchronize()
    classes = json.loads(b.describe())
    assert sum(c["ensembles"] for c in classes) == len(ens)
    lanes = {m: l for c in classes for m, l in zip(c["members"], c["member_lanes"])}
    for i, e in enumerate(ens):
        lattice = e.model == rosen.ROSEN_MODEL_LATTICE
        out, st = single(rosen, e, 0 if lattice else lanes[i])
        mine = b.lattice_outputs(i) if lattice else b.offlattice_outputs(i)
        torch.cuda.synchronize()
        assert torch.equal(got[i], st), (i, rosen.stats_dict(got[i]), rosen.stats_dict(st))
        for key, v in mine.items():
            assert torch.equal(v, out[key]), (i, key)
        if not lattice:
            # With the default lanes per chain: same paths, FP32-close values.
            out2, st2 = single(rosen, e)
            torch.cuda.synchronize()
            assert torch.equal(out2["alive"], mine["alive"])
            al = mine["alive"].bool()
            lw = out2["logw"][al].double()
            err = (mine["logw"][al].double() - lw).abs()
            assert (err <= (e.N - 1) * (2e-6 + 2e-7 * lw.abs() + 1e-5 * e.beta_eps)).all()
            a, b2 = rosen.stats_dict(got[i]), rosen.stats_dict(st2)
            for key in ("mean_r2", "mean_rg2", "logZ"):
                assert abs(a[key] - b2[key]) <= 1e-5 * abs(b2[key]), (i, key)
    b.close()


def test_repeated_runs_are_identical_and_match_the_oracle(rosen):
    ens = mixed_ensembles(rosen)[:2] + mixed_ensembles(rosen)[4:6]
    b = rosen.RosenBatch(ens)
    b.tune()
    b.run()
    first = b.stats().clone()
    b.run()
    second = b.stats()
    torch.cuda.synchronize()
    assert torch.equal(first, second)
    # Lattice chains are bit-exact with the oracle; real-space chains agree
    # within the FP32 bounds of the single-ensemble tests.
    e = ens[1]
    o = oracle.lattice_run(e.seed, e.N, e.C, beta_eps=e.beta_eps, ensemble=e.ensemble)
    g = {k: v.cpu().numpy() for k, v in b.lattice_outputs(1).items()}
    assert np.array_equal(g["r2"].astype(np.int64), o["r2"])
    assert np.array_equal(g["counts"].astype(np.int64), o["counts"].astype(np.int64))
    e = ens[3]
    o = oracle.offlattice_run(e.seed, e.N, e.C, e.k, potential=oracle.LJ, beta_eps=e.beta_eps,
                              ensemble=e.ensemble)
    g = {k: v.cpu().numpy() for k, v in b.offlattice_outputs(3).items()}
    assert (g["alive"] == o["alive"]).mean() >= 0.999
    al = (g["alive"] == 1) & (o["alive"] == 1)
    lw = o["logw"][al]
    ok = np.abs(g["logw"][al] - lw) <= (e.N - 1) * (2e-6 + 2e-7 * np.abs(lw) + 1e-5 * e.beta_eps)
    assert ok.mean() >= 0.999
    b.close()


def test_large_members_get_their_own_launch(rosen):
    # A member with several waves of resident chains runs as its own
    # single-ensemble launch inside the graph; its outputs are those of
    # rosen_*_grow with the default lanes, bit for bit, and the small members
    # of its class still share the class kernel.
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    ens = [rosen.ensemble(R, 60, 300_000, 21, 0, k=32, potential=rosen.ROSEN_LJ, beta_eps=0.6),
           rosen.ensemble(R, 50, 700, 22, 1, k=32, potential=rosen.ROSEN_LJ, beta_eps=0.3),
           rosen.ensemble(R, 64, 400_000, 23, 2, k=32),
           rosen.ensemble(L, 64, 3_000_000, 24, 3, beta_eps=0.2),
           rosen.ensemble(L, 60, 2_000, 25, 4, beta_eps=0.1)]
    b = rosen.RosenBatch(ens)
    b.tune()
    b.run()
    b.run()
    got = b.stats()
    torch.cuda.synchronize()
    classes = json.loads(b.describe())
    own = {m: o for c in classes for m, o in zip(c["members"], c["own_launch"])}
    assert own[0] == own[2] == own[3] == 1 and own[1] == own[4] == 0
    lanes = {m: l for c in classes for m, l in zip(c["members"], c["member_lanes"])}
    for i, e in enumerate(ens):
        lattice = e.model == rosen.ROSEN_MODEL_LATTICE
        out, st = single(rosen, e, 0 if (lattice or own[i]) else lanes[i])
        mine = b.lattice_outputs(i) if lattice else b.offlattice_outputs(i)
        torch.cuda.synchronize()
        assert torch.equal(got[i], st), i
        for key, v in mine.items():
            assert torch.equal(v, out[key]), (i, key)
    b.close()


def test_config_like_batch_runs(rosen):
    # A scaled-down draw of the batched configuration: N uniform in [8, 256],
    # chain counts log-uniform, half lattice ISAW, half LJ with k in {16,32,64}.
    rng = np.random.default_rng(4)
    ens = []
    for e in range(24):
        N = int(rng.integers(8, 257))
        C = int(10 ** rng.uniform(2, 3.5))
        if e % 2 == 0:
            ens.append(rosen.ensemble(rosen.ROSEN_MODEL_LATTICE, N, C, 1000 + e, e,
                                      beta_eps=float(rng.uniform(0, 0.5))))
        else:
            ens.append(rosen.ensemble(rosen.ROSEN_MODEL_OFFLATTICE, N, C, 1000 + e, e,
                                      k=int(rng.choice([16, 32, 64])), potential=rosen.ROSEN_LJ,
                                      beta_eps=float(rng.uniform(0, 1))))
    b = rosen.RosenBatch(ens)
    b.run()
    st = b.stats().cpu().numpy()
    assert np.isfinite(st[:, 11]).all()          # logZ
    assert (st[:, 1] > 0).all()                   # live chains in every ensemble
    lanes = {m: l for c in json.loads(b.describe())
             for m, l in zip(c["members"], c["member_lanes"])}
    for i in (0, 1, 7):
        lat = ens[i].model == rosen.ROSEN_MODEL_LATTICE
        _, s1 = single(rosen, ens[i], 0 if lat else lanes[i])
        torch.cuda.synchronize()
        assert np.array_equal(s1.cpu().numpy(), st[i])
    b.close()
