"""Long chains in batches and in the serving loop.

Ensembles too long for the shared-memory kernels (lattice N > 512, real
space N > 1024) run in long-chain classes of a batch, and long requests run
through the long-chain entry points in the server.  Their statistics and
per-chain outputs must equal growing the ensemble alone through
rosen_lattice_grow_long / rosen_offlattice_grow_long, bit for bit.
"""
import json

import numpy as np
import pytest
import torch

from paper_1704_04381_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def alone(rosen, e):
    """Grow and reduce ensemble e alone through the long-chain entry points."""
    if e.model == rosen.ROSEN_MODEL_LATTICE:
        out = rosen.lattice_outputs(e.N, e.C)
        p = rosen.lattice_params(e.seed, e.N, e.C, beta_eps=e.beta_eps, ensemble=e.ensemble)
        rosen.rosen_lattice_grow_long(p, out, rosen.lattice_long_workspace(e.N, e.C))
        rin = rosen.lattice_reduce_in(out, e.N, use_counts=int(e.beta_eps == 0.0))
    else:
        out = rosen.offlattice_outputs(e.N, e.C)
        p = rosen.offlattice_params(e.seed, e.N, e.C, e.k, potential=e.potential,
                                    beta_eps=e.beta_eps, sigma=e.sigma, cutoff=e.cutoff,
                                    ensemble=e.ensemble)
        rosen.rosen_offlattice_grow_long(p, out, rosen.offlattice_long_workspace(e.N, e.C))
        rin = rosen.offlattice_reduce_in(out, e.N, e.k)
    st = rosen.stats_tensor()
    rosen.rosen_reduce(rin, st, rosen.reduce_workspace(e.C))
    torch.cuda.synchronize()
    return out, rosen.stats_dict(st)


def equal_stats(a, b, keys):
    for k in keys:
        assert a[k] == b[k] or (np.isnan(a[k]) and np.isnan(b[k])), (k, a[k], b[k])


def test_batch_with_long_chains(rosen):
    L, O = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    ens = [rosen.ensemble(L, 700, 3000, 61, 0, beta_eps=0.2),
           rosen.ensemble(L, 64, 5000, 62, 1),
           rosen.ensemble(O, 1500, 200, 63, 2, k=16),
           rosen.ensemble(O, 1200, 100, 64, 3, k=16, potential=rosen.ROSEN_LJ, beta_eps=0.7),
           rosen.ensemble(L, 2000, 800, 65, 4)]
    b = rosen.RosenBatch(ens)
    b.tune()
    b.run()
    torch.cuda.synchronize()
    classes = json.loads(b.describe())
    assert sorted(m for c in classes if c["long"] for m in c["members"]) == [0, 2, 3, 4]
    stats = b.stats().cpu().numpy()
    for e in (0, 2, 3, 4):
        out, st = alone(rosen, ens[e])
        got = dict(zip(rosen.STAT_KEYS, stats[e].tolist()))
        equal_stats(got, st, rosen.STAT_KEYS)
        mine = b.lattice_outputs(e) if ens[e].model == L else b.offlattice_outputs(e)
        torch.cuda.synchronize()
        for k in mine:
            np.testing.assert_array_equal(mine[k].cpu().numpy(), out[k].cpu().numpy(), err_msg=k)
    b.close()


def test_served_long_requests(rosen):
    srv = rosen.RosenServer(mem_budget_bytes=8 << 30, max_slots=4, max_queue=16)
    try:
        reqs = [rosen.request(rosen.ROSEN_MODEL_LATTICE, 1000, 2000, 71, 0, beta_eps=0.3),
                rosen.request(rosen.ROSEN_MODEL_OFFLATTICE, 1500, 100, 72, 1, k=32)]
        tickets = [srv.submit(r) for r in reqs]
        for r, t in zip(reqs, tickets):
            st, res = srv.wait(t, timeout_s=120)
            assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK, res.get("message")
            e = rosen.ensemble(r.model, r.N, r.C, r.seed, r.ensemble, k=r.k,
                               potential=r.potential, beta_eps=r.beta_eps, sigma=r.sigma,
                               cutoff=r.cutoff)
            _, ref = alone(rosen, e)
            equal_stats(res["stats"], ref, rosen.STAT_KEYS)
    finally:
        srv.close()
