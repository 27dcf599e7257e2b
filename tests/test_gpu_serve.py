"""The request loop (rosen_serve_*).

- Each request's result is the same alone and in the mix: the chains of a
  request are a pure function of its parameters, and the server runs them
  with the single-ensemble kernels, so the statistics must be bitwise equal
  to a request served on its own.
- Requests that arrive while others run are admitted and overlap with them.
- Failures are made on the host: a request larger than the whole budget, a
  full queue, a cancelled ticket, a wait that times out, an unknown ticket, a
  client thread that submits and leaves, a server destroyed with work pending.
"""
import threading
import time

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


def mix(rosen):
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    return [
        rosen.request(L, 64, 200_000, 2, 0, beta_eps=0.2),
        rosen.request(R, 48, 20_000, 3, 1, k=32, potential=rosen.ROSEN_HARD_SPHERE),
        rosen.request(L, 16, 50_000, 4, 2),
        rosen.request(R, 30, 10_000, 5, 3, k=16, potential=rosen.ROSEN_LJ, beta_eps=0.7),
        rosen.request(L, 200, 3_000, 6, 4, beta_eps=0.4, store_coords=True),
        rosen.request(R, 64, 2_000, 7, 5, k=64, potential=rosen.ROSEN_LJ, beta_eps=1.0,
                      store_coords=True),
    ]


@pytest.mark.parametrize("shortest_first", [False, True])
def test_alone_and_in_the_mix(rosen, shortest_first):
    # With shortest_first the streams carry priorities by work; the results
    # are the same either way.
    srv = rosen.RosenServer(mem_budget_bytes=8 << 30, max_slots=8, shortest_first=shortest_first)
    alone = []
    for r in mix(rosen):
        t = srv.submit(r)
        st, res = srv.wait(t, 120)
        assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK, res
        alone.append(res["stats"])
        assert srv.release(t) == rosen.ROSEN_OK
    tickets = [srv.submit(r) for r in mix(rosen)]
    admitted = []
    for t, a in zip(tickets, alone):
        st, res = srv.wait(t, 120)
        assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK
        assert res["stats"] == a            # bitwise: same kernels, same chains
        admitted.append((res["t_admit_ns"], res["t_done_ns"]))
    # Continuous admission: requests submitted together were on the GPU together.
    overlaps = sum(1 for i, (a0, d0) in enumerate(admitted) for (a1, d1) in admitted[i + 1:]
                   if a1 < d0 and a0 < d1)
    assert overlaps >= 1
    info = srv.info()
    assert info["completed"] == 12 and info["running"] == 0
    # Stored conformations stay until release.
    assert info["bytes_in_use"] > 0
    for t in tickets:
        assert srv.release(t) == rosen.ROSEN_OK
    time.sleep(0.05)
    assert srv.info()["bytes_in_use"] == 0
    srv.close()


def test_admission_respects_the_budget(rosen):
    L = rosen.ROSEN_MODEL_LATTICE
    big = rosen.request(L, 64, 2_000_000, 9, 0, beta_eps=0.3)
    srv = rosen.RosenServer(mem_budget_bytes=100 << 20, max_slots=8)   # fits one at a time
    tickets = [srv.submit(big) for _ in range(3)]
    res = [srv.wait(t, 120)[1] for t in tickets]
    spans = sorted((r["t_admit_ns"], r["t_done_ns"]) for r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 2_000_000         # next admitted only after the previous finished
    assert res[0]["stats"] == res[1]["stats"] == res[2]["stats"]
    srv.close()


def test_host_side_failures(rosen):
    L = rosen.ROSEN_MODEL_LATTICE
    srv = rosen.RosenServer(mem_budget_bytes=64 << 20, max_slots=1, max_queue=2)
    # Larger than the whole budget: rejected at submit.
    st, _ = srv.try_submit(rosen.request(L, 64, 10_000_000, 1))
    assert st == rosen.ROSEN_EINVAL and "budget" in rosen.last_error()
    # Invalid parameters.
    assert srv.try_submit(rosen.request(L, 1, 100, 1))[0] == rosen.ROSEN_EINVAL
    # A long request occupies the only slot; two more fill the queue; the next is EBUSY.
    long_req = rosen.request(L, 512, 2_000_000, 2, beta_eps=0.2)
    t0 = srv.submit(long_req)
    deadline = time.time() + 10
    while srv.info()["running"] < 1 and time.time() < deadline:
        time.sleep(0.001)
    assert srv.info()["running"] == 1
    t1 = srv.submit(rosen.request(L, 32, 1000, 3))
    t2 = srv.submit(rosen.request(L, 32, 1000, 4))
    assert srv.try_submit(rosen.request(L, 32, 1000, 5))[0] == rosen.ROSEN_EBUSY
    # A queued request can be cancelled; a running one cannot.
    assert srv.cancel(t2) == rosen.ROSEN_OK
    assert srv.cancel(t0) == rosen.ROSEN_EBUSY
    st, res = srv.poll(t2)
    assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_ECLOSED
    # A bounded wait that runs out.
    st, _ = srv.wait(t1, 0.001)
    assert st in (rosen.ROSEN_ETIMEOUT, rosen.ROSEN_OK)
    assert srv.poll(12345)[0] == rosen.ROSEN_ENOTFOUND
    assert srv.wait(t1, 120)[0] == rosen.ROSEN_OK
    assert srv.wait(t0, 120)[0] == rosen.ROSEN_OK
    # A client thread that submits and leaves without waiting: the work still
    # completes and another thread collects it.
    box = {}
    th = threading.Thread(target=lambda: box.setdefault("t", srv.submit(rosen.request(L, 32, 500, 6))))
    th.start()
    th.join()
    st, res = srv.wait(box["t"], 60)
    assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK
    # Destroy with work queued: queued requests are cancelled, running ones finish.
    srv.submit(long_req)
    srv.submit(rosen.request(L, 32, 1000, 7))
    srv.close()
    assert srv.handle is None


def test_results_match_the_single_ensemble_path(rosen):
    R = rosen.ROSEN_MODEL_OFFLATTICE
    r = rosen.request(R, 40, 5_000, 11, 2, k=32, potential=rosen.ROSEN_LJ, beta_eps=0.5)
    srv = rosen.RosenServer(mem_budget_bytes=1 << 30)
    st, res = srv.wait(srv.submit(r), 60)
    srv.close()
    out = rosen.offlattice_outputs(40, 5_000)
    rosen.rosen_offlattice_grow(rosen.offlattice_params(11, 40, 5_000, 32, potential=rosen.ROSEN_LJ,
                                                        beta_eps=0.5, ensemble=2), out)
    s = rosen.stats_tensor()
    rosen.rosen_reduce(rosen.offlattice_reduce_in(out, 40, 32), s, rosen.reduce_workspace(5_000))
    assert np.array_equal(s.cpu().numpy(), np.array([res["stats"][k] for k in rosen.STAT_KEYS]))


def test_served_results_match_the_oracle(rosen):
    # A mix served together, every request checked against the FP64 oracle
    # (Eq. 2 / Eq. 9 estimator): per-chain conformations from the server's
    # stored coordinates, ensemble statistics from oracle.reduce.
    import oracle
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    reqs = [
        # lattice ISAW, conformations stored: bit-exact
        ("isaw", rosen.request(L, 48, 3000, 21, 4, beta_eps=0.3, store_coords=True)),
        # athermal lattice: exact counts, statistics to FP64 rounding
        ("athermal", rosen.request(L, 40, 4000, 22, 5, store_coords=True)),
        # hard spheres and Lennard-Jones: the oracle's paths
        ("hs", rosen.request(R, 40, 2000, 23, 6, k=32, store_coords=True)),
        ("lj", rosen.request(R, 32, 1500, 24, 7, k=16, potential=rosen.ROSEN_LJ, beta_eps=0.8,
                             store_coords=True)),
        # long chains: the long-chain kernels inside the server
        ("long", rosen.request(L, 600, 300, 25, 8, beta_eps=0.2, store_coords=True)),
    ]
    srv = rosen.RosenServer(mem_budget_bytes=4 << 30, max_slots=8)
    try:
        tickets = [srv.submit(r) for _, r in reqs]
        for (kind, r), t in zip(reqs, tickets):
            st, res = srv.wait(t, 180)
            assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK, res
            N, C = r.N, r.C
            xyz = rosen.served_coords(res, r.model, N, C).cpu().numpy()   # [N][3][C]
            xyz = np.transpose(xyz, (2, 0, 1))                               # [C][N][3]
            got = res["stats"]
            if r.model == L:
                o = oracle.lattice_run(r.seed, N, C, beta_eps=r.beta_eps, ensemble=r.ensemble,
                                       coords=True)
                assert np.array_equal(xyz.astype(np.float64), o["coords"]), kind
                ref = oracle.reduce(o["logw"], o["r2"].astype(np.float64), o["n2rg2"] / N ** 2,
                                    N)
                assert got["n"] == ref["n"] and got["n_alive"] == ref["n_alive"]
                if r.beta_eps == 0.0:
                    # log W from the exact counts in FP64: sums of non-negative
                    # terms, within 4 n 2^-53 relative.
                    tol = 4.0 * C * 2.0 ** -53
                    for key in ("mean_r2", "mean_rg2", "ess"):
                        assert abs(got[key] - ref[key]) <= tol * abs(ref[key]), (kind, key)
                    assert abs(got["logZ"] - ref["logZ"]) <= tol * max(1.0, abs(ref["logZ"]))
                else:
                    # FP32 log W: (N-1)(1e-6 + 6e-8 |log W|) per chain.
                    lwmax = np.abs(o["logw"][o["alive"] == 1]).max()
                    dlw = (N - 1) * (1e-6 + 6e-8 * lwmax)
                    assert abs(got["logZ"] - ref["logZ"]) <= dlw, kind
                    for key in ("mean_r2", "mean_rg2"):
                        assert abs(got[key] - ref[key]) <= 4 * dlw * abs(ref[key]), (kind, key)
            else:
                pot = oracle.LJ if r.potential == rosen.ROSEN_LJ else oracle.HARD_SPHERE
                o = oracle.offlattice_run(r.seed, N, C, r.k, potential=pot, beta_eps=r.beta_eps,
                                          ensemble=r.ensemble, coords=True)
                # A chain on the oracle's path carries only the FP32 drift;
                # any other path differs by O(1) somewhere.
                alive = o["alive"] == 1
                d = np.abs(xyz.astype(np.float64) - o["coords"]).reshape(C, -1).max(1)
                same = d <= (N - 1) * 4e-7 + 1e-6
                assert same.mean() >= 0.999, (kind, same.mean())
                ref = oracle.reduce(o["logw"], o["r2"], o["rg2"], N, r.k)
                assert got["n"] == ref["n"]
                assert abs(got["n_alive"] - ref["n_alive"]) <= 0.001 * C
                for key, se in (("mean_r2", "se_r2"), ("mean_rg2", "se_rg2")):
                    dd = abs(got[key] - ref[key])
                    assert dd <= 1e-3 * abs(ref[key]) and dd <= 3 * ref[se] + 1e-12, (kind, key)
                assert abs(got["logZ"] - ref["logZ"]) <= 1e-3 * max(1.0, abs(ref["logZ"]))
                assert alive.any()
        for t in tickets:
            assert srv.release(t) == rosen.ROSEN_OK
    finally:
        srv.close()


def test_time_slices_let_a_small_request_pass_a_large_one(rosen):
    # A large request is grown in slices of a few milliseconds; with the
    # shortest-remaining-work policy a small request submitted while it runs
    # gets the next slice and finishes first.  Both results equal those of
    # the requests served alone, bit for bit.
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    big = rosen.request(R, 64, 2_000_000, 31, 0, k=32)
    small = rosen.request(L, 32, 1000, 32, 1, beta_eps=0.2)
    srv = rosen.RosenServer(mem_budget_bytes=4 << 30, max_slots=8, shortest_first=True)
    try:
        alone = {}
        for name, r in (("big", big), ("small", small)):
            st, res = srv.wait(srv.submit(r), 120)
            assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK
            alone[name] = res["stats"]
        tb = srv.submit(big)
        deadline = time.time() + 10
        while srv.info()["running"] < 1 and time.time() < deadline:
            time.sleep(0.0005)
        time.sleep(0.01)                    # the large request is on the GPU
        ts = srv.submit(small)
        st_s, rs = srv.wait(ts, 120)
        st_b, rb = srv.wait(tb, 120)
        assert st_s == st_b == rosen.ROSEN_OK
        assert rs["stats"] == alone["small"] and rb["stats"] == alone["big"]
        assert rs["t_done_ns"] < rb["t_done_ns"]
        # The small request waited about a slice or two, not the large one's time.
        assert rs["t_done_ns"] - rs["t_submit_ns"] < 0.5 * (rb["t_done_ns"] - rb["t_admit_ns"])
    finally:
        srv.close()


def test_admission_passes_a_request_that_does_not_fit(rosen):
    # A request that does not fit the budget next to a running one may be
    # passed by a later request that does fit; it is admitted once memory
    # frees up.
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    a = rosen.request(R, 256, 20_000, 41, 0, k=32, potential=rosen.ROSEN_LJ, beta_eps=0.5,
                      store_coords=True)                       # ~62 MB, tens of ms
    b = rosen.request(L, 128, 60_000, 42, 1, store_coords=True)   # ~94 MB
    c = rosen.request(L, 32, 1000, 43, 2)                          # < 1 MB
    srv = rosen.RosenServer(mem_budget_bytes=140 << 20, max_slots=8)   # 146.8 MB
    try:
        ta = srv.submit(a)
        deadline = time.time() + 10
        while srv.info()["running"] < 1 and time.time() < deadline:
            time.sleep(0.0005)
        tb = srv.submit(b)
        tc = srv.submit(c)
        res = {}
        # c fits next to a and is served while b waits; a's conformations
        # stay reserved until it is released, and only then does b fit.
        for name, t in (("c", tc), ("a", ta)):
            st, r = srv.wait(t, 120)
            assert st == rosen.ROSEN_OK and r["status"] == rosen.ROSEN_OK, r
            res[name] = r
        assert srv.poll(tb)[0] == rosen.ROSEN_EAGAIN
        srv.release(ta)
        st, r = srv.wait(tb, 120)
        assert st == rosen.ROSEN_OK and r["status"] == rosen.ROSEN_OK, r
        res["b"] = r
        assert res["c"]["t_admit_ns"] < res["b"]["t_admit_ns"]     # c passed b
        assert res["b"]["t_admit_ns"] >= res["a"]["t_done_ns"]
        for t in (tb, tc):
            srv.release(t)
        time.sleep(0.05)
        assert srv.info()["bytes_in_use"] == 0
    finally:
        srv.close()


def test_pool_failure_returns_the_reservation(rosen):
    # The server's pool is capped below what a request needs while the budget
    # admits it: its allocation fails on the host (ROSEN_ENOMEM, no GPU work),
    # its reservation goes back to the budget, and later requests still run.
    L = rosen.ROSEN_MODEL_LATTICE
    srv = rosen.RosenServer(mem_budget_bytes=1 << 30, max_slots=4, pool_max_bytes=32 << 20)
    try:
        big = rosen.request(L, 64, 100, 51, 0, store_coords=True)
        big.C = 200_000                     # 12 B x 64 x 2e5 = 154 MB of conformations
        for _ in range(3):
            st, res = srv.wait(srv.submit(big), 60)
            assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_ENOMEM, res
        info = srv.info()
        assert info["failed"] == 3 and info["bytes_in_use"] == 0
        small = rosen.request(L, 32, 2000, 52, 1)
        st, res = srv.wait(srv.submit(small), 60)
        assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK
        assert srv.info()["bytes_in_use"] == 0
    finally:
        srv.close()


def test_sliced_requests_equal_the_single_ensemble_path(rosen):
    # Requests large enough for several slices (chain ranges on two streams
    # per request) equal the single-ensemble entry points bit for bit:
    # lattice in restart mode (the retry kernel over ranges that start above
    # chain 0), two-pass hard spheres (the deferral mask shared by the
    # slices), and real space in restart mode.
    L, R = rosen.ROSEN_MODEL_LATTICE, rosen.ROSEN_MODEL_OFFLATTICE
    cases = [
        rosen.request(L, 64, 12_000_000, 61, 0, beta_eps=0.3, max_attempts=8),
        rosen.request(R, 64, 1_500_000, 62, 1, k=32),
        rosen.request(R, 48, 600_000, 63, 2, k=16, sigma=1.2, max_attempts=4),
    ]
    srv = rosen.RosenServer(mem_budget_bytes=8 << 30, max_slots=4)
    try:
        tickets = [srv.submit(r) for r in cases]
        got = []
        for t in tickets:
            st, res = srv.wait(t, 300)
            assert st == rosen.ROSEN_OK and res["status"] == rosen.ROSEN_OK, res
            got.append(res["stats"])
    finally:
        srv.close()
    for r, g in zip(cases, got):
        st = rosen.stats_tensor()
        ws = rosen.reduce_workspace(r.C)
        if r.model == L:
            out = rosen.lattice_outputs(r.N, r.C, attempts=True)
            rosen.rosen_lattice_grow(rosen.lattice_params(r.seed, r.N, r.C, beta_eps=r.beta_eps,
                                                          ensemble=r.ensemble,
                                                          max_attempts=r.max_attempts), out)
            rosen.rosen_reduce(rosen.lattice_reduce_in(out, r.N, 0), st, ws)
        else:
            out = rosen.offlattice_outputs(r.N, r.C, attempts=r.max_attempts > 1)
            rosen.rosen_offlattice_grow(
                rosen.offlattice_params(r.seed, r.N, r.C, r.k, potential=r.potential,
                                        sigma=r.sigma, ensemble=r.ensemble,
                                        max_attempts=r.max_attempts), out)
            rosen.rosen_reduce(rosen.offlattice_reduce_in(out, r.N, r.k), st, ws)
        ref = rosen.stats_dict(st)
        for key in rosen.STAT_KEYS:
            assert g[key] == ref[key] or (np.isnan(g[key]) and np.isnan(ref[key])), (r.N, key)
        del out
        torch.cuda.empty_cache()
