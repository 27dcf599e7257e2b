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
