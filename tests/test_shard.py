"""Splitting an ensemble over ranks (no GPU needed).

Each rank grows a contiguous chain range.  The ranks exchange only their 18
statistics, which are merged as the reduction merges its tiles.  Checked here:
- The merge of shard statistics equals the reduction of all chains at once.
  The merge is the library's rosen_stats_merge (host code, no GPU); the
  per-shard and whole-ensemble statistics come from the FP64 oracle, so this
  pins the library's merge against the oracle's single reduction.
- Two gloo ranks on CPU gather and merge to the same answer on every rank.
- Timing takes the maximum over ranks.
- The chain ranges tile the ensemble.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1704_04381_gb300 import build as pkg_build
from paper_1704_04381_gb300 import shard


@pytest.fixture(scope="module", autouse=True)
def library():
    # rosen_stats_merge lives in librosen.so (host code; no device needed).
    pkg_build.build()

KEYS = [k for k in shard.STAT_KEYS]


def close(a, b, keys=KEYS):
    for key in keys:
        x, y = a[key], b[key]
        if isinstance(y, float) and math.isnan(y):
            assert math.isnan(x), key
        elif math.isinf(y):
            assert x == y, key
        else:
            assert abs(x - y) <= 1e-12 * max(1.0, abs(y)), (key, x, y)


def test_chain_ranges_tile_the_ensemble():
    for C in (1, 7, 1000, 10 ** 7 + 3):
        for world in (1, 2, 3, 8):
            spans = [shard.chain_range(r, world, C) for r in range(world)]
            assert spans[0][0] == 0
            assert sum(n for _, n in spans) == C
            assert all(spans[r][0] + spans[r][1] == spans[r + 1][0] for r in range(world - 1))


@pytest.mark.parametrize("kind", ["lattice", "offlattice"])
def test_merge_equals_one_reduction(kind):
    N, C = 40, 6000
    if kind == "lattice":
        o = oracle.lattice_run(7, N, C, beta_eps=0.3)
        A1, A2, k = o["r2"].astype(np.float64), o["n2rg2"] / N ** 2, 0
    else:
        o = oracle.offlattice_run(7, N, C, 8, sigma=1.2)
        A1, A2, k = o["r2"], o["rg2"], 8
    whole = oracle.reduce(o["logw"], A1, A2, N, k)
    for world in (2, 3, 5):
        parts = []
        for r in range(world):
            c0, n = shard.chain_range(r, world, C)
            s = slice(c0, c0 + n)
            parts.append(oracle.reduce(o["logw"][s], A1[s], A2[s], N, k))
        close(shard.merge_stats(parts, N, k), whole)


def test_merge_with_an_empty_shard():
    # A shard whose chains all died has log_max = -inf and adds only counts.
    N = 20
    o = oracle.offlattice_run(9, N, 2000, 4, sigma=1.6)
    assert (o["alive"] == 0).any()
    dead = np.flatnonzero(o["alive"] == 0)[:50]
    live = np.flatnonzero(o["alive"] == 1)
    idx = np.concatenate([dead, live])
    lw, a1, a2 = o["logw"][idx], o["r2"][idx], o["rg2"][idx]
    whole = oracle.reduce(lw, a1, a2, N, 4)
    parts = [oracle.reduce(lw[:50], a1[:50], a2[:50], N, 4),
             oracle.reduce(lw[50:], a1[50:], a2[50:], N, 4)]
    assert parts[0]["log_max"] == -math.inf
    close(shard.merge_stats(parts, N, 4), whole)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, N, C, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c0, n = shard.chain_range(rank, world, C)
        o = oracle.lattice_run(3, N, n, beta_eps=0.2, chain0=c0, threads=1)
        st = oracle.reduce(o["logw"], o["r2"].astype(np.float64), o["n2rg2"] / N ** 2, N)
        merged = shard.gather_stats(st, N)
        slowest = shard.max_over_ranks(10.0 * (rank + 1))
        q.put((rank, merged, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_merge():
    N, C, world = 32, 4000, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, N, C, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    o = oracle.lattice_run(3, N, C, beta_eps=0.2)
    whole = oracle.reduce(o["logw"], o["r2"].astype(np.float64), o["n2rg2"] / N ** 2, N)
    for rank, merged, slowest in results:
        close(merged, whole)
        assert slowest == 20.0
