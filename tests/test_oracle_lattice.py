"""Pins for the cubic-lattice oracle (Algorithm 1 with the weight of Eq. 3).

The Rosenbluth weight is an unbiased estimator of the number of walks
(athermal) or of the partition function sum_walks exp(beta_eps * contacts)
(interacting SAW), and W-weighted means are ratio estimators of the exact
walk averages (Eq. 2).  Exact enumeration fixes all of them for n <= 10.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle

DIRS = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                dtype=np.int64)
Z_SIGMAS = 4.5


@pytest.fixture(scope="module")
def enum10():
    return oracle.enumerate_saw(10)


@pytest.fixture(scope="module")
def athermal16():
    # Lattice athermal SAW, N = 16 monomers, 100,000 chains, seed 1.
    return oracle.lattice_run(1, 16, 100_000, beta_eps=0.0, trace=True, coords=True)


def prefix_walks(trace):
    """Per-step factors m_i and positions r_i of every chain, decoded from its trace."""
    t = trace.astype(np.int64)
    m = t >> 3
    d = t & 7
    steps = DIRS[np.minimum(d, 5)]
    pos = np.cumsum(steps, axis=1)
    return m, pos


def ratio_mean_se(w, a):
    """W-weighted mean of a and the standard error of that ratio estimator."""
    S = w.sum()
    mean = (w * a).sum() / S
    se = np.sqrt((w ** 2 * (a - mean) ** 2).sum()) / S
    return mean, se


def test_mean_prefix_weight_is_exact_walk_count(athermal16, enum10):
    cnt, sr2, _ = enum10
    m, pos = prefix_walks(athermal16["trace"])
    assert (m[:, :10] > 0).all(), "no cubic SAW is trapped before 11 steps"
    W = np.cumprod(m.astype(np.float64), axis=1)
    for n in range(1, 11):
        w = W[:, n - 1]
        c_n = cnt[n].sum()
        se = w.std(ddof=1) / np.sqrt(len(w))
        if se == 0:
            assert w.mean() == c_n
        else:
            assert abs(w.mean() - c_n) < Z_SIGMAS * se, (n, w.mean(), c_n, se)
        r2 = (pos[:, n - 1] ** 2).sum(1).astype(np.float64)
        mean, se_r = ratio_mean_se(w, r2)
        exact = sr2[n].sum() / c_n
        assert abs(mean - exact) < Z_SIGMAS * se_r + 1e-12, (n, mean, exact, se_r)


def test_radius_of_gyration_matches_enumeration(enum10):
    cnt, _, sg2 = enum10
    n = 10
    o = oracle.lattice_run(11, n + 1, 100_000, beta_eps=0.0)
    w = np.exp(oracle.lattice_logw_from_counts(o["counts"]))
    rg2 = o["n2rg2"] / float((n + 1) ** 2)
    mean, se = ratio_mean_se(w, rg2)
    exact = sg2[n].sum() / cnt[n].sum() / (n + 1) ** 2
    assert abs(mean - exact) < Z_SIGMAS * se


@pytest.mark.parametrize("beta_eps", [0.2, 0.4])
def test_isaw_weight_is_partition_function(enum10, beta_eps):
    cnt, sr2, sg2 = enum10
    n = 8
    o = oracle.lattice_run(2, n + 1, 200_000, beta_eps=beta_eps)
    w = np.exp(o["logw"])
    c = np.arange(cnt.shape[1])
    boltz = np.exp(beta_eps * c)
    Z = (cnt[n] * boltz).sum()
    se = w.std(ddof=1) / np.sqrt(len(w))
    assert abs(w.mean() - Z) < Z_SIGMAS * se, (w.mean(), Z, se)
    exact_r2 = (sr2[n] * boltz).sum() / Z
    mean, se_r = ratio_mean_se(w, o["r2"].astype(np.float64))
    assert abs(mean - exact_r2) < Z_SIGMAS * se_r
    exact_g2 = (sg2[n] * boltz).sum() / Z / (n + 1) ** 2
    mean, se_g = ratio_mean_se(w, o["n2rg2"] / float((n + 1) ** 2))
    assert abs(mean - exact_g2) < Z_SIGMAS * se_g


def test_athermal_logw_equals_factor_counts(athermal16):
    lw = oracle.lattice_logw_from_counts(athermal16["counts"])
    alive = athermal16["alive"].astype(bool)
    np.testing.assert_allclose(athermal16["logw"][alive], lw[alive], rtol=0, atol=1e-12)
    assert (athermal16["counts"][alive, 1:7].sum(1) == 15).all()
    assert (athermal16["counts"][alive, 6] >= 1).all()   # the first step has 6 options


def test_lattice_invariants(athermal16):
    o = athermal16
    alive = o["alive"].astype(bool)
    n = 15
    # Parity: R^2 has the parity of the number of steps.
    assert ((o["r2"][alive] - n) % 2 == 0).all()
    # Weight bounds for survivors: 6 <= W <= 6 * 5^(n-1).
    W = np.exp(o["logw"][alive])
    assert (W >= 6 * (1 - 1e-12)).all() and (W <= 6 * 5 ** (n - 1) * (1 + 1e-12)).all()
    # Coordinates: unit steps, self-avoiding, end matches R^2, Rg from positions.
    xyz = o["coords"][alive].astype(np.int64)
    steps = np.abs(np.diff(xyz, axis=1)).sum(-1)
    assert (steps == 1).all()
    assert ((xyz[:, -1] ** 2).sum(1) == o["r2"][alive]).all()
    g2 = 16 * (xyz ** 2).sum((1, 2)) - (xyz.sum(1) ** 2).sum(1)
    assert (g2 == o["n2rg2"][alive]).all()
    keys = (xyz[..., 0] + 64) * 16384 + (xyz[..., 1] + 64) * 128 + (xyz[..., 2] + 64)
    srt = np.sort(keys, axis=1)
    assert (np.diff(srt, axis=1) > 0).all()
    # Cubic symmetry of the W-weighted end vector.
    w = W / W.sum()
    end = xyz[:, -1].astype(np.float64)
    for a in range(3):
        mean = (w * end[:, a]).sum()
        se = np.sqrt((w ** 2 * (end[:, a] - mean) ** 2).sum())
        assert abs(mean) < Z_SIGMAS * se
    m2 = [(w * end[:, a] ** 2).sum() for a in range(3)]
    assert max(m2) / min(m2) < 1.05


def rosenbluth_tree(n):
    """Exact probability of every step sequence the athermal rule can produce.

    Enumerates the growth tree of Eq. 3: at each step the free neighbours of
    the end are equally likely, so a completed walk has probability 1/W.
    Returns {trace tuple: probability} for walks that survive n steps.
    """
    out = {}

    def rec(path, occ, prob, tr):
        if len(path) - 1 == n:
            out[tuple(tr)] = prob
            return
        end = path[-1]
        free = [d for d in range(6) if tuple(end + DIRS[d]) not in occ]
        for d in free:
            nxt = end + DIRS[d]
            occ.add(tuple(nxt))
            rec(path + [nxt], occ, prob / len(free), tr + [(len(free) << 3) | d])
            occ.remove(tuple(nxt))

    rec([np.zeros(3, np.int64)], {(0, 0, 0)}, 1.0, [])
    return out


def test_path_distribution_is_the_rosenbluth_law():
    n = 4
    law = rosenbluth_tree(n)
    assert abs(sum(law.values()) - 1.0) < 1e-12 and len(law) == 726
    C = 300_000
    o = oracle.lattice_run(7, n + 1, C, trace=True)
    keys = [tuple(r) for r in o["trace"].tolist()]
    uniq, counts = np.unique(np.array(keys, dtype=np.int64), axis=0, return_counts=True)
    seen = {tuple(u.tolist()): c for u, c in zip(uniq, counts)}
    assert set(seen) <= set(law)
    order = sorted(law)
    obs = np.array([seen.get(k, 0) for k in order], dtype=np.float64)
    exp = np.array([law[k] * C for k in order])
    chi2 = stats.chisquare(obs, exp)
    assert chi2.pvalue > 1e-4, chi2


def test_selection_uses_the_documented_draw():
    # Recompute the first step by hand from the Philox draw: all six neighbours
    # are free, so idx = floor(x * 6 / 2^32) is the chosen direction.
    seed, N = 99, 3
    o = oracle.lattice_run(seed, N, 64, trace=True)
    for c in range(64):
        x = oracle.philox4x32_10([c, 0, 1, 0], [seed & 0xFFFFFFFF, seed >> 32])[0]
        assert o["trace"][c, 0] == (6 << 3) | ((int(x) * 6) >> 32)
