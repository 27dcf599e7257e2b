"""Pins for the oracle's PERM (pruned-enriched Rosenbluth growth, breadth
first; Grassberger, Phys. Rev. E 56, 3682 (1997)).

Enrichment (two copies sharing the weight) and pruning (removal with
probability 1/2, the survivor's weight doubled) keep the expected total
weight of every length, so the mean over independent populations of Eq. 9's
estimate (1/M0) sum W is the exact number of walks c_n (athermal) or the
exact partition function Z_n(beta eps) (interacting SAW).  Checked here:
- without thresholds the method is plain Rosenbluth growth: the same chains
  as orc_lattice_run, bit for bit (no dead end happens before 11 steps);
- with pruning and enrichment both active (and with the population cap
  binding), the mean estimate equals the exact c_n for n <= 12 (published
  c_11, c_12 beyond the enumeration) and the exact Z_n(0.4) for n <= 10;
- the W-weighted <R^2>_n pooled over populations equals the exact walk
  average;
- the fates follow the thresholds: no final weight exceeds c_hi mu^n when
  the cap does not bind (a reversed comparison would break this), and the
  population actually grows and shrinks.
"""
import math

import numpy as np
import pytest

import oracle

Z_SIGMAS = 4.5
C11, C12 = 41934150, 198842742       # published cubic SAW counts


@pytest.fixture(scope="module")
def enum10():
    return oracle.enumerate_saw(10)


def log_weights(o):
    return np.log(o["w_m"]) + o["w_e"] * math.log(2.0)


@pytest.mark.parametrize("beta_eps", [0.0, 0.3])
def test_without_thresholds_it_is_plain_rosenbluth(beta_eps):
    N, C = 11, 2000
    p = oracle.perm_run(3, N, C, C, beta_eps=beta_eps, c_hi=math.inf, c_lo=0.0, positions=True)
    ref = oracle.lattice_run(3, N, C, beta_eps=beta_eps, coords=True)
    assert (p["pop"] == C).all() and p["n"] == C
    assert np.array_equal(p["pos"].astype(np.float64), ref["coords"])
    # W as a product of the step factors vs log W as a sum of logs.
    assert np.abs(log_weights(p) - ref["logw"]).max() < 1e-12
    whole = math.log(np.exp(ref["logw"]).mean())
    assert abs(p["logz"][N - 1] - whole) < 1e-12


def population_runs(runs, N, M0, max_pop, beta_eps, mu, c_hi, c_lo):
    z, pops, r2 = [], [], []
    for s in range(runs):
        o = oracle.perm_run(1000 + s, N, M0, max_pop, beta_eps=beta_eps, mu=mu, c_hi=c_hi,
                            c_lo=c_lo)
        z.append(np.exp(o["logz"]))
        pops.append(o["pop"])
        r2.append(o["r2"])
    return np.array(z), np.array(pops), np.array(r2)


def assert_unbiased(z, exact, label):
    for n, zn in exact.items():
        col = z[:, n]
        se = col.std(ddof=1) / math.sqrt(len(col))
        assert abs(col.mean() - zn) <= Z_SIGMAS * se + 1e-9 * zn, (label, n, col.mean(), zn, se)


def test_athermal_counts_are_unbiased_with_pruning_and_enrichment(enum10):
    cnt, _, _ = enum10
    N = 13                                   # up to n = 12 steps
    z, pops, _ = population_runs(400, N, 200, 800, 0.0, 4.684, 1.3, 0.6)
    # Both operations happened: the population grew (enrichment) and shrank
    # from one step to the next (pruning).
    assert pops.max() > 200 and (np.diff(pops, axis=1) < 0).any()
    exact = {n: float(cnt[n].sum()) for n in range(1, 11)}
    exact[11], exact[12] = float(C11), float(C12)
    assert_unbiased(z, exact, "athermal")


def test_the_population_cap_binds_and_stays_unbiased(enum10):
    cnt, _, _ = enum10
    N, M0 = 11, 150
    z, pops, _ = population_runs(400, N, M0, M0, 0.0, 4.684, 1.1, 0.6)
    assert pops.max() == M0                  # enrichment was denied at the cap
    assert_unbiased(z, {n: float(cnt[n].sum()) for n in range(1, 11)}, "cap")


def test_interacting_partition_function_is_unbiased(enum10):
    cnt, _, _ = enum10
    beta_eps = 0.4
    c = np.arange(cnt.shape[1])
    exact = {n: float((cnt[n] * np.exp(beta_eps * c)).sum()) for n in range(1, 11)}
    z, pops, _ = population_runs(400, 11, 200, 800, beta_eps, 5.3, 1.3, 0.6)
    assert pops.max() > 200 and (np.diff(pops, axis=1) < 0).any()
    assert_unbiased(z, exact, "isaw")


def test_weighted_r2_matches_the_exact_walk_average(enum10):
    cnt, sr2, _ = enum10
    z, _, r2 = population_runs(400, 11, 300, 1200, 0.0, 4.684, 1.3, 0.6)
    for n in (4, 7, 10):
        exact = sr2[n].sum() / cnt[n].sum()
        w = z[:, n]
        pooled = (w * r2[:, n]).sum() / w.sum()
        # Jackknife over the independent populations.
        jk = np.array([np.delete(w * r2[:, n], q).sum() / np.delete(w, q).sum()
                       for q in range(len(w))])
        se = math.sqrt((len(w) - 1) * ((jk - jk.mean()) ** 2).mean())
        assert abs(pooled - exact) <= Z_SIGMAS * se, (n, pooled, exact, se)


def test_final_weights_respect_the_enrichment_threshold():
    # With mu > 3 and c_lo <= c_hi / 2, every weight after a step's fates is
    # at most c_hi mu^i: kept chains lie below the threshold, enriched copies
    # carry half a weight of at most 6 c_hi mu^(i-1), pruning survivors
    # twice a weight below c_lo mu^i.
    N, mu, c_hi, c_lo = 40, 4.684, 1.3, 0.6
    o = oracle.perm_run(5, N, 2000, 10 ** 6, mu=mu, c_hi=c_hi, c_lo=c_lo)
    assert o["n"] > 0
    lw = log_weights(o)
    assert lw.max() <= math.log(c_hi) + (N - 1) * math.log(mu) + 1e-12
    # Plain Rosenbluth weights spread far wider than PERM's.
    plain = oracle.lattice_run(5, N, 2000)["logw"]
    plain = plain[np.isfinite(plain)]
    assert np.ptp(lw) < 0.5 * np.ptp(plain)
