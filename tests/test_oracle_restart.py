"""Pins for restart mode in the oracle (Sections 3.3.2 and 3.3.3).

The paper throws a trapped chain away and grows it again from the first
monomer.  Attempt a of chain c draws from the step word i + 2^16 a, so
attempt 0 is the plain stream.  Every attempt is an independent Rosenbluth
growth.  The mean weight over all attempts, counting the discarded ones as 0,
therefore estimates Z, using Eq. 9 with the number of growths started.  The
surviving chains are ordinary Rosenbluth samples.

The trimer fixes all of this in closed form.  For hard spheres of diameter
sigma and bond length 1 at N = 3:
- The end overlaps bead 0 iff 2 + 2c < sigma^2, where c = cos of the bond
  angle is uniform on [-1, 1].
- One trial is therefore free with probability p = 1 - sigma^2/4.
- All k trials of step 2 overlap with probability q = (1 - p)^k.
- The number of attempts a made under a cap A is geometric, truncated at A:
  P(a = j) = q^(j-1)(1 - q) for j < A, and P(a = A) = q^(A-1).
- E[W / k^2] = p per attempt.
- <R^2> = E[2 + 2c | c >= sigma^2/2 - 1] = 2 + sigma^2/2.
"""
import numpy as np
from scipy import stats

import oracle

Z_SIGMAS = 4.5

# Number of 12-step self-avoiding walks on the simple cubic lattice (series
# A001412 of the OEIS; Fisher & Sykes, Phys. Rev. 114 (1959) 45).
CUBIC_SAW_C12 = 198842742


def test_trimer_attempt_law_weight_and_size():
    sigma, k, A, C = 1.8, 2, 4, 60_000
    p = 1.0 - sigma ** 2 / 4.0
    q = (1.0 - p) ** k
    o = oracle.offlattice_run(11, 3, C, k, sigma=sigma, max_attempts=A)
    a = o["attempts"].astype(np.int64)
    assert a.min() >= 1 and a.max() <= A

    # Attempts: geometric law truncated at A (chi-square, 3 degrees of freedom).
    expect = np.array([q ** (j - 1) * (1 - q) for j in range(1, A)] + [q ** (A - 1)]) * C
    seen = np.bincount(a, minlength=A + 1)[1:]
    chi2 = ((seen - expect) ** 2 / expect).sum()
    assert stats.chi2.sf(chi2, A - 1) > 1e-4, (seen, expect)

    # A chain is alive iff its last attempt survived; only a = A can be dead.
    alive = o["alive"].astype(bool)
    assert alive[a < A].all()
    frac, p_alive = alive.mean(), 1.0 - q ** A
    assert abs(frac - p_alive) < Z_SIGMAS * np.sqrt(p_alive * (1 - p_alive) / C)

    # Eq. 9 over the attempts: sum W / sum a estimates E[W] = p k^2 per growth.
    wn = np.where(alive, np.exp(o["logw"] - 2 * np.log(k)), 0.0)
    R = wn.sum() / a.sum()
    se = np.sqrt(((wn - R * a) ** 2).sum()) / a.sum()
    assert abs(R - p) < Z_SIGMAS * se, (R, p, se)
    # The per-chain mean instead (dead attempts not counted) is biased upwards:
    # E[W | survived] / E[a] differs from p by far more than the error here.
    assert wn.sum() / C > p + 10 * se

    # The oracle's reduction with n = the number of attempts gives the same.
    st = oracle.reduce(o["logw"], o["r2"], o["rg2"], 3, k=k, n=a.sum())
    assert st["n"] == a.sum()
    assert abs(np.exp(st["logZ_norm"]) - R) < 1e-12 * R

    # Size of the survivors: 2 + sigma^2 / 2.
    w = wn[alive]
    r2 = o["r2"][alive]
    S = w.sum()
    mean = (w * r2).sum() / S
    se_r = np.sqrt((w ** 2 * (r2 - mean) ** 2).sum()) / S
    assert abs(mean - (2 + sigma ** 2 / 2)) < Z_SIGMAS * se_r, mean
    assert abs(st["mean_r2"] - mean) < 1e-12 * mean


def test_single_attempt_is_the_plain_run():
    plain = oracle.offlattice_run(12, 3, 5000, 2, sigma=1.8)
    one = oracle.offlattice_run(12, 3, 5000, 2, sigma=1.8, max_attempts=1)
    for key in ("logw", "r2", "rg2", "alive"):
        np.testing.assert_array_equal(plain[key], one[key])
    assert (one["attempts"] == 1).all()


def test_lattice_restart_continues_the_plain_stream():
    # Attempt 0 of restart mode is the plain run: the chains that survive it
    # are untouched, and exactly the chains the plain run loses are regrown.
    N, C = 64, 40_000
    plain = oracle.lattice_run(21, N, C, beta_eps=0.2, trace=True, coords=True)
    rs = oracle.lattice_run(21, N, C, beta_eps=0.2, trace=True, coords=True, max_attempts=16)
    first = plain["alive"].astype(bool)
    assert 0 < (~first).sum() < C // 20
    np.testing.assert_array_equal(rs["attempts"] == 1, first)
    for key in ("counts", "logw", "r2", "n2rg2", "trace", "coords"):
        np.testing.assert_array_equal(rs[key][first], plain[key][first])
    # A trapped attempt has probability < 1%, so sixteen in a row never happen.
    assert rs["alive"].all()
    # Regrown chains are self-avoiding walks with consistent outputs.
    re = np.flatnonzero(~first)
    pos = rs["coords"][re].astype(np.int64)                    # [R, N, 3]
    steps = np.diff(pos, axis=1)
    assert (np.abs(steps).sum(-1) == 1).all()
    keys = pos[..., 0] * 10 ** 6 + pos[..., 1] * 10 ** 3 + pos[..., 2]
    assert all(len(np.unique(kk)) == N for kk in keys)
    np.testing.assert_array_equal(rs["r2"][re], (pos[:, -1] ** 2).sum(-1))
    g2 = N * (pos ** 2).sum((1, 2)) - (pos.sum(1) ** 2).sum(-1)
    np.testing.assert_array_equal(rs["n2rg2"][re], g2)
    cnt = rs["counts"][re].astype(np.int64)
    assert (cnt[:, 0] == 0).all() and (cnt[:, 1:7].sum(1) == N - 1).all()
    tr = rs["trace"][re].astype(np.int64)
    np.testing.assert_array_equal(cnt[:, 1:7],
                                  np.stack([(tr >> 3 == m).sum(1) for m in range(1, 7)], 1))


def test_lattice_restart_estimates_the_walk_count():
    # Eq. 9 over all attempts at n = 12 steps: sum W / sum a -> c_12.
    N, C = 13, 200_000
    o = oracle.lattice_run(22, N, C, max_attempts=8)
    a = o["attempts"].astype(np.float64)
    w = np.where(o["alive"].astype(bool), np.exp(o["logw"]), 0.0)
    R = w.sum() / a.sum()
    se = np.sqrt(((w - R * a) ** 2).sum()) / a.sum()
    assert abs(R - CUBIC_SAW_C12) < Z_SIGMAS * se, (R, CUBIC_SAW_C12, se)
