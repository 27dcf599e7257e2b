"""Pins for the oracle's ensemble reduction (Eq. 2 with W as importance weight, Eq. 9).

Athermal lattice weights are exact integers W = prod_m m^counts[m], so every
sum the reduction forms can be computed exactly with Python integers and
fractions; the FP64 log-sum-exp result must agree to rounding.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lattice16():
    return oracle.lattice_run(1, 16, 20_000)


def exact_stats(counts, r2, n2rg2, N):
    W = [0 if c[0] else (2 ** int(c[2]) * 3 ** int(c[3]) * 4 ** int(c[4]) * 5 ** int(c[5])
                        * 6 ** int(c[6])) for c in counts]
    A = [Fraction(int(a)) for a in r2]
    B = [Fraction(int(b), N * N) for b in n2rg2]
    S0 = sum(W)
    S1 = sum(w * a for w, a in zip(W, A))
    S2 = sum(w * b for w, b in zip(W, B))
    m1, m2 = S1 / S0, S2 / S0
    v1 = sum(w * w * (a - m1) ** 2 for w, a in zip(W, A))
    v2 = sum(w * w * (b - m2) ** 2 for w, b in zip(W, B))
    Q0 = sum(w * w for w in W)
    return {
        "logZ": math.log(S0) - math.log(len(W)),
        "mean_r2": float(m1), "mean_rg2": float(m2),
        "se_r2": math.sqrt(float(v1)) / float(S0),
        "se_rg2": math.sqrt(float(v2)) / float(S0),
        "ess": float(Fraction(S0 * S0, Q0)),
        "n_alive": sum(1 for w in W if w > 0),
    }


def test_reduce_matches_exact_rational_sums(lattice16):
    o = lattice16
    N = 16
    st = oracle.reduce(o["logw"], o["r2"], o["n2rg2"] / float(N * N), N)
    ex = exact_stats(o["counts"], o["r2"], o["n2rg2"], N)
    assert st["n"] == len(o["logw"]) and st["n_alive"] == ex["n_alive"]
    for key in ("mean_r2", "mean_rg2", "se_r2", "se_rg2", "ess"):
        assert st[key] == pytest.approx(ex[key], rel=1e-12), key
    assert st["logZ"] == pytest.approx(ex["logZ"], rel=0, abs=1e-11)


def test_reduce_counts_dead_chains_in_z():
    # Eq. 9 averages W over every generated chain: a dead chain (W = 0) lowers Z
    # but leaves ratio means unchanged.
    lw = np.array([0.0, np.log(3.0), -np.inf, np.log(2.0)])
    a = np.array([1.0, 2.0, 123.0, 4.0])
    st = oracle.reduce(lw, a, a, 5)
    assert st["n_alive"] == 3
    assert st["logZ"] == pytest.approx(math.log(6.0 / 4.0), abs=1e-15)
    assert st["mean_r2"] == pytest.approx((1 + 6 + 8) / 6.0, rel=1e-15)
    assert st["ess"] == pytest.approx(36.0 / 14.0, rel=1e-15)


def test_reduce_is_shift_invariant_over_huge_range():
    # Weights spanning hundreds of orders of magnitude: log-sum-exp keeps them.
    rng = np.random.default_rng(3)
    lw = rng.uniform(500, 900, size=1000)
    a = rng.uniform(0, 10, size=1000)
    st = oracle.reduce(lw, a, a, 64)
    st2 = oracle.reduce(lw - 700.0, a, a, 64)
    assert st["logZ"] - st2["logZ"] == pytest.approx(700.0, abs=1e-9)
    assert st["mean_r2"] == pytest.approx(st2["mean_r2"], rel=1e-14)
    top = np.argmax(lw)
    w = np.exp(lw - lw[top])
    assert st["mean_r2"] == pytest.approx((w * a).sum() / w.sum(), rel=1e-12)


def test_reduce_all_dead():
    st = oracle.reduce(np.full(4, -np.inf), np.zeros(4), np.zeros(4), 8)
    assert st["n_alive"] == 0 and st["logZ"] == -math.inf and st["ess"] == 0.0
    assert math.isnan(st["mean_r2"])


def test_logz_norm_uses_trials_per_step():
    lw = np.full(10, 7.0)
    st = oracle.reduce(lw, np.ones(10), np.ones(10), N=5, k=4)
    assert st["logZ_norm"] == pytest.approx(7.0 - 4 * math.log(4.0), abs=1e-14)
