"""Pins for the scaling fits (Section 5.1, Eq. 7-10) on the host.

The fits are plain weighted least squares. They are pinned by:
- exact recovery of known exponents from noise-free power laws;
- agreement with numpy's polyfit and scipy's curve_fit (library routines);
- Monte Carlo calibration of the reported errors;
- the error of log Z-hat checked against the spread of independent oracle
  ensembles;
- the exact SAW counts of the enumeration.
"""
import os

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_1704_04381_gb300 import scaling

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table4.txt")


def table4():
    vals = {}
    for line in open(GOLDEN):
        f = line.split("#")[0].split()
        if f:
            vals[f[0]] = [float(x) for x in f[1:]]
    return vals


def test_golden_table_is_the_papers():
    t = table4()
    assert t["mu"] == [4.684, 4.6856, 0.0001]
    assert t["gamma"][1] == 1.1592 and t["nu"][1] == 0.5880


def test_exact_power_laws_are_recovered():
    n = np.array(scaling.lengths(8, 511, 14), dtype=np.float64)
    logz = n * np.log(4.684) + 0.1608 * np.log(n) + 0.31
    r = scaling.fit_mu_gamma(n, logz, np.full(len(n), 1e-3))
    assert abs(r["mu"] - 4.684) < 1e-10 and abs(r["gamma"] - 1.1608) < 1e-9
    assert abs(r["c"] - 0.31) < 1e-8 and r["chi2_dof"] < 1e-12
    r2 = 1.37 * n ** (2 * 0.5877)
    f = scaling.fit_nu(n, r2, 0.01 * r2)
    assert abs(f["nu"] - 0.5877) < 1e-12 and abs(f["a"] - 1.37) < 1e-10


def test_corrected_fit_recovers_exponent_and_amplitude():
    n = np.array(scaling.lengths(8, 511, 14), dtype=np.float64)
    r2 = 1.25 * n ** (2 * 0.5877) * (1 - 0.4 * n ** -0.528)
    f = scaling.fit_nu_corrected(n, r2, 1e-3 * r2)
    assert abs(f["nu"] - 0.5877) < 1e-7 and abs(f["b"] + 0.4) < 1e-5, f
    # The bare power law is biased on the same data; the corrected fit is not.
    assert abs(scaling.fit_nu(n, r2, 1e-3 * r2)["nu"] - 0.5877) > 5e-3
    # With noise: agrees with scipy's curve_fit on the full nonlinear model.
    rng = np.random.default_rng(5)
    se = 2e-3 * r2
    y = r2 + rng.normal(0, se)
    f = scaling.fit_nu_corrected(n, y, se)
    p, cov = optimize.curve_fit(lambda x, a, nu, b: a * x ** (2 * nu) * (1 + b * x ** -0.528),
                                n, y, p0=[1.2, 0.59, -0.3], sigma=se, absolute_sigma=True)
    assert abs(f["nu"] - p[1]) < 1e-6
    infl = max(1.0, f["chi2_dof"]) ** 0.5
    assert abs(f["nu_se"] - np.sqrt(cov[1, 1]) * infl) < 0.02 * f["nu_se"]


def test_fits_agree_with_library_routines():
    rng = np.random.default_rng(3)
    n = np.array(scaling.lengths(8, 511, 12), dtype=np.float64)
    se = 0.002 + 0.0004 * np.sqrt(n)
    logz = n * np.log(4.68) + 0.17 * np.log(n) + 0.2 + rng.normal(0, se)
    r = scaling.fit_mu_gamma(n, logz, se)
    p, cov = optimize.curve_fit(lambda x, a, b, c: a * x + b * np.log(x) + c, n, logz,
                                sigma=se, absolute_sigma=True)
    # curve_fit iterates (Levenberg-Marquardt) to about 1e-7; a wrong weight or
    # a dropped term would move gamma by ~1e-2.
    assert abs(r["mu"] - np.exp(p[0])) < 1e-7 * r["mu"]
    assert abs(r["gamma"] - (p[1] + 1)) < 1e-6
    infl = max(1.0, r["chi2_dof"]) ** 0.5
    assert abs(r["gamma_se"] - np.sqrt(cov[1, 1]) * infl) < 1e-4 * r["gamma_se"]
    r2 = 1.2 * n ** 1.18 * np.exp(rng.normal(0, 0.003, len(n)))
    f = scaling.fit_nu(n, r2, 0.003 * r2)
    slope, _ = np.polyfit(np.log(n), np.log(r2), 1, w=np.full(len(n), 1 / 0.003))
    assert abs(f["nu"] - slope / 2) < 1e-10


def test_reported_errors_are_calibrated():
    # Repeat a noisy fit many times: the spread of the estimates matches the
    # reported standard errors, and the estimates are unbiased.
    rng = np.random.default_rng(11)
    n = np.array(scaling.lengths(16, 511, 10), dtype=np.float64)
    se = 0.003 * np.sqrt(n / 16)
    truth = n * np.log(4.684) + 0.16 * np.log(n) - 0.1
    mus, gams, se_mu, se_g = [], [], [], []
    for _ in range(2000):
        r = scaling.fit_mu_gamma(n, truth + rng.normal(0, se), se)
        mus.append(r["mu"]); gams.append(r["gamma"])
        se_mu.append(r["mu_se"] / max(1.0, r["chi2_dof"]) ** 0.5)
        se_g.append(r["gamma_se"] / max(1.0, r["chi2_dof"]) ** 0.5)
    assert abs(np.std(mus) / np.mean(se_mu) - 1) < 0.08
    assert abs(np.std(gams) / np.mean(se_g) - 1) < 0.08
    assert abs(np.mean(gams) - 1.16) < 4 * np.std(gams) / np.sqrt(len(gams))


def test_log_z_error_matches_the_spread_of_independent_ensembles():
    # 150 oracle ensembles of 2000 athermal chains at N = 40: the standard
    # deviation of log Z-hat across them agrees with the per-ensemble error.
    N, C, E = 40, 2000, 150
    o = oracle.lattice_run(5, N, C * E)
    lz, se = [], []
    for e in range(E):
        s = slice(e * C, (e + 1) * C)
        st = oracle.reduce(o["logw"][s], o["r2"][s].astype(np.float64),
                           o["n2rg2"][s] / N ** 2, N)
        lz.append(st["logZ"])
        se.append(scaling.log_z_se(st))
    ratio = np.std(lz, ddof=1) / np.mean(se)
    assert 0.8 < ratio < 1.2, ratio


def test_fit_of_exact_walk_counts():
    # c_n for n <= 10 from the exact enumeration: even at these short lengths
    # the three-parameter fit of Eq. 10 lands near the connective constant.
    cnt, _, _ = oracle.enumerate_saw(10)
    n = np.arange(4, 11)
    logc = np.log([cnt[k].sum() for k in n])
    r = scaling.fit_mu_gamma(n, logc, np.full(len(n), 1e-3))
    assert abs(r["mu"] - table4()["mu"][0]) < 0.08, r
    assert 1.0 < r["gamma"] < 1.4, r
