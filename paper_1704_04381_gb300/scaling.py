"""Scaling analysis of Rosenbluth ensembles (Section 5.1, Eq. 7-10).

From a series of ensembles grown on the GPU at several chain lengths this
module estimates:
- the size exponent nu, by a weighted least-squares fit of
  log <R^2_n> = log a + 2 nu log n (Eq. 7), and by the same law with the
  leading correction to scaling, a n^(2 nu) (1 + b n^-Delta);
- the connective constant mu and the entropic exponent gamma, by a weighted
  least-squares fit of log Z_n = n log mu + (gamma - 1) log n + c (Eq. 8 with
  Eq. 9's estimate of Z_n, in the logarithmic form of Eq. 10).

n = N - 1 is the number of steps.  The literature quotes mu and gamma per
step of an n-step walk, and Z_n is then the number of n-step walks.  Every
point carries its own standard error:
- the ratio standard error of <R^2>;
- for log Z, the relative error of the mean weight, sqrt(1/ESS - 1/n_growths).

Ensembles at different lengths are independent (their own ensemble ids), so
the points are uncorrelated.  Parameter errors come from the weighted normal
equations, inflated by sqrt(chi^2/dof) when the fit is worse than the errors
allow.

The chains are grown and reduced by the CUDA library (one batch, one graph
launch).  Only the fits -- a few dozen numbers -- run on the host.
"""
import argparse
import json
import math
import time

import numpy as np


def log_z_se(stats):
    """Standard error of log Z-hat from one ensemble's statistics (delta method).

    Z-hat = exp(log_max) S0 / n, and its relative variance is
    (n Q0 / S0^2 - 1) / n = 1/ESS - 1/n.
    """
    n, ess = stats["n"], stats["ess"]
    if not (ess > 0):
        return math.inf
    return math.sqrt(max(1.0 / ess - 1.0 / n, 0.0))


def weighted_lsq(X, y, se):
    """Weighted least squares y ~ X beta with independent errors se.

    Returns (beta, cov, chi2_dof), where cov is inflated by chi2/dof when that
    exceeds 1.
    """
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = 1.0 / np.asarray(se, dtype=np.float64) ** 2
    A = X.T @ (w[:, None] * X)
    b = X.T @ (w * y)
    cov = np.linalg.inv(A)
    beta = cov @ b
    r = y - X @ beta
    dof = max(len(y) - X.shape[1], 1)
    chi2_dof = float((w * r * r).sum() / dof)
    return beta, cov * max(1.0, chi2_dof), chi2_dof


def fit_nu(n, r2, r2_se):
    """Eq. 7: <R^2_n> = a n^(2 nu).  Fits log <R^2> against log n."""
    n = np.asarray(n, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    se = np.asarray(r2_se, dtype=np.float64) / r2          # error of log <R^2>
    X = np.stack([np.ones_like(n), np.log(n)], axis=1)
    beta, cov, chi2 = weighted_lsq(X, np.log(r2), se)
    return {"nu": beta[1] / 2.0, "nu_se": math.sqrt(cov[1, 1]) / 2.0, "a": math.exp(beta[0]),
            "chi2_dof": chi2, "points": len(n)}


# Leading correction-to-scaling exponent of the 3D self-avoiding walk
# (N. Clisby, Phys. Rev. Lett. 104 (2010) 055702: Delta_1 = 0.528).  The
# paper fits the bare power law of Eq. 7; at chain lengths of tens to
# hundreds of steps the correction shifts that fit's nu by ~0.01.
DELTA_SAW = 0.528


def fit_nu_corrected(n, r2, r2_se, delta=DELTA_SAW):
    """Eq. 7 with the leading correction: <R^2_n> = a n^(2 nu) (1 + b n^-delta).

    For fixed nu the model is linear in (a, a b), so nu minimises the
    profiled chi^2 (weighted by the standard errors of <R^2>); its error is
    where chi^2 has risen by 1 (curvature), inflated by sqrt(chi^2/dof) when
    that exceeds 1.
    """
    from scipy import optimize

    n = np.asarray(n, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    w = 1.0 / np.asarray(r2_se, dtype=np.float64) ** 2

    def chi2(nu):
        X = np.stack([n ** (2 * nu), n ** (2 * nu - delta)], axis=1)
        A = X.T @ (w[:, None] * X)
        coef = np.linalg.solve(A, X.T @ (w * r2))
        r = r2 - X @ coef
        return float((w * r * r).sum()), coef

    res = optimize.minimize_scalar(lambda v: chi2(v)[0], bounds=(0.4, 0.8), method="bounded",
                                   options={"xatol": 1e-10})
    nu = float(res.x)
    c0, coef = chi2(nu)
    h = 1e-4
    curv = (chi2(nu + h)[0] - 2 * c0 + chi2(nu - h)[0]) / (h * h)
    dof = max(len(n) - 3, 1)
    se = math.sqrt(2.0 / curv) if curv > 0 else math.inf
    return {"nu": nu, "nu_se": se * math.sqrt(max(1.0, c0 / dof)), "a": coef[0],
            "b": coef[1] / coef[0], "delta": delta, "chi2_dof": c0 / dof, "points": len(n)}


def fit_mu_gamma(n, log_z, log_z_se_):
    """Eq. 8 and Eq. 10: log Z_n = n log mu + (gamma - 1) log n + c."""
    n = np.asarray(n, dtype=np.float64)
    X = np.stack([n, np.log(n), np.ones_like(n)], axis=1)
    beta, cov, chi2 = weighted_lsq(X, log_z, log_z_se_)
    mu = math.exp(beta[0])
    return {"mu": mu, "mu_se": mu * math.sqrt(cov[0, 0]), "gamma": beta[1] + 1.0,
            "gamma_se": math.sqrt(cov[1, 1]), "c": beta[2], "chi2_dof": chi2, "points": len(n)}


def lengths(n_min, n_max, points):
    """About `points` step counts spaced evenly in log n, from n_min to n_max."""
    g = np.unique(np.round(np.geomspace(n_min, n_max, points)).astype(int))
    return [int(v) for v in g]


def run_series(model, steps, chains, seed=7, k=32, beta_eps=0.0, sigma=1.0, cutoff=2.5,
               tune=True):
    """Grow and reduce one ensemble per step count in a single batch.

    model: "lattice" or "hard_sphere" / "lj" (real space, k trials).  Returns
    (rows, seconds), one row per step count n with the ensemble's statistics,
    and the wall time of the batch run (growth and reduction of every
    ensemble, one graph launch; tuning and set-up excluded).
    """
    import torch

    from . import rosen
    ens = []
    for e, n in enumerate(steps):
        if model == "lattice":
            ens.append(rosen.ensemble(rosen.ROSEN_MODEL_LATTICE, n + 1, chains, seed, e,
                                      beta_eps=beta_eps))
        else:
            pot = rosen.ROSEN_LJ if model == "lj" else rosen.ROSEN_HARD_SPHERE
            ens.append(rosen.ensemble(rosen.ROSEN_MODEL_OFFLATTICE, n + 1, chains, seed, e, k=k,
                                      potential=pot, beta_eps=beta_eps, sigma=sigma,
                                      cutoff=cutoff))
    b = rosen.RosenBatch(ens)
    try:
        if tune:
            b.tune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run()
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
        st = b.stats().cpu().numpy()
    finally:
        b.close()
    rows = []
    for e, n in enumerate(steps):
        d = dict(zip(rosen.STAT_KEYS, (float(v) for v in st[e])))
        d["steps"] = n
        d["logZ_se"] = log_z_se(d)
        rows.append(d)
    return rows, seconds


def analyse(rows, n_fit_min=1):
    """Fits of Eq. 7 and Eq. 10 over the rows with at least n_fit_min steps."""
    use = [r for r in rows if r["steps"] >= n_fit_min and r["n_alive"] > 1]
    n = [r["steps"] for r in use]
    r2 = [r["mean_r2"] for r in use]
    se = [r["se_r2"] for r in use]
    out = {"nu_fit": fit_nu(n, r2, se)}
    if len(use) >= 4:
        out["nu_corrected_fit"] = fit_nu_corrected(n, r2, se)
        out["mu_gamma_fit"] = fit_mu_gamma(n, [r["logZ"] for r in use],
                                           [r["logZ_se"] for r in use])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="Scaling exponents from Rosenbluth ensembles")
    ap.add_argument("--model", default="lattice", choices=["lattice", "hard_sphere", "lj"])
    ap.add_argument("--n-min", type=int, default=8, help="fewest steps")
    ap.add_argument("--n-max", type=int, default=511, help="most steps")
    ap.add_argument("--points", type=int, default=16)
    ap.add_argument("--chains", type=int, default=1_000_000, help="chains per length")
    ap.add_argument("--fit-from", type=int, default=16, help="fit step counts >= this")
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--beta-eps", type=float, default=0.0)
    ap.add_argument("--sigma", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=7)
    a = ap.parse_args(argv)
    steps = lengths(a.n_min, a.n_max, a.points)
    rows, secs = run_series(a.model, steps, a.chains, seed=a.seed, k=a.k, beta_eps=a.beta_eps,
                            sigma=a.sigma)
    res = analyse(rows, a.fit_from)
    res.update({"model": a.model, "chains_per_length": a.chains, "steps": steps,
                "batch_seconds": secs,
                "series": [{k: r[k] for k in ("steps", "logZ", "logZ_se", "mean_r2", "se_r2",
                                              "mean_rg2", "se_rg2", "ess", "n_alive")}
                           for r in rows]})
    print(json.dumps(res))
    return res


if __name__ == "__main__":
    main()
