"""Pins for the real-space oracle (Algorithm 2, weight = sum of trial weights).

With k trials per step the normalised weight W / k^(N-1) is an unbiased
estimator of the mean Boltzmann factor of an ideal (freely jointed) chain:
the fraction of self-avoiding ideal chains for hard spheres, E[exp(-beta U)]
for Lennard-Jones beads.  Closed forms (trimer, ideal limit), a quadrature
and simple sampling with an independent generator fix these values.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle

Z_SIGMAS = 4.5


def ratio_mean_se(w, a):
    S = w.sum()
    mean = (w * a).sum() / S
    se = np.sqrt((w ** 2 * (a - mean) ** 2).sum()) / S
    return mean, se


def mean_se(x):
    return x.mean(), x.std(ddof=1) / np.sqrt(len(x))


def lj(d2, beta_eps, cutoff=2.5):
    s3 = (1.0 / d2) ** 3
    u = 4.0 * s3 * (s3 - 1.0)
    return np.where(d2 < cutoff ** 2, beta_eps * u, 0.0)


def test_hard_sphere_trimer_closed_form():
    # N = 3: cos of the bond angle is uniform on [-1, 1]; the end bead overlaps
    # the first one iff r02^2 = 2 + 2c < 1, i.e. c < -1/2.  So E[W/k^2] = 3/4
    # and <R^2> = E[(2 + 2c) | c >= -1/2] = 5/2.
    k = 32
    o = oracle.offlattice_run(5, 3, 200_000, k)
    wn = np.exp(o["logw"] - 2 * np.log(k))
    m, se = mean_se(wn)
    assert abs(m - 0.75) < Z_SIGMAS * se
    mean, se_r = ratio_mean_se(wn, o["r2"])
    assert abs(mean - 2.5) < Z_SIGMAS * se_r


def test_directions_are_uniform_on_the_sphere():
    # Step 1 has no non-bonded bead, so the chosen trial is one of k uniform
    # directions: r_1 = u with E[u] = 0, E[u_a^2] = 1/3, |u| = 1.
    o = oracle.offlattice_run(3, 2, 200_000, 8, coords=True)
    u = o["coords"][:, 1, :]
    np.testing.assert_allclose((u ** 2).sum(1), 1.0, rtol=0, atol=1e-14)
    for a in range(3):
        m, se = mean_se(u[:, a])
        assert abs(m) < Z_SIGMAS * se
        m2, se2 = mean_se(u[:, a] ** 2)
        assert abs(m2 - 1.0 / 3.0) < Z_SIGMAS * se2
    m, se = mean_se(u[:, 0] * u[:, 1])
    assert abs(m) < Z_SIGMAS * se


@pytest.mark.parametrize("N", [2, 8, 32])
def test_lj_at_zero_coupling_is_the_ideal_chain(N):
    k = 16
    o = oracle.offlattice_run(9, N, 50_000, k, potential=oracle.LJ, beta_eps=0.0, coords=True)
    np.testing.assert_allclose(o["logw"], (N - 1) * np.log(k), rtol=1e-13)
    m, se = mean_se(o["r2"])
    assert abs(m - (N - 1)) < Z_SIGMAS * se
    m, se = mean_se(o["rg2"])
    assert abs(m - (N * N - 1) / (6.0 * N)) < Z_SIGMAS * se
    xyz = o["coords"]
    bonds = np.sqrt((np.diff(xyz, axis=1) ** 2).sum(-1))
    np.testing.assert_allclose(bonds, 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("beta_eps", [0.3, 1.0])
def test_lj_trimer_quadrature(beta_eps):
    # N = 3: only the pair (0, 2) interacts, at r02 = sqrt(2 + 2c), c ~ U[-1, 1].
    f = lambda c: np.exp(-lj(2 + 2 * c, beta_eps))
    Z = 0.5 * integrate.quad(f, -1, 1, points=[-0.5], limit=200)[0]
    R2 = 0.5 * integrate.quad(lambda c: (2 + 2 * c) * f(c), -1, 1, points=[-0.5],
                              limit=200)[0] / Z
    k = 16
    o = oracle.offlattice_run(21, 3, 200_000, k, potential=oracle.LJ, beta_eps=beta_eps)
    wn = np.exp(o["logw"] - 2 * np.log(k))
    m, se = mean_se(wn)
    assert abs(m - Z) < Z_SIGMAS * se
    mean, se_r = ratio_mean_se(wn, o["r2"])
    assert abs(mean - R2) < Z_SIGMAS * se_r


def ideal_chains(rng, C, N):
    """Freely jointed chains with unit bonds, drawn with numpy's own generator."""
    z = rng.uniform(-1, 1, size=(C, N - 1))
    phi = rng.uniform(0, 2 * np.pi, size=(C, N - 1))
    s = np.sqrt(1 - z * z)
    steps = np.stack([s * np.cos(phi), s * np.sin(phi), z], -1)
    return np.concatenate([np.zeros((C, 1, 3)), np.cumsum(steps, 1)], 1)


def pair_d2(pos):
    return ((pos[:, :, None, :] - pos[:, None, :, :]) ** 2).sum(-1)


def test_hard_sphere_rosenbluth_matches_simple_sampling():
    N, k = 6, 16
    rng = np.random.default_rng(1234)
    pos = ideal_chains(rng, 400_000, N)
    d2 = pair_d2(pos)
    far = np.triu(np.ones((N, N), bool), k=2)
    saw = ~((d2 < 1.0) & far).any((1, 2))
    r2_ss = (pos[:, -1] ** 2).sum(-1)
    p_ss, se_p = mean_se(saw.astype(float))
    r2_mean_ss, se_r2_ss = mean_se(r2_ss[saw])

    o = oracle.offlattice_run(17, N, 100_000, k)
    wn = np.exp(o["logw"] - (N - 1) * np.log(k))
    m, se = mean_se(wn)
    assert abs(m - p_ss) < Z_SIGMAS * np.hypot(se, se_p)
    mean, se_r = ratio_mean_se(wn, o["r2"])
    assert abs(mean - r2_mean_ss) < Z_SIGMAS * np.hypot(se_r, se_r2_ss)


def test_lj_rosenbluth_matches_simple_sampling():
    N, k, beta_eps = 5, 16, 0.5
    rng = np.random.default_rng(99)
    pos = ideal_chains(rng, 400_000, N)
    d2 = pair_d2(pos)
    far = np.triu(np.ones((N, N), bool), k=2)
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        bu = np.where(far, lj(np.where(far, d2, 1.0), beta_eps), 0.0).sum((1, 2))
        boltz = np.exp(-bu)
    r2 = (pos[:, -1] ** 2).sum(-1)
    z_ss, se_z = mean_se(boltz)
    r2_ss, se_r_ss = ratio_mean_se(boltz, r2)

    o = oracle.offlattice_run(31, N, 100_000, k, potential=oracle.LJ, beta_eps=beta_eps)
    wn = np.exp(o["logw"] - (N - 1) * np.log(k))
    m, se = mean_se(wn)
    assert abs(m - z_ss) < Z_SIGMAS * np.hypot(se, se_z)
    mean, se_r = ratio_mean_se(wn, o["r2"])
    assert abs(mean - r2_ss) < Z_SIGMAS * np.hypot(se_r, se_r_ss)


def test_hard_sphere_geometry_of_grown_chains():
    N, k = 16, 32
    o = oracle.offlattice_run(4, N, 2000, k, coords=True, trace=True)
    alive = o["alive"].astype(bool)
    xyz = o["coords"][alive]
    bonds = np.sqrt((np.diff(xyz, axis=1) ** 2).sum(-1))
    np.testing.assert_allclose(bonds, 1.0, rtol=0, atol=1e-12)
    d2 = pair_d2(xyz)
    far = np.triu(np.ones((N, N), bool), k=2)
    assert (d2[:, far] >= 1.0).all()
    np.testing.assert_allclose(o["r2"][alive], (xyz[:, -1] ** 2).sum(-1), rtol=1e-12)
    cm = xyz.mean(1, keepdims=True)
    np.testing.assert_allclose(o["rg2"][alive], ((xyz - cm) ** 2).sum(-1).mean(1),
                               rtol=1e-12)
    # Weight bounds: 1 <= W / k^(N-1) ... each factor m_i <= k, first one = k.
    lw = o["logw"][alive]
    assert (lw <= (N - 1) * np.log(k) + 1e-9).all() and (lw >= np.log(k) - 1e-9).all()


def test_zero_diameter_hard_spheres_are_ideal():
    o = oracle.offlattice_run(8, 12, 1000, 8, sigma=0.0)
    np.testing.assert_allclose(o["logw"], 11 * np.log(8), rtol=1e-13)
