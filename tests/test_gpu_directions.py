"""Exhaustive accuracy of the FP32 trial directions (rosen_sphere_points).

The real-space kernels re-decide a step in FP64 whenever an FP32 decision
lies within its error band; the band assumes every direction component is
within 2.7e-7 of the exact (s cos phi, s sin phi, z).  Here every one of the
2^24 possible angles and every one of the 2^24 possible polar words is
checked against FP64 on the host, so the bound is measured, not assumed.
"""
import numpy as np
import pytest
import torch

from paper_1704_04381_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu
COMPONENT_BOUND = 2.7e-7


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def points(rosen, a, b):
    words = torch.from_numpy(np.stack([a, b], 1).astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty((len(a), 3), dtype=torch.float32, device="cuda")
    rosen.rosen_sphere_points(words, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_every_angle(rosen):
    V = np.arange(1 << 24, dtype=np.uint64)
    a = np.full(len(V), 0x80000000, dtype=np.uint64)        # z = 0, s = 1 exactly
    u = points(rosen, a, V << np.uint64(8))
    phi = 2.0 * np.pi * V.astype(np.float64) / 2.0 ** 24
    ex = np.abs(u[:, 0] - np.cos(phi)).max()
    ey = np.abs(u[:, 1] - np.sin(phi)).max()
    assert (u[:, 2] == 0.0).all()
    assert ex < 1.5e-7 and ey < 1.5e-7, (ex, ey)


def test_every_polar_word(rosen):
    A = np.arange(1 << 24, dtype=np.uint64)
    u = points(rosen, A << np.uint64(8), np.zeros(len(A), dtype=np.uint64))   # phi = 0
    z = 1.0 - 2.0 * A.astype(np.float64) / 2.0 ** 24
    assert (u[:, 2] == z).all()                              # z is exact
    s = np.sqrt((1.0 - z) * (1.0 + z))
    assert np.abs(u[:, 0] - s).max() < 1.2e-7
    assert (u[:, 1] == 0.0).all()


def test_random_pairs_within_the_band_bound(rosen):
    rng = np.random.default_rng(0)
    n = 1 << 23
    a = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
    b = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
    u = points(rosen, a, b)
    z = 1.0 - 2.0 * (a >> np.uint64(8)).astype(np.float64) / 2.0 ** 24
    phi = 2.0 * np.pi * (b >> np.uint64(8)).astype(np.float64) / 2.0 ** 24
    s = np.sqrt((1.0 - z) * (1.0 + z))
    err = np.abs(u - np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)).max(0)
    assert (err < COMPONENT_BOUND).all(), err


# The float-float directions the Lennard-Jones kernels commit (dir_ff).
FF_BOUND = 1.5e-12


def points_ff(rosen, a, b):
    words = torch.from_numpy(np.stack([a, b], 1).astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty((len(a), 5), dtype=torch.float32, device="cuda")
    rosen.rosen_sphere_points_ff(words, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    return np.stack([o[:, 0] + o[:, 1], o[:, 2] + o[:, 3], o[:, 4]], 1)


def test_float_float_every_angle(rosen):
    V = np.arange(1 << 24, dtype=np.uint64)
    a = np.full(len(V), 0x80000000, dtype=np.uint64)
    u = points_ff(rosen, a, V << np.uint64(8))
    phi = 2.0 * np.pi * V.astype(np.float64) / 2.0 ** 24
    ex = np.abs(u[:, 0] - np.cos(phi)).max()
    ey = np.abs(u[:, 1] - np.sin(phi)).max()
    assert (u[:, 2] == 0.0).all()
    assert ex < FF_BOUND and ey < FF_BOUND, (ex, ey)


def test_float_float_every_polar_word(rosen):
    A = np.arange(1 << 24, dtype=np.uint64)
    u = points_ff(rosen, A << np.uint64(8), np.zeros(len(A), dtype=np.uint64))
    z = 1.0 - 2.0 * A.astype(np.float64) / 2.0 ** 24
    assert (u[:, 2] == z).all()
    s = np.sqrt((1.0 - z) * (1.0 + z))
    assert np.abs(u[:, 0] - s).max() < FF_BOUND
    assert (u[:, 1] == 0.0).all()


def test_float_float_random_pairs(rosen):
    rng = np.random.default_rng(1)
    n = 1 << 23
    a = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
    b = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
    u = points_ff(rosen, a, b)
    z = 1.0 - 2.0 * (a >> np.uint64(8)).astype(np.float64) / 2.0 ** 24
    phi = 2.0 * np.pi * (b >> np.uint64(8)).astype(np.float64) / 2.0 ** 24
    s = np.sqrt((1.0 - z) * (1.0 + z))
    err = np.abs(u - np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)).max(0)
    assert (err < FF_BOUND).all(), err
