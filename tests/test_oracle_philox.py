"""CPU checks of the oracle's Philox4x32-10.

The definitive pin -- equality with cuRAND's Philox4_32_10 generator for the
same key and counter -- needs a GPU and lives in test_gpu_philox.py.  Here:
properties any correct counter-based generator has (distinct counters give
unrelated outputs, uniform words, balanced bits, key dependence).
"""
import numpy as np
from scipy import stats

import oracle


def words(n, key=(1, 0), step=0):
    out = np.empty((n, 4), np.uint32)
    for c in range(n):
        out[c] = oracle.philox4x32_10([c, 0, step, 0], key)
    return out


def test_outputs_are_uniform_and_balanced():
    w = words(20_000)
    u = (w.astype(np.float64) + 0.5) / 2.0 ** 32
    for col in range(4):
        assert stats.kstest(u[:, col], "uniform").pvalue > 1e-4
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 128).mean(0)
    assert np.abs(bits - 0.5).max() < 0.02


def test_key_and_counter_dependence():
    a = oracle.philox4x32_10([0, 0, 0, 0], [0, 0])
    b = oracle.philox4x32_10([0, 0, 0, 0], [1, 0])
    c = oracle.philox4x32_10([0, 0, 0, 1], [0, 0])
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    # Avalanche: one counter bit flips about half of the 128 output bits.
    flips = []
    for bit in range(32):
        x = oracle.philox4x32_10([1 << bit, 0, 0, 0], [7, 9])
        y = oracle.philox4x32_10([0, 0, 0, 0], [7, 9])
        flips.append(np.unpackbits((x ^ y).view(np.uint8)).sum())
    assert 50 < np.mean(flips) < 78


def test_no_collisions_over_many_counters():
    w = words(50_000)
    packed = w[:, 0].astype(np.uint64) << 32 | w[:, 1].astype(np.uint64)
    assert len(np.unique(packed)) == len(packed)
