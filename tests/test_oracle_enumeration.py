"""Pins for the exact SAW enumerator (oracle.enumerate_saw).

The enumerator is the exact answer the Rosenbluth weight is unbiased for
(Eq. 3 with Eq. 1): it is pinned here against brute force over all 6^n random
walks (a different algorithm) and against the published SAW counts of the
simple cubic lattice.
"""
import itertools

import numpy as np
import pytest

import oracle

DIRS = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                dtype=np.int64)

# Number of n-step self-avoiding walks on the simple cubic lattice, n = 1..10
# (Fisher & Sykes, Phys. Rev. 114 (1959) 45; series A001412 of the OEIS).
CUBIC_SAW_COUNTS = [6, 30, 150, 726, 3534, 16926, 81390, 387966, 1853886, 8809878]


def brute_force(n):
    """Walk every one of the 6^n direction sequences; keep the self-avoiding ones.

    Returns dicts keyed by contact number: count, sum R^2, sum (n+1)^2 Rg^2.
    """
    cnt, sr2, sg2 = {}, {}, {}
    seqs = np.array(list(itertools.product(range(6), repeat=n)), dtype=np.int64)
    for lo in range(0, len(seqs), 50000):
        s = seqs[lo:lo + 50000]
        steps = DIRS[s]                                     # [M, n, 3]
        pos = np.concatenate([np.zeros((len(s), 1, 3), np.int64), np.cumsum(steps, 1)], 1)
        l1 = np.abs(pos[:, :, None, :] - pos[:, None, :, :]).sum(-1)   # [M, n+1, n+1]
        iu = np.triu_indices(n + 1, k=1)
        saw = (l1[:, iu[0], iu[1]] > 0).all(1)
        far = np.triu(np.ones((n + 1, n + 1), bool), k=2)   # pairs with j - i >= 2
        contacts = ((l1 == 1) & far).sum((1, 2))
        r2 = (pos[:, -1] ** 2).sum(1)
        g2 = (n + 1) * (pos ** 2).sum((1, 2)) - (pos.sum(1) ** 2).sum(1)
        for c in np.unique(contacts[saw]):
            sel = saw & (contacts == c)
            cnt[int(c)] = cnt.get(int(c), 0) + int(sel.sum())
            sr2[int(c)] = sr2.get(int(c), 0) + int(r2[sel].sum())
            sg2[int(c)] = sg2.get(int(c), 0) + int(g2[sel].sum())
    return cnt, sr2, sg2


@pytest.fixture(scope="module")
def enum10():
    return oracle.enumerate_saw(10)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_enumerator_matches_brute_force(enum10, n):
    cnt, sr2, sg2 = enum10
    bc, br, bg = brute_force(n)
    for c in range(n + 1):
        assert cnt[n, c] == bc.get(c, 0), (n, c)
        assert sr2[n, c] == br.get(c, 0), (n, c)
        assert sg2[n, c] == bg.get(c, 0), (n, c)


def test_enumerator_counts_match_literature(enum10):
    cnt, _, _ = enum10
    assert cnt.sum(1)[1:].tolist() == CUBIC_SAW_COUNTS


def test_enumerator_closed_forms(enum10):
    cnt, sr2, sg2 = enum10
    # One step: 6 walks, R^2 = 1, N^2 Rg^2 = 2*1 - 1 = 1 each.
    assert cnt[1, 0] == 6 and sr2[1, 0] == 6 and sg2[1, 0] == 6
    # No walk of at most 3 steps can revisit a site: c_n = 6 * 5^(n-1).
    for n in (1, 2, 3):
        assert cnt[n].sum() == 6 * 5 ** (n - 1)
    # Contacts first appear at n = 3: the 6 x 4 U-shapes end next to the origin.
    assert cnt[1, 1:].sum() == 0 and cnt[2, 1:].sum() == 0
    assert cnt[3, 1] == 24 and cnt[3, 2:].sum() == 0
    # Each U-shape has exactly one fourth step that lands on the origin.
    assert cnt[4].sum() == 6 * 5 ** 3 - 24
    # n = 2: per first step, 1 straight continuation (R^2 = 4) and 4 turns (R^2 = 2).
    assert sr2[2].sum() * 5 == cnt[2].sum() * 12
