"""The 14-electron gas in 358 spin-orbitals (179 plane waves, six-word
determinants), the system of the paper's CCSDTQ calculation (Sec. III.B).

The size of its truncated, momentum- and S_z-conserving space is counted
here from the oracle's plane-wave basis by a generating-function count over
particle sets (holes enumerated), independently of the oracle's own code,
and compared with the size the paper prints, 2.6(1) x 10^8.  The same
counter reproduces the exactly printed 22,969 of the 66 spin-orbital CISDT
space, which pins the counter itself.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def truncated_sector_size(kvecs: np.ndarray, nel: int, lmax: int) -> int:
    """Number of determinants with at most lmax holes among the nel lowest
    spin-orbitals (spin-orbital 2p = alpha, 2p+1 = beta of plane wave p) and
    as many particles above, with the reference's total momentum and S_z."""
    nso = 2 * len(kvecs)
    span = lmax * int(np.abs(kvecs).max())
    side = 2 * span + 1
    # c[n, a, kx, ky, kz]: particle sets of n spin-orbitals, a of them alpha
    c = np.zeros((lmax + 1, lmax + 1, side, side, side), dtype=np.int64)
    c[0, 0, span, span, span] = 1
    for q in range(nel, nso):
        k = kvecs[q // 2]
        alpha = 1 if q % 2 == 0 else 0
        for n in range(lmax, 0, -1):
            src = c[n - 1, : lmax + 1 - alpha]
            dst = c[n, alpha:]
            sl = tuple(slice(max(0, d), side + min(0, d)) for d in k)
            ss = tuple(slice(max(0, -d), side - max(0, d)) for d in k)
            dst[(slice(None),) + sl] += src[(slice(None),) + ss]
    total = 0
    for h in range(lmax + 1):
        for holes in itertools.combinations(range(nel), h):
            kk = np.sum([kvecs[q // 2] for q in holes], axis=0) if h else np.zeros(3, dtype=int)
            a = sum(1 for q in holes if q % 2 == 0)
            idx = tuple(int(x) + span for x in kk)
            total += int(c[h, a][idx])
    return total


def test_counter_reproduces_the_exact_66_orbital_size():
    s = oracle.System.ueg(14, 66, 1.0, 3)
    assert truncated_sector_size(s.kvecs(), 14, 3) == 22969


def test_358_orbital_ccsdtq_space_matches_paper():
    f = [ln.split() for ln in open(os.path.join(GOLDEN, "ueg358_space_size.txt")) if not ln.startswith("#")][0]
    nel, nso, lmax, size, err = (int(x) for x in f[:5])
    s = oracle.System.ueg(nel, nso, 1.0, lmax)
    k = s.kvecs()
    assert s.nw == 6 and len(k) == 179 and int((k ** 2).sum(1).max()) == 12   # the |n|^2 <= 12 shell
    n = truncated_sector_size(k, nel, lmax)
    assert abs(n - size) <= err, n


def test_358_orbital_rank_key_and_signs():
    """Six-word determinants through the oracle's rank key and signs: the key
    is order-preserving and invertible on random determinants of levels 0-4."""
    s = oracle.System.ueg(14, 358, 1.0, 4)
    rng = np.random.default_rng(4)
    dets = {s.hf()}
    for _ in range(400):
        lev = int(rng.integers(1, 5))
        holes = rng.choice(14, size=lev, replace=False)
        parts = 14 + rng.choice(344, size=lev, replace=False)
        d = s.hf()
        for q in list(holes) + list(parts):
            d ^= 1 << int(q)
        dets.add(d)
    dets = sorted(dets)
    keys = [s.rank(d) for d in dets]
    assert keys[0] == 0 and all(a < b for a, b in zip(keys, keys[1:]))
    assert all(s.unrank(k) == d for k, d in zip(keys, dets))
    assert keys[-1] < s.key_bound() < 2 ** 40
