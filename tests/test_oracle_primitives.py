"""Pins of the oracle's random-number, sampling and rounding primitives."""
import numpy as np
import pytest

import oracle

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _numpy_block(ctr, key):
    """Philox-4x64-10 block from numpy's generator.  numpy advances its 256-bit
    counter before producing a block, so start it one below."""
    v = sum(int(ctr[i]) << (64 * i) for i in range(4))
    v = (v - 1) % (1 << 256)
    words = np.array([(v >> (64 * i)) & (2 ** 64 - 1) for i in range(4)], dtype=np.uint64)
    g = np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64))
    return g.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 7, 9, 11], [1, 0]),
    ([199, (2 << 56) | 123456, 17, 0], [1, 0]),
    ([2 ** 64 - 1, 2 ** 63 + 5, 3, 0], [1000 + 63, 63]),
])
def test_philox_matches_numpy(ctr, key):
    assert np.array_equal(oracle.philox(ctr, key), _numpy_block(ctr, key))


def test_numpy_counter_convention_is_preincrement():
    # the same counter without the decrement must NOT match: the convention is checked, not assumed
    ctr, key = [5, 7, 9, 11], [1, 0]
    g = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    assert not np.array_equal(oracle.philox(ctr, key), g.random_raw(4))


def _golden_psize():
    from fractions import Fraction

    out = {}
    for line in open(f"{GOLDEN}/p_size.txt"):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out[int(f[0])] = [Fraction(x) for x in f[1:]]
    return out


@pytest.mark.parametrize("lmax", [1, 2, 3, 4])
def test_size_distribution_exact(lmax):
    """Counting all 2^16 leading-bit patterns reproduces p_size exactly,
    including the remainder in the last bin (Sec. II footnote)."""
    want = _golden_psize()[lmax]
    assert sum(want) == 1
    counts = np.zeros(lmax + 3, dtype=np.int64)
    counts_fnc = np.zeros(lmax + 3, dtype=np.int64)
    low = 0x0123456789AB
    for v in range(1 << 16):
        r = (v << 48) | low
        counts[oracle.size_draw(r, lmax, False)] += 1
        counts_fnc[oracle.size_draw(r, lmax, True)] += 1
    for s in range(lmax + 3):
        assert counts[s] == want[s] * (1 << 16)
    # full non-composite: s >= 2 with p(s)/(1 - p(0) - p(1)) (Sec. IV.B)
    norm = 1 - want[0] - want[1]
    assert counts_fnc[0] == counts_fnc[1] == 0
    for s in range(2, lmax + 3):
        assert counts_fnc[s] == want[s] / norm * (1 << 16)


def test_selection_counts_equal_weights():
    """Every position x in [0, N_ex) maps to one excitor, and excitor i owns
    exactly |t_i| positions: selection probabilities |t_i|/N_ex sum to 1."""
    rng = np.random.default_rng(0)
    for trial in range(20):
        n = int(rng.integers(2, 12))
        pops = rng.integers(-40, 40, size=n)
        pops[pops == 0] = 1
        w = np.abs(pops).astype(np.int64)
        w[0] = 0
        prefix = np.cumsum(w)
        nex = int(prefix[-1])
        counts = np.zeros(n, dtype=np.int64)
        for x in range(nex):
            counts[oracle.pick_index(prefix, x)] += 1
        assert counts[0] == 0
        assert np.array_equal(counts[1:], np.abs(pops[1:]))
        assert counts.sum() == nex


def test_below_is_floor_of_product():
    rng = np.random.default_rng(1)
    for _ in range(200):
        r = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        n = int(rng.integers(1, 2 ** 40))
        assert oracle.below(r, n) == (r * n) >> 64


@pytest.mark.parametrize("x", [0.3, -2.75, 17.000001, 1e-3, -5e-4, 0.0078125, 123456.789])
def test_stochastic_rounding_unbiased(x):
    """E_u[round(x)] = x: floor plus one with probability of the remainder;
    below the spawn cutoff, +-cutoff with probability |x|/cutoff."""
    cutoff = 2.0 ** -7
    ax = abs(x)
    sgn = -1 if x < 0 else 1
    if ax < cutoff:
        p = ax / cutoff
        lo, hi = 0, 512
    else:
        q = ax * 65536.0
        p = q - np.floor(q)
        lo, hi = int(np.floor(q)), int(np.floor(q)) + 1
    eps = 1e-12
    if p - eps > 0:
        assert oracle.stoch_round(x, p - eps, cutoff) == sgn * hi
    assert oracle.stoch_round(x, min(p + eps, 1 - 1e-16), cutoff) == sgn * lo
    # the mean over a fine uniform grid of u equals x on the fixed-point grid
    us = (np.arange(4096) + 0.5) / 4096
    mean = np.mean([oracle.stoch_round(x, u, cutoff) for u in us])
    assert abs(mean / 65536.0 - x) <= (hi - lo) / 65536.0 / 4096 + 1e-15


def test_rounding_without_cutoff_is_plain_stochastic():
    assert oracle.stoch_round(1e-6, 0.0, 0.0) == 1
    assert oracle.stoch_round(1e-6, 0.9, 0.0) == 0
    assert oracle.stoch_round(-2.5 / 65536, 0.4, 0.0) == -3
    assert oracle.stoch_round(-2.5 / 65536, 0.6, 0.0) == -2
