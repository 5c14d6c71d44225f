"""Pins of the reblocking analysis used for statistical error bars."""
import math

import numpy as np

from oracle import brute


def test_reblock_iid():
    rng = np.random.default_rng(0)
    x = rng.normal(size=2 ** 14)
    mean, se, opt, table = brute.reblock(x)
    want = 1.0 / math.sqrt(len(x))
    assert abs(se - want) < 4 * table[opt][3]
    # every level agrees for uncorrelated data
    for b, n, se_b, ee in table[:8]:
        assert abs(se_b - want) < 4 * ee


def test_reblock_ar1_matches_closed_form():
    """For x_t = phi x_{t-1} + e_t the variance of the mean is
    var(x) (1 + phi)/((1 - phi) n) asymptotically."""
    rng = np.random.default_rng(1)
    phi, n = 0.9, 2 ** 17
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    var = 1.0 / (1 - phi * phi)
    want = math.sqrt(var * (1 + phi) / ((1 - phi) * n))
    mean, se, opt, table = brute.reblock(x)
    assert abs(se - want) < 4 * table[opt][3]
    # the unblocked estimate underestimates by sqrt((1 + phi)/(1 - phi))
    assert table[0][2] < 0.3 * want
    assert opt >= 3
