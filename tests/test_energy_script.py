"""The blocking analysis of energy.py (Flyvbjerg-Petersen) on series with
known standard errors of the mean, and its projected-energy estimator."""
import numpy as np

import energy


def test_blocking_iid():
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.standard_normal(1 << 14)
    se, levels = energy.blocking(x)
    assert abs(se * np.sqrt(len(x)) - 1.0) < 0.15
    assert levels[0][0] == len(x)


def test_blocking_ar1():
    # AR(1) with phi = 0.8: the error of the mean is sqrt((1+phi)/(1-phi)) / sqrt(n)
    rng = np.random.Generator(np.random.PCG64(5))
    phi, n = 0.8, 1 << 16
    e = rng.standard_normal(n) * np.sqrt(1 - phi ** 2)
    y = np.zeros(n)
    for i in range(1, n):
        y[i] = phi * y[i - 1] + e[i]
    se, _ = energy.blocking(y)
    expect = np.sqrt((1 + phi) / (1 - phi)) / np.sqrt(n)
    assert 0.75 < se / expect < 1.3


def test_projected_energy_ratio_of_means():
    rng = np.random.Generator(np.random.PCG64(7))
    n0 = 1000.0 + 10.0 * rng.standard_normal(4096)
    en = -0.5 * n0 + rng.standard_normal(4096)
    recs = [{"e_num": a, "n0": int(b * 65536), "shift": -0.5 + 0.01 * c}
            for a, b, c in zip(en, n0, rng.standard_normal(4096))]
    e, se, es, ses = energy.projected_energy(recs)
    assert abs(e + 0.5) < 4 * se and se < 1e-3
    assert abs(es + 0.5) < 4 * ses
