"""The benchmark's own arithmetic on the CPU: blocked error estimates,
algorithmic bytes per phase and the profile-file reader."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_blocked_error_iid_and_correlated():
    rng = np.random.Generator(np.random.PCG64(11))
    x = rng.standard_normal(4096)
    se = bench.blocked_error(x)
    assert abs(se / (1.0 / np.sqrt(4096)) - 1.0) < 0.5          # iid: close to sigma / sqrt(n)
    # AR(1) with phi = 0.9: the error of the mean is sqrt((1+phi)/(1-phi)) larger
    phi, y = 0.9, np.zeros(1 << 15)
    e = rng.standard_normal(len(y)) * np.sqrt(1 - phi ** 2)
    for i in range(1, len(y)):
        y[i] = phi * y[i - 1] + e[i]
    expect = np.sqrt((1 + phi) / (1 - phi)) / np.sqrt(len(y))
    assert 0.6 < bench.blocked_error(y) / expect < 1.5
    assert bench.blocked_error(np.ones(5)) == 0.0                # too short for 8 blocks


def test_algorithmic_bytes_per_phase():
    r = dict(n_visit=0, nocc_after=1000, n_spawned=300, n_sel=2000, n_attempts=5000, n_keys=200)
    nw = 2
    be = 8 * nw + 16
    assert bench.algorithmic_bytes("scan", [r], nw) == 1000 * 16
    assert bench.algorithmic_bytes("sample", [r], nw) == 2000 * 0.97 * be + 300 * 16
    assert bench.algorithmic_bytes("attempts", [r], nw) == 5000 * be + 300 * 16
    assert bench.algorithmic_bytes("sort", [r], nw) == 300 * 32
    assert bench.algorithmic_bytes("reduce", [r], nw) == 300 * 16 + 200 * 16
    assert bench.algorithmic_bytes("merge", [r], nw) == 1000 * be + 200 * 16 + 1000 * be
    # averaged over records
    r2 = dict(r, n_sel=4000)
    assert bench.algorithmic_bytes("sample", [r, r2], nw) == 3000 * 0.97 * be + 300 * 16


def test_read_traffic_from_profiles():
    b, issue = bench.read_traffic("ueg14_m114_ccsdt_fnc_ms", "attempts")
    assert b is not None and b > 0 and 0 < issue <= 100
    assert bench.read_traffic("no_such_workload", "sample") == (None, None)


def test_oracle_on_several_cores_small_workload():
    """The CPU baseline's process pool (spawned processes, a barrier, slices
    of one full step) on the 38 spin-orbital gas with two processes."""
    from ccmc_inputs import workload

    w = workload("ueg14_m38_ccsd")
    v, kps, cores, secs, nslices = bench.oracle_all_cores(w, 0, 2, cores=2, per_slice=2000)
    assert cores == 2 and v > 0 and secs > 0 and nslices >= 1 and kps >= 0
