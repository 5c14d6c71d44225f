"""The shoulder-plot diagnostic (Sec. IV.A): its analysis on the CPU, and a
short run of the three samplers through the CUDA library."""
import numpy as np
import pytest

import shoulder


def test_shoulder_of_rising_then_falling_ratio():
    # N_0 grows slowly at first and then at the rate of N_total: the ratio
    # N_total / N_0 peaks where N_0 starts to catch up
    steps = np.arange(400)
    ntot = 100.0 * np.exp(0.03 * steps)
    n0 = 100.0 * np.exp(0.03 * np.clip(steps - 150, 0, None) + 0.005 * np.minimum(steps, 150))
    n0[200:] = n0[200:] * np.exp(0.01 * (steps[200:] - 200))   # the reference overtakes: the ratio falls
    res = shoulder.shoulder_of(ntot, n0, window=5)
    ratio = ntot / n0
    assert res["found"]
    assert abs(res["step"] - int(np.argmax(ratio))) <= 5
    assert res["n_total"] == pytest.approx(ntot[res["step"]])


def test_shoulder_of_run_cut_off_while_rising():
    steps = np.arange(100)
    res = shoulder.shoulder_of(100.0 * np.exp(0.05 * steps), np.full(100, 100.0), window=5)
    assert not res["found"] and res["step"] == 99


def test_shoulder_of_dead_reference():
    res = shoulder.shoulder_of([10.0, 20.0], [0.0, 0.0], window=1)
    assert res == {"found": False, "step": None, "n_total": None, "ratio": None}


def test_running_median_window():
    x = [1.0, 9.0, 2.0, 8.0, 3.0]
    assert list(shoulder.running_median(x, 3)) == [1.0, 5.0, 2.0, 8.0, 3.0]


@pytest.mark.gpu
def test_shoulder_runs_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import workload

    w = workload("ueg14_m38_ccsd")
    for name, (fnc, ms) in shoulder.SAMPLERS.items():
        ntot, n0, status = shoulder.run_sampler(ccmc, w, fnc, ms, 0.01, 20.0, 5e4, 3000)
        assert status == "ok" and len(ntot) == len(n0) > 0
        assert ntot[-1] > 5e4 or len(ntot) >= 3000
        res = shoulder.shoulder_of(ntot, n0)
        assert res["ratio"] is not None and res["ratio"] >= 1.0
