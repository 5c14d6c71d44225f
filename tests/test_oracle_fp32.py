"""Pins of the oracle's FP32 form: matrix elements and diagonal energies in
single precision from tables rounded from the FP64 ones, with spawn and death
values still formed in FP64 and populations exact."""
import numpy as np
import pytest

import oracle
from oracle import brute
from _systems import tiny_molecule


@pytest.mark.parametrize("kind", ["ueg", "mol"])
def test_fp32_matrix_elements_match_second_quantisation(kind):
    if kind == "ueg":
        ham = brute.UEGBrute(3, 38, 1.0)
        s = oracle.System.ueg(3, 38, 1.0, 2).set_fp32()
    else:
        h1, eri = tiny_molecule(norb=5, nocc=2, seed=4, scale=0.5)
        ham = brute.GenericBrute(4, h1, eri)
        s = oracle.System.generic(4, h1, eri, 4).set_fp32()
    dets = brute.sector(ham)
    H = brute.hamiltonian_matrix(ham, dets)
    Hf = np.array([[s.hij_f(a, b) for b in dets] for a in dets])
    scale = np.max(np.abs(H))
    err = np.max(np.abs(H - Hf))
    assert err < 4e-7 * scale * max(1, ham.nel)      # single-precision rounding of sums of <= N terms
    assert err > 0.0                                   # genuinely single precision


def test_fp32_long_run_energy_matches_deterministic_cc():
    """The FP32 form stays within the statistical error of the exact CCSD energy."""
    ham = brute.UEGBrute(3, 38, 1.0)
    efci, dets, H = brute.fci_energy(ham)
    ecc, _, _ = brute.solve_cc(ham, dets, H, 2)
    s = oracle.System.ueg(3, 38, 1.0, 2)
    ehf = s.ehf()
    s.set_fp32()
    sim = oracle.Sim(s, tau=0.02, target_pop=500, d0_init=20, seed=9)
    recs = sim.run(30000)
    en = np.array([r["e_num"] for r in recs[5000:]])
    n0 = np.array([r["n0"] / 65536.0 for r in recs[5000:]])
    e = en.mean() / n0.mean()
    _, se, _, _ = brute.reblock(en - e * n0)
    se /= n0.mean()
    assert abs(e - (ecc - ehf)) < 4 * se + 1e-6
