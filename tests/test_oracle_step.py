"""Pins of the oracle's whole CCMC step against exact results.

* the mean change of one step equals the exact action of the linearised
  propagator on t_HF exp(T/t_HF)|HF> (Sec. II, Eq. CCMC) for the original,
  full non-composite (Sec. IV.B) and multi-spawn (Sec. IV.C) samplers;
* annihilation conserves the summed weights exactly before the threshold;
* the deterministic CC fixed point equals FCI at full truncation;
* the long-run projected energy (Sec. II, Eq. E_proj) reproduces the
  deterministic CC energy within reblocked error bars.
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from _systems import tiny_molecule


def _random_list(s, dets, rng, scale, frac=0.7):
    nel = s.nel
    hf = (1 << nel) - 1
    lst = sorted((d for d in dets if brute.level(d, nel) <= s.lmax), key=s.rank)
    assert lst[0] == hf
    keep, pops = [hf], [int(scale * 65536)]
    for d in lst[1:]:
        if rng.random() < frac:
            keep.append(d)
            v = int(rng.normal() * scale / 3 * 65536)
            pops.append(v if v != 0 else 65536)
    return lst, keep, pops


def _mean_step(s, keep, pops, lst, K, tau, shift, fnc, ms):
    sim = oracle.Sim(s, tau=tau, fnc=fnc, multispawn=ms, a_thresh=1.0, seed=11)
    sim.set_list(keep, pops)
    keys = {s.rank(d): i for i, d in enumerate(lst)}
    pos = {d: i for i, d in enumerate(lst)}
    acc = np.zeros((K, len(lst)))
    for k in range(K):
        sim.set_state(k, shift, False, 1.0)
        sim.step(propagate_only=True)
        dk, dp = sim.spawned()
        de = sim.death()
        np.add.at(acc[k], [keys[int(x)] for x in dk], dp / 65536.0)
        for d, v in zip(keep, de):
            acc[k, pos[d]] += v / 65536.0
    return acc.mean(0), acc.std(0, ddof=1) / np.sqrt(K)


CASES = [
    ("mol", 0, 0), ("mol", 1, 0), ("mol", 1, 1), ("mol", 0, 1),
    ("ueg", 0, 0), ("ueg", 1, 1),
    ("mol-negref", 0, 0), ("mol-negref", 1, 1),
]


@pytest.mark.parametrize("kind,fnc,ms", CASES)
def test_one_step_mean_equals_exact_action(kind, fnc, ms):
    tau, shift = 0.01, 0.3
    if kind.startswith("mol"):
        h1, eri = tiny_molecule(norb=5, nocc=2, seed=11, scale=0.3)
        ham = brute.GenericBrute(4, h1, eri)
        s = oracle.System.generic(4, h1, eri, 2)
        K = 3000
    else:
        ham = brute.UEGBrute(3, 38, 1.0)
        s = oracle.System.ueg(3, 38, 1.0, 2)
        K = 3000
    efci, dets, H = brute.fci_energy(ham)
    rng = np.random.default_rng(3)
    lst, keep, pops = _random_list(s, dets, rng, 40.0)
    if kind == "mol-negref":
        pops[0] = -pops[0]          # a negative reference weight (overall sign of Psi)
    amps = {d: p / 65536 for d, p in zip(keep[1:], pops[1:])}
    exact = brute.exact_step_change(ham, dets, H, amps, pops[0] / 65536, tau, shift, s.ehf(), s.lmax)
    mean, se = _mean_step(s, keep, pops, lst, K, tau, shift, fnc, ms)
    ex = np.array([exact[d] for d in lst])
    z = (mean - ex) / np.maximum(se, 1e-12)
    # deterministic seeds: the outcome is fixed; 5 sigma over <= 60 components
    assert np.max(np.abs(z)) < 5.0, (np.max(np.abs(z)), np.argmax(np.abs(z)))
    # the step changed a good fraction of the space
    assert np.count_nonzero(se) > len(lst) // 2


@pytest.mark.parametrize("fnc,ms", [(0, 0), (1, 1)])
def test_annihilation_conserves_weight(fnc, ms):
    """After a step, every excitor holds exactly old + death + spawned weight,
    except entries below one particle, which become 0 or +-1 with their sign.
    The list stays sorted by key, unique, HF first, within the truncation."""
    s = oracle.System.ueg(14, 38, 1.0, 2)
    sim = oracle.Sim(s, tau=0.01, fnc=fnc, multispawn=ms, seed=5)
    sim.run(60)
    bits, keys, pops = sim.get_list()
    it, shift, vary, nprev = sim.get_state()
    probe = oracle.Sim(s, tau=0.01, fnc=fnc, multispawn=ms, seed=5)
    probe.set_list_words(bits, pops)
    probe.set_state(it, shift, vary, nprev)
    probe.step(propagate_only=True)
    dk, dp = probe.spawned()
    death = probe.death()
    want = {}
    for k, p, d in zip(keys, pops, death):
        want[int(k)] = int(p) + int(d)
    for k, p in zip(dk, dp):
        want[int(k)] = want.get(int(k), 0) + int(p)
    sim.step()
    b2, k2, p2 = sim.get_list()
    assert k2[0] == 0 and all(int(a) < int(b) for a, b in zip(k2, k2[1:]))
    got = {int(k): int(p) for k, p in zip(k2, p2)}
    for k, v in want.items():
        if k == 0 or abs(v) >= 65536:
            assert got.get(k, 0) == v
        elif v == 0:
            assert k not in got
        else:
            assert got.get(k, 0) in (0, 65536 if v > 0 else -65536)
    assert set(got) <= set(want)
    for w, k in zip(b2, k2):
        d = s.from_words(w)
        assert s.rank(d) == int(k) and s.level(d) <= s.lmax


def test_fnc_estimator_equals_list_sum():
    """In FNC mode for the UEG, composite clusters cannot reach level <= 2, so
    the sampled numerator equals sum_i <HF|H|D_i> s_D(i) t_i over the list."""
    s = oracle.System.ueg(14, 38, 1.0, 2)
    sim = oracle.Sim(s, tau=0.01, fnc=1, multispawn=1, seed=2)
    sim.run(40)
    bits, keys, pops = sim.get_list()
    hf = s.hf()
    want = 0.0
    for w, p in zip(bits, pops):
        d = s.from_words(w)
        if 1 <= s.level(d) <= 2:
            want += s.hij(hf, d) * s.excitor_sign(d) * p / 65536.0
    rec = sim.step()
    assert abs(rec.e_num - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("nel,nso,lmax", [(2, 14, 2), (3, 14, 3), (2, 38, 2)])
def test_deterministic_cc_equals_fci_ueg(nel, nso, lmax):
    ham = brute.UEGBrute(nel, nso, 1.0)
    efci, dets, H = brute.fci_energy(ham)
    ecc, amps, res = brute.solve_cc(ham, dets, H, lmax)
    assert res < 1e-10
    assert abs(ecc - efci) < 1e-10


def test_deterministic_cc_full_truncation_is_an_eigenstate():
    """Full-truncation CC on a random molecule gives an exact eigenpair of H."""
    h1, eri = tiny_molecule(norb=4, nocc=2, seed=1, scale=0.3)
    ham = brute.GenericBrute(4, h1, eri)
    efci, dets, H = brute.fci_energy(ham)
    ecc, amps, res = brute.solve_cc(ham, dets, H, 4)
    psi = brute.cc_wavefunction(amps, 4)
    v = np.array([psi.get(d, 0.0) for d in dets])
    assert np.linalg.norm(H @ v - ecc * v) < 1e-9 * np.linalg.norm(v)
    assert abs(ecc - efci) < 1e-10


def _projected_energy(recs, skip):
    en = np.array([r["e_num"] for r in recs[skip:]])
    n0 = np.array([r["n0"] / 65536.0 for r in recs[skip:]])
    e = en.mean() / n0.mean()
    _, se, _, _ = brute.reblock(en - e * n0)
    return e, se / n0.mean()


@pytest.mark.parametrize("nel,fnc,ms", [(3, 0, 0), (3, 1, 1), (2, 0, 0)])
def test_long_run_energy_matches_deterministic_cc(nel, fnc, ms):
    """CCMC E_proj over a long run agrees with the deterministic CCSD energy
    (14 or 38 spin-orbital UEG) within four reblocked standard errors."""
    nso, lmax = 38, 2
    ham = brute.UEGBrute(nel, nso, 1.0)
    efci, dets, H = brute.fci_energy(ham)
    ecc, _, _ = brute.solve_cc(ham, dets, H, lmax)
    s = oracle.System.ueg(nel, nso, 1.0, lmax)
    sim = oracle.Sim(s, tau=0.02, target_pop=500, d0_init=20, fnc=fnc, multispawn=ms, seed=9)
    recs = sim.run(30000)
    e, se = _projected_energy(recs, 5000)
    assert abs(e - (ecc - s.ehf())) < 4 * se
    assert se < 3e-5


def test_shift_held_then_varied():
    """S stays 0 (i.e. at E_HF) until the population first exceeds the target
    at a report boundary, then moves every A steps by
    -(zeta/(A tau)) ln(N(t)/N(t - A tau)) (Sec. II)."""
    s = oracle.System.ueg(14, 38, 1.0, 2)
    tau, A, zeta, target = 0.01, 10, 0.05, 800.0
    sim = oracle.Sim(s, tau=tau, target_pop=target, shift_a=A, zeta=zeta, seed=4)
    recs = sim.run(400)
    vary_from = None
    nprev = 100.0
    shift = 0.0
    for k, r in enumerate(recs):
        assert r["shift"] == shift
        if (k + 1) % A == 0:
            nt = r["ntot_after"] / 65536.0
            if vary_from is not None:
                shift = shift - (zeta / (A * tau)) * np.log(nt / nprev)
            if vary_from is None and nt > target:
                vary_from = k
            nprev = nt
    assert vary_from is not None and vary_from < 350
    assert all(r["shift"] == 0.0 for r in recs[: vary_from + 1])
    assert any(r["shift"] != 0.0 for r in recs[vary_from + 1:])
