"""Pins of the oracle's systems and Slater-Condon matrix elements against
closed forms and against the Hamiltonian built by literal second quantisation."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from _systems import tiny_molecule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("npw", [7, 19, 27, 33, 57, 81, 93])
def test_ueg_basis_closes_shells(npw):
    """Plane-wave counts 7/19/27/33/57/81/93 close the |n|^2 <= 1,2,3,4,5,6,8 shells."""
    s = oracle.System.ueg(2, 2 * npw, 1.0, 2)
    kv = s.kvecs()
    n2 = (kv ** 2).sum(1)
    assert np.all(np.diff(n2) >= 0)
    b = brute.UEGBrute(2, 2 * npw, 1.0)
    assert np.array_equal(kv, np.array(b.kv))


def test_ueg_rejects_open_shell_basis():
    with pytest.raises(ValueError):
        oracle.System.ueg(14, 40, 1.0, 2)


@pytest.mark.parametrize("nel,nso,rs", [(14, 38, 1.0), (14, 66, 0.5), (54, 162, 1.0), (14, 114, 5.0)])
def test_ueg_closed_forms(nel, nso, rs):
    """L = r_s (4 pi N/3)^(1/3); T = |k|^2/2; v(q) = 4 pi/(Omega |q|^2) for k = 2 pi n/L."""
    s = oracle.System.ueg(nel, nso, rs, 2)
    L = rs * (4.0 * math.pi * nel / 3.0) ** (1.0 / 3.0)
    assert abs(s.length() / L - 1) < 1e-14
    kv = s.kvecs()
    for p in range(0, nso, 3):
        k = 2 * math.pi * kv[p // 2] / L
        assert abs(s.tkin(p) - 0.5 * float(k @ k)) <= 1e-13 * max(1.0, s.tkin(p))
    for n2 in range(1, 13):
        q2 = (2 * math.pi / L) ** 2 * n2
        assert abs(s.vq(n2) / (4 * math.pi / (L ** 3 * q2)) - 1) < 1e-13
    assert s.vq(0) == 0.0


def test_ueg_hf_energy_closed_form():
    """E_HF = sum_occ |k|^2/2 - sum_{same-spin pairs} v(k_i - k_j)."""
    s = oracle.System.ueg(14, 38, 1.0, 2)
    b = brute.UEGBrute(14, 38, 1.0)
    e = 0.0
    for p in range(14):
        e += b.h1(p, p)
    for p in range(14):
        for q in range(p + 1, 14):
            if p % 2 == q % 2:
                dk = b.kvec(p) - b.kvec(q)
                e -= 4 * math.pi / (b.omega * float(dk @ dk))
    assert abs(s.ehf() - e) < 1e-12 * abs(e)


@pytest.mark.parametrize("nel,nso,lmax", [(2, 14, 2), (3, 14, 3), (4, 14, 4), (3, 38, 2), (2, 38, 2)])
def test_ueg_slater_condon_vs_second_quantisation(nel, nso, lmax):
    ham = brute.UEGBrute(nel, nso, 1.0)
    s = oracle.System.ueg(nel, nso, 1.0, lmax)
    dets = brute.sector(ham)
    H = brute.hamiltonian_matrix(ham, dets)
    Ho = np.array([[s.hij(a, b) for b in dets] for a in dets])
    assert np.max(np.abs(H - Ho)) < 1e-12 * max(1.0, np.max(np.abs(H)))


@pytest.mark.parametrize("nel,norb,seed", [(2, 4, 1), (3, 4, 2), (4, 4, 3), (4, 5, 4), (3, 5, 5)])
def test_generic_slater_condon_vs_second_quantisation(nel, norb, seed):
    h1, eri = tiny_molecule(norb=norb, nocc=max(1, nel // 2), seed=seed, scale=0.5)
    ham = brute.GenericBrute(nel, h1, eri)
    s = oracle.System.generic(nel, h1, eri, min(nel, 4))
    dets = brute.sector(ham)
    H = brute.hamiltonian_matrix(ham, dets)
    Ho = np.array([[s.hij(a, b) for b in dets] for a in dets])
    assert np.max(np.abs(H - Ho)) < 1e-12 * max(1.0, np.max(np.abs(H)))


def test_synthetic_molecule_reference_is_hartree_fock():
    """With h chosen so the Fock matrix is diagonal, Brillouin's theorem makes
    <HF|H|single> vanish and E_HF = sum_i (h_ii + e_i) over occupied orbitals."""
    from ccmc_inputs import molecule_fock_levels, molecule_integrals

    norb, nocc = 12, 3
    h1, eri = molecule_integrals(norb=norb, nocc=nocc, seed=7)
    s = oracle.System.generic(2 * nocc, h1, eri, 2)
    eps = molecule_fock_levels(norb, nocc)
    e = sum(h1[i, i] + eps[i] for i in range(nocc))
    assert abs(s.ehf() - e) < 1e-10 * max(1, abs(e))
    hf = s.hf()
    for i in range(2 * nocc):
        for a in range(2 * nocc, 2 * norb):
            if i % 2 != a % 2:
                continue
            d = hf ^ (1 << i) ^ (1 << a)
            assert abs(s.hij(hf, d)) < 1e-10


def _golden_sizes():
    out = []
    for line in open(os.path.join(GOLDEN, "ueg_space_sizes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out.append(tuple(int(x) for x in f[:4]))
    return out


@pytest.mark.parametrize("nel,nso,lmax,size", _golden_sizes())
def test_ueg_space_size_matches_paper(nel, nso, lmax, size):
    """Closing HF under the excitation generator (every draw visited) reaches
    exactly the truncated space sizes the paper prints."""
    s = oracle.System.ueg(nel, nso, 1.0, lmax)
    # at CCSD every double is one draw from HF, so the top level need not be expanded
    assert s.generator_closure(lmax, expand_top=(lmax > 2)) == size


def _random_excited(nel, nso, level, rng):
    """A determinant (int bit string) with `level` holes in the lowest nel
    spin-orbitals and `level` particles above them, any spins."""
    holes = rng.choice(nel, size=level, replace=False)
    parts = nel + rng.choice(nso - nel, size=level, replace=False)
    d = (1 << nel) - 1
    for q in list(holes) + list(parts):
        d ^= 1 << int(q)
    return d


@pytest.mark.parametrize("kind", ["ueg", "molecule", "molecule41"])
def test_excitation_form_diagonal_equals_slater_condon(kind):
    """H_DD - E_HF in the excitation form (Fock diagonal of the reference plus
    pair corrections among holes and particles) equals the difference of the
    two plain Slater-Condon diagonals <D|H|D> - <HF|H|HF>, for determinants
    of every excitation level up to 6 (spins not conserved: the identity
    holds for any determinant)."""
    from ccmc_inputs import molecule_integrals

    rng = np.random.Generator(np.random.PCG64(17))
    if kind == "ueg":
        s, nel, nso = oracle.System.ueg(14, 66, 1.0, 4), 14, 66
    elif kind == "molecule":
        h1, eri = molecule_integrals(norb=8, nocc=3, seed=5)
        s, nel, nso = oracle.System.generic(6, h1, eri, 4), 6, 16
    else:
        h1, eri = molecule_integrals(norb=41, nocc=10, seed=7)
        s, nel, nso = oracle.System.generic(20, h1, eri, 4), 20, 82
    hf = (1 << nel) - 1
    ehf = s.hij(hf, hf)
    for level in range(1, 7):
        for _ in range(40):
            d = _random_excited(nel, nso, min(level, nel, nso - nel), rng)
            direct = s.hij(d, d) - ehf
            assert abs(s.hdiag_rel(d) - direct) <= 1e-12 * max(1.0, abs(ehf)), (level, d)


def test_excitation_form_diagonal_fp32_within_single_precision():
    """The FP32 form of H_DD - E_HF agrees with the FP64 one to single
    precision of the summed terms (a dozen terms of at most a few hartree)."""
    from ccmc_inputs import molecule_integrals

    rng = np.random.Generator(np.random.PCG64(18))
    h1, eri = molecule_integrals(norb=41, nocc=10, seed=7)
    for s, nel, nso in [(oracle.System.ueg(54, 162, 1.0, 2).set_fp32(), 54, 162),
                        (oracle.System.generic(20, h1, eri, 4).set_fp32(), 20, 82)]:
        for level in range(1, 5):
            for _ in range(40):
                d = _random_excited(nel, nso, level, rng)
                e64, e32 = s.hdiag_rel(d), s.hdiag_rel_f(d)
                assert abs(e32 - e64) <= 2e-6 * (1.0 + 8 * level * 25.0), (level, e64, e32)
