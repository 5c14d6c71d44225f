"""Pins of the excitation generators by exhaustive enumeration of every draw."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from _systems import tiny_molecule


def _draw_outcomes(s, dj, n0, n1, n2_of):
    """Visit every (type, first, second) draw; returns {det: Fraction} with None for null."""
    out = {}
    for t, pt in n0:
        for i1 in range(n1(t)):
            n2 = n2_of(t, i1)
            for i2 in range(n2):
                r = [t, brute.r_for_index(i1, n1(t)), brute.r_for_index(i2, n2), 0]
                res = s.excite(dj, r)
                key = None if res is None else res[0]
                out[key] = out.get(key, Fraction(0)) + pt / (n1(t) * n2)
                if res is not None:
                    assert abs(res[1] - s.hij(res[0], dj)) == 0.0
    return out


def _connected_doubles_ueg(b, dj, nel, nso):
    occ = [p for p in range(nso) if (dj >> p) & 1]
    vir = [p for p in range(nso) if not (dj >> p) & 1]
    out = set()
    for i, j in itertools.combinations(occ, 2):
        for a, c in itertools.combinations(vir, 2):
            d = dj ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << c)
            if brute.sz_of(d) == brute.sz_of(dj) and b.total_momentum(d) == b.total_momentum(dj):
                out.add(d)
    return out


@pytest.mark.parametrize("nel,nso", [(4, 14), (3, 38), (14, 38)])
def test_ueg_generator_exhaustive(nel, nso):
    """Every momentum- and spin-conserving double excitation is produced with
    p_gen = 2/(C(N,2)(M-N)) exactly; the rest of the probability is null."""
    s = oracle.System.ueg(nel, nso, 1.0, 4 if nel < 14 else 2)
    b = brute.UEGBrute(nel, nso, 1.0)
    npairs, nvirt = nel * (nel - 1) // 2, nso - nel
    pgen = Fraction(2, npairs * nvirt)
    hf = (1 << nel) - 1
    starts = [hf]
    for d in sorted(_connected_doubles_ueg(b, hf, nel, nso))[:3]:
        starts.append(d)
    for dj in starts:
        out = _draw_outcomes(s, dj, [(0, Fraction(1))], lambda t: npairs, lambda t, i1: nvirt)
        want = _connected_doubles_ueg(b, dj, nel, nso)
        got = {k for k in out if k is not None}
        assert got == want
        for k in got:
            assert out[k] == pgen
        assert sum(out.values()) == 1
        # 1/p_gen reported by the generator
        for i1 in range(npairs):
            r = [0, brute.r_for_index(i1, npairs), brute.r_for_index(0, nvirt), 0]
            res = s.excite(dj, r)
            if res is not None:
                assert res[2] == float(1 / pgen)


def _spin_orbitals(dj, nso, spin, occupied):
    return [p for p in range(nso) if p % 2 == spin and bool((dj >> p) & 1) == occupied]


@pytest.mark.parametrize("nel,norb", [(4, 5), (3, 5), (6, 6)])
def test_generic_generator_exhaustive(nel, norb):
    """Singles with probability p_s/(N n_virt(spin)) and doubles with
    (1-p_s)/(C(N,2) n_pairs(spins)), p_s = n_S/(n_S+n_D) counted at HF; all
    spin-conserving singles and doubles are reachable; sums to one exactly."""
    h1, eri = tiny_molecule(norb=norb, nocc=max(1, nel // 2), seed=norb, scale=0.3)
    s = oracle.System.generic(nel, h1, eri, min(nel, 4))
    nso = 2 * norb
    hf = (1 << nel) - 1
    no = [len(_spin_orbitals(hf, nso, sg, True)) for sg in (0, 1)]
    nv = [norb - no[0], norb - no[1]]
    from math import comb

    ns = no[0] * nv[0] + no[1] * nv[1]
    nd = comb(no[0], 2) * comb(nv[0], 2) + comb(no[1], 2) * comb(nv[1], 2) + no[0] * no[1] * nv[0] * nv[1]
    ps = Fraction(ns, ns + nd)
    npairs = comb(nel, 2)
    r_single = brute.r_for_index(0, ns + nd)
    r_double = brute.r_for_index(ns, ns + nd)

    va = nel if nel % 2 == 0 else nel + 1      # first alpha virtual
    vb = nel if nel % 2 == 1 else nel + 1      # first beta virtual
    # HF, an alpha single and an alpha-beta double: all in the reference's S_z sector
    for dj in [hf, hf ^ 1 ^ (1 << va), hf ^ 0b11 ^ (1 << va) ^ (1 << vb)]:
        occ = [p for p in range(nso) if (dj >> p) & 1]

        def n1(t):
            return nel if t == r_single else npairs

        def n2_of(t, i1):
            if t == r_single:
                return nv[occ[i1] % 2]
            x, y = _pair(i1)
            si, sj = occ[x] % 2, occ[y] % 2
            if si == sj:
                return comb(nv[si], 2)
            return nv[0] * nv[1]

        out = _draw_outcomes(s, dj, [(r_single, ps), (r_double, 1 - ps)], n1, n2_of)
        assert sum(out.values()) == 1
        # expected probabilities by direct counting
        want = {}
        for i in occ:
            for a in _spin_orbitals(dj, nso, i % 2, False):
                d = dj ^ (1 << i) ^ (1 << a)
                want[d] = want.get(d, 0) + ps / (nel * nv[i % 2])
        for i, j in itertools.combinations(occ, 2):
            si, sj = i % 2, j % 2
            if si == sj:
                pairs = list(itertools.combinations(_spin_orbitals(dj, nso, si, False), 2))
            else:
                pairs = list(itertools.product(_spin_orbitals(dj, nso, 0, False), _spin_orbitals(dj, nso, 1, False)))
            for a, c in pairs:
                d = dj ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << c)
                want[d] = want.get(d, 0) + (1 - ps) / (npairs * len(pairs))
        got = {k: v for k, v in out.items() if k is not None}
        assert got == want


def _pair(idx):
    y = 1
    while (y + 1) * y // 2 <= idx:
        y += 1
    return idx - y * (y - 1) // 2, y
