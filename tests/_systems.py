"""Tiny systems shared by the oracle pin tests."""
import numpy as np

from ccmc_inputs import molecule_integrals


def tiny_molecule(norb=4, nocc=2, seed=3, scale=0.1):
    """A small 8-fold symmetric random Hamiltonian (weak coupling)."""
    return molecule_integrals(norb=norb, nocc=nocc, seed=seed, scale=scale)


def all_dets(nel, nso):
    import itertools

    return sorted(sum(1 << p for p in occ) for occ in itertools.combinations(range(nso), nel))
