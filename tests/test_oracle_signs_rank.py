"""Pins of excitor signs, cluster collapse and the order-preserving rank key."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import brute
from _systems import all_dets


@pytest.mark.parametrize("nel,nso", [(2, 8), (3, 8), (4, 10), (5, 12)])
def test_excitor_sign_matches_operator_string(nel, nso):
    """s_D(i) = <D_i|c_i|D_HF> with c_i = a+_a a+_b ... a_j a_i (Sec. II Eq. 3-5)."""
    h1 = np.eye(nso // 2)
    eri = np.zeros((nso // 2,) * 4)
    s = oracle.System.generic(nel, h1, eri, min(nel, 4))
    for d in all_dets(nel, nso):
        if brute.level(d, nel) > min(nel, 4):
            continue
        assert s.excitor_sign(d) == brute.excitor_sign(d, nel)
        assert s.level(d) == brute.level(d, nel)


def _tiny_system(nel=4, nso=10, lmax=4):
    h1 = np.eye(nso // 2)
    eri = np.zeros((nso // 2,) * 4)
    return oracle.System.generic(nel, h1, eri, lmax)


def test_collapse_matches_operator_product_and_is_order_independent():
    """prod_e c_e |HF> = sigma |D>: same result as applying the literal excitor
    strings, zero when excitors share an orbital, and the same for every order
    of the excitors (excitors are products of an even number of operators)."""
    nel, nso = 4, 10
    s = _tiny_system(nel, nso)
    hf = (1 << nel) - 1
    exc = [d for d in all_dets(nel, nso) if 1 <= brute.level(d, nel) <= 2]
    rng = np.random.default_rng(0)
    nonzero = 0
    for trial in range(1200):
        k = int(rng.integers(2, 4))
        picks = [exc[i] for i in rng.choice(len(exc), size=k, replace=False)]
        res = s.collapse(picks)
        ops = []
        for e in picks:
            ops += brute.excitor_ops(e, nel)
        sg, d = brute.apply_ops(ops, hf)
        if sg == 0:
            assert res is None
            continue
        nonzero += 1
        assert res == (d, sg)
        for perm in itertools.permutations(picks):
            assert s.collapse(list(perm)) == res
    assert nonzero > 60


@pytest.mark.parametrize("nel,nso,lmax", [(4, 12, 2), (4, 12, 3), (4, 12, 4), (3, 14, 2), (6, 14, 3)])
def test_rank_key_is_order_isomorphism(nel, nso, lmax):
    """Keys of all determinants of level <= l increase strictly with the
    bit-string order, HF has key 0, and unrank inverts rank."""
    s = _tiny_system(nel, nso, lmax)
    dets = [d for d in all_dets(nel, nso) if brute.level(d, nel) <= lmax]
    keys = [s.rank(d) for d in dets]
    assert keys[0] == 0 and dets[0] == (1 << nel) - 1
    assert all(a < b for a, b in zip(keys, keys[1:]))
    assert max(keys) < s.key_bound()
    for d, k in zip(dets, keys):
        assert s.unrank(k) == d


def test_rank_key_large_words():
    """Across word boundaries (M = 162, three words) rank order still follows
    bit-string order on random determinants."""
    s = oracle.System.ueg(54, 162, 1.0, 2)
    rng = np.random.default_rng(2)
    dets = set()
    hf = (1 << 54) - 1
    while len(dets) < 400:
        n = int(rng.integers(0, 3))
        holes = rng.choice(54, size=n, replace=False)
        parts = rng.choice(np.arange(54, 162), size=n, replace=False)
        d = hf
        for h in holes:
            d ^= 1 << int(h)
        for p in parts:
            d |= 1 << int(p)
        dets.add(d)
    dets = sorted(dets)
    keys = [s.rank(d) for d in dets]
    assert all(a < b for a, b in zip(keys, keys[1:]))
    assert all(s.unrank(k) == d for d, k in zip(dets, keys))
