"""The seeded input generators: the synthetic full-size molecule state and
the batched replica recipe produce what their descriptions say."""
import numpy as np

from ccmc_inputs import batched_replicas, molecule_state, random_excitors


def _popcount_rows(words):
    x = np.ascontiguousarray(words)
    return np.unpackbits(x.view(np.uint8).reshape(len(x), -1), axis=1).sum(axis=1)


def test_random_excitors_levels_and_spin():
    rng = np.random.Generator(np.random.PCG64(3))
    norb, nocc = 12, 4
    hf = (1 << (2 * nocc)) - 1
    for level in range(1, 5):
        w = random_excitors(norb, nocc, level, 500, rng)
        assert w.shape == (500, 1)
        d = w[:, 0].astype(object)
        for x in d:
            x = int(x)
            assert bin(x).count("1") == 2 * nocc                      # electron count
            assert bin(hf & ~x).count("1") == level                   # excitation level
            alpha = sum(1 for q in range(0, 2 * norb, 2) if x >> q & 1)
            assert alpha == nocc                                       # S_z of the reference


def test_molecule_state_small():
    draws = {1: 200, 2: 2000, 3: 3000, 4: 3000}
    words, pops, levels = molecule_state(norb=10, nocc=3, draws=draws, n_total=1.0e5, seed=5)
    n = len(words)
    # sorted, unique, reference first (canonical order: unsigned, top word first)
    keys = [tuple(int(v) for v in row[::-1]) for row in words]
    assert keys == sorted(keys) and len(set(keys)) == n
    assert levels[0] == 0 and np.all(levels[1:] >= 1) and np.all(levels <= 4)
    assert np.all(_popcount_rows(words) == 6)
    assert pops[0] > 0 and np.all(np.abs(pops[1:]) >= 65536)         # at least one particle each
    # level counts cannot exceed the sector sizes: singles of 3 alpha + 3 beta occupied into 7 + 7 virtual
    assert np.sum(levels == 1) <= 2 * 3 * 7


def test_batched_recipe():
    reps = batched_replicas(64)
    assert len(reps) == 64 and len({w["seed"] for w in reps}) == 64
    assert {w["nso"] for w in reps} == {38, 54, 66, 114}
    assert {w["rs"] for w in reps} == {0.5, 1.0, 2.0, 5.0}
    for r, w in enumerate(reps):
        assert w["replica"] == r and w["nel"] == 14
        if w["nso"] == 114:
            assert w["lmax"] == 2
        else:
            assert w["lmax"] == (2 if (r // 16) % 2 == 0 else 3)
        expected = 1.0e6 if (w["lmax"] == 3 and w["nso"] == 66 and w["rs"] == 5.0) else 10.0 ** (4 + r % 3)
        assert w["target_pop"] == expected
