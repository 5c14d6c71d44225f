"""Pins of the oracle's simulation of the paper's distribution of excitors
over processors (Sec. III, Eq. ccmc_dist; Fig. excitdistrib; Fig. bias).

* the determinant hash is Philox-4x64-10 (numpy's generator, a library
  routine) applied to the bit string, chained three words at a time;
* the owner reduces to hash(D) mod N_p when excitors never move (the paper's
  reduction of Eq. ccmc_dist to Eq. fciqmc_dist), is constant over aligned
  runs of 2^nu_move iterations, and is uniform over the processors;
* the pair co-location sums agree with a direct count, have the unbiased
  mean 1/N_p and the spread of a binomial law over the iterations whose
  terms are correlated by the moves: sqrt((N_p - 1) / N_p^2 * F / T), F the
  phased-moves factor (about 2^(nu+1)/3, against the 2^nu of moves aligned
  across excitors);
* the restricted sampler reduces to the plain one for N_p = 1 and, averaged
  over iterations (owners), its one-step mean equals the exact propagator
  action (Sec. II, Eq. CCMC): drawing the later excitors of a composite from
  the first one's processor with the weight (N_q N_p / N_ex)^(s-1) is right.
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from _systems import tiny_molecule

HASH_KEY = [0x243F6A8885A308D3, 0x13198A2E03707344]


def _numpy_block(ctr, key):
    v = sum(int(ctr[i]) << (64 * i) for i in range(4))
    v = (v - 1) % (1 << 256)
    words = np.array([(v >> (64 * i)) & (2 ** 64 - 1) for i in range(4)], dtype=np.uint64)
    return np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64)).random_raw(4)


def _numpy_hash(words):
    h = 0
    for g in range(0, len(words), 3):
        c = [int(words[g + q]) if g + q < len(words) else 0 for q in range(3)] + [h]
        h = int(_numpy_block(c, HASH_KEY)[0])
    return h


@pytest.mark.parametrize("words", [[7], [(1 << 14) - 1, 3], [2 ** 64 - 1, 5, 9], [1, 2, 3, 4, 5, 6], [0]])
def test_hash_is_chained_philox(words):
    assert oracle.det_hash(words) == _numpy_hash(words)


def test_owner_without_moves_is_the_static_hash():
    rng = np.random.default_rng(2)
    for _ in range(50):
        w = [int(x) for x in rng.integers(0, 2 ** 63, size=2)]
        for np_ in (2, 7, 32):
            p0 = oracle.owner(w, 0, 64, np_)
            assert p0 == oracle.det_hash(w) % np_
            assert all(oracle.owner(w, t, 64, np_) == p0 for t in (1, 17, 1000))


def test_owner_moves_only_every_two_to_the_nu_iterations():
    rng = np.random.default_rng(3)
    for nu in (0, 2, 4):
        for _ in range(20):
            w = [int(x) for x in rng.integers(0, 2 ** 63, size=2)]
            h = oracle.det_hash(w)
            own = [oracle.owner(w, t, nu, 97) for t in range(64)]
            for t in range(1, 64):
                if ((h + t) >> nu) == ((h + t - 1) >> nu):
                    assert own[t] == own[t - 1]
            # the phase of the moves is set by the hash: the first move is at
            # the first t with (h + t) a multiple of 2^nu
            if nu > 0:
                first = next(t for t in range(1, 64) if (h + t) % (1 << nu) == 0)
                assert all(own[t] == own[0] for t in range(first))


def test_owners_are_uniform_over_processors():
    rng = np.random.default_rng(4)
    np_ = 16
    counts = np.zeros(np_)
    for _ in range(8000):
        w = [int(x) for x in rng.integers(0, 2 ** 63, size=2)]
        counts[oracle.owner(w, int(rng.integers(0, 1000)), 3, np_)] += 1
    chi2 = (((counts - 500.0) ** 2) / 500.0).sum()
    assert chi2 < 40.0      # 15 degrees of freedom: p ~ 5e-4


def _ueg_excitors(nel, nso, lmax):
    s = oracle.System.ueg(nel, nso, 1.0, lmax)
    keys = s.space_keys(lmax, expand_top=False)[1:]
    return np.stack([s.to_words(s.unrank(int(k))) for k in keys])


def test_colocation_sums_match_direct_count():
    dets = _ueg_excitors(14, 38, 2)[:60]
    np_, nu, ck = 5, 2, [1, 7, 16, 33]
    s1, s2 = oracle.colocation(dets, np_, nu, ck)
    own = np.array([[oracle.owner(d, t, nu, np_) for d in dets] for t in range(ck[-1])])
    for k, T in enumerate(ck):
        same = (own[:T, :, None] == own[:T, None, :]).sum(axis=0)
        iu = np.triu_indices(len(dets), 1)
        c = same[iu]
        assert int(s1[k]) == int(c.sum()) and int(s2[k]) == int((c.astype(np.int64) ** 2).sum())


def _phased_moves_factor(L: int, T: int) -> float:
    """T x the variance of a pair's co-location average over T iterations,
    in units of p(1 - p), p = 1/N_p.  The owner of each excitor changes every
    L = 2^nu iterations at a phase set by its own hash (Eq. ccmc_dist), so
    the co-location of two excitors is unchanged over d iterations only when
    neither has moved: with independent uniform phases that has probability
    (1 - d/L)^2, and once either moves the new co-location is independent of
    the old.  Hence Var = p(1-p)/T^2 [T + 2 sum_{d=1}^{L-1} (T - d)(1 - d/L)^2],
    which tends to (2L^2 + 1)/(3L) for T >> L (the binomial argument with
    moves aligned across excitors would give L)."""
    return (T + 2.0 * sum((T - d) * (1.0 - d / L) ** 2 for d in range(1, min(L, T)))) / T


def test_phased_moves_factor_limits():
    assert _phased_moves_factor(1, 100) == 1.0
    for L in (2, 16, 64):
        assert abs(_phased_moves_factor(L, 10 ** 7) - (2 * L * L + 1) / (3 * L)) < 1e-3 * L


@pytest.mark.parametrize("np_,nu", [(8, 0), (8, 3), (32, 2), (5, 4)])
def test_colocation_mean_and_spread_scaling(np_, nu):
    """Fig. excitdistrib: the mean co-location probability is unbiased (1/N_p)
    and its spread over pairs follows the binomial law of p = 1/N_p over the
    iterations, with the moves every 2^nu iterations correlating them (the
    phased-moves factor above; an aligned-moves or an uncorrelated law would
    be off by 22 % or more for nu >= 3)."""
    dets = _ueg_excitors(14, 38, 2)[:200]
    T = 512
    s1, s2 = oracle.colocation(dets, np_, nu, [T])
    P = len(dets) * (len(dets) - 1) / 2
    mean = float(s1[0]) / (P * T)
    var = float(s2[0]) / (P * T * T) - mean * mean
    assert abs(mean * np_ - 1.0) < 0.05
    p = 1.0 / np_
    expect = np.sqrt(p * (1 - p) * _phased_moves_factor(2 ** nu, T) / T)
    assert abs(np.sqrt(var) / expect - 1.0) < 0.03


def test_one_rank_is_the_plain_step():
    h1, eri = tiny_molecule(norb=5, nocc=2, seed=11, scale=0.3)
    s = oracle.System.generic(4, h1, eri, 2)
    a = oracle.Sim(s, tau=0.01, target_pop=300, d0_init=50, seed=3)
    b = oracle.Sim(s, tau=0.01, target_pop=300, d0_init=50, seed=3, n_ranks=1, nu_move=0)
    assert a.run(300) == b.run(300)


def test_distributed_step_mean_equals_exact_action():
    """With 3 simulated processors moving every iteration, the mean of one
    step over many iterations (owner configurations) and Philox keys equals
    the exact action of the propagator: a composite cluster's later excitors
    come from the first one's processor q only, and its amplitude carries
    (N_q N_p / N_ex)^(s-1) (selection within q, co-location probability
    N_p^-(s-1) averaged over owners)."""
    tau, shift = 0.01, 0.3
    h1, eri = tiny_molecule(norb=5, nocc=2, seed=11, scale=0.3)
    ham = brute.GenericBrute(4, h1, eri)
    s = oracle.System.generic(4, h1, eri, 2)
    efci, dets, H = brute.fci_energy(ham)
    rng = np.random.default_rng(3)
    hf = (1 << 4) - 1
    lst = sorted((d for d in dets if brute.level(d, 4) <= 2), key=s.rank)
    keep, pops = [hf], [int(40.0 * 65536)]
    for d in lst[1:]:
        if rng.random() < 0.7:
            keep.append(d)
            v = int(rng.normal() * 40.0 / 3 * 65536)
            pops.append(v if v != 0 else 65536)
    amps = {d: p / 65536 for d, p in zip(keep[1:], pops[1:])}
    exact = brute.exact_step_change(ham, dets, H, amps, pops[0] / 65536, tau, shift, s.ehf(), s.lmax)
    keys = {s.rank(d): i for i, d in enumerate(lst)}
    pos = {d: i for i, d in enumerate(lst)}
    K = 4000
    acc = np.zeros((K, len(lst)))
    sim = oracle.Sim(s, tau=tau, seed=11, n_ranks=3, nu_move=0)
    sim.set_list(keep, pops)
    dropped = 0
    for k in range(K):
        sim.set_state(k, shift, False, 1.0)
        sim.step(propagate_only=True)
        dk, dp = sim.spawned()
        np.add.at(acc[k], [keys[int(x)] for x in dk], dp / 65536.0)
        for d, v in zip(keep, sim.death()):
            acc[k, pos[d]] += v / 65536.0
    mean, se = acc.mean(0), acc.std(0, ddof=1) / np.sqrt(K)
    ex = np.array([exact[d] for d in lst])
    z = (mean - ex) / np.maximum(se, 1e-12)
    assert np.max(np.abs(z)) < 5.0, (np.max(np.abs(z)), np.argmax(np.abs(z)))
