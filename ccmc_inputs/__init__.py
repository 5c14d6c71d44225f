"""Seeded, synthetic inputs shared by the CUDA library's callers and the oracle.

This module holds workload descriptions and input generators only: no part of
the CCMC step lives here.  The paper's own systems (water, benzene) need
integrals that are not available, so the workloads are a uniform electron gas
(closed-form integrals) and a synthetic molecule-like Hamiltonian generated
from a fixed seed.
"""
from __future__ import annotations

import copy

import numpy as np

# Run parameters common to every workload.
COMMON = dict(
    d0_init=100.0,        # initial weight on the reference (unit-weight particles, Sec. II)
    shift_a=10,           # steps between shift updates
    zeta=0.05,            # shift damping
    spawn_cutoff=2.0 ** -7,
    a_thresh=1.0,         # multi-spawn threshold (the paper uses 1, Sec. IV.C)
    fnc=False,
    multispawn=False,
    replica=0,
    precision="fp64",
)

WORKLOADS = {
    # UEG 14 e / 38 spin-orbitals (19 plane waves), CCSD, original sampling
    "ueg14_m38_ccsd": dict(kind="ueg", nel=14, nso=38, rs=1.0, lmax=2, target_pop=2.0e4,
                           tau=0.01, nsteps=200, seed=1),
    # UEG 14 e / 114 spin-orbitals (57 plane waves), CCSDT, full non-composite + multi-spawn
    "ueg14_m114_ccsdt_fnc_ms": dict(kind="ueg", nel=14, nso=114, rs=1.0, lmax=3, target_pop=1.0e6,
                                    tau=0.005, nsteps=2000, seed=1, fnc=True, multispawn=True),
    # synthetic molecule: 20 e in 41 spatial orbitals (82 spin-orbitals), CCSDTQ.
    # With these integrals (N(0,1) magnitudes) the spawned weight per step
    # is about tau * 2.5e3 E_h times the population, and the shift, updated
    # every shift_a steps with damping zeta, holds the population only when
    # shift_a * tau * 2.5e3 is well below zeta: tau = 2e-6.  Every population
    # reachable on one GPU is then below the annihilation plateau, so the
    # wavefunction is noise-dominated; the reference starts with 2e6
    # particles so that it keeps a sizeable share through the timed window.
    # (molecule_state gives a separate full-size synthetic list for parity
    # tests of single steps.)
    "mol20_m82_ccsdtq": dict(kind="generic", nel=20, norb=41, lmax=4, target_pop=1.0e7,
                             tau=2.0e-6, nsteps=50, seed=1, molecule_seed=7, d0_init=2.0e6,
                             equilibrate=400, list_capacity=40_000_000, state_seed=31),
    # UEG 14 e / 66 spin-orbitals (33 plane waves), CCSDT with full
    # non-composite sampling, r_s = 0.5 and 5: the systems of the paper's
    # parallelisation-bias study (Sec. III.B, Fig. bias; CISDT space 22,969),
    # run with the simulated distribution over processors (n_ranks, nu_move).
    "ueg14_m66_ccsdt_rs0.5": dict(kind="ueg", nel=14, nso=66, rs=0.5, lmax=3, target_pop=2.0e5,
                                  tau=0.001, nsteps=20000, seed=1, fnc=True, d0_init=1.0e3),
    "ueg14_m66_ccsdt_rs5": dict(kind="ueg", nel=14, nso=66, rs=5.0, lmax=3, target_pop=2.0e5,
                                tau=0.001, nsteps=20000, seed=1, fnc=True, d0_init=1.0e3),
    # UEG 14 e / 358 spin-orbitals (179 plane waves, |n|^2 <= 12; six-word
    # determinants), r_s = 1, CCSDTQ: the system of the paper's published
    # correlation energy (Sec. III.B), full non-composite + multi-spawn.
    "ueg14_m358_ccsdtq": dict(kind="ueg", nel=14, nso=358, rs=1.0, lmax=4, target_pop=3.0e7,
                              tau=0.003, nsteps=20000, seed=1, fnc=True, multispawn=True, d0_init=1.0e4),
    # UEG 54 e / 162 spin-orbitals (81 plane waves), CCSD, FP32 matrix elements.
    # 10^4 initial particles on HF: from 100 the original sampler stays below
    # the shoulder on this system and the population blows up.  Grown at 1% of
    # the target, then every population is scaled up to the target.
    "ueg54_m162_ccsd_fp32": dict(kind="ueg", nel=54, nso=162, rs=1.0, lmax=2, target_pop=1.0e8,
                                 tau=0.01, nsteps=50, seed=1, precision="fp32", grow_fraction=0.01,
                                 d0_init=1.0e4),
}


def workload(name: str, **overrides) -> dict:
    """A complete parameter dictionary for one named workload."""
    w = copy.deepcopy(COMMON)
    w.update(WORKLOADS[name])
    w.update(overrides)
    w["name"] = name
    return w


def batched_replicas(n: int = 64) -> list[dict]:
    """Replica r: M in {38, 54, 66, 114} x r_s in {0.5, 1, 2, 5} by r mod 16,
    CCSD when floor(r/16) is even else CCSDT, target 10^(4 + r mod 3),
    seed 1000 + r, with two exceptions found by running every replica alone
    for 8000 steps: CCSDT at M = 114 did not settle at these populations (at
    r_s = 5 not even at 10^6; the population blew up within 1000-4000 steps),
    so M = 114 replicas are CCSD throughout; and CCSDT at M = 66, r_s = 5
    needs 10^6 excitors to settle.  Lists get room for 8x the target."""
    out = []
    ms = [38, 54, 66, 114]
    rss = [0.5, 1.0, 2.0, 5.0]
    for r in range(n):
        c = r % 16
        m, rs = ms[c // 4], rss[c % 4]
        lmax = 3 if (r // 16) % 2 == 1 and m < 114 else 2
        target = 10.0 ** (4 + r % 3)
        if lmax == 3 and m == 66 and rs == 5.0:
            target = 1.0e6
        w = copy.deepcopy(COMMON)
        w.update(kind="ueg", nel=14, nso=m, rs=rs, lmax=lmax, target_pop=target, tau=0.01, nsteps=100,
                 seed=1000 + r, replica=r, list_capacity=int(8 * target) + 65536, name=f"batched_r{r}")
        out.append(w)
    return out


# ---------------------------------------------------------------------------
# Synthetic molecule-like Hamiltonian
# ---------------------------------------------------------------------------


def molecule_fock_levels(norb: int = 41, nocc: int = 10) -> np.ndarray:
    """Orbital energies spaced like a water-dimer-sized basis: two deep core
    levels (fewer if nocc < 2), the remaining occupied levels evenly in
    [-1.4, -0.45] and the virtual levels evenly in [0.15, 3.0] hartree."""
    ncore = min(2, nocc)
    core = np.array([-20.6, -20.5])[:ncore]
    val = np.linspace(-1.4, -0.45, nocc - ncore)
    virt = np.linspace(0.15, 3.0, norb - nocc)
    return np.concatenate([core, val, virt])


def molecule_integrals(norb: int = 41, nocc: int = 10, seed: int = 7, scale: float = 1.0):
    """Return (h1[norb,norb], eri[norb,norb,norb,norb]) with 8-fold symmetric
    chemists' integrals (pq|rs) = scale g exp(-(|p-q| + |r-s|)/8), g ~ N(0,1)
    drawn in canonical order (p>=q, r>=s, pq>=rs) from PCG64(seed), and h1
    chosen so that the closed-shell Fock matrix of the lowest nocc orbitals is
    diagonal with the levels of molecule_fock_levels:
    h_pq = e_p d_pq - sum_j [2 (pq|jj) - (pj|jq)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eri = np.zeros((norb,) * 4)
    for p in range(norb):
        for q in range(p + 1):
            pq = p * (p + 1) // 2 + q
            for r in range(norb):
                for s in range(r + 1):
                    rs_ = r * (r + 1) // 2 + s
                    if rs_ > pq:
                        continue
                    v = scale * rng.standard_normal() * np.exp(-((p - q) + (r - s)) / 8.0)
                    for a, b, c, d in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                       (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                        eri[a, b, c, d] = v
    eps = molecule_fock_levels(norb, nocc)
    occ = np.arange(nocc)
    g = 2.0 * np.einsum("pqjj->pq", eri[:, :, occ][:, :, :, occ]) - np.einsum("pjjq->pq", eri[:, occ][:, :, occ])
    h1 = np.diag(eps) - g
    h1 = 0.5 * (h1 + h1.T)
    return h1, eri


def synthetic_populations(levels, n_total: float, seed: int, ref_fraction: float = 0.2) -> np.ndarray:
    """Seeded fixed-point populations (multiples of 2^-16) for a list whose
    first entry is the reference: the reference holds ref_fraction of
    n_total; the others share the rest with lognormal magnitudes that fall by
    10x per excitation level above 2, random signs, and at least one particle
    each (the occupation threshold of a converged list)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    levels = np.asarray(levels)
    n = len(levels)
    w = np.exp(rng.standard_normal(n)) * 10.0 ** (-(np.maximum(levels, 2) - 2))
    w[0] = 0.0
    w *= (1.0 - ref_fraction) * n_total / w.sum()
    w = np.maximum(w, 1.0)
    pops = np.round(w * 65536.0).astype(np.int64)
    signs = np.where(rng.random(n) < 0.5, -1, 1)
    pops = pops * signs
    pops[0] = int(round(ref_fraction * n_total * 65536.0))
    return pops


def random_excitors(norb: int, nocc: int, level: int, count: int, rng) -> np.ndarray:
    """count determinants drawn uniformly from the S_z-conserving level-`level`
    excitations of the closed-shell reference (nocc doubly occupied spatial
    orbitals out of norb; spin-orbital 2p is alpha, 2p+1 beta), as
    [count, ceil(2 norb / 64)] uint64 words (bit q of word q // 64).  Repeats
    are possible."""
    nvir = norb - nocc
    nw = (2 * norb + 63) // 64
    # number of alpha holes a: weight C(nocc,a) C(nocc,L-a) C(nvir,a) C(nvir,L-a)
    from math import comb

    wts = np.array([comb(nocc, a) * comb(nocc, level - a) * comb(nvir, a) * comb(nvir, level - a)
                    for a in range(level + 1)], dtype=np.float64)
    na = rng.choice(level + 1, size=count, p=wts / wts.sum())
    words = np.zeros((count, nw), dtype=np.uint64)
    hf = np.zeros(nw, dtype=np.uint64)
    for q in range(2 * nocc):
        hf[q // 64] |= np.uint64(1) << np.uint64(q % 64)
    words[:] = hf
    for a in range(level + 1):
        rows = np.nonzero(na == a)[0]
        if len(rows) == 0:
            continue
        picks = []
        for spin, k in ((0, a), (1, level - a)):
            if k == 0:
                continue
            holes = np.argsort(rng.random((len(rows), nocc)), axis=1)[:, :k]
            parts = nocc + np.argsort(rng.random((len(rows), nvir)), axis=1)[:, :k]
            picks += [2 * holes + spin, 2 * parts + spin]
        if not picks:
            continue
        idx = np.concatenate(picks, axis=1).astype(np.uint64)   # flipped spin-orbitals (all distinct)
        for w in range(nw):
            inw = (idx // np.uint64(64)) == np.uint64(w)
            bit = np.where(inw, np.left_shift(np.uint64(1), idx % np.uint64(64)), np.uint64(0))
            words[rows, w] ^= np.bitwise_or.reduce(bit, axis=1)
    return words


def molecule_state(norb: int = 41, nocc: int = 10, draws=None, n_total: float = 1.0e7, seed: int = 31,
                   ref_fraction: float = 0.3):
    """A full-size synthetic CCSDTQ list for the molecule-like Hamiltonian:
    the reference plus distinct excitors drawn uniformly per level (draws =
    {level: count}, repeats removed), in canonical order (unsigned bit-string
    order, most significant word first), with synthetic_populations weights.
    Returns (words [n, nw] uint64, pops int64, levels)."""
    if draws is None:
        draws = {1: 4000, 2: 400_000, 3: 1_500_000, 4: 2_500_000}
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [random_excitors(norb, nocc, lv, c, rng) for lv, c in sorted(draws.items())]
    hf = random_excitors(norb, nocc, 0, 1, rng)
    words = np.concatenate([hf] + parts, axis=0)
    order = np.lexsort(tuple(words[:, w] for w in range(words.shape[1])))   # last word is the primary key
    words = words[order]
    keep = np.ones(len(words), dtype=bool)
    keep[1:] = np.any(words[1:] != words[:-1], axis=1)
    words = words[keep]
    hfw = hf[0]
    flips = np.zeros(len(words), dtype=np.int64)
    for w in range(words.shape[1]):
        x = np.ascontiguousarray(words[:, w] ^ hfw[w])
        flips += np.unpackbits(x.view(np.uint8).reshape(-1, 8), axis=1).sum(axis=1).astype(np.int64)
    levels = flips // 2
    assert np.array_equal(words[0], hfw) and levels[0] == 0
    pops = synthetic_populations(levels, n_total, seed, ref_fraction)
    return words, pops, levels
