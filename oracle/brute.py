"""Brute-force references that pin the oracle (test infrastructure only).

Nothing here calls the C oracle; these are independent, literal restatements
of the textbook definitions the paper relies on, for tiny systems only:

* second quantisation on occupation-number bit strings (Sec. II, Eq. 3-4:
  determinants are a+_{i1} a+_{i2} ... |0> with i1 < i2 < ..., excitors are
  a+_a a+_b ... a_j a_i with i < j < ..., a < b < ...);
* the Hamiltonian H = sum h_pq a+_p a_q + 1/2 sum <pq|rs> a+_p a+_q a_s a_r
  built by applying operator strings, and its lowest eigenvalue (FCI);
* the coupled cluster wavefunction t_HF exp(T/t_HF)|HF> (Sec. II, Eq. 2) by
  repeated application of T, the deterministic truncated CC equations, and
  the exact expected change of one propagator step (Sec. II, Eq. CCMC);
* reblocking (Flyvbjerg & Petersen, J. Chem. Phys. 91, 461 (1989)) with the
  optimal-block rule of Lee, Needs & Foulkes, Phys. Rev. E 83, 066706 (2011).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Operator strings on bit-string determinants (python ints, bit p = orbital p)
# ---------------------------------------------------------------------------


def apply_ops(ops, det):
    """Apply an operator product written left to right, e.g.
    [('+', a), ('+', b), ('-', j), ('-', i)] = a+_a a+_b a_j a_i; the rightmost
    operator acts first.  Returns (sign, det) or (0, None) if it vanishes."""
    sign = 1
    for kind, p in reversed(ops):
        occ = (det >> p) & 1
        below = bin(det & ((1 << p) - 1)).count("1")
        if kind == "-":
            if not occ:
                return 0, None
            det ^= 1 << p
        else:
            if occ:
                return 0, None
            det |= 1 << p
        if below & 1:
            sign = -sign
    return sign, det


def excitor_ops(det, nel):
    """Operator string of the excitor c_i that maps HF to det (Sec. II Eq. 3):
    creators of the particles a<b<..<e, then annihilators of holes l..j i."""
    hf = (1 << nel) - 1
    holes = [p for p in range(nel) if not (det >> p) & 1]
    parts = [p for p in range(det.bit_length()) if (det >> p) & 1 and not (hf >> p) & 1]
    ops = [("+", a) for a in parts] + [("-", i) for i in reversed(holes)]
    return ops


def excitor_sign(det, nel):
    """s_D(i) = <D_i|c_i|D_HF> (Sec. II, Eq. 5)."""
    sg, d = apply_ops(excitor_ops(det, nel), (1 << nel) - 1)
    assert d == det
    return sg


def popcount(x):
    return bin(x).count("1")


def level(det, nel):
    return nel - popcount(det & ((1 << nel) - 1))


# ---------------------------------------------------------------------------
# Hamiltonians
# ---------------------------------------------------------------------------


class UEGBrute:
    """Uniform electron gas: plane waves k = 2 pi n/L sorted by (|n|^2, n),
    Coulomb 4 pi/(Omega |q|^2) without q = 0, kinetic |k|^2/2."""

    def __init__(self, nel, nso, rs):
        self.nel, self.nso, self.rs = nel, nso, rs
        npw = nso // 2
        vecs = []
        r = 4
        for v in itertools.product(range(-r, r + 1), repeat=3):
            vecs.append(v)
        vecs.sort(key=lambda v: (v[0] ** 2 + v[1] ** 2 + v[2] ** 2, v))
        self.kv = vecs[:npw]
        n2last = sum(c * c for c in self.kv[-1])
        n2next = sum(c * c for c in vecs[npw])
        assert n2next > n2last, "basis size does not close a shell"
        self.L = rs * (4.0 * math.pi * nel / 3.0) ** (1.0 / 3.0)
        self.omega = self.L ** 3

    def kvec(self, p):
        n = self.kv[p // 2]
        return np.array([2.0 * math.pi * c / self.L for c in n])

    def h1(self, p, q):
        if p != q:
            return 0.0
        k = self.kvec(p)
        return 0.5 * float(k @ k)

    def g(self, p, q, r, s):
        """<pq|rs> for spin-orbitals."""
        if p % 2 != r % 2 or q % 2 != s % 2:
            return 0.0
        np_, nq, nr, ns = (np.array(self.kv[x // 2]) for x in (p, q, r, s))
        if not np.array_equal(np_ + nq, nr + ns):
            return 0.0
        qv = self.kvec(p) - self.kvec(r)
        q2 = float(qv @ qv)
        if q2 == 0.0:
            return 0.0
        return 4.0 * math.pi / (self.omega * q2)

    def g_items(self):
        """Nonzero <pq|rs>, using momentum conservation to find s."""
        where = {tuple(v): i for i, v in enumerate(self.kv)}
        out = {}
        for p, q, r in itertools.product(range(self.nso), repeat=3):
            ns = tuple(np.array(self.kv[p // 2]) + np.array(self.kv[q // 2]) - np.array(self.kv[r // 2]))
            if ns not in where:
                continue
            for sp in (0, 1):
                t = 2 * where[ns] + sp
                v = self.g(p, q, r, t)
                if v != 0.0:
                    out[(p, q, r, t)] = v
        return out

    def total_momentum(self, det):
        t = np.zeros(3, dtype=int)
        for p in range(self.nso):
            if (det >> p) & 1:
                t += np.array(self.kv[p // 2])
        return tuple(int(c) for c in t)


class GenericBrute:
    """Spin-orbital integrals from spatial h1[p,q] and chemists' (pq|rs)."""

    def __init__(self, nel, h1, eri):
        self.nel = nel
        self.h = np.asarray(h1)
        self.eri = np.asarray(eri)
        self.nso = 2 * self.h.shape[0]

    def h1(self, p, q):
        if p % 2 != q % 2:
            return 0.0
        return float(self.h[p // 2, q // 2])

    def g(self, p, q, r, s):
        if p % 2 != r % 2 or q % 2 != s % 2:
            return 0.0
        return float(self.eri[p // 2, r // 2, q // 2, s // 2])

    def g_items(self):
        out = {}
        for p, q, r, t in itertools.product(range(self.nso), repeat=4):
            v = self.g(p, q, r, t)
            if v != 0.0:
                out[(p, q, r, t)] = v
        return out

    def total_momentum(self, det):
        return (0, 0, 0)


def sz_of(det):
    na = sum(1 for p in range(0, det.bit_length(), 2) if (det >> p) & 1)
    nb = sum(1 for p in range(1, det.bit_length(), 2) if (det >> p) & 1)
    return na - nb


def sector(ham):
    """All N-electron determinants with the reference's S_z and momentum."""
    nel, nso = ham.nel, ham.nso
    hf = (1 << nel) - 1
    want = (sz_of(hf), ham.total_momentum(hf))
    dets = []
    for occ in itertools.combinations(range(nso), nel):
        d = sum(1 << p for p in occ)
        if (sz_of(d), ham.total_momentum(d)) == want:
            dets.append(d)
    dets.sort()
    return dets


def hamiltonian_matrix(ham, dets):
    """<D_a|H|D_b> by literal application of every operator string."""
    index = {d: i for i, d in enumerate(dets)}
    n = len(dets)
    H = np.zeros((n, n))
    nso = ham.nso
    g = ham.g_items()
    for b, d in enumerate(dets):
        occ = [p for p in range(nso) if (d >> p) & 1]
        for p in range(nso):
            for q in occ:
                v = ham.h1(p, q)
                if v == 0.0:
                    continue
                sg, d2 = apply_ops([("+", p), ("-", q)], d)
                if sg and d2 in index:
                    H[index[d2], b] += v * sg
        for (p, q, r, s), v in g.items():
            if not ((d >> r) & 1 and (d >> s) & 1) or r == s:
                continue
            sg, d2 = apply_ops([("+", p), ("+", q), ("-", s), ("-", r)], d)
            if sg and d2 in index:
                H[index[d2], b] += 0.5 * v * sg
    return H


def fci_energy(ham):
    dets = sector(ham)
    H = hamiltonian_matrix(ham, dets)
    w, v = np.linalg.eigh(H)
    return float(w[0]), dets, H


# ---------------------------------------------------------------------------
# Coupled cluster wavefunction by explicit cluster expansion
# ---------------------------------------------------------------------------


def apply_T(amps, vec, nel):
    """T|phi> with T = sum_e t_e c_e; amps: {det_e: t_e}; vec: {det: coeff}."""
    out = {}
    ops = {e: excitor_ops(e, nel) for e in amps}
    for d, c in vec.items():
        for e, t in amps.items():
            sg, d2 = apply_ops(ops[e], d)
            if sg:
                out[d2] = out.get(d2, 0.0) + sg * t * c
    return out


def cc_wavefunction(amps, nel, t_hf=1.0, max_order=None):
    """t_HF exp(T/t_HF)|HF> in the determinant basis (Sec. II, Eq. 2)."""
    hf = (1 << nel) - 1
    scaled = {e: t / t_hf for e, t in amps.items() if t != 0.0 and e != hf}
    psi = {hf: t_hf}
    term = {hf: t_hf}
    n = 0
    while term and (max_order is None or n < max_order):
        n += 1
        term = apply_T(scaled, term, nel)
        term = {d: c / n for d, c in term.items() if c != 0.0}
        for d, c in term.items():
            psi[d] = psi.get(d, 0.0) + c
    return psi


def exact_step_change(ham, dets, H, amps, t_hf, tau, shift, ehf, lmax):
    """Expected change of every excitor amplitude of level <= l in one step:
    dt_i = -tau s_D(i) sum_j (H_ij - (E_HF + S) delta_ij) <D_j|Psi>
    (Sec. II Eq. CCMC, with determinant coefficients converted to excitor
    amplitudes by s_D)."""
    nel = ham.nel
    psi = cc_wavefunction(amps, nel, t_hf)
    index = {d: i for i, d in enumerate(dets)}
    vec = np.zeros(len(dets))
    for d, c in psi.items():
        if d in index:
            vec[index[d]] += c
    hv = H @ vec - (ehf + shift) * vec
    out = {}
    for d in dets:
        if level(d, nel) <= lmax:
            out[d] = -tau * excitor_sign(d, nel) * hv[index[d]]
    return out


def solve_cc(ham, dets, H, lmax, tol=1e-12):
    """Deterministic truncated CC: <D_i|(H - E) exp(T)|HF> = 0 for every
    excitor i of level 1..l, E = <HF|H exp(T)|HF>."""
    import scipy.optimize

    nel = ham.nel
    hf = (1 << nel) - 1
    index = {d: i for i, d in enumerate(dets)}
    exc = [d for d in dets if 1 <= level(d, nel) <= lmax]

    def psi_vec(t):
        amps = dict(zip(exc, t))
        psi = cc_wavefunction(amps, nel, 1.0)
        v = np.zeros(len(dets))
        for d, c in psi.items():
            if d in index:
                v[index[d]] += c
        return v

    def resid(t):
        v = psi_vec(t)
        hv = H @ v
        e = hv[index[hf]]
        return np.array([hv[index[d]] - e * v[index[d]] for d in exc])

    sol = scipy.optimize.root(resid, np.zeros(len(exc)), method="hybr", tol=tol)
    v = psi_vec(sol.x)
    e = (H @ v)[index[hf]]
    return float(e), dict(zip(exc, sol.x)), float(np.max(np.abs(resid(sol.x)))) if exc else 0.0


# ---------------------------------------------------------------------------
# Generation probabilities by exhaustive enumeration
# ---------------------------------------------------------------------------


def r_for_index(idx, n):
    """A 64-bit value r with floor(r * n / 2^64) == idx."""
    return -((-idx << 64) // n)


def enumerate_ueg_generation(nel, nso, excite_fn, dj):
    """Probability of each outcome of the uniform UEG double-excitation
    generator from dj, by visiting every (pair, virtual) draw once."""
    npairs = nel * (nel - 1) // 2
    nvirt = nso - nel
    counts = {}
    total = npairs * nvirt
    for pi in range(npairs):
        for ai in range(nvirt):
            r = [0, r_for_index(pi, npairs), r_for_index(ai, nvirt), 0]
            res = excite_fn(dj, r)
            key = None if res is None else res[0]
            counts[key] = counts.get(key, 0) + 1
    return {k: Fraction(c, total) for k, c in counts.items()}


# ---------------------------------------------------------------------------
# Reblocking
# ---------------------------------------------------------------------------


def reblock(x):
    """Returns (mean, standard error, optimal block level, table).  Each level
    averages neighbouring pairs; the standard error at each level is
    sqrt(var/(n-1)) of the block means; the chosen level is the smallest B
    (block size 2^b) with B^3 > 2 n (se_b/se_0)^4."""
    x = np.asarray(x, dtype=np.float64)
    n0 = len(x)
    table = []
    y = x.copy()
    b = 0
    while len(y) >= 4:
        n = len(y)
        var = float(np.var(y, ddof=1))
        se = math.sqrt(var / n)
        table.append((b, n, se, se / math.sqrt(2.0 * (n - 1))))
        if n % 2:
            y = y[:-1]
        y = 0.5 * (y[0::2] + y[1::2])
        b += 1
    se0 = table[0][2]
    opt = len(table) - 1
    for b, n, se, _ in table:
        if se0 == 0.0 or (2 ** b) ** 3 > 2 * n0 * (se / se0) ** 4:
            opt = b
            break
    return float(np.mean(x)), table[opt][2], opt, table
