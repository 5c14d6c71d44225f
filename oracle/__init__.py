"""Plain CPU oracle of one CCMC time step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it shares
no code with the CUDA library, and the two meet only through the seeded input
generators in ``ccmc_inputs``.

The arithmetic lives in ``ccmc_oracle.c`` (plain C, FP64, no fused
multiply-add); this module compiles it with gcc and wraps it with ctypes.
The brute-force references that pin the oracle live in ``oracle.brute``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccmc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libccmc_oracle.so")

FIX_ONE = 1 << 16

# Philox counter tags (bits 56..63 of counter word 1)
TAG_SAMPLE, TAG_SAMPLE_ATT, TAG_VISIT, TAG_VISIT_ATT, TAG_THRESH = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("tau", c_double),
        ("target_pop", c_double),
        ("d0_init", c_double),
        ("shift_a", c_int32),
        ("fnc", c_int32),
        ("zeta", c_double),
        ("spawn_cutoff", c_double),
        ("multispawn", c_int32),
        ("n_ranks", c_int32),
        ("a_thresh", c_double),
        ("seed", c_uint64),
        ("replica", c_uint64),
        ("nu_move", c_int32),
        ("pad1", c_int32),
    ]


class Record(ctypes.Structure):
    _fields_ = [
        ("iter", c_uint64),
        ("shift", c_double),
        ("n0", c_int64),
        ("ntot", c_int64),
        ("n_sel", c_int64),
        ("n_visit", c_int64),
        ("n_attempts", c_int64),
        ("n_spawned", c_int64),
        ("e_num", c_double),
        ("ntot_after", c_int64),
        ("nocc_after", c_int64),
        ("n_keys", c_int64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u64p, i64p, dp, i32p = POINTER(c_uint64), POINTER(c_int64), POINTER(c_double), POINTER(c_int32)
        sig = {
            "orc_ueg_new": (c_void_p, [c_int, c_int, c_double, c_int]),
            "orc_generic_new": (c_void_p, [c_int, c_int, dp, dp, c_double, c_int]),
            "orc_system_free": (None, [c_void_p]),
            "orc_sys_info": (None, [c_void_p, i32p]),
            "orc_ehf": (c_double, [c_void_p]),
            "orc_ueg_length": (c_double, [c_void_p]),
            "orc_hf": (None, [c_void_p, u64p]),
            "orc_ueg_kvec": (None, [c_void_p, i32p]),
            "orc_ueg_tkin": (c_double, [c_void_p, c_int]),
            "orc_ueg_vq": (c_double, [c_void_p, c_int]),
            "orc_hij": (c_double, [c_void_p, u64p, u64p]),
            "orc_hij_f": (c_double, [c_void_p, u64p, u64p]),
            "orc_system_set_fp32": (c_int, [c_void_p]),
            "orc_hdiag_rel": (c_double, [c_void_p, u64p]),
            "orc_hdiag_rel_f": (c_double, [c_void_p, u64p]),
            "orc_excitor_sign": (c_int, [c_void_p, u64p]),
            "orc_level": (c_int, [c_void_p, u64p]),
            "orc_collapse": (c_int, [c_void_p, c_int, u64p, u64p, i32p]),
            "orc_rank": (c_uint64, [c_void_p, u64p]),
            "orc_unrank": (None, [c_void_p, c_uint64, u64p]),
            "orc_key_bound": (c_uint64, [c_void_p]),
            "orc_excite": (c_int, [c_void_p, u64p, u64p, u64p, dp, dp]),
            "orc_philox": (None, [u64p, u64p, u64p]),
            "orc_det_hash": (c_uint64, [u64p, c_int]),
            "orc_owner": (c_uint64, [u64p, c_int, c_uint64, c_int, c_uint64]),
            "orc_colocation": (None, [u64p, c_int64, c_int, c_int64, c_int, c_int64, i64p, c_int, u64p, u64p]),
            "orc_size_draw": (c_int, [c_uint64, c_int, c_int]),
            "orc_pick_index": (c_int64, [i64p, c_int64, c_uint64]),
            "orc_below": (c_uint64, [c_uint64, c_uint64]),
            "orc_stoch_round": (c_int64, [c_double, c_double, c_double]),
            "orc_sim_new": (c_void_p, [c_void_p, POINTER(Params)]),
            "orc_sim_free": (None, [c_void_p]),
            "orc_sim_step": (c_int, [c_void_p, c_int]),
            "orc_sim_run": (c_int, [c_void_p, c_int, POINTER(Record)]),
            "orc_sim_set_list": (c_int, [c_void_p, c_int64, u64p, i64p]),
            "orc_sim_size": (c_int64, [c_void_p]),
            "orc_sim_get_list": (None, [c_void_p, u64p, u64p, i64p]),
            "orc_sim_nspawned": (c_int64, [c_void_p]),
            "orc_sim_get_spawned": (None, [c_void_p, u64p, i64p]),
            "orc_sim_get_death": (None, [c_void_p, i64p]),
            "orc_sim_ndeath": (c_int64, [c_void_p]),
            "orc_sim_get_record": (None, [c_void_p, POINTER(Record)]),
            "orc_sim_set_state": (None, [c_void_p, c_uint64, c_double, c_int32, c_double]),
            "orc_sim_get_state": (None, [c_void_p, u64p, dp, i32p, dp]),
            "orc_sim_sample_range": (c_int, [c_void_p, c_int64, c_int64, c_int64, c_int64]),
            "orc_generator_closure": (c_int64, [c_void_p, c_int, c_int, u64p, c_int64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(POINTER(c_uint64))


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(POINTER(c_int64))


def det_hash(words) -> int:
    """The determinant hash of the simulated distribution (Sec. III)."""
    w, wp = _u64(words)
    return int(lib().orc_det_hash(wp, len(w)))


def owner(words, it: int, nu_move: int, n_ranks: int) -> int:
    """Processor of an excitor at iteration it (Sec. III, Eq. ccmc_dist)."""
    w, wp = _u64(words)
    return int(lib().orc_owner(wp, len(w), c_uint64(it), nu_move, c_uint64(n_ranks)))


def colocation(dets: np.ndarray, n_ranks: int, nu_move: int, checkpoints) -> tuple:
    """Sums over excitor pairs of C_ij(T) and C_ij(T)^2 at each checkpoint T,
    C_ij(T) = iterations t < T with i and j on the same processor."""
    d = np.ascontiguousarray(dets, dtype=np.uint64)
    ck = np.ascontiguousarray(checkpoints, dtype=np.int64)
    s1 = np.zeros(len(ck), dtype=np.uint64)
    s2 = np.zeros(len(ck), dtype=np.uint64)
    lib().orc_colocation(d.ctypes.data_as(POINTER(c_uint64)), d.shape[0], d.shape[1], n_ranks, nu_move,
                         int(ck[-1]), ck.ctypes.data_as(POINTER(c_int64)), len(ck),
                         s1.ctypes.data_as(POINTER(c_uint64)), s2.ctypes.data_as(POINTER(c_uint64)))
    return s1, s2


def philox(ctr, key) -> np.ndarray:
    """Philox-4x64-10 block for a 4-word counter and a 2-word key."""
    c, cp = _u64(ctr)
    k, kp = _u64(key)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox(cp, kp, out.ctypes.data_as(POINTER(c_uint64)))
    return out


def size_draw(r0: int, lmax: int, fnc: bool) -> int:
    return lib().orc_size_draw(c_uint64(r0), lmax, int(fnc))


def below(r: int, n: int) -> int:
    return int(lib().orc_below(c_uint64(r), c_uint64(n)))


def pick_index(prefix, x: int) -> int:
    p, pp = _i64(prefix)
    return int(lib().orc_pick_index(pp, len(p), c_uint64(x)))


def stoch_round(x: float, u: float, cutoff: float) -> int:
    return int(lib().orc_stoch_round(x, u, cutoff))


class System:
    """A Hamiltonian with its Hartree-Fock reference and truncation level."""

    def __init__(self, handle):
        if not handle:
            raise ValueError("oracle rejected the system description")
        self._h = c_void_p(handle)
        info = np.zeros(5, dtype=np.int32)
        lib().orc_sys_info(self._h, info.ctypes.data_as(POINTER(c_int32)))
        self.nel, self.nso, self.nw, self.lmax, self.kind = (int(v) for v in info)

    @classmethod
    def ueg(cls, nel: int, nso: int, rs: float, lmax: int) -> "System":
        return cls(lib().orc_ueg_new(nel, nso, rs, lmax))

    @classmethod
    def generic(cls, nel: int, h1: np.ndarray, eri: np.ndarray, lmax: int, ecore: float = 0.0) -> "System":
        norb = h1.shape[0]
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64).reshape(norb ** 4)
        obj = cls(lib().orc_generic_new(nel, norb, h1.ctypes.data_as(POINTER(c_double)),
                                        eri.ctypes.data_as(POINTER(c_double)), ecore, lmax))
        return obj

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().orc_system_free(self._h)
                self._h = None
        except Exception:
            pass

    # --- helpers: determinants are python ints (bit p = spin-orbital p) ---
    def to_words(self, d: int) -> np.ndarray:
        return np.array([(d >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(self.nw)], dtype=np.uint64)

    def from_words(self, w) -> int:
        return sum(int(w[i]) << (64 * i) for i in range(self.nw))

    def hf(self) -> int:
        return (1 << self.nel) - 1

    def ehf(self) -> float:
        return lib().orc_ehf(self._h)

    def length(self) -> float:
        return lib().orc_ueg_length(self._h)

    def kvecs(self) -> np.ndarray:
        out = np.zeros((self.nso // 2, 3), dtype=np.int32)
        lib().orc_ueg_kvec(self._h, out.ctypes.data_as(POINTER(c_int32)))
        return out

    def tkin(self, p: int) -> float:
        return lib().orc_ueg_tkin(self._h, p)

    def vq(self, n2: int) -> float:
        return lib().orc_ueg_vq(self._h, n2)

    def hij(self, bra: int, ket: int) -> float:
        b, bp = _u64(self.to_words(bra))
        k, kp = _u64(self.to_words(ket))
        return lib().orc_hij(self._h, bp, kp)

    def hij_f(self, bra: int, ket: int) -> float:
        """<bra|H|ket> of the FP32 form (after set_fp32)."""
        b, bp = _u64(self.to_words(bra))
        k, kp = _u64(self.to_words(ket))
        return lib().orc_hij_f(self._h, bp, kp)

    def set_fp32(self):
        """Matrix elements and generation probabilities in single precision."""
        if lib().orc_system_set_fp32(self._h):
            raise MemoryError("orc_system_set_fp32 failed")
        self.fp32 = True
        return self

    def hdiag_rel(self, d: int) -> float:
        """H_DD - E_HF in the excitation form the step uses."""
        w, wp = _u64(self.to_words(d))
        return lib().orc_hdiag_rel(self._h, wp)

    def hdiag_rel_f(self, d: int) -> float:
        """The same in single precision (FP32 form; the system must be set_fp32)."""
        w, wp = _u64(self.to_words(d))
        return lib().orc_hdiag_rel_f(self._h, wp)

    def excitor_sign(self, d: int) -> int:
        w, wp = _u64(self.to_words(d))
        return lib().orc_excitor_sign(self._h, wp)

    def level(self, d: int) -> int:
        w, wp = _u64(self.to_words(d))
        return lib().orc_level(self._h, wp)

    def collapse(self, excitors):
        ex = np.concatenate([self.to_words(e) for e in excitors])
        e, ep = _u64(ex)
        out = np.zeros(self.nw, dtype=np.uint64)
        sg = c_int32(0)
        ok = lib().orc_collapse(self._h, len(excitors), ep, out.ctypes.data_as(POINTER(c_uint64)), ctypes.byref(sg))
        if not ok:
            return None
        return self.from_words(out), int(sg.value)

    def rank(self, d: int) -> int:
        w, wp = _u64(self.to_words(d))
        return int(lib().orc_rank(self._h, wp))

    def unrank(self, key: int) -> int:
        out = np.zeros(self.nw, dtype=np.uint64)
        lib().orc_unrank(self._h, c_uint64(key), out.ctypes.data_as(POINTER(c_uint64)))
        return self.from_words(out)

    def generator_closure(self, max_level: int, expand_top: bool = True) -> int:
        """Determinants reached from HF by repeated excitation-generator draws."""
        return int(lib().orc_generator_closure(self._h, max_level, int(expand_top), None, 0))

    def space_keys(self, max_level: int, expand_top: bool = True) -> np.ndarray:
        """Sorted rank keys of every determinant reached by the closure."""
        n = self.generator_closure(max_level, expand_top)
        out = np.zeros(n, dtype=np.uint64)
        lib().orc_generator_closure(self._h, max_level, int(expand_top), out.ctypes.data_as(POINTER(c_uint64)), n)
        return out

    def key_bound(self) -> int:
        return int(lib().orc_key_bound(self._h))

    def excite(self, dj: int, r):
        w, wp = _u64(self.to_words(dj))
        rr, rp = _u64(r)
        out = np.zeros(self.nw, dtype=np.uint64)
        h = c_double(0.0)
        ip = c_double(0.0)
        ok = lib().orc_excite(self._h, wp, rp, out.ctypes.data_as(POINTER(c_uint64)), ctypes.byref(h), ctypes.byref(ip))
        if not ok:
            return None
        return self.from_words(out), h.value, ip.value


def default_params(**kw) -> Params:
    p = Params()
    p.tau = kw.get("tau", 0.01)
    p.target_pop = kw.get("target_pop", 1e4)
    p.d0_init = kw.get("d0_init", 100.0)
    p.shift_a = kw.get("shift_a", 10)
    p.fnc = int(kw.get("fnc", 0))
    p.zeta = kw.get("zeta", 0.05)
    p.spawn_cutoff = kw.get("spawn_cutoff", 2.0 ** -7)
    p.multispawn = int(kw.get("multispawn", 0))
    p.n_ranks = int(kw.get("n_ranks", 1))
    p.nu_move = int(kw.get("nu_move", 64))
    p.pad1 = 0
    p.a_thresh = kw.get("a_thresh", 1.0)
    p.seed = kw.get("seed", 1)
    p.replica = kw.get("replica", 0)
    return p


class Sim:
    """One CCMC walker population evolving under the oracle step."""

    def __init__(self, system: System, **params):
        self.system = system
        self.params = default_params(**params)
        h = lib().orc_sim_new(system._h, ctypes.byref(self.params))
        if not h:
            raise MemoryError("orc_sim_new failed")
        self._h = c_void_p(h)

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().orc_sim_free(self._h)
                self._h = None
        except Exception:
            pass

    def set_list(self, dets, pops):
        s = self.system
        bits = np.concatenate([s.to_words(d) for d in dets]) if len(dets) else np.zeros(0, np.uint64)
        b, bp = _u64(bits)
        p, pp = _i64(pops)
        rc = lib().orc_sim_set_list(self._h, len(dets), bp, pp)
        if rc:
            raise ValueError(f"orc_sim_set_list failed ({rc})")

    def set_list_words(self, bits: np.ndarray, pops: np.ndarray):
        b, bp = _u64(bits.reshape(-1))
        p, pp = _i64(pops)
        rc = lib().orc_sim_set_list(self._h, len(p), bp, pp)
        if rc:
            raise ValueError(f"orc_sim_set_list failed ({rc})")

    def size(self) -> int:
        return int(lib().orc_sim_size(self._h))

    def get_list(self):
        """Returns (bits[n, nw] uint64, keys[n] uint64, pop[n] int64)."""
        n = self.size()
        bits = np.zeros((n, self.system.nw), dtype=np.uint64)
        keys = np.zeros(n, dtype=np.uint64)
        pop = np.zeros(n, dtype=np.int64)
        lib().orc_sim_get_list(self._h, bits.ctypes.data_as(POINTER(c_uint64)),
                               keys.ctypes.data_as(POINTER(c_uint64)), pop.ctypes.data_as(POINTER(c_int64)))
        return bits, keys, pop

    def step(self, propagate_only: bool = False) -> Record:
        rc = lib().orc_sim_step(self._h, int(propagate_only))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")
        return self.record()

    def sample_range(self, i_lo: int, i_hi: int, g_lo: int, g_hi: int) -> Record:
        """Propagate only the visits [i_lo, i_hi) and samples [g_lo, g_hi)."""
        rc = lib().orc_sim_sample_range(self._h, i_lo, i_hi, g_lo, g_hi)
        if rc:
            raise RuntimeError(f"oracle sample_range failed ({rc})")
        return self.record()

    def run(self, nsteps: int):
        recs = (Record * nsteps)()
        rc = lib().orc_sim_run(self._h, nsteps, recs)
        if rc:
            raise RuntimeError(f"oracle run failed ({rc})")
        return [r.as_dict() for r in recs]

    def record(self) -> Record:
        r = Record()
        lib().orc_sim_get_record(self._h, ctypes.byref(r))
        return r

    def spawned(self):
        n = int(lib().orc_sim_nspawned(self._h))
        keys = np.zeros(n, dtype=np.uint64)
        pop = np.zeros(n, dtype=np.int64)
        lib().orc_sim_get_spawned(self._h, keys.ctypes.data_as(POINTER(c_uint64)), pop.ctypes.data_as(POINTER(c_int64)))
        return keys, pop

    def death(self) -> np.ndarray:
        """Death deltas of the latest step, for the list at that step's start."""
        out = np.zeros(int(lib().orc_sim_ndeath(self._h)), dtype=np.int64)
        lib().orc_sim_get_death(self._h, out.ctypes.data_as(POINTER(c_int64)))
        return out

    def set_state(self, it: int, shift: float, vary: bool, nprev: float):
        lib().orc_sim_set_state(self._h, c_uint64(it), shift, int(vary), nprev)

    def get_state(self):
        it = c_uint64(0)
        sh = c_double(0.0)
        vy = c_int32(0)
        npv = c_double(0.0)
        lib().orc_sim_get_state(self._h, ctypes.byref(it), ctypes.byref(sh), ctypes.byref(vy), ctypes.byref(npv))
        return int(it.value), sh.value, bool(vy.value), npv.value
