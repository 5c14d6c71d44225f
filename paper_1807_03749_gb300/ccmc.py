"""Thin ctypes binding of the C ABI in include/ccmc.h (argument marshalling only).

Every step of the CCMC time step runs in the CUDA kernels of libccmc.so; this
module converts Python/numpy arguments to the C structs and back.  Loading
fails loudly when the library has not been built or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64,
                    c_void_p)

import numpy as np

from . import build as _build

CCMC_UEG, CCMC_GENERIC = 0, 1
CCMC_FP64, CCMC_FP32 = 0, 1

STATUS = {
    0: "CCMC_OK", 1: "CCMC_ERR_ARG", 2: "CCMC_ERR_CUDA", 3: "CCMC_ERR_OOM", 4: "CCMC_ERR_SPAWN_OVERFLOW",
    5: "CCMC_ERR_TIMEOUT", 6: "CCMC_ERR_NUMERIC", 7: "CCMC_ERR_LIST_OVERFLOW", 8: "CCMC_ERR_STATE",
    9: "CCMC_ERR_RUNAWAY",
}

ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p)


class Hamiltonian(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("n_electrons", c_int32), ("n_spinorb", c_int32), ("reserved", c_int32),
                ("rs", c_double), ("h1", POINTER(c_double)), ("eri", POINTER(c_double)), ("e_core", c_double)]


class Reference(ctypes.Structure):
    _fields_ = [("bits", POINTER(c_uint64))]


class Params(ctypes.Structure):
    _fields_ = [("tau", c_double), ("target_pop", c_double), ("d0_init", c_double), ("shift_a", c_int32),
                ("fnc", c_int32), ("zeta", c_double), ("spawn_cutoff", c_double), ("multispawn", c_int32),
                ("precision", c_int32), ("a_thresh", c_double), ("seed", c_uint64), ("replica", c_uint64),
                ("list_capacity", c_uint64), ("spawn_capacity", c_uint64), ("cuda_stream", c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", c_void_p), ("radix_bits", c_int32),
                ("flags", c_int32), ("n_ranks", c_int32), ("nu_move", c_int32)]


class Record(ctypes.Structure):
    _fields_ = [("iter", c_uint64), ("shift", c_double), ("n0", c_int64), ("ntot", c_int64), ("n_sel", c_int64),
                ("n_visit", c_int64), ("n_attempts", c_int64), ("n_spawned", c_int64), ("e_num", c_double),
                ("ntot_after", c_int64), ("nocc_after", c_int64), ("n_keys", c_int64), ("n_clusters", c_int64),
                ("n_direct", c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class CCMCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

EXPORTS = [
    "ccmc_init", "ccmc_step", "ccmc_energy", "ccmc_reference_energy", "ccmc_get_records", "ccmc_list_size",
    "ccmc_get_list", "ccmc_set_list", "ccmc_get_spawned", "ccmc_get_death", "ccmc_set_state", "ccmc_get_state",
    "ccmc_save", "ccmc_load", "ccmc_sync", "ccmc_last_error", "ccmc_free", "ccmc_profile", "ccmc_phase_times",
    "ccmc_reduce_records_noalloc", "ccmc_batch_create", "ccmc_step_batched", "ccmc_batch_info", "ccmc_batch_free",
    "ccmc_batch_profile", "ccmc_batch_phase_times", "ccmc_colocation",
]

PHASES = ["scan", "sample", "attempts", "sort", "reduce", "merge", "finalize"]


def load(path: str | None = None):
    """Loads libccmc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    L = ctypes.CDLL(path)
    u64p, i64p, dp, i32p = POINTER(c_uint64), POINTER(c_int64), POINTER(c_double), POINTER(c_int32)
    vp = c_void_p
    sig = {
        "ccmc_init": (c_int, [POINTER(Hamiltonian), POINTER(Reference), c_int, POINTER(Params), POINTER(c_void_p)]),
        "ccmc_step": (c_int, [vp, c_int]),
        "ccmc_energy": (c_int, [vp, dp, dp, dp, dp, dp]),
        "ccmc_reference_energy": (c_int, [vp, dp]),
        "ccmc_get_records": (c_int, [vp, POINTER(Record), c_size_t, POINTER(c_size_t)]),
        "ccmc_list_size": (c_int, [vp, POINTER(c_size_t)]),
        "ccmc_get_list": (c_int, [vp, u64p, u64p, i64p, c_size_t, POINTER(c_size_t)]),
        "ccmc_set_list": (c_int, [vp, u64p, i64p, c_size_t]),
        "ccmc_get_spawned": (c_int, [vp, u64p, i64p, c_size_t, POINTER(c_size_t)]),
        "ccmc_get_death": (c_int, [vp, i64p, c_size_t, POINTER(c_size_t)]),
        "ccmc_set_state": (c_int, [vp, c_uint64, c_double, c_int32, c_double]),
        "ccmc_get_state": (c_int, [vp, u64p, dp, i32p, dp]),
        "ccmc_save": (c_int, [vp, c_char_p]),
        "ccmc_load": (c_int, [vp, c_char_p]),
        "ccmc_sync": (c_int, [vp]),
        "ccmc_last_error": (c_char_p, [vp]),
        "ccmc_free": (None, [vp]),
        "ccmc_profile": (c_int, [vp, c_int32]),
        "ccmc_phase_times": (c_int, [vp, dp, i64p, c_int32, i64p]),
        "ccmc_reduce_records_noalloc": (c_int, [vp, vp, c_size_t, c_int32, vp, vp, POINTER(c_size_t), vp]),
        "ccmc_batch_create": (c_int, [POINTER(c_void_p), c_int32, vp, POINTER(c_void_p)]),
        "ccmc_step_batched": (c_int, [vp, c_int32]),
        "ccmc_batch_info": (c_int, [vp, i32p, i32p, i32p, i32p, i32p]),
        "ccmc_batch_free": (None, [vp]),
        "ccmc_batch_profile": (c_int, [vp, c_int32]),
        "ccmc_batch_phase_times": (c_int, [vp, dp, i64p, c_int32, i64p]),
        "ccmc_colocation": (c_int, [u64p, c_size_t, c_int32, c_int64, c_int32, i64p, c_int32, u64p, u64p, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(POINTER(ct)) if a is not None else None


def torch_allocator():
    """(alloc, free) callbacks that take device memory from PyTorch's caching
    allocator on the current device and stream."""
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), FREE_FN(_free)


class Context:
    """One CCMC wavefunction on the GPU (a ccmc_ctx)."""

    def __init__(self, kind: str, nel: int, nso: int, lmax: int, *, rs: float = 1.0, h1=None, eri=None,
                 e_core: float = 0.0, tau: float = 0.01, target_pop: float = 1e4, d0_init: float = 100.0,
                 shift_a: int = 10, zeta: float = 0.05, spawn_cutoff: float = 2.0 ** -7, fnc: bool = False,
                 multispawn: bool = False, a_thresh: float = 1.0, seed: int = 1, replica: int = 0,
                 precision: str = "fp64", list_capacity: int = 0, spawn_capacity: int = 0, stream=None,
                 use_torch_allocator: bool = False, radix_bits: int = 0, use_graph: bool = True,
                 sort_all: bool = False, n_ranks: int = 1, nu_move: int = 64, **_ignored):
        L = load()
        self._lib = L
        self.nel, self.nso, self.lmax = nel, nso, lmax
        self.nw = (nso + 63) // 64
        ham = Hamiltonian()
        ham.kind = CCMC_UEG if kind == "ueg" else CCMC_GENERIC
        ham.n_electrons = nel
        ham.n_spinorb = nso
        ham.rs = rs
        ham.e_core = e_core
        self._keep = []
        if ham.kind == CCMC_GENERIC:
            h1 = np.ascontiguousarray(h1, dtype=np.float64)
            eri = np.ascontiguousarray(eri, dtype=np.float64)
            self._keep += [h1, eri]
            ham.h1 = _ptr(h1, c_double)
            ham.eri = _ptr(eri, c_double)
        p = Params()
        p.tau, p.target_pop, p.d0_init = tau, target_pop, d0_init
        p.shift_a, p.fnc, p.zeta, p.spawn_cutoff = shift_a, int(fnc), zeta, spawn_cutoff
        p.multispawn, p.a_thresh = int(multispawn), a_thresh
        p.precision = CCMC_FP32 if precision == "fp32" else CCMC_FP64
        p.seed, p.replica = seed, replica
        p.list_capacity, p.spawn_capacity = list_capacity, spawn_capacity
        p.radix_bits = radix_bits
        p.flags = (0 if use_graph else 1) | (2 if sort_all else 0)
        p.n_ranks, p.nu_move = n_ranks, nu_move
        if stream is not None:
            p.cuda_stream = c_void_p(int(stream))
        if use_torch_allocator:
            fa, ff = torch_allocator()
            self._keep += [fa, ff]
            p.alloc, p.free = fa, ff
        self._params = p
        h = c_void_p(0)
        st = L.ccmc_init(ctypes.byref(ham), None, lmax, ctypes.byref(p), ctypes.byref(h))
        if st != 0:
            raise CCMCError(st, "ccmc_init failed")
        self._h = h

    # -- helpers -----------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            msg = self._lib.ccmc_last_error(self._h)
            raise CCMCError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.ccmc_free(self._h)
            self._h = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI mirrors ---------------------------------------------------------
    def step(self, nsteps: int = 1):
        self._check(self._lib.ccmc_step(self._h, nsteps))

    def energy(self) -> dict:
        v = [c_double(0.0) for _ in range(5)]
        self._check(self._lib.ccmc_energy(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(["e_proj", "e_num", "n0", "shift", "n_total"], [x.value for x in v]))

    def reference_energy(self) -> float:
        e = c_double(0.0)
        self._check(self._lib.ccmc_reference_energy(self._h, ctypes.byref(e)))
        return e.value

    def records(self, cap: int = 1 << 14) -> list[dict]:
        buf = (Record * cap)()
        n = c_size_t(0)
        self._check(self._lib.ccmc_get_records(self._h, buf, cap, ctypes.byref(n)))
        return [buf[i].as_dict() for i in range(n.value)]

    def list_size(self) -> int:
        n = c_size_t(0)
        self._check(self._lib.ccmc_list_size(self._h, ctypes.byref(n)))
        return n.value

    def get_list(self, out=None, with_keys: bool = True):
        """(bits[n, K] uint64, keys[n] uint64, pop[n] int64) in key order.
        With out = (bits, keys, pop) of room for the list (for instance pinned
        host buffers), those are filled and views of their first n rows
        returned.  with_keys=False skips the keys (None in their place): a
        list uploaded again with set_list has its keys recomputed anyway."""
        n = self.list_size()
        if out is None:
            bits = np.zeros((n, self.nw), dtype=np.uint64)
            keys = np.zeros(n, dtype=np.uint64) if with_keys else None
            pop = np.zeros(n, dtype=np.int64)
        else:
            bits, keys, pop = out
            if not with_keys:
                keys = None
            if len(pop) < n or (keys is not None and len(keys) < n) or bits.shape[0] < n or bits.shape[1] != self.nw:
                raise ValueError("output buffers too small")
            if not (bits.flags.c_contiguous and pop.flags.c_contiguous and (keys is None or keys.flags.c_contiguous)):
                raise ValueError("output buffers must be contiguous")
        m = c_size_t(0)
        kp = _ptr(keys, c_uint64) if keys is not None else None
        self._check(self._lib.ccmc_get_list(self._h, _ptr(bits, c_uint64), kp, _ptr(pop, c_int64), n, ctypes.byref(m)))
        return bits[:n], (keys[:n] if keys is not None else None), pop[:n]

    def set_list(self, bits: np.ndarray, pop: np.ndarray):
        bits = np.ascontiguousarray(bits, dtype=np.uint64).reshape(-1, self.nw)
        pop = np.ascontiguousarray(pop, dtype=np.int64)
        self._check(self._lib.ccmc_set_list(self._h, _ptr(bits, c_uint64), _ptr(pop, c_int64), len(pop)))

    def get_spawned(self):
        """Sorted (keys, pops) of the spawned records of the latest step."""
        n = c_size_t(0)
        cap = self._spawned_count()
        keys = np.zeros(cap, dtype=np.uint64)
        pop = np.zeros(cap, dtype=np.int64)
        self._check(self._lib.ccmc_get_spawned(self._h, _ptr(keys, c_uint64), _ptr(pop, c_int64), cap,
                                               ctypes.byref(n)))
        return keys[: n.value], pop[: n.value]

    def _spawned_count(self) -> int:
        n = c_size_t(0)
        st = self._lib.ccmc_get_spawned(self._h, None, None, 0, ctypes.byref(n))
        if st not in (0, 1):
            self._check(st)
        return n.value

    def get_death(self):
        n = c_size_t(0)
        st = self._lib.ccmc_get_death(self._h, None, 0, ctypes.byref(n))
        if st not in (0, 1):
            self._check(st)
        out = np.zeros(n.value, dtype=np.int64)
        self._check(self._lib.ccmc_get_death(self._h, _ptr(out, c_int64), n.value, ctypes.byref(n)))
        return out

    def set_state(self, it: int, shift: float, vary: bool, nprev: float):
        self._check(self._lib.ccmc_set_state(self._h, it, shift, int(vary), nprev))

    def get_state(self):
        it, sh, vy, npv = c_uint64(0), c_double(0.0), c_int32(0), c_double(0.0)
        self._check(self._lib.ccmc_get_state(self._h, ctypes.byref(it), ctypes.byref(sh), ctypes.byref(vy),
                                             ctypes.byref(npv)))
        return int(it.value), sh.value, bool(vy.value), npv.value

    def save(self, path: str):
        self._check(self._lib.ccmc_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        self._check(self._lib.ccmc_load(self._h, os.fsencode(path)))

    def sync(self):
        self._check(self._lib.ccmc_sync(self._h))

    def profile(self, enable: bool = True):
        self._check(self._lib.ccmc_profile(self._h, int(enable)))

    def phase_times(self):
        """({phase: ms}, {phase: launches}, total kernel launches)."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        la = np.zeros(len(PHASES), dtype=np.int64)
        tot = c_int64(0)
        self._check(self._lib.ccmc_phase_times(self._h, _ptr(ms, c_double), _ptr(la, c_int64), len(PHASES),
                                               ctypes.byref(tot)))
        return dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, la.tolist())), int(tot.value)


class Batch:
    """Several contexts stepped together (one launch per phase over all of
    them, replayed from a CUDA graph).  The contexts stay usable for reading
    results and checkpoints but must not be stepped on their own."""

    def __init__(self, contexts, stream):
        L = load()
        self._lib = L
        self.contexts = list(contexts)
        arr = (c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = c_void_p(0)
        st = L.ccmc_batch_create(arr, len(self.contexts), c_void_p(int(stream)), ctypes.byref(h))
        if st != 0:
            raise CCMCError(st, "ccmc_batch_create failed")
        self._h = h

    def step(self, nsteps: int = 1):
        st = self._lib.ccmc_step_batched(self._h, nsteps)
        if st != 0:
            why = []
            for i, c in enumerate(self.contexts):
                msg = self._lib.ccmc_last_error(c._h)
                if msg:
                    why.append(f"context {i}: {msg.decode()}")
            raise CCMCError(st, "ccmc_step_batched failed" + ("; " + "; ".join(why) if why else ""))

    def info(self) -> dict:
        w, t, d, g, n = c_int32(0), c_int32(0), c_int32(0), c_int32(0), c_int32(0)
        self._lib.ccmc_batch_info(self._h, ctypes.byref(w), ctypes.byref(t), ctypes.byref(d), ctypes.byref(g),
                                  ctypes.byref(n))
        return {"work_blocks": w.value, "sample_tile": t.value, "digit_bits": d.value, "groups": g.value,
                "tunings": n.value}

    def profile(self, enable: bool = True):
        if self._lib.ccmc_batch_profile(self._h, int(enable)):
            raise CCMCError(2, "ccmc_batch_profile failed")

    def phase_times(self):
        ms = np.zeros(len(PHASES), dtype=np.float64)
        la = np.zeros(len(PHASES), dtype=np.int64)
        tot = c_int64(0)
        self._lib.ccmc_batch_phase_times(self._h, _ptr(ms, c_double), _ptr(la, c_int64), len(PHASES),
                                         ctypes.byref(tot))
        return dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, la.tolist())), int(tot.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.ccmc_batch_free(self._h)
            self._h = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def colocation(dets: np.ndarray, n_ranks: int, nu_move: int, checkpoints, stream=None):
    """Co-location sums of the simulated distribution (ccmc_colocation): for
    each checkpoint T, (sum over pairs of C_ij(T), sum of C_ij(T)^2)."""
    L = load()
    d = np.ascontiguousarray(dets, dtype=np.uint64)
    if d.ndim == 1:
        d = d.reshape(-1, 1)
    ck = np.ascontiguousarray(checkpoints, dtype=np.int64)
    s1 = np.zeros(len(ck), dtype=np.uint64)
    s2 = np.zeros(len(ck), dtype=np.uint64)
    st = L.ccmc_colocation(_ptr(d, c_uint64), d.shape[0], d.shape[1], n_ranks, nu_move, _ptr(ck, c_int64), len(ck),
                           _ptr(s1, c_uint64), _ptr(s2, c_uint64), c_void_p(int(stream)) if stream else None)
    if st != 0:
        raise CCMCError(st, "ccmc_colocation failed")
    return s1, s2


def from_workload(w: dict, **overrides) -> Context:
    """A context for a workload description (see ccmc_inputs)."""
    w = dict(w)
    w.update(overrides)
    if w["kind"] == "generic" and "h1" not in w:
        from ccmc_inputs import molecule_integrals

        h1, eri = molecule_integrals(norb=w["norb"], nocc=w["nel"] // 2, seed=w.get("molecule_seed", 7),
                                     scale=w.get("eri_scale", 1.0))
        w["h1"], w["eri"] = h1, eri
    nso = w.get("nso", 2 * w.get("norb", 0))
    return Context(w["kind"], w["nel"], nso, w["lmax"], **{k: v for k, v in w.items()
                                                            if k not in ("kind", "nel", "nso", "lmax", "norb")})
